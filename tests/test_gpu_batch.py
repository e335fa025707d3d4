"""GPU tests of the batched solver (independent 2-D problems, mixed precision).

The batch runs the same blocked FP32 sweep, FP64 residual and FP64 update as a
single mixed-precision plan, chunks each cycle the same way and scales the
defect by the same power of two, so every problem's iterate must equal the
single-plan solve bit for bit (same cycle count).  Residuals are re-checked
with the oracle.
"""
import numpy as np
import pytest

import oracle
import srj_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1511_04292_gb300 as srj  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _problem(n, P, seed):
    row = srj.schedules.lookup(2, n, P)
    f, u0 = W.random_smooth_problem_2d(n, seed)
    return dict(dims=(n, n), h=1.0 / (n + 1), omega=row["omega"], q=row["q"], order=row["order"]), f, u0


def test_batch_matches_single_plan_solves_bit_for_bit():
    specs = [(64, 5, 1), (128, 7, 3), (256, 6, 5), (64, 10, 7), (128, 5, 9), (512, 8, 11)]
    probs, fs, u0s = zip(*[_problem(*s) for s in specs])
    T = 8
    batch = srj.Batch(list(probs), temporal_depth=T)
    fd = [torch.from_numpy(f).cuda() for f in fs]
    ud = [torch.from_numpy(u).cuda() for u in u0s]
    stats, ms, rc = batch.solve(fd, ud, 1e-10, 200)
    assert rc == 0 and ms > 0
    for (n, P, _), pr, f, u0, u, st in zip(specs, probs, fs, u0s, ud, stats):
        plan = srj.Plan.from_table((n, n), P, "mixed")
        plan.set_temporal_depth(T)
        ref = torch.from_numpy(u0).cuda()
        st1 = plan.solve(torch.from_numpy(f).cuda(), ref, 1e-10, 200)
        assert st["cycles"] == st1["cycles"], (n, P)
        assert torch.equal(u, ref), (n, P)
        r0, _ = oracle.residual((n, n), pr["h"], f, u0)
        l2, _ = oracle.residual((n, n), pr["h"], f, u.cpu().numpy())
        assert l2 <= 1e-10 * r0 * (1 + 1e-9)


def test_more_problems_than_one_step_block():
    """300 problems: the per-phase step kernel (one thread per problem, 256
    per block) runs on more than one block, and the row blocks due at a cycle
    end come from both.  Sampled problems equal their single-plan solves bit
    for bit; every residual is re-checked by the oracle."""
    rng = np.random.default_rng(17)
    specs = [(64, int(P), 2000 + i) for i, P in enumerate(rng.integers(5, 11, size=300))]
    probs, fs, u0s = zip(*[_problem(*s) for s in specs])
    T = 8
    batch = srj.Batch(list(probs), temporal_depth=T)
    ud = [torch.from_numpy(u).cuda() for u in u0s]
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda() for f in fs], ud, 1e-10, 200)
    assert rc == 0
    for i in range(0, len(specs), 23):
        n, P, _ = specs[i]
        plan = srj.Plan.from_table((n, n), P, "mixed")
        plan.set_temporal_depth(T)
        ref = torch.from_numpy(u0s[i]).cuda()
        st1 = plan.solve(torch.from_numpy(fs[i]).cuda(), ref, 1e-10, 200)
        assert stats[i]["cycles"] == st1["cycles"] and torch.equal(ud[i], ref), (i, P)
    for (n, P, _), pr, f, u0, u in zip(specs, probs, fs, u0s, ud):
        r0, _ = oracle.residual((n, n), pr["h"], f, u0)
        l2, _ = oracle.residual((n, n), pr["h"], f, u.cpu().numpy())
        assert l2 <= 1e-10 * r0 * (1 + 1e-9)


def test_batch_ragged_sizes_and_own_orders():
    """Non-square and non-table grids with schedules from the oracle's solver and
    the library's own order (order=None)."""
    from oracle import schedule as S
    probs, fs, u0s = [], [], []
    for i, dims in enumerate([(37, 23), (200, 3), (1, 1), (129, 250)]):
        km = oracle.kappa_min_dirichlet(dims)
        P = 1 if dims == (1, 1) else 4
        if P == 1:
            omega, q = np.array([1.0]), np.array([1])
        else:
            omega, beta, _ = S.solve_optimal(P, km)
            q = S.q_floor(beta)
        probs.append(dict(dims=dims, h=1.0 / (max(dims) + 1), omega=omega, q=q, order=None))
        fs.append(W.random_field(dims, 50 + i))
        u = W.random_field(dims, 60 + i); u[1:-1, 1:-1] = 0
        u0s.append(u)
    batch = srj.Batch(probs, temporal_depth=5)
    ud = [torch.from_numpy(u).cuda() for u in u0s]
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda() for f in fs], ud, 1e-10, 5000)
    assert rc == 0
    for pr, f, u0, u in zip(probs, fs, u0s, ud):
        r0, _ = oracle.residual(pr["dims"], pr["h"], f, u0)
        l2, _ = oracle.residual(pr["dims"], pr["h"], f, u.cpu().numpy())
        assert l2 <= 1e-10 * r0 * (1 + 1e-9)


def test_batch_statuses():
    pr, f, u0 = _problem(64, 5, 1)
    batch = srj.Batch([pr, pr], temporal_depth=4)
    bad = f.copy(); bad[3, 3] = np.inf
    ud = [torch.from_numpy(u0).cuda(), torch.from_numpy(u0).cuda()]
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda(), torch.from_numpy(bad).cuda()], ud, 1e-10, 100,
                                raise_on_fail=False)
    assert rc == -4 and stats[0]["rel_res"] <= 1e-10
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda()] * 2, ud, 1e-14, 1, raise_on_fail=False)
    assert rc == -3 and all(s["cycles"] == 1 for s in stats)


def test_full_batched_workload_converges():
    """Workload 4: 256 problems, n in {64..1024}, P in 5..10, random smooth f and
    polynomial boundary data, tol 1e-10; every residual re-checked by the oracle."""
    specs = W.batch_specs()
    probs, fs, u0s = zip(*[_problem(n, P, seed) for n, P, seed in specs])
    batch = srj.Batch(list(probs))
    ud = [torch.from_numpy(u).cuda() for u in u0s]
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda() for f in fs], ud, 1e-10, 500)
    assert rc == 0
    for pr, f, u0, u in zip(probs, fs, u0s, ud):
        r0, _ = oracle.residual(pr["dims"], pr["h"], f, u0)
        l2, _ = oracle.residual(pr["dims"], pr["h"], f, u.cpu().numpy())
        assert l2 <= 1e-10 * r0 * (1 + 1e-9)


def test_batch_stagnation_flag():
    pr, f, u0 = _problem(128, 6, 2)
    batch = srj.Batch([pr, pr], temporal_depth=6)
    ud = [torch.from_numpy(u0).cuda() for _ in range(2)]
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda()] * 2, ud, 1e-30, 10000, raise_on_fail=False)
    assert rc == -3 and all(s["stagnated"] == 1 and s["cycles"] < 200 and s["rel_res"] < 1e-11 for s in stats)


def test_many_grid_sizes_use_the_tile_list_sweep_bit_for_bit():
    """More distinct grid sizes than the grouped sweep takes (16): the batch runs
    the tile-list sweep, and every problem still equals its single-plan solve
    bit for bit."""
    from oracle import schedule as S
    T = 6
    dims_list = [(30 + 3 * i, 20 + 2 * i) for i in range(18)]
    probs, fs, u0s, plans = [], [], [], []
    for i, dims in enumerate(dims_list):
        km = oracle.kappa_min_dirichlet(dims)
        omega, beta, _ = S.solve_optimal(4, km)
        q = S.q_floor(beta)
        order = S.order_drift(omega, q, km)
        h = 1.0 / (max(dims) + 1)
        probs.append(dict(dims=dims, h=h, omega=omega, q=q, order=order))
        fs.append(W.random_field(dims, 80 + i))
        u = W.random_field(dims, 90 + i); u[1:-1, 1:-1] = 0
        u0s.append(u)
        plan = srj.Plan(dims, h, omega, q, order, "mixed")
        plan.set_temporal_depth(T)
        plans.append(plan)
    batch = srj.Batch(probs, temporal_depth=T)
    ud = [torch.from_numpy(u).cuda() for u in u0s]
    stats, ms, rc = batch.solve([torch.from_numpy(f).cuda() for f in fs], ud, 1e-10, 2000)
    assert rc == 0
    for plan, f, u0, u, st in zip(plans, fs, u0s, ud, stats):
        ref = torch.from_numpy(u0).cuda()
        st1 = plan.solve(torch.from_numpy(f).cuda(), ref, 1e-10, 2000)
        assert st["cycles"] == st1["cycles"]
        assert torch.equal(u, ref)


def test_repeated_solve_reuses_the_graph_bit_for_bit():
    """A second solve with the same tolerance reuses the captured graph, whose
    launches the first solve narrowed to its last unfinished problems: it must
    launch every problem again and give the same bits and cycle counts."""
    specs = [(64, 5, 21), (256, 10, 23), (128, 6, 25), (64, 9, 27)]
    probs, fs, u0s = zip(*[_problem(*s) for s in specs])
    batch = srj.Batch(list(probs), temporal_depth=8)
    fd = [torch.from_numpy(f).cuda() for f in fs]
    runs = []
    for _ in range(2):
        ud = [torch.from_numpy(u).cuda() for u in u0s]
        stats, ms, rc = batch.solve(fd, ud, 1e-10, 200)
        assert rc == 0
        runs.append((ud, [(s["cycles"], s["sweeps"]) for s in stats]))
    # the problems finish after different numbers of phases, so the first solve narrows its launches
    assert runs[0][1] == runs[1][1] and len({sw for _, sw in runs[0][1]}) > 1
    for a, b in zip(runs[0][0], runs[1][0]):
        assert torch.equal(a, b)


def test_depth_tuner_picks_a_valid_depth_and_leaves_the_inputs():
    """srj_batch_tune_depth times one cycle of every problem for each depth and
    returns the fastest; the caller's u is untouched (the trial solves run on
    copies), and a batch built with the tuned depth converges."""
    specs = [(64, 5, 21), (256, 6, 23), (128, 8, 25), (512, 7, 27)]
    probs, fs, u0s = zip(*[_problem(*s) for s in specs])
    fd = [torch.from_numpy(f).cuda() for f in fs]
    ud = [torch.from_numpy(u).cuda() for u in u0s]
    T, ms = srj.Batch.tune_depth(list(probs), fd, ud, 4, 8)
    assert 4 <= T <= 8 and ms > 0
    for u, u0 in zip(ud, u0s):
        assert np.array_equal(u.cpu().numpy(), u0)
    batch = srj.Batch(list(probs), temporal_depth=T)
    stats, _, rc = batch.solve(fd, ud, 1e-10, 200)
    assert rc == 0 and batch.info()["temporal_depth"] == T
