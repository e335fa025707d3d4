"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances:
* FP64 sweeps and the FP64 residual use the oracle's operation order without
  FMA contraction, so iterates and residual vectors must be bit-identical.
  Norms are parallel reductions: relative 1e-12 (at the full sizes, against a
  pairwise sum of the identical residual field; the oracle's one-by-one sum of
  N squares is then held to the recursive-summation bound (N - 1) 2^-53).
* FP32 sweep: per point, |gpu - oracle| <= 8 eps32 * (|u| + c (sum|nbrs| + |h^2 f| + 2d |u|))
  (a handful of FP32 roundings of the terms of one step).
* Mixed-precision solves: final relative residual, recomputed by the oracle
  from the returned u, <= tol.
"""
import math

import numpy as np
import pytest

import oracle
import srj_workloads as W
from oracle import schedule as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1511_04292_gb300 as srj  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def small_schedule(dims, P=3):
    km = oracle.kappa_min_dirichlet(dims)
    omega, beta, _ = S.solve_optimal(P, km)
    q = S.q_floor(beta)
    return omega, q, S.order_drift(omega, q, km)


def random_problem(dims, seed):
    f = W.random_field(dims, seed)
    u = W.random_field(dims, seed + 1)
    return f, u


SHAPES_2D = [(37, 23), (128, 128), (200, 3), (1, 1), (1, 7), (5, 1), (130, 67)]
SHAPES_3D = [(13, 11, 9), (1, 1, 1), (32, 5, 3), (6, 1, 4)]


@pytest.mark.parametrize("dims", SHAPES_2D + SHAPES_3D)
def test_fp64_sweeps_bit_identical(dims):
    omega, q, order = small_schedule(dims)
    seq = oracle.omega_sequence(omega, order)
    h = 1.0 / (max(dims) + 1)
    f, u = random_problem(dims, 100 + len(dims))
    plan = srj.Plan(dims, h, omega, q, order, "fp64")
    for first, count in [(0, 1), (1, 2), (0, len(seq)), (len(seq) - 1, 3)]:
        ud = dev(u)
        plan.steps(dev(f), ud, first, count)
        ref = u.copy()
        oracle.steps(dims, h, seq, f, ref, first=first, count=count)
        assert np.array_equal(ud.cpu().numpy(), ref), (dims, first, count)


@pytest.mark.parametrize("dims", SHAPES_2D + SHAPES_3D)
def test_fused_fp64_sweeps_within_rounding_of_the_oracle(dims):
    """SRJ_PREC_FP64_FMA (each step as fma(c, fma(-2d, u, t), u)): after one
    full cycle and after a few steps the iterates stay within 1e-12 relative
    (max norm) of the oracle's at equal sweep count; a full solve converges to
    the same tolerance in the same cycles as the bit-exact FP64 plan."""
    omega, q, order = small_schedule(dims)
    seq = oracle.omega_sequence(omega, order)
    h = 1.0 / (max(dims) + 1)
    f, u = random_problem(dims, 300 + len(dims))
    plan = srj.Plan(dims, h, omega, q, order, "fp64fma")
    for first, count in [(0, 3), (0, len(seq))]:
        ud = dev(u)
        plan.steps(dev(f), ud, first, count)
        ref = u.copy()
        oracle.steps(dims, h, seq, f, ref, first=first, count=count)
        got = ud.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), (dims, first, count)
    if min(dims) >= 3:
        u0 = u.copy(); u0[tuple(slice(1, -1) for _ in dims)] = 0.0
        exact = srj.Plan(dims, h, omega, q, order, "fp64")
        st_e = exact.solve(dev(f), dev(u0), 1e-10, 500)
        ud = dev(u0)
        st_f = plan.solve(dev(f), ud, 1e-10, 500)
        assert st_f["cycles"] == st_e["cycles"] and st_f["rel_res"] <= 1e-10
        r0, _ = oracle.residual(dims, h, f, u0)
        l2, _ = oracle.residual(dims, h, f, ud.cpu().numpy())
        assert l2 <= 1e-10 * r0 * (1 + 1e-9)


@pytest.mark.parametrize("case", ["2d_4096_P10", "3d_512_P12"])
def test_full_size_fp64_steps_and_residual_bit_identical(case):
    """The FP64 path at the workloads' full sizes, in the launch configuration of
    the FP64 comparator (table schedule, plan order): a few steps from the
    start of the cycle and around its largest weight give the oracle's iterate
    bit for bit, and so does the residual field of the result."""
    if case == "2d_4096_P10":
        n, P = 4096, 10
        dims = (n, n)
        f, u = W.random_smooth_problem_2d(n, 2)
    else:
        n, P = 512, 12
        dims = (n, n, n)
        f, u = W.gaussian_blobs_3d(n, 3)
    plan = srj.Plan.from_table(dims, P, "fp64")
    row = srj.schedules.lookup(len(dims), n, P)
    seq = oracle.omega_sequence(row["omega"], row["order"])
    k = int(np.argmax(seq))
    fd = dev(f)
    ref = u.copy()
    ud = dev(u)
    for first, count in [(0, 2), (max(k - 1, 0), 3)]:
        plan.steps(fd, ud, first, count)
        oracle.steps(dims, plan.h, seq, f, ref, first=first, count=count)
        assert np.array_equal(ud.cpu().numpy(), ref), (case, first, count)
    rd = torch.empty_like(ud)
    l2, linf = plan.residual(fd, ud, rd)
    l2o, linfo, r = oracle.residual(dims, plan.h, f, ref, want_r=True)
    assert np.array_equal(rd.cpu().numpy(), r)
    assert linf == linfo
    # The norms sum ~N squares in different orders.  Against a pairwise sum of the
    # (identical) residual field: the library's blocked reduction within 1e-12, the
    # oracle's one-by-one sum within the recursive-summation bound (N - 1) * 2^-53.
    acc = math.sqrt(float(np.sum(np.square(r))))
    assert math.isclose(l2, acc, rel_tol=1e-12), (l2, acc)
    assert math.isclose(l2o, acc, rel_tol=r.size * 2.0 ** -53), (l2o, acc)


@pytest.mark.parametrize("dims", [(37, 23), (1, 1), (64, 64), (13, 11, 9), (2, 3, 1)])
def test_fp64_residual_bit_identical(dims):
    h = 0.37
    f, u = random_problem(dims, 7)
    plan = srj.Plan(dims, h, [1.0], [1], None, "fp64")
    rd = torch.empty_like(dev(u))
    l2, linf = plan.residual(dev(f), dev(u), rd)
    l2o, linfo, r = oracle.residual(dims, h, f, u, want_r=True)
    assert np.array_equal(rd.cpu().numpy(), r)
    assert math.isclose(l2, l2o, rel_tol=1e-12) and linf == linfo


@pytest.mark.parametrize("dims", [(37, 23), (130, 67), (1, 1), (3, 9), (13, 11, 9), (17, 4, 3)])
def test_fp32_sweep_within_rounding_bound(dims):
    omega, q, order = small_schedule(dims)
    h = 1.0 / (max(dims) + 1)
    f, u = random_problem(dims, 31)
    nd = len(dims)
    plan = srj.Plan(dims, h, omega, q, order, "mixed")
    inner = tuple(slice(1, -1) for _ in dims)
    for k in range(len(order)):
        c = omega[order[k]] / (2 * nd)
        ud = dev(u)
        plan.steps(dev(f), ud, k, 1)
        # oracle on the float32-rounded inputs the GPU sweep starts from
        u32 = u.astype(np.float32).astype(np.float64)
        f32 = (h * h * f).astype(np.float32).astype(np.float64) / (h * h)
        ref = oracle.sweep(dims, h, omega[order[k]], f32, u32)
        got = ud.cpu().numpy()
        nb = np.zeros_like(u32)
        for ax in range(nd):
            for sh in (-1, 1):
                nb += np.abs(np.roll(u32, sh, axis=ax))
        bound = 8 * 2.0 ** -24 * (np.abs(u32) + c * (nb + np.abs(h * h * f32) + 2 * nd * np.abs(u32)))
        assert np.all(np.abs(got[inner] - ref[inner]) <= bound[inner]), (dims, k)
        # the ghost layer of u is never written
        g = got.copy(); g[inner] = 0
        g0 = u.copy(); g0[inner] = 0
        assert np.array_equal(g, g0)


def test_fp64_solve_matches_oracle_cycle_for_cycle():
    """Workload 1 (128^2, P = 5, FP64, tol 1e-10): same cycle count and a
    bit-identical solution."""
    n = 128
    dims = (n, n)
    f, _, u0 = W.manufactured_2d(n)
    row = srj.schedules.lookup(2, n, 5)
    plan = srj.Plan.from_table(dims, 5, "fp64")
    ud = dev(u0)
    st = plan.solve(dev(f), ud, 1e-10, 1000)
    seq = oracle.omega_sequence(row["omega"], row["order"])
    ref = u0.copy()
    so = oracle.solve(dims, 1.0 / (n + 1), seq, f, ref, 1e-10, 1000)
    assert so["status"] == oracle.CONVERGED and st["cycles"] == so["cycles"]
    assert np.array_equal(ud.cpu().numpy(), ref)
    assert math.isclose(st["rel_res"], so["rel"], rel_tol=1e-10)


@pytest.mark.parametrize("case", ["2d_128_P5", "2d_257x255", "3d_33", "2d_1x1"])
def test_mixed_solve_reaches_tolerance(case):
    if case == "2d_128_P5":
        n = 128; dims = (n, n)
        f, _, u0 = W.manufactured_2d(n)
        plan = srj.Plan.from_table(dims, 5, "mixed")
    elif case == "2d_257x255":
        dims = (257, 255)
        f, u0 = W.random_smooth_problem_2d(256, 5)[0], None
        f = W.random_field(dims, 9)
        u0 = W.random_field(dims, 10); u0[1:-1, 1:-1] = 0
        omega, q, order = small_schedule(dims, 6)
        plan = srj.Plan(dims, 1.0 / 257, omega, q, order, "mixed")
    elif case == "3d_33":
        dims = (33, 33, 33)
        f, u0 = W.gaussian_blobs_3d(33, 3)
        omega, q, order = small_schedule(dims, 5)
        plan = srj.Plan(dims, 1.0 / 34, omega, q, order, "mixed")
    else:
        dims = (1, 1)
        f = W.random_field(dims, 1); u0 = W.random_field(dims, 2)
        plan = srj.Plan(dims, 0.5, [1.0], [1], None, "mixed")
    ud = dev(u0)
    st = plan.solve(dev(f), ud, 1e-10, 2000)
    r0, _ = oracle.residual(dims, plan.h, f, u0)
    l2, _ = oracle.residual(dims, plan.h, f, ud.cpu().numpy())
    assert l2 <= 1e-10 * r0 * (1 + 1e-9), (case, l2 / r0, st)
    assert math.isclose(st["rel_res"], l2 / r0, rel_tol=1e-6, abs_tol=1e-13)


def test_stagnation_stops_at_the_floating_point_floor():
    """A tolerance below the FP64 floor of the residual stops after a few
    non-improving cycles with NOT_CONVERGED and the stagnated flag, instead of
    running max_cycles."""
    n = 256
    f, u0 = W.random_smooth_problem_2d(n, 4)
    for prec in ("fp64", "mixed"):
        plan = srj.Plan.from_table((n, n), 6, prec)
        st = plan.solve(dev(f), dev(u0), 1e-30, 10000, raise_on_fail=False)
        assert st["status"] == -3 and st["stagnated"] == 1 and st["cycles"] < 200, st
        assert st["rel_res"] < 1e-11
        # the rounding-floor estimate is reported
        assert 0 < st["res_floor"] < st["r0_l2"], st
    # a tolerance just above the floor is met, so the floor rule does not end a solve early
    plan = srj.Plan.from_table((n, n), 6, "fp64")
    st = plan.solve(dev(f), dev(u0), 1e-10, 10000)
    assert st["status"] == 0 and st["rel_res"] <= 1e-10 and st["stagnated"] == 0


def test_zero_problem_converges_immediately():
    dims = (16, 16)
    plan = srj.Plan.from_table((64, 64), 5, "mixed")
    z = torch.zeros(plan.shape, dtype=torch.float64, device="cuda")
    st = plan.solve(z, z.clone(), 1e-10, 10)
    assert st["cycles"] == 0 and st["r0_l2"] == 0.0


def test_not_converged_and_diverged_statuses():
    dims = (64, 64)
    f = W.random_field(dims, 3)
    plan = srj.Plan.from_table(dims, 5, "fp64")
    st = plan.solve(dev(f), dev(W.zero_field(dims)), 1e-14, 1, raise_on_fail=False)
    assert st["status"] == -3 and st["cycles"] == 1
    bad = f.copy(); bad[5, 5] = np.nan
    st = plan.solve(dev(bad), dev(W.zero_field(dims)), 1e-10, 3, raise_on_fail=False)
    assert st["status"] == -4


def test_boundary_adjoint_matches_dense_transpose():
    """b depends on the ghost values g through b_p = h^2 f_p + sum of ghost
    neighbours; the adjoint kernel must equal B^T lambda with B built densely."""
    for dims in [(7, 5), (4, 3, 5)]:
        nd = len(dims)
        shape = tuple(n + 2 for n in reversed(dims))
        plan = srj.Plan(dims, 0.1, [1.0], [1], None, "fp64")
        lam = W.random_field(dims, 77)
        got = torch.empty(shape, dtype=torch.float64, device="cuda")
        plan.boundary_adjoint(dev(lam), got)
        got = got.cpu().numpy()
        ref = np.zeros(shape)
        inner = tuple(slice(1, -1) for _ in dims)
        it = np.ndindex(*shape)
        for idx in it:
            if all(1 <= idx[a] <= shape[a] - 2 for a in range(nd)):
                continue
            # perturb ghost idx by 1: b changes at interior neighbours by 1
            g = np.zeros(shape); g[idx] = 1.0
            acc = np.zeros(shape)
            for ax in range(nd):
                for sh in (-1, 1):
                    acc += np.roll(g, sh, axis=ax)
            ref[idx] = np.sum(acc[inner] * lam[inner])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_solve_host_equals_device_solve(prec):
    """srj_solve_host (host arrays, copies inside the call) gives the device
    solve's iterate bit for bit, for numpy and pinned CPU tensors, and copies
    the iterate back also when the solve stops unconverged."""
    n = 256
    dims = (n, n)
    f, u0 = W.random_smooth_problem_2d(n, 2)
    plan = srj.Plan.from_table(dims, 8, prec)
    for tol, cycles in [(1e-10, 200), (1e-30, 1)]:
        ud = dev(u0)
        st = plan.solve(dev(f), ud, tol, cycles, raise_on_fail=False)
        ref = ud.cpu().numpy()
        uh = u0.copy()
        sth = plan.solve_host(f, uh, tol, cycles, raise_on_fail=False)
        assert sth["status"] == st["status"] and sth["cycles"] == st["cycles"]
        assert np.array_equal(uh, ref)
        ut = torch.from_numpy(u0.copy()).pin_memory()
        plan.solve_host(torch.from_numpy(f).pin_memory(), ut, tol, cycles, raise_on_fail=False)
        assert np.array_equal(ut.numpy(), ref)
    with pytest.raises(TypeError):
        plan.solve_host(dev(f), u0.copy(), 1e-10, 10)


def test_full_size_workload2_mixed_solve():
    """Workload 2 at full size (4096^2, P = 10, mixed, tol 1e-10) in the launch
    configuration the benchmark times (the autotuner's temporal depth and sweep
    variant, as the benchmark picks them): one full cycle of that configuration
    gives the bits of single steps, the oracle's residual of the returned u is
    within tolerance, and one FP32 sweep at this size agrees with the oracle on
    every point within the rounding bound."""
    n = 4096
    dims = (n, n)
    f, u0 = W.random_smooth_problem_2d(n, 2)
    plan = srj.Plan.from_table(dims, 10, "mixed")
    T, _ = plan.autotune()
    V = plan.sweep_variant()
    M = plan.info()["M"]
    fd = dev(f)
    got = dev(u0)
    plan.steps(fd, got, 0, M)
    plan.set_temporal_depth(1)
    ref = dev(u0)
    plan.steps(fd, ref, 0, M)
    assert torch.isfinite(ref).all() and torch.equal(got, ref), (T, V)
    del got, ref
    plan.set_temporal_depth(T)
    plan.set_sweep_variant(V)
    ud = dev(u0)
    st = plan.solve(fd, ud, 1e-10, 100)
    u = ud.cpu().numpy()
    r0, _ = oracle.residual(dims, plan.h, f, u0)
    l2, _ = oracle.residual(dims, plan.h, f, u)
    assert l2 <= 1e-10 * r0 * (1 + 1e-9), (l2 / r0, st)
    # one sweep of the largest weight on the converged field
    row = srj.schedules.lookup(2, n, 10)
    k = int(np.argmax(row["omega"][row["order"]]))
    ud2 = dev(u)
    plan.steps(dev(f), ud2, k, 1)
    h = plan.h
    u32 = u.astype(np.float32).astype(np.float64)
    f32 = (h * h * f).astype(np.float32).astype(np.float64) / (h * h)
    ref = oracle.sweep(dims, h, row["omega"][row["order"][k]], f32, u32)
    got = ud2.cpu().numpy()
    c = row["omega"][row["order"][k]] / 4
    nb = sum(np.abs(np.roll(u32, s, axis=a)) for a in (0, 1) for s in (-1, 1))
    bound = 8 * 2.0 ** -24 * (np.abs(u32) + c * (nb + np.abs(h * h * f32) + 4 * np.abs(u32)))
    assert np.all(np.abs(got - ref)[1:-1, 1:-1] <= bound[1:-1, 1:-1])


def test_full_size_workload3_mixed_solve():
    """Workload 3 at full size (512^3, 8 Gaussian blobs, P = 12, mixed, tol 1e-9)
    in the launch configuration the benchmark times (the autotuner's temporal
    depth): the oracle's residual of the returned u is within tolerance; at this
    size the blocked steps give the bits of single steps; and one FP32 step
    agrees with the oracle within the rounding bound on sampled z planes
    (first, last, and both sides of the boundaries between the first two z
    segments for both blocked depths: 64 planes long with T = 2, 86 with T = 3)."""
    n = 512
    dims = (n, n, n)
    f, u0 = W.gaussian_blobs_3d(n, 3)
    plan = srj.Plan.from_table(dims, 12, "mixed")
    assert plan.temporal_depth() == 2
    T, _ = plan.autotune()
    assert T in (1, 2, 3) and plan.temporal_depth() == T
    fd = dev(f)
    ud = dev(u0)
    st = plan.solve(fd, ud, 1e-9, 200)
    u = ud.cpu().numpy()
    del ud
    r0, _ = oracle.residual(dims, plan.h, f, u0)
    l2, _ = oracle.residual(dims, plan.h, f, u)
    assert l2 <= 1e-9 * r0 * (1 + 1e-9), (l2 / r0, st)
    # blocked (both depths) against single steps, from u0, even and ragged counts
    for first, count, depth in [(0, 8, 2), (3, 7, 2), (0, 12, 3), (5, 7, 3)]:
        plan.set_temporal_depth(depth)
        got = dev(u0)
        plan.steps(fd, got, first, count)
        plan.set_temporal_depth(1)
        ref = dev(u0)
        plan.steps(fd, ref, first, count)
        assert torch.equal(got, ref), (first, count, depth)
        del got, ref
    plan.set_temporal_depth(T)
    # one step of the largest weight on the converged field, against the oracle on z slabs
    row = srj.schedules.lookup(3, n, 12)
    k = int(np.argmax(row["omega"][row["order"]]))
    w = row["omega"][row["order"][k]]
    ud2 = dev(u)
    plan.steps(fd, ud2, k, 1)
    got = ud2.cpu().numpy()
    del ud2
    h = plan.h
    c = w / 6
    for z in (1, 2, 64, 65, 86, 87, 257, n - 1, n):
        sl = slice(z - 1, z + 2)
        u32 = np.ascontiguousarray(u[sl]).astype(np.float32).astype(np.float64)
        f32 = (h * h * np.ascontiguousarray(f[sl])).astype(np.float32).astype(np.float64) / (h * h)
        ref = oracle.sweep((n, n, 1), h, w, f32, u32)[1]
        nb = sum(np.abs(np.roll(u32, s, axis=a)) for a in (0, 1, 2) for s in (-1, 1))[1]
        bound = 8 * 2.0 ** -24 * (np.abs(u32[1]) + c * (nb + np.abs(h * h * f32[1]) + 6 * np.abs(u32[1])))
        diff = np.abs(got[z] - ref)
        assert np.all(diff[1:-1, 1:-1] <= bound[1:-1, 1:-1]), (z, float(diff[1:-1, 1:-1].max()))


@pytest.mark.parametrize("dims", [(37, 23), (130, 67), (1, 1), (5, 300), (129, 129), (300, 5), (1000, 700)])
def test_blocked_fp32_sweep_bit_identical_to_single_steps(dims):
    """Temporal blocking (T steps per launch on register-resident tiles) must give
    exactly the bits of T single-step launches, for every T, for step counts that
    are not multiples of T, and on grids smaller or ragged against the tile."""
    omega, q, order = small_schedule(dims, 4)
    h = 1.0 / (max(dims) + 1)
    f, u = random_problem(dims, 41)
    u[tuple(slice(1, -1) for _ in dims)] *= 1e-3  # keep the iterates moderate
    plan = srj.Plan(dims, h, omega, q, order, "mixed")
    fd = dev(f)
    for count, first in [(len(order), 0), (13, 5)]:
        plan.set_sweep_variant(0)
        plan.set_temporal_depth(1)
        ref = dev(u)
        plan.steps(fd, ref, first, count)
        for variant in range(6):
            plan.set_sweep_variant(variant)
            for T in range(2, 9):
                plan.set_temporal_depth(T)
                got = dev(u)
                plan.steps(fd, got, first, count)
                assert torch.equal(got, ref), (dims, variant, T, count, first)


@pytest.mark.parametrize("dims", [(37, 23, 19), (130, 67, 70), (1, 1, 1), (5, 300, 3), (129, 29, 65), (250, 2, 130)])
def test_blocked_fp32_sweep_3d_bit_identical_to_single_steps(dims):
    """3-D temporal blocking (T = 2 or 3 steps per launch, tiles streamed through
    z segments whose length the launcher picks per grid) must give exactly the
    bits of single-step launches, for step counts that are not multiples of T,
    on grids ragged against the tile centre and spanning more than one z
    segment."""
    omega, q, order = small_schedule(dims, 4)
    h = 1.0 / (max(dims) + 1)
    f, u = random_problem(dims, 43)
    u[tuple(slice(1, -1) for _ in dims)] *= 1e-3
    plan = srj.Plan(dims, h, omega, q, order, "mixed")
    fd = dev(f)
    for count, first in [(len(order), 0), (13, 5), (2, 1), (3, 2)]:
        plan.set_temporal_depth(1)
        ref = dev(u)
        plan.steps(fd, ref, first, count)
        for T in (2, 3):
            plan.set_temporal_depth(T)
            got = dev(u)
            plan.steps(fd, got, first, count)
            assert torch.equal(got, ref), (dims, T, count, first)


def test_bounded_wait_runs_out_and_is_reported():
    """The prefetching sweep's waits are bounded: in the self-test mode no
    prefetch copy is issued, every wait runs out after the limit, the blocks
    report it through the device status word and return, and the context stays
    usable (a plan created afterwards still reproduces the oracle)."""
    L = srj.lib()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        rc = L.srj_selftest_wait_timeout(20000, stream)
        assert rc == -5, L.srj_last_error()
        assert b"self-test passed" in L.srj_last_error()
    assert L.srj_selftest_wait_timeout(0, stream) == -1
    dims = (40, 33)
    omega, q, order = small_schedule(dims)
    f, u = random_problem(dims, 5)
    plan = srj.Plan(dims, 1.0 / 41, omega, q, order, "fp64")
    ud = dev(u)
    plan.steps(dev(f), ud, 0, len(order))
    ref = u.copy()
    oracle.steps(dims, 1.0 / 41, oracle.omega_sequence(omega, order), f, ref)
    assert np.array_equal(ud.cpu().numpy(), ref)


def test_autotune_picks_a_valid_depth_and_solve_still_converges():
    n = 512
    dims = (n, n)
    f, u0 = W.random_smooth_problem_2d(n, 8)
    plan = srj.Plan.from_table(dims, 8, "mixed")
    T, us = plan.autotune()
    assert 1 <= T <= 8 and plan.temporal_depth() == T and us > 0
    ud = dev(u0)
    plan.solve(dev(f), ud, 1e-10, 200)
    r0, _ = oracle.residual(dims, plan.h, f, u0)
    l2, _ = oracle.residual(dims, plan.h, f, ud.cpu().numpy())
    assert l2 <= 1e-10 * r0 * (1 + 1e-9)


def test_temporal_depth_rules():
    p64 = srj.Plan((16, 16), 0.1, [1.0], [1], None, "fp64")
    with pytest.raises(srj.SRJError):
        p64.set_temporal_depth(4)
    p3 = srj.Plan((8, 8, 8), 0.1, [1.0], [1], None, "mixed")
    assert p3.temporal_depth() == 2
    p3.set_temporal_depth(1)
    p3.set_temporal_depth(3)
    with pytest.raises(srj.SRJError):
        p3.set_temporal_depth(4)
    p2 = srj.Plan((16, 16), 0.1, [1.0], [1], None, "mixed")
    assert p2.temporal_depth() == 8
    with pytest.raises(srj.SRJError):
        p2.set_temporal_depth(9)


def test_auto_plan_from_native_planner_converges():
    """A plan built entirely by the library (native planner + its own cycle order)
    on a ragged grid solves to tolerance (mixed and FP64)."""
    dims = (300, 211)
    f = W.random_field(dims, 71)
    u0 = W.random_field(dims, 72); u0[1:-1, 1:-1] = 0
    for prec in ("mixed", "fp64"):
        plan = srj.Plan.auto(dims, 8, prec)
        ud = dev(u0)
        plan.solve(dev(f), ud, 1e-10, 500)
        r0, _ = oracle.residual(dims, plan.h, f, u0)
        l2, _ = oracle.residual(dims, plan.h, f, ud.cpu().numpy())
        assert l2 <= 1e-10 * r0 * (1 + 1e-9)


def test_full_size_2pow15_sweeps():
    """The 32768^2 throughput line's launch configurations at full size: the
    blocked FP32 sweep (T = 8, the 4096^2 grid's scheme, as the benchmark runs
    it) gives the bits of single steps, one FP32 step agrees with the oracle
    within the rounding bound on sampled rows, and the FP64 sweep is
    bit-identical to the oracle on sampled rows."""
    n = 32768
    dims = (n, n)
    h = 1.0 / (n + 1)
    f, u0 = W.random_smooth_problem_2d_device(n, 2)
    # a nonzero interior, so that every term of the update is exercised
    u0[1:-1, 1:-1] = 0.25 * f[1:-1, 1:-1]
    row = srj.schedules.lookup(2, 4096, 10)
    plan = srj.Plan(dims, h, row["omega"], row["q"], row["order"], "mixed")
    plan.set_temporal_depth(8)
    plan.set_sweep_variant(0)
    first, count = 5, 16
    got = u0.clone()
    plan.steps(f, got, first, count)
    plan.set_temporal_depth(1)
    ref = u0.clone()
    plan.steps(f, ref, first, count)
    assert torch.isfinite(ref).all() and torch.equal(got, ref)
    del got, ref
    sample_rows = (1, 2, 48, 49, 12345, n - 1, n)
    # one FP32 step of the cycle's first weight against the oracle, on 3-row slabs
    w = float(row["omega"][row["order"][0]])
    one = u0.clone()
    plan.steps(f, one, 0, 1)
    for y in sample_rows:
        us = u0[y - 1:y + 2].cpu().numpy()
        fs = f[y - 1:y + 2].cpu().numpy()
        u32 = us.astype(np.float32).astype(np.float64)
        f32 = (h * h * fs).astype(np.float32).astype(np.float64) / (h * h)
        refrow = oracle.sweep((n, 1), h, w, f32, u32)[1]
        c = w / 4
        nb = sum(np.abs(np.roll(u32, s, axis=a)) for a in (0, 1) for s in (-1, 1))[1]
        bound = 8 * 2.0 ** -24 * (np.abs(u32[1]) + c * (nb + np.abs(h * h * f32[1]) + 4 * np.abs(u32[1])))
        diff = np.abs(one[y].cpu().numpy() - refrow)
        assert np.all(diff[1:-1] <= bound[1:-1]), (y, float(diff[1:-1].max()))
    del one, plan
    torch.cuda.empty_cache()
    # FP64 sweep (the benchmark times it on a one-weight plan): bit-identical rows
    p64 = srj.Plan(dims, h, [1.0], [1], None, "fp64")
    u64 = u0.clone()
    p64.steps(f, u64, 0, 1)
    for y in sample_rows:
        us = u0[y - 1:y + 2].cpu().numpy()
        fs = f[y - 1:y + 2].cpu().numpy()
        refrow = oracle.sweep((n, 1), h, 1.0, fs, us)[1]
        assert np.array_equal(u64[y].cpu().numpy(), refrow), y
