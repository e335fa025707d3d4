"""Parity of the spherical-operator path (Sect. 5.2) with the oracle: FP64
sweeps and residual fields bit for bit, FP64 solves cycle for cycle, mixed-
precision solves to tolerance (checked by the oracle's residual), and the
paper's analytic test at the oracle's discretisation error."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import oracle  # noqa: E402
import paper_1511_04292_gb300.schedules as sch  # noqa: E402
from paper_1511_04292_gb300 import spherical as sp  # noqa: E402

from test_oracle_spherical import paper_problem_2d  # noqa: E402

pytestmark = pytest.mark.gpu

SHAPES = [(37, 23), (2, 2), (1, 4), (130, 67), (5, 300), (13, 11, 9), (2, 3, 1), (32, 5, 7), (3, 8, 2)]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def schedule(P=5):
    row = sch.lookup(2, 64, P)
    return row["omega"], row["q"], row["order"]


def problem(dims, seed):
    rng = np.random.default_rng(seed)
    shape = oracle.padded_shape(dims)
    return rng.standard_normal(shape), rng.standard_normal(shape)


@pytest.mark.parametrize("dims", SHAPES)
def test_sweeps_bit_identical(dims):
    omega, q, order = schedule(5)
    coef = sp.coefficients(dims)
    plan = sp.SphericalPlan(dims, omega, q, order, coef=coef)
    b, u = problem(dims, 3)
    seq = oracle.omega_sequence(omega, order)
    ref = u.copy()
    for k in range(7):
        ref = oracle.sph_sweep(dims, coef, seq[(2 + k) % len(seq)], b, ref)
    ud = dev(u)
    plan.steps(dev(b), ud, 2, 7)
    assert np.array_equal(ud.cpu().numpy(), ref)


@pytest.mark.parametrize("dims", SHAPES)
def test_residual_field_bit_identical(dims):
    omega, q, order = schedule(5)
    coef = sp.coefficients(dims)
    plan = sp.SphericalPlan(dims, omega, q, order, coef=coef)
    b, u = problem(dims, 5)
    l2, linf, r = oracle.sph_residual(dims, coef, b, u, want_r=True)
    rd = torch.empty_like(dev(u))
    gl2, glinf = plan.residual(dev(b), dev(u), rd)
    assert np.array_equal(rd.cpu().numpy(), r)
    assert glinf == linf
    assert gl2 == pytest.approx(l2, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("dims", [(40, 30), (12, 10, 8), (1, 3)])
def test_solve_matches_oracle_cycle_for_cycle(dims):
    omega, q, order = schedule(6)
    coef = sp.coefficients(dims)
    plan = sp.SphericalPlan(dims, omega, q, order, coef=coef)
    b, u0 = problem(dims, 7)
    seq = oracle.omega_sequence(omega, order)
    ref = u0.copy()
    so = oracle.sph_solve(dims, coef, seq, b, ref, 1e-10, 500)
    ud = dev(u0)
    st = plan.solve(dev(b), ud, 1e-10, 500)
    assert so["status"] == oracle.CONVERGED and st["cycles"] == so["cycles"]
    assert np.array_equal(ud.cpu().numpy(), ref)
    assert st["rel_res"] == pytest.approx(so["rel"], rel=1e-10, abs=1e-300)


@pytest.mark.parametrize("dims", [(300, 200), (40, 30, 20), (64, 64)])
def test_mixed_solve_reaches_tolerance(dims):
    """FP32 cycles inside FP64 defect correction: the oracle's own residual of
    the returned field meets the tolerance, within a few cycles of FP64."""
    n = max(dims)
    row = sch.lookup(2, 256 if n > 128 else 64, 8 if n > 128 else 6)
    b, u0 = problem(dims, 9)
    coef = sp.coefficients(dims)
    r0, _ = oracle.sph_residual(dims, coef, b, u0)
    mixed = sp.SphericalPlan(dims, row["omega"], row["q"], row["order"], coef=coef, precision="mixed")
    ud = dev(u0)
    st = mixed.solve(dev(b), ud, 1e-10, 500)
    l2, _ = oracle.sph_residual(dims, coef, b, ud.cpu().numpy())
    assert l2 / r0 <= 1.5e-10
    fp64 = sp.SphericalPlan(dims, row["omega"], row["q"], row["order"], coef=coef)
    st64 = fp64.solve(dev(b), dev(u0), 1e-10, 500)
    assert st["cycles"] <= st64["cycles"] + 3, (st, st64)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_paper_problem_reaches_the_discretisation_error(precision):
    """Sect. 5.2 axisymmetric test (l = 0, 2 terms), N = 256: the GPU solve
    reaches the oracle's discretisation error (second order: 1.5e-5)."""
    N = 256
    dims = (N, N)
    ua, b = paper_problem_2d(N, N)
    u0 = np.zeros_like(ua)
    u0[:, -1] = ua[:, -1]
    row = sch.lookup(2, 256, 8)
    plan = sp.SphericalPlan(dims, row["omega"], row["q"], row["order"], precision=precision)
    ud = dev(u0)
    st = plan.solve(dev(b), ud, 1e-12, 2000)
    u = ud.cpu().numpy()
    err = np.abs(u - ua)[1:-1, 2:-1].max()
    assert 1.0e-5 < err < 2.5e-5, (err, st)
    # prescriptions hold on the returned field
    assert np.array_equal(u[1:-1, 1], u[1:-1, 2]) and np.array_equal(u[1:-1, 0], u[1:-1, 2])
    assert np.array_equal(u[0], u[1]) and np.array_equal(u[-1], u[-2])


def test_bad_schedule_and_bad_arguments_are_rejected():
    with pytest.raises(Exception):
        sp.SphericalPlan((8, 8), [3.0], [1])  # 1 - 3 kappa reaches -5 at kappa = 2: no contraction
    with pytest.raises(Exception):
        sp.SphericalPlan((0, 8), [1.0], [1])
    plan = sp.SphericalPlan((8, 8), [1.0], [1])
    with pytest.raises(Exception):
        plan.solve(dev(np.zeros((10, 10))), dev(np.zeros((9, 10))), 1e-8, 10)


@pytest.mark.parametrize("dims", [(300, 200), (37, 23), (2, 5), (130, 67), (129, 200), (1000, 9), (3, 1), (200, 1), (121, 2)])
def test_blocked_fp32_cycles_bit_identical(dims):
    """Mixed 2-D plans run their FP32 cycles T steps per launch on register-
    resident tiles; T = 3 and 8 must give the bits of single steps (three
    cycles, ragged grids, tiles holding the r = 0 prescription and the theta
    mirrors)."""
    row = sch.lookup(2, 64, 6)
    b, u0 = problem(dims, 13)
    plan = sp.SphericalPlan(dims, row["omega"], row["q"], row["order"], precision="mixed")
    assert plan.temporal_depth() == 8
    outs = []
    for T in (1, 3, 8):
        plan.set_temporal_depth(T)
        ud = dev(u0)
        st = plan.solve(dev(b), ud, 1e-30, 3, check_status=False)
        assert st["cycles"] == 3
        outs.append(ud.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_spherical_temporal_depth_rules():
    row = sch.lookup(2, 64, 5)
    p64 = sp.SphericalPlan((16, 16), row["omega"], row["q"], row["order"])
    assert p64.temporal_depth() == 1
    with pytest.raises(Exception):
        p64.set_temporal_depth(2)
    p3 = sp.SphericalPlan((8, 8, 8), row["omega"], row["q"], row["order"], precision="mixed")
    with pytest.raises(Exception):
        p3.set_temporal_depth(2)
    p2 = sp.SphericalPlan((16, 16), row["omega"], row["q"], row["order"], precision="mixed")
    with pytest.raises(Exception):
        p2.set_temporal_depth(9)


def test_bench_size_mixed_solve():
    """The spherical benchmark problem at its size (Sect. 5.2 test, 1024^2,
    P = 10, mixed, tol 1e-10) with the default blocked depth: the oracle's
    residual of the returned field meets the tolerance, and the solve gives the
    bits of the same solve with single-step launches."""
    import srj_workloads as W
    n = 1024
    dims = (n, n)
    b, u0 = W.spherical_problem_2d(n, 5)
    row = sch.lookup(2, n, 10)
    coef = sp.coefficients(dims)
    plan = sp.SphericalPlan(dims, row["omega"], row["q"], row["order"], coef=coef, precision="mixed")
    assert plan.temporal_depth() == 8
    outs, stats = [], []
    for T in (8, 1):
        plan.set_temporal_depth(T)
        ud = dev(u0)
        stats.append(plan.solve(dev(b), ud, 1e-10, 400))
        outs.append(ud.cpu().numpy())
    assert stats[0]["cycles"] == stats[1]["cycles"]
    assert np.array_equal(outs[0], outs[1])
    r0, _ = oracle.sph_residual(dims, coef, b, u0)
    l2, _ = oracle.sph_residual(dims, coef, b, outs[0])
    assert l2 <= 1e-10 * r0 * (1 + 1e-9), (l2 / r0, stats[0])
