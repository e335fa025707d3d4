"""GPU parity of the masked / diagonally shifted operator (Sect. 5.3 test B
setting) against the oracle.  FP64: bit-identical iterates and residuals (same
operation order, no FMA); mixed precision: tolerance reached, checked by the
oracle's residual."""
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


def random_mask(dims, seed, frac=0.75):
    rng = np.random.default_rng(seed)
    m = (rng.random(tuple(n + 2 for n in reversed(dims))) < frac).astype(np.uint8)
    inner = np.zeros_like(m); inner[tuple(slice(1, -1) for _ in dims)] = 1
    return m * inner


def region_mask_2d(n):
    """A Cartesian stand-in for the test-B region: a wavy disc minus a hole."""
    x = np.arange(n + 2) / (n + 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    th = np.arctan2(Y - 0.5, X - 0.5)
    rr = np.hypot(X - 0.5, Y - 0.45)
    inside = rr < 0.38 * (1 - 0.15 * np.cos(3 * th) + 0.08 * np.cos(5 * th))
    hole = np.hypot(X - 0.62, Y - 0.55) < 0.08
    m = (inside & ~hole).astype(np.uint8)
    m[0, :] = m[-1, :] = 0; m[:, 0] = m[:, -1] = 0
    return m


def schedule_for(dims, sigma, P=4):
    nd = len(dims)
    km = oracle.shifted_kappa(oracle.kappa_min_dirichlet(dims), nd, sigma)
    omega, beta, _ = S.solve_optimal(P, km)
    q = S.q_floor(beta)
    return omega, q, S.order_drift(omega, q, km)


@pytest.mark.parametrize("dims,sigma", [((37, 23), -0.01), ((64, 64), 0.2), ((13, 11, 9), -0.005), ((1, 1), 0.0)])
def test_fp64_operator_sweeps_and_residual_bit_identical(dims, sigma):
    omega, q, order = schedule_for(dims, sigma)
    seq = oracle.omega_sequence(omega, order)
    h = 1.0 / (max(dims) + 1)
    mask = random_mask(dims, 3)
    f = W.random_field(dims, 4); u = W.random_field(dims, 5)
    plan = srj.Plan(dims, h, omega, q, order, "fp64")
    plan.set_operator(sigma, dev(mask))
    ud = dev(u)
    plan.steps(dev(f), ud, 0, len(seq))
    ref = u.copy()
    for om in seq:
        ref = oracle.sweep_op(dims, h, om, sigma, mask, f, ref)
    assert np.array_equal(ud.cpu().numpy(), ref)
    rd = torch.empty_like(dev(u))
    l2, linf = plan.residual(dev(f), dev(u), rd)
    l2o, linfo, r = oracle.residual_op(dims, h, sigma, mask, f, u, want_r=True)
    assert np.array_equal(rd.cpu().numpy(), r) and linf == linfo
    assert abs(l2 - l2o) <= 1e-12 * l2o


def test_region_solve_fp64_matches_oracle_and_mixed_converges():
    """GS_linear-type operator (sigma = -C^2 h^2, C = 3) on an irregular region of a
    256^2 grid with fixed data outside it: FP64 solve bit-identical to the oracle's
    cycle for cycle; the mixed-precision solve reaches the tolerance."""
    n = 256
    dims = (n, n)
    h = 1.0 / (n + 1)
    sigma = -9.0 * h * h
    mask = region_mask_2d(n)
    f = W.smooth_random_2d(n, 6)
    u0 = W.poly_boundary_2d(n, 7)
    outside = (mask == 0)
    u0[1:-1, 1:-1] = 0.0
    u0[outside] = W.poly_boundary_2d(n, 8)[outside] * 0 + 0.3  # fixed value outside the region
    u0[0, :] = u0[-1, :] = 0.3; u0[:, 0] = u0[:, -1] = 0.3
    omega, q, order = schedule_for(dims, sigma, 6)
    seq = oracle.omega_sequence(omega, order)
    p64 = srj.Plan(dims, h, omega, q, order, "fp64")
    p64.set_operator(sigma, dev(mask))
    ud = dev(u0)
    st = p64.solve(dev(f), ud, 1e-10, 2000)
    ref = u0.copy()
    so = oracle.solve_op(dims, h, sigma, mask, seq, f, ref, 1e-10, 2000)
    assert so["status"] == oracle.CONVERGED and so["cycles"] == st["cycles"]
    assert np.array_equal(ud.cpu().numpy(), ref)
    pm = srj.Plan(dims, h, omega, q, order, "mixed")
    pm.set_operator(sigma, dev(mask))
    assert pm.temporal_depth() == 1
    um = dev(u0)
    pm.solve(dev(f), um, 1e-10, 2000)
    r0, _ = oracle.residual_op(dims, h, sigma, mask, f, u0)
    l2, _ = oracle.residual_op(dims, h, sigma, mask, f, um.cpu().numpy())
    assert l2 <= 1e-10 * r0 * (1 + 1e-9)
    assert np.array_equal(um.cpu().numpy()[outside], u0[outside])


def test_plain_operator_restored_bit_for_bit():
    dims = (64, 64)
    plan = srj.Plan.from_table(dims, 5, "fp64")
    f = W.random_field(dims, 1); u = W.random_field(dims, 2)
    a = dev(u); plan.steps(dev(f), a, 0, 50)
    plan.set_operator(0.1, dev(random_mask(dims, 9)))
    plan.set_operator(0.0, None)
    b = dev(u); plan.steps(dev(f), b, 0, 50)
    assert torch.equal(a, b)


def test_indefinite_shift_rejected():
    dims = (64, 64)
    plan = srj.Plan.from_table(dims, 5, "fp64")
    with pytest.raises(srj.SRJError):
        plan.set_operator(-0.5, None)  # below the smallest eigenvalue: not positive definite
