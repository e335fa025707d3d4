"""Pins of the oracle's masked / diagonally shifted operator (the Sect. 5.3
test B setting: SRJ applied inside a mask, Eq. GS_linear's linear term as a
shift of the diagonal)."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import srj_workloads as W
from oracle import schedule as S
from test_oracle import laplacian_matrix, sine_mode, mode_kappa


def _mask(dims, seed, frac=0.7):
    rng = np.random.default_rng(seed)
    m = (rng.random(tuple(n + 2 for n in reversed(dims))) < frac).astype(np.uint8)
    g = np.zeros_like(m); g[tuple(slice(1, -1) for _ in dims)] = 1
    return m * g  # ghosts never active


@pytest.mark.parametrize("dims", [(9, 7), (5, 6, 4)])
def test_unshifted_unmasked_is_the_plain_sweep(dims):
    f = W.random_field(dims, 1); u = W.random_field(dims, 2)
    for om in (0.6, 7.25, 1234.5):
        assert np.array_equal(oracle.sweep_op(dims, 0.1, om, 0.0, None, f, u), oracle.sweep(dims, 0.1, om, f, u))
    l2a, _, ra = oracle.residual_op(dims, 0.1, 0.0, None, f, u, want_r=True)
    l2b, _, rb = oracle.residual(dims, 0.1, f, u, want_r=True)
    assert np.array_equal(ra, rb) and l2a == l2b


@pytest.mark.parametrize("dims,sigma", [((9, 7), -0.05), ((9, 7), 0.3), ((5, 6, 4), -0.02)])
def test_masked_shifted_sweep_matches_sparse_submatrix(dims, sigma):
    """x_S' = x_S + omega/(2d+sigma) (b_S - A_SS x_S - A_SF x_F) on the active set S,
    with the inactive interior points F and the ghosts held fixed."""
    nd = len(dims)
    h = 0.125
    inner = tuple(slice(1, -1) for _ in dims)
    mask = _mask(dims, 3)
    f = W.random_field(dims, 4); u = W.random_field(dims, 5)
    A = laplacian_matrix(dims) + sigma * sp.identity(int(np.prod(dims)))
    A = A.tocsr()
    act = mask[inner].reshape(-1).astype(bool)
    x = u[inner].reshape(-1)
    g = u.copy(); g[inner] = 0
    bnd = np.zeros_like(g)
    for ax in range(nd):
        for s in (-1, 1):
            bnd += np.roll(g, s, axis=ax)
    b = h * h * f[inner].reshape(-1) + bnd[inner].reshape(-1)
    r = b - A @ x
    for om in (0.7, 33.0):
        ref = x.copy()
        ref[act] = x[act] + om / (2 * nd + sigma) * r[act]
        got = oracle.sweep_op(dims, h, om, sigma, mask, f, u)[inner].reshape(-1)
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    l2, linf, rr = oracle.residual_op(dims, h, sigma, mask, f, u, want_r=True)
    np.testing.assert_allclose(rr[inner].reshape(-1)[act], r[act], rtol=1e-12, atol=1e-12 * np.abs(r).max())
    assert np.all(rr[inner].reshape(-1)[~act] == 0)
    assert math.isclose(l2, np.linalg.norm(r[act]), rel_tol=1e-12)


@pytest.mark.parametrize("dims,sigma", [((16, 12), -0.01), ((16, 12), 0.5), ((8, 7, 6), -0.005)])
def test_shifted_eigenmode_decay(dims, sigma):
    """With the diagonal shift the sine modes stay eigenvectors; D^-1 A has
    eigenvalue kappa' = (2d kappa + sigma)/(2d + sigma) and a cycle multiplies a
    mode by prod (1 - omega_i kappa')^{q_i} (Eq. cycleAmplFact)."""
    nd = len(dims)
    kmin = oracle.shifted_kappa(oracle.kappa_min_dirichlet(dims), nd, sigma)
    omega, beta, _ = S.solve_optimal(3, kmin)
    q = S.q_floor(beta)
    seq = oracle.omega_sequence(omega, S.order_drift(omega, q, kmin))
    f = np.zeros(tuple(n + 2 for n in reversed(dims)))
    for m in [tuple(1 for _ in dims), tuple(dims), tuple(max(1, n // 2) for n in dims)]:
        e = sine_mode(dims, m)
        kp = oracle.shifted_kappa(mode_kappa(dims, m), nd, sigma)
        lam = float(np.prod((1.0 - omega * kp) ** q))
        u = e.copy()
        for om in seq:
            u = oracle.sweep_op(dims, 0.1, om, sigma, None, f, u)
        assert np.max(np.abs(u - lam * e)) <= 1e-10 * max(1.0, abs(lam)), (m, lam)


def test_masked_shifted_solve_equals_dense_solve():
    dims = (14, 11)
    h = 1.0 / 15
    sigma = -0.02
    inner = (slice(1, -1), slice(1, -1))
    # an annulus-like active region: points inside a disc, outside a smaller disc
    yy, xx = np.meshgrid(np.arange(dims[1] + 2), np.arange(dims[0] + 2), indexing="ij")
    rr = np.hypot(xx - 7.5, yy - 6.0)
    mask = ((rr < 6.2) & (rr > 1.8)).astype(np.uint8)
    mask[0, :] = mask[-1, :] = 0; mask[:, 0] = mask[:, -1] = 0
    f = W.random_field(dims, 7); u0 = W.random_field(dims, 8)
    u0[inner] *= (1 - mask[inner])  # fixed values outside the region, 0 inside
    A = (laplacian_matrix(dims) + sigma * sp.identity(np.prod(dims))).toarray()
    act = mask[inner].reshape(-1).astype(bool)
    x_all = u0[inner].reshape(-1)
    g = u0.copy(); g[inner] = 0
    bnd = sum(np.roll(g, s, axis=a) for a in (0, 1) for s in (-1, 1))[inner].reshape(-1)
    b = h * h * f[inner].reshape(-1) + bnd - A[:, ~act] @ x_all[~act]
    xs = np.linalg.solve(A[np.ix_(act, act)], b[act])
    kmin = oracle.shifted_kappa(oracle.kappa_min_dirichlet(dims), 2, sigma)
    omega, beta, _ = S.solve_optimal(4, kmin)
    q = S.q_floor(beta)
    seq = oracle.omega_sequence(omega, S.order_drift(omega, q, kmin))
    u = u0.copy()
    st = oracle.solve_op(dims, h, sigma, mask, seq, f, u, 1e-13, 20000)
    assert st["status"] == oracle.CONVERGED
    got = u[inner].reshape(-1)
    np.testing.assert_allclose(got[act], xs, rtol=0, atol=1e-11 * np.abs(xs).max())
    assert np.array_equal(got[~act], x_all[~act])
