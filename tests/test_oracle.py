"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test pins the oracle's sweep, residual or cycle loop to something other
than itself: a sparse-matrix formulation of weighted Jacobi (scipy), the exact
eigenmode decay of Eq. cycleAmplFact, a dense direct solve (numpy/LAPACK), and
the O(h^2) convergence of manufactured solutions (Sect. 5.1).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import srj_workloads as W
from oracle import schedule as S


def laplacian_matrix(dims):
    """A_h = 2d I - (neighbour sum) on the interior, built from 1-D tridiagonal
    blocks with Kronecker products; the unknowns are ordered x fastest."""
    mats = [sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) for n in dims]
    eye = [sp.identity(n) for n in dims]
    A = None
    for k in range(len(dims)):
        term = None
        for j in reversed(range(len(dims))):  # slowest dimension first in kron
            blk = mats[j] if j == k else eye[j]
            term = blk if term is None else sp.kron(term, blk)
        A = term if A is None else A + term
    return A.tocsr()


def boundary_vector(dims, u):
    """Contribution of the ghost values of u to b: for each interior point, the sum
    of its ghost neighbours (computed by applying the full padded-grid operator to
    the ghost-only field)."""
    g = u.copy()
    inner = tuple(slice(1, -1) for _ in dims)
    g[inner] = 0.0
    acc = np.zeros_like(g[inner])
    nd = len(dims)
    for ax in range(nd):
        for sh in (-1, 1):
            acc += np.roll(g, sh, axis=ax)[inner]
    return acc.reshape(-1)


def interior(a, nd):
    return a[tuple(slice(1, -1) for _ in range(nd))].reshape(-1)


@pytest.mark.parametrize("dims", [(7, 5), (6, 5, 4)])
def test_sweep_matches_sparse_weighted_jacobi(dims):
    """Eq. 2nd-order_CD with source: x' = x + (omega/2d) D^-1-normalised residual,
    written with a scipy sparse matrix, for random u, f, boundary data and weights."""
    nd = len(dims)
    h = 1.0 / 7.0
    rng = np.random.default_rng(1)
    A = laplacian_matrix(dims)
    for omega in (1.0, 0.71, 37.5, 1234.5):
        u = W.random_field(dims, int(rng.integers(1 << 30)))
        f = W.random_field(dims, int(rng.integers(1 << 30)))
        out = oracle.sweep(dims, h, omega, f, u)
        x = interior(u, nd)
        b = h * h * interior(f, nd) + boundary_vector(dims, u)
        ref = x + (omega / (2 * nd)) * (b - A @ x)
        np.testing.assert_allclose(interior(out, nd), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
        # ghost layer untouched
        g = out.copy(); g[tuple(slice(1, -1) for _ in dims)] = 0
        g0 = u.copy(); g0[tuple(slice(1, -1) for _ in dims)] = 0
        assert np.array_equal(g, g0)
        l2, linf, r = oracle.residual(dims, h, f, u, want_r=True)
        rr = b - A @ x
        np.testing.assert_allclose(interior(r, nd), rr, rtol=1e-12, atol=1e-12 * np.abs(rr).max())
        assert math.isclose(l2, np.linalg.norm(rr), rel_tol=1e-12)
        assert math.isclose(linf, np.abs(rr).max(), rel_tol=1e-12)


def sine_mode(dims, m):
    idx = [np.arange(n + 2) for n in dims]
    parts = [np.sin(mi * math.pi * ix / (n + 1)) for mi, ix, n in zip(m, idx, dims)]
    e = parts[0]
    for p in parts[1:]:
        e = p[:, None] * e[None, ...] if e.ndim == 1 else np.multiply.outer(p, e)
    return np.ascontiguousarray(e)


def mode_kappa(dims, m):
    d = len(dims)
    return (2.0 / d) * sum(math.sin(mi * math.pi / (2 * (n + 1))) ** 2 for mi, n in zip(m, dims))


@pytest.mark.parametrize("dims,P", [((16, 12), 3), ((20, 20), 4), ((8, 7, 6), 3)])
def test_eigenmode_decay_per_cycle(dims, P):
    """Eq. cycleAmplFact: with f = 0 and zero boundary data, a discrete sine mode
    of the Dirichlet grid is multiplied by exactly prod_i (1 - omega_i kappa)^q_i
    per M-cycle, whatever the order of the weights."""
    km = oracle.kappa_min_dirichlet(dims)
    omega, beta, _ = S.solve_optimal(P, km)
    q = S.q_floor(beta)
    order = S.order_drift(omega, q, km)
    seq = oracle.omega_sequence(omega, order)
    h = 1.0 / (dims[0] + 1)
    f = np.zeros(tuple(n + 2 for n in reversed(dims)))
    rng = np.random.default_rng(7)
    modes = [tuple(1 for _ in dims), tuple(dims), tuple(int(rng.integers(1, n + 1)) for n in dims),
             tuple(int(rng.integers(1, n + 1)) for n in dims)]
    for m in modes:
        e = sine_mode(dims, m)
        lam = float(np.prod((1.0 - omega * mode_kappa(dims, m)) ** q))
        u = e.copy()
        oracle.steps(dims, h, seq, f, u)
        assert np.max(np.abs(u - lam * e)) <= 1e-11 * max(1.0, abs(lam)), (m, lam)
        # a reversed order gives the same product (order independence of Eq. cycleAmplFact)
        u2 = e.copy()
        oracle.steps(dims, h, seq[::-1].copy(), f, u2)
        assert np.max(np.abs(u2 - lam * e)) <= 1e-10 * max(1.0, abs(lam))


@pytest.mark.parametrize("dims", [(16, 16), (13, 9), (6, 6, 6), (5, 7, 4)])
def test_fixed_point_equals_dense_solve(dims):
    """SRJ run to a relative residual of 1e-13 reproduces the direct solution of
    A_h u = h^2 f + (boundary terms) computed by LAPACK."""
    nd = len(dims)
    h = 1.0 / (max(dims) + 1)
    f = W.random_field(dims, 11)
    u0 = W.random_field(dims, 12)
    u0[tuple(slice(1, -1) for _ in dims)] = 0.0
    A = laplacian_matrix(dims).toarray()
    b = h * h * interior(f, nd) + boundary_vector(dims, u0)
    x = np.linalg.solve(A, b)
    km = oracle.kappa_min_dirichlet(dims)
    omega, beta, _ = S.solve_optimal(3, km)
    q = S.q_floor(beta)
    seq = oracle.omega_sequence(omega, S.order_drift(omega, q, km))
    u = u0.copy()
    st = oracle.solve(dims, h, seq, f, u, 1e-13, 10000)
    assert st["status"] == oracle.CONVERGED and st["rel"] <= 1e-13
    np.testing.assert_allclose(interior(u, nd), x, rtol=0, atol=1e-11 * np.abs(x).max())


def test_plain_jacobi_special_case():
    """P = 1, omega = 1 is textbook Jacobi: x' = D^-1 (b - (A - D) x)."""
    dims = (9, 8)
    h = 0.1
    A = laplacian_matrix(dims)
    D = A.diagonal()
    f = W.random_field(dims, 3)
    u = W.random_field(dims, 4)
    x = interior(u, 2)
    b = h * h * interior(f, 2) + boundary_vector(dims, u)
    for _ in range(5):
        x = (b - (A @ x - D * x)) / D
    oracle.steps(dims, h, np.array([1.0]), f, u, first=0, count=5)
    np.testing.assert_allclose(interior(u, 2), x, rtol=1e-12, atol=1e-13)


def _solve_to(dims, f, u0, tol=1e-12, P=5):
    km = oracle.kappa_min_dirichlet(dims)
    omega, beta, _ = S.solve_optimal(P, km)
    q = S.q_floor(beta)
    seq = oracle.omega_sequence(omega, S.order_drift(omega, q, km))
    u = u0.copy()
    st = oracle.solve(dims, 1.0 / (dims[0] + 1), seq, f, u, tol, 100000)
    assert st["status"] == oracle.CONVERGED
    return u


def test_manufactured_solution_second_order():
    """Discretisation error of the converged SRJ solution falls as h^2 (ratio ~4
    per halving of h) for the workload-1 field and for u = -exp(xy) (Sect. 5.1)."""
    errs_a, errs_b = [], []
    for n in (15, 31, 63):
        f, ue, u0 = W.manufactured_2d(n)
        u = _solve_to((n, n), f, u0)
        errs_a.append(np.abs(u - ue).max())
        f, ue, u0 = W.exp_xy_2d(n, n)
        u = _solve_to((n, n), f, u0)
        errs_b.append(np.abs(u - ue).max())
    for errs in (errs_a, errs_b):
        r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
        assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs


def test_solve_reports_divergence():
    """A non-contracting weight (omega = 3 > 1 amplifies the kappa = 2 mode by 5)
    makes the residual blow up; the oracle reports it instead of looping."""
    dims = (8, 8)
    f = W.random_field(dims, 5)
    u = W.zero_field(dims)
    st = oracle.solve(dims, 0.1, np.array([3.0]), f, u, 1e-12, 5000)
    assert st["status"] in (oracle.DIVERGED, oracle.NOT_CONVERGED)
    assert not (st["rel"] <= 1.0)
