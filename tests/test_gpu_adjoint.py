"""GPU tests of the differentiable solve (srj_gradient / SRJSolve).

L = 1/2 sum_interior (u - u_t)^2 with u = S(f, g).  u is linear in (f, g), so L is
exactly quadratic and central differences with a unit step are exact up to the
solves' tolerance.  Small grids are checked against a dense LAPACK adjoint.
"""
import numpy as np
import pytest

import oracle
import srj_workloads as W
from oracle import schedule as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1511_04292_gb300 as srj  # noqa: E402
from paper_1511_04292_gb300.autograd import SRJSolve  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _laplacian(dims):
    import scipy.sparse as sp
    mats = [sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) for n in dims]
    eye = [sp.identity(n) for n in dims]
    A = None
    for k in range(len(dims)):
        term = None
        for j in reversed(range(len(dims))):
            blk = mats[j] if j == k else eye[j]
            term = blk if term is None else sp.kron(term, blk)
        A = term if A is None else A + term
    return A.toarray()


@pytest.mark.parametrize("dims,prec", [((12, 9), "fp64"), ((5, 4, 6), "fp64"), ((12, 9), "mixed"),
                                       ((12, 9), "fp64fma")])
def test_gradient_matches_dense_adjoint(dims, prec):
    nd = len(dims)
    shape = tuple(n + 2 for n in reversed(dims))
    inner = tuple(slice(1, -1) for _ in dims)
    h = 1.0 / (max(dims) + 1)
    km = oracle.kappa_min_dirichlet(dims)
    omega, beta, _ = S.solve_optimal(3, km)
    q = S.q_floor(beta)
    plan = srj.Plan(dims, h, omega, q, S.order_drift(omega, q, km), prec)
    f = W.random_field(dims, 1)
    g = W.random_field(dims, 2)
    ut = W.random_field(dims, 3)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    u = SRJSolve.apply(ft, gt, plan, 1e-14, 100000)
    loss = 0.5 * ((u - torch.from_numpy(ut).cuda())[inner] ** 2).sum()
    loss.backward()
    # dense reference: b = h^2 f + B g
    A = _laplacian(dims)
    gz = g.copy(); gz[inner] = 0
    acc = np.zeros(shape)
    for ax in range(nd):
        for sh in (-1, 1):
            acc += np.roll(gz, sh, axis=ax)
    b = h * h * f[inner].reshape(-1) + acc[inner].reshape(-1)
    x = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, x - ut[inner].reshape(-1))
    gf_ref = np.zeros(shape); gf_ref[inner] = (h * h * lam).reshape(f[inner].shape)
    L = np.zeros(shape); L[inner] = lam.reshape(f[inner].shape)
    gg_ref = np.zeros(shape)
    for ax in range(nd):
        for sh in (-1, 1):
            gg_ref += np.roll(L, sh, axis=ax)
    gg_ref[inner] = 0
    np.testing.assert_allclose(u.detach().cpu().numpy()[inner].reshape(-1), x, rtol=0, atol=1e-10 * np.abs(x).max())
    np.testing.assert_allclose(ft.grad.cpu().numpy(), gf_ref, rtol=0, atol=1e-10 * np.abs(gf_ref).max())
    np.testing.assert_allclose(gt.grad.cpu().numpy(), gg_ref, rtol=0, atol=1e-10 * np.abs(gg_ref).max())


def test_full_size_adjoint_against_central_differences():
    """Workload 5: 2048^2 FP64, L = 1/2 ||u - u_t||^2, gradients w.r.t. f and the
    boundary data from the adjoint backward, against central differences on 32
    seeded random directions in (f, g) (relative error <= 1e-5), every solve in
    FP64.  L is quadratic in (f, g), so the central difference has no truncation
    error; solves go to tol 1e-12 or to their floating-point floor (relative
    residual ~1e-12 at this size), which bounds the error of u by about
    cond(A) x 1e-12 ~ 2e-6 relative."""
    n = 2048
    dims = (n, n)
    shape = (n + 2, n + 2)
    inner = (slice(1, -1), slice(1, -1))
    f, g = W.random_smooth_problem_2d(n, 21)
    ut = W.smooth_target_2d(n, 22)
    plan = srj.Plan.from_table(dims, 10, "fp64")
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    gt = torch.from_numpy(g).cuda().requires_grad_(True)
    utd = torch.from_numpy(ut).cuda()
    u = SRJSolve.apply(ft, gt, plan, 1e-12, 200)
    loss = 0.5 * ((u - utd)[inner] ** 2).sum()
    loss.backward()
    grad_f = ft.grad.cpu().numpy()
    grad_g = gt.grad.cpu().numpy()
    rng = np.random.default_rng(23)
    ghost = np.ones(shape, bool); ghost[inner] = False
    dirs = []
    for k in range(32):
        df = np.zeros(shape); df[inner] = 0.2 * rng.standard_normal((n, n))
        dg = np.zeros(shape); dg[ghost] = rng.standard_normal(ghost.sum())
        dirs.append((df, dg))
    worst = 0.0
    for k, (df, dg) in enumerate(dirs):
        sol = []
        for sgn in (1.0, -1.0):
            u0 = g + sgn * dg
            u0[inner] = 0.0
            ud = torch.from_numpy(u0).cuda()
            st = plan.solve(torch.from_numpy(f + sgn * df).cuda(), ud, 1e-12, 200, raise_on_fail=False)
            assert st["rel_res"] <= 1e-12 or st["stagnated"], st
            assert st["rel_res"] < 1e-11, st
            sol.append(ud.cpu().numpy())
        up, um = sol
        Lp = 0.5 * np.sum((up - ut)[inner] ** 2)
        Lm = 0.5 * np.sum((um - ut)[inner] ** 2)
        fd = (Lp - Lm) / 2.0
        an = np.sum(grad_f * df) + np.sum(grad_g * dg)
        worst = max(worst, abs(fd - an) / abs(an))
    assert worst <= 1e-5, worst
