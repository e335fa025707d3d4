"""Pins of the spherical-coordinate oracle (Sect. 5.2) against facts it does not
compute itself: closed forms of the difference coefficients, exact images of
low-order functions, a dense solve of the effective system, and second-order
convergence to the paper's analytic solution (Eqs. grav:source, grav:sol)."""
import math

import numpy as np
import pytest

import oracle
import paper_1511_04292_gb300.schedules as sch

scipy_special = pytest.importorskip("scipy.special")
from scipy.optimize import brentq  # noqa: E402


def seq_for(P=6):
    row = sch.lookup(2, 64, P)
    return oracle.omega_sequence(row["omega"], row["order"])


def paper_problem_2d(nr, nt):
    """Axisymmetric test of Sect. 5.2 truncated to the l = 0 and l = 2 terms
    (a_l = 2^-l, k_l the first root of j_l; b_l = c_l from continuity at r = 1):
    returns (u_analytic, b = r^2 s) in the padded (theta, r) layout."""
    jn = scipy_special.spherical_jn
    dr, dt = 1.0 / nr, math.pi / nt
    r = (np.arange(nr + 2) - 0.5) * dr
    t = (np.arange(nt + 2) - 0.5) * dt
    R, Th = np.meshgrid(r, t)
    P2 = 0.5 * (3 * np.cos(Th) ** 2 - 1)
    k0, k2 = math.pi, brentq(lambda x: jn(2, x), 5.0, 6.5)
    a0, a2 = 1.0, 0.25
    b0 = -a0 * (0 * jn(0, k0) - k0 * jn(1, k0))
    b2 = -a2 / 5 * (2 * jn(2, k2) - k2 * jn(3, k2))
    Rin = np.where(R <= 1, R, 1.0)
    u_in = (a0 * jn(0, k0 * Rin) + b0) + (a2 * jn(2, k2 * Rin) + b2 * Rin ** 2) * P2
    u_out = b0 / R + b2 / R ** 3 * P2
    s = np.where(R <= 1, -a0 * k0 ** 2 * jn(0, k0 * Rin) - a2 * k2 ** 2 * jn(2, k2 * Rin) * P2, 0.0)
    return np.where(R <= 1, u_in, u_out), R ** 2 * s


def test_radial_coefficients_closed_form_and_effective_row():
    """With r_i = (i - 1/2) dr the radial coefficients are dimensionless:
    cr_m = (i - 3/2)(i - 1/2), cr_p = (i - 1/2)(i + 1/2), cr_0 = 2 (i - 1/2)^2.
    Under u_1 = u_2 the effective row 2 is (-15/4, +15/4): weakly diagonally
    dominant, as Sect. 5.2 requires of the prescription."""
    for nr in (4, 17, 100):
        radial, _, _ = oracle.spherical_coefficients((nr, 8))
        for i in range(1, nr + 1):
            assert radial[0, i] == pytest.approx((i - 1.5) * (i - 0.5), rel=1e-12, abs=1e-12)
            assert radial[1, i] == pytest.approx((i - 0.5) * (i + 0.5), rel=1e-12)
            assert radial[2, i] == pytest.approx(2 * (i - 0.5) ** 2, rel=1e-12)
        assert radial[2, 2] - radial[0, 2] == pytest.approx(15 / 4) and radial[1, 2] == pytest.approx(15 / 4)


def test_polar_and_azimuthal_coefficients():
    nt = 24
    _, polar, azim = oracle.spherical_coefficients((8, nt, 6))
    dt, dp = math.pi / nt, 2 * math.pi / 6
    for j in range(1, nt + 1):
        t = (j - 0.5) * dt
        assert polar[0, j] + polar[1, j] == pytest.approx(polar[2, j], rel=1e-14)
        assert (polar[1, j] - polar[0, j]) * dt == pytest.approx(1 / math.tan(t), rel=1e-9, abs=1e-12)
        assert polar[0, j] > 0 and polar[1, j] > 0  # diagonal dominance holds down to the poles
        assert azim[j] * (math.sin(t) * dp) ** 2 == pytest.approx(1.0, rel=1e-12)


def test_constants_are_in_the_kernel():
    """Row sums vanish and the boundary prescriptions keep constants: L(1) = 0."""
    for dims in [(9, 7), (6, 5, 4)]:
        coef = oracle.spherical_coefficients(dims)
        u = np.full(oracle.padded_shape(dims), 3.0)
        b = np.zeros_like(u)
        l2, linf = oracle.sph_residual(dims, coef, b, u)
        assert linf <= 1e-12 * 3.0 * np.max(np.abs(coef[0]))


def test_exact_images_of_r2_cos_theta_cos_phi():
    """Central differences are exact on r^2 (L r^2 = 6 r^2 away from r = 0), and on
    cos(theta) / cos(phi) the discrete operator has the closed forms
    cos(t) [(2 cos dt - 2) / dt^2 - sin(dt) / dt] and cp (2 cos dp - 2) cos(phi)."""
    nr, nt, nph = 12, 10, 8
    dims = (nr, nt, nph)
    coef = oracle.spherical_coefficients(dims)
    dr, dt, dp = 1.0 / nr, math.pi / nt, 2 * math.pi / nph
    r = (np.arange(nr + 2) - 0.5) * dr
    t = (np.arange(nt + 2) - 0.5) * dt
    ph = (np.arange(nph + 2) - 0.5) * dp
    P, T, R = np.meshgrid(ph, t, r, indexing="ij")
    b = np.zeros(oracle.padded_shape(dims))
    # r^2: residual = L u - b = L u
    _, _, res = oracle.sph_residual(dims, coef, b, np.ascontiguousarray(R ** 2), want_r=True)
    ii = slice(3, nr + 1)
    np.testing.assert_allclose(res[1:-1, 1:-1, ii], (6 * R ** 2)[1:-1, 1:-1, ii], rtol=1e-9, atol=1e-9)
    # cos(theta): interior polar rows (no mirror substitution), r-independent so only theta terms act
    _, _, res = oracle.sph_residual(dims, coef, b, np.ascontiguousarray(np.cos(T)), want_r=True)
    ref = np.cos(T) * ((2 * math.cos(dt) - 2) / dt ** 2 - math.sin(dt) / dt)
    np.testing.assert_allclose(res[1:-1, 2:-2, 2:-1], ref[1:-1, 2:-2, 2:-1], rtol=1e-9, atol=1e-9)
    # cos(phi): periodic wrap included (all k)
    _, _, res = oracle.sph_residual(dims, coef, b, np.ascontiguousarray(np.cos(P)), want_r=True)
    cp = coef[2][None, :, None]
    ref = cp * (2 * math.cos(dp) - 2) * np.cos(P)
    np.testing.assert_allclose(res[1:-1, 1:-1, 2:-1], ref[1:-1, 1:-1, 2:-1], rtol=1e-9, atol=1e-9)


def dense_effective_solve(dims, coef, b, ughost):
    """Solve L u = b on the active points by a dense LU, the matrix assembled
    point by point from the boundary rules (independent of the C code)."""
    nr, nt = dims[0], dims[1]
    nph = dims[2] if len(dims) == 3 else 1
    radial, polar, azim = coef
    act = [(k, j, i) for k in range(nph) for j in range(nt) for i in range(2, nr + 1)]
    index = {p: n for n, p in enumerate(act)}
    A = np.zeros((len(act), len(act)))
    rhs = np.zeros(len(act))
    for n, (k, j, i) in enumerate(act):
        kk = k + 1 if len(dims) == 3 else None
        bp = b[kk, j + 1, i] if kk is not None else b[j + 1, i]
        rhs[n] = bp
        d = radial[2, i] + polar[2, j + 1] + (2 * azim[j + 1] if len(dims) == 3 else 0.0)
        A[n, n] -= d

        def add(kq, jq, iq, c):
            if iq == nr + 1:  # Dirichlet ghost
                g = ughost[kq + 1, jq + 1, iq] if len(dims) == 3 else ughost[jq + 1, iq]
                rhs[n] -= c * g
                return
            A[n, index[(kq, jq, iq)]] += c
        add(k, j, i if i == 2 else i - 1, radial[0, i])          # u_1 = u_2
        add(k, j, i + 1, radial[1, i])
        add(k, j if j == 0 else j - 1, i, polar[0, j + 1])        # theta mirrors
        add(k, j if j == nt - 1 else j + 1, i, polar[1, j + 1])
        if len(dims) == 3:
            add((k - 1) % nph, j, i, azim[j + 1])                 # periodic phi
            add((k + 1) % nph, j, i, azim[j + 1])
    x = np.linalg.solve(A, rhs)
    return act, x


@pytest.mark.parametrize("dims", [(7, 6), (5, 4, 6)])
def test_srj_fixed_point_equals_dense_solve(dims):
    rng = np.random.default_rng(11)
    shape = oracle.padded_shape(dims)
    coef = oracle.spherical_coefficients(dims)
    b = rng.standard_normal(shape)
    u = np.zeros(shape)
    u[..., -1] = rng.standard_normal(shape[:-1])  # Dirichlet data at r_{N+1}
    ug = u.copy()
    st = oracle.sph_solve(dims, coef, seq_for(5), b, u, 1e-14, 5000)
    assert st["status"] == oracle.CONVERGED
    act, x = dense_effective_solve(dims, coef, b, ug)
    got = np.array([u[(k + 1, j + 1, i) if len(dims) == 3 else (j + 1, i)] for (k, j, i) in act])
    np.testing.assert_allclose(got, x, rtol=1e-9, atol=1e-9 * np.max(np.abs(x)))
    # finalize: the prescription u_0 = u_1 = u_2 and the mirrors hold on the returned field
    if len(dims) == 2:
        assert np.array_equal(u[1:-1, 0], u[1:-1, 2]) and np.array_equal(u[1:-1, 1], u[1:-1, 2])
        assert np.array_equal(u[0, :], u[1, :]) and np.array_equal(u[-1, :], u[-2, :])
    else:
        assert np.array_equal(u[0], u[-2]) and np.array_equal(u[-1], u[1])


def test_second_order_convergence_to_the_analytic_solution():
    """Sect. 5.2: the discretisation error dominates at convergence and falls
    as N^-2 (two halvings of dr and dtheta)."""
    errs = []
    for N in (32, 64, 128):
        dims = (N, N)
        ua, b = paper_problem_2d(N, N)
        u = np.zeros_like(ua)
        u[:, -1] = ua[:, -1]
        st = oracle.sph_solve(dims, oracle.spherical_coefficients(dims), seq_for(6), b, u, 1e-12, 3000)
        assert st["status"] == oracle.CONVERGED
        errs.append(np.abs(u - ua)[1:-1, 2:-1].max())
    for a, c in zip(errs, errs[1:]):
        assert 3.5 < a / c < 4.5, errs


def test_printed_matrix_entries_do_not_discretise_the_equation():
    """Reading of Sect. 5.2: the printed matrix (r_i +- 2 dr) doubles the
    first-derivative term; SRJ still converges on it, but not to the analytic
    solution, while the printed difference equation (r_i +- dr) does."""
    N = 64
    dims = (N, N)
    ua, b = paper_problem_2d(N, N)
    coef = list(oracle.spherical_coefficients(dims))
    r = (np.arange(N + 2) - 0.5) / N
    rad = coef[0].copy()
    rad[0] = r * (r - 2.0 / N) * N * N
    rad[1] = r * (r + 2.0 / N) * N * N
    coef[0] = rad
    u = np.zeros_like(ua)
    u[:, -1] = ua[:, -1]
    st = oracle.sph_solve(dims, coef, seq_for(6), b, u, 1e-12, 3000)
    assert st["status"] == oracle.CONVERGED
    assert np.abs(u - ua)[1:-1, 2:-1].max() > 0.1


def test_3d_converges_at_second_order():
    errs = []
    for N in (12, 24):
        ua2, b2 = paper_problem_2d(N, N)
        ua = np.repeat(ua2[None], N + 2, axis=0)
        b = np.ascontiguousarray(np.repeat(b2[None], N + 2, axis=0))
        dims = (N, N, N)
        u = np.zeros_like(ua)
        u[:, :, -1] = ua[:, :, -1]
        st = oracle.sph_solve(dims, oracle.spherical_coefficients(dims), seq_for(6), b, u, 1e-12, 3000)
        assert st["status"] == oracle.CONVERGED
        errs.append(np.abs(u - ua)[1:-1, 1:-1, 2:-1].max())
    assert errs[0] / errs[1] > 3.0, errs
