"""Pins of the oracle-side schedule tools against the paper's printed values.

Fixtures: tests/golden/paper_schedules.json holds Table 1 (P = 2..5), the P = 14
and P = 15 tables of Sect. 4.2 and the Sect. 5.1 worked example, as printed.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle
from oracle import schedule as S

GOLDEN = json.loads((Path(__file__).parent / "golden" / "paper_schedules.json").read_text())
ROWS = GOLDEN["rows"]
# Table 1 P=4 rows at these N are not equal-ripple as printed (see the
# equal-ripple test); they are not used as pins.
P4_IRREGULAR = {150, 250, 400, 450, 500}


def printed(P, N):
    for r in ROWS:
        if r["P"] == P and r["N"] == N:
            return np.array(r["omega"]), np.array(r["beta"]), r["rho"]
    raise KeyError((P, N))


def maxima_levels(omega, beta, km):
    beta = beta / beta.sum()
    kap = np.concatenate([[km], S.interior_maxima(omega, beta), [2.0]])
    return S.log_gamma(kap, omega, beta)


def test_worked_example_neff():
    """Eq. effectiveNDirichlet on the 585 x 280 grid of Sect. 5.1 gives 252.56."""
    ex = GOLDEN["worked_example"]
    assert round(oracle.neff_dirichlet(ex["zones"]), 2) == ex["n_eff"]


def test_worked_example_p10_n550():
    """Sect. 5.1: the optimal P=10, N=550 scheme gives q = {1,1,3,9,21,49,116,268,587,1014},
    M = 2069, omega_1..3 = 106105, 40577.2, 10230.6 and rho = 125.85."""
    ex = GOLDEN["worked_example"]
    omega, beta, _ = S.solve_optimal(ex["P"], oracle.kappa_min_neumann(ex["N"]))
    q = S.q_floor(beta)
    assert q.tolist() == ex["q"] and int(q.sum()) == ex["M"]
    for got, want in zip(omega[:3], ex["omega_leading"]):
        assert abs(got / want - 1) < 5e-6, (got, want)
    assert round(S.rho(omega, beta), 2) == ex["rho"]


@pytest.mark.parametrize("row", [r for r in ROWS if not (r["P"] == 4 and r["N"] in P4_IRREGULAR)],
                         ids=lambda r: "P%d_N%d" % (r["P"], r["N"]))
def test_printed_rows_are_equal_ripple_and_satisfy_theorem2(row):
    """Every printed optimal row has equal maxima of Gamma at kappa_m, at its P-1
    interior maxima and at kappa_M = 2 (Eq. equMax), its beta is Theorem 2 of the
    interior maxima (Eq. betai), and its rho is sum omega beta (Eq. rho) — to
    the 6-digit precision of the tables."""
    omega, beta = np.array(row["omega"]), np.array(row["beta"])
    km = oracle.kappa_min_neumann(row["N"])
    lv = maxima_levels(omega, beta, km)
    # first-order effect on log Gamma of rounding every printed value to 6
    # significant digits (relative error <= 5e-6), at each maximum
    kap = np.concatenate([[km], S.interior_maxima(omega, beta / beta.sum()), [2.0]])
    x = np.outer(kap, omega)
    bound = 5e-6 * ((beta * np.abs(x / (1 - x))).sum(axis=1) + (beta * np.abs(np.log(np.abs(1 - x)))).sum(axis=1))
    assert np.ptp(lv) <= 2 * bound.max() + 1e-12, (lv, bound)
    kint = S.interior_maxima(omega, beta / beta.sum())
    b2 = S.beta_theorem2(omega, kint)
    np.testing.assert_allclose(b2, beta, rtol=1e-3)
    assert abs(S.rho(omega, beta) - row["rho"]) <= 0.011 + 2e-5 * row["rho"]


@pytest.mark.parametrize("P,N", [(2, 100), (2, 500), (3, 100), (3, 350), (5, 100), (5, 300), (5, 500),
                                 (4, 100), (4, 300)])
def test_solver_reproduces_table1(P, N):
    """The solver of Sect. 3 reproduces the printed Table 1 rows: weights and beta
    to the tables' rounding, and a level max Gamma no higher than the printed row's."""
    w_tab, b_tab, rho_tab = printed(P, N)
    km = oracle.kappa_min_neumann(N)
    omega, beta, _ = S.solve_optimal(P, km)
    np.testing.assert_allclose(omega, w_tab, rtol=1e-3)
    np.testing.assert_allclose(beta, b_tab, rtol=1e-3, atol=2e-6)
    assert abs(S.rho(omega, beta) - rho_tab) <= 0.011
    ours = maxima_levels(omega, beta, km).max()
    theirs = maxima_levels(w_tab, b_tab, km).max()
    assert ours <= theirs + 1e-9
    np.testing.assert_allclose(maxima_levels(omega, beta, km), ours, rtol=0, atol=1e-11)


@pytest.mark.parametrize("P,N", [(14, 256), (14, 1024), (14, 4096), (15, 256), (15, 2048)])
def test_solver_reproduces_large_p_tables(P, N):
    """P = 14 and P = 15 tables of Sect. 4.2: the solver's scheme has the same rho
    (to 1e-3 relative) and a lower maximum of Gamma than the printed row.  The
    printed large-P rows are close to, but not at, the minimax optimum: some
    middle weights differ by up to ~10% while the level differs by ~1e-3 of
    log Gamma, which is why only rho and the level are pinned here."""
    w_tab, b_tab, rho_tab = printed(P, N)
    km = oracle.kappa_min_neumann(N)
    omega, beta, _ = S.solve_optimal(P, km)
    assert abs(S.rho(omega, beta) / rho_tab - 1) <= 1.5e-3
    np.testing.assert_allclose(omega[[0, 1, -1]], w_tab[[0, 1, -1]], rtol=5e-3)
    ours = maxima_levels(omega, beta, km).max()
    theirs = maxima_levels(w_tab, b_tab, km).max()
    assert ours < theirs


def test_guess_exponents_match_equations():
    """Eq. omegaaprox1 (odd P) / omegaaprox2 (even P): first and last exponents 0
    and 1, the middle one 1/2 for odd P, symmetric about 1/2."""
    for P in range(3, 16):
        e = S.guess_exponents(P)
        assert e[0] == 0.0 and e[-1] == 1.0 and len(e) == P
        assert np.allclose(np.array(e) + np.array(e[::-1]), 1.0)
        if P % 2:
            assert e[P // 2] == 0.5


def test_q_floor_rule():
    """Sect. 4.3: q_i = floor(beta_i / beta_1), q_1 = 1."""
    q = S.q_floor([0.1, 0.25, 0.65])
    assert q.tolist() == [1, 2, 6]


@pytest.mark.parametrize("P,N", [(5, 100), (10, 550), (12, 362.75)])
def test_drift_order_is_a_valid_cycle_with_bounded_growth(P, N):
    """The ordering is a permutation of the multiset {omega_i x q_i}; its worst
    in-cycle window growth stays within one decade of the unavoidable single-step
    factor |1 - 2 omega_1| at kappa = 2, while the plain even spread (Sect. 5.1)
    grows by many more decades."""
    km = oracle.kappa_min_neumann(N)
    omega, beta, _ = S.solve_optimal(P, km)
    q = S.q_floor(beta)
    order = S.order_drift(omega, q, km)
    assert np.bincount(order, minlength=P).tolist() == q.tolist()
    window, suffix = S.window_growth(omega, order, km)
    floor = math.log10(2 * omega[0] - 1)
    assert floor - 1e-9 <= window <= floor + 1.0
    assert suffix <= floor
    even = sorted(((j + 0.5) / qi, i) for i, qi in enumerate(q) for j in range(qi))
    w_even, _ = S.window_growth(omega, [i for _, i in even], km)
    assert w_even > window + 3.0


def test_fp32_order_is_a_valid_cycle_with_no_more_modelled_noise():
    """order_fp32 permutes the same multiset as the drift order (same cycle
    polynomial, Sect. 2) and never raises the modelled FP32 cycle noise; an
    order that moves many small weights out of the body is flagged."""
    km = oracle.kappa_min_dirichlet((4096, 4096))
    row = __import__("paper_1511_04292_gb300").schedules.lookup(2, 4096, 10)
    omega, q = row["omega"], row["q"]
    base = S.order_drift(omega, q, km)
    tuned = S.order_fp32(omega, q, km)
    assert np.bincount(tuned, minlength=len(q)).tolist() == list(q)
    assert np.array_equal(np.sort(base), np.sort(tuned))
    nb, nt = S.fp32_cycle_noise(omega, base, km), S.fp32_cycle_noise(omega, tuned, km)
    assert nt <= nb
    # 28 of the smallest weights pulled out of the start of the body: unbalanced
    body = list(base[:-4])
    drop = set([i for i, v in enumerate(body) if v == len(q) - 1][:28])
    bad = np.array([v for i, v in enumerate(body) if i not in drop] + [len(q) - 1] * 32)
    assert S.fp32_cycle_noise(omega, bad, km) > 1.0


def _cycle_float(seq, r, dtype):
    """One SRJ cycle on the 2-D defect equation A e = r from e = 0 (e = 0 on the
    boundary), every operation rounded to `dtype` (numpy does not contract)."""
    e = np.zeros_like(r, dtype=dtype)
    rr = r.astype(dtype)
    four = dtype(4.0)
    for w in seq:
        nb = ((e[1:-1, :-2] + e[1:-1, 2:]) + e[:-2, 1:-1]) + e[2:, 1:-1]
        t = (nb + rr[1:-1, 1:-1]) - four * e[1:-1, 1:-1]
        e2 = e.copy()
        e2[1:-1, 1:-1] = e[1:-1, 1:-1] + dtype(w / 4.0) * t
        e = e2
    return e


def test_fp32_noise_model_against_brute_force_fp32_cycles():
    """The FP32 noise model that picks the cycle order, against brute force: one
    cycle in float32 and in float64 on a 128^2 grid from a white residual; the
    residual of the difference, ||A (e32 - e64)|| / ||r||, for the drift order
    with m = 0..36 copies of omega_P moved to the tail and for the reversed
    order.  The measured noise spans 20 decades; the model must rank the orders
    as measured (Spearman >= 0.95), stay within a factor 10 of every measurement,
    and the order order_fp32 picks must be within 1.5x of the quietest one."""
    import paper_1511_04292_gb300.schedules as sch
    from scipy.stats import spearmanr
    n, P = 128, 7
    row = sch.lookup(2, n, P)
    omega, q = np.asarray(row["omega"]), np.asarray(row["q"])
    km = oracle.kappa_min_dirichlet((n, n))
    base = [int(v) for v in S.order_drift(omega, q, km)]
    small = P - 1
    body = base[:-min(S.TAIL_STEPS, int(q[-1]))]
    tail0 = len(base) - len(body)
    pos = [i for i, v in enumerate(body) if v == small]
    cands = {"reversed": base[::-1]}
    for m in range(0, 40, 4):
        drop = set(pos[:m])
        cands[m] = [v for i, v in enumerate(body) if i not in drop] + [small] * (tail0 + m)
    rng = np.random.default_rng(5)
    r = np.zeros((n + 2, n + 2))
    r[1:-1, 1:-1] = rng.standard_normal((n, n))
    r = r.astype(np.float32).astype(np.float64)

    def A(e):
        return 4 * e[1:-1, 1:-1] - (((e[1:-1, :-2] + e[1:-1, 2:]) + e[:-2, 1:-1]) + e[2:, 1:-1])

    model, meas = [], []
    for o in cands.values():
        seq = omega[np.asarray(o)]
        d = _cycle_float(seq, r, np.float32).astype(np.float64) - _cycle_float(seq, r, np.float64)
        meas.append(np.linalg.norm(A(d)) / np.linalg.norm(r[1:-1, 1:-1]))
        model.append(S.fp32_cycle_noise(omega, o, km))
    model, meas = np.array(model), np.array(meas)
    assert np.all(np.isfinite(meas)) and meas.max() / meas.min() > 1e15
    assert spearmanr(model, meas).correlation >= 0.95
    assert np.all((meas / model > 0.1) & (meas / model < 10.0)), meas / model
    pick = [int(v) for v in S.order_fp32(omega, q, km)]
    seq = omega[np.asarray(pick)]
    d = _cycle_float(seq, r, np.float32).astype(np.float64) - _cycle_float(seq, r, np.float64)
    assert np.linalg.norm(A(d)) / np.linalg.norm(r[1:-1, 1:-1]) <= 1.5 * meas.min()


def test_cycle_factor_bounds_the_dense_cycle_matrix():
    """Brute force on a 12 x 10 Dirichlet grid: the error of one SRJ cycle is
    multiplied by E = prod_k (I - omega_k D^-1 A) (dense, in the cycle order).
    Its spectral radius equals the largest |prod_i (1 - omega_i kappa)^q_i| over
    the grid's eigenvalues kappa, and max_cycle_factor, which samples the whole
    interval [kappa_min, 2], bounds it from above."""
    nx, ny = 12, 10
    N = nx * ny
    A = np.zeros((N, N))
    for y in range(ny):
        for x in range(nx):
            i = y * nx + x
            A[i, i] = 4.0
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                if 0 <= x + dx < nx and 0 <= y + dy < ny:
                    A[i, (y + dy) * nx + x + dx] = -1.0
    J = A / 4.0  # D^-1 A
    kap = np.linalg.eigvalsh(J)
    km = oracle.kappa_min_dirichlet((nx, ny))
    assert abs(kap.min() - km) < 1e-12
    omega, beta, _ = S.solve_optimal(3, km)
    q = S.q_floor(beta)
    order = S.order_drift(omega, q, km)
    E = np.eye(N)
    for k in order:
        E = (np.eye(N) - omega[k] * J) @ E
    rho = np.max(np.abs(np.linalg.eigvals(E)))
    per_mode = np.max(np.abs(np.prod([(1.0 - w * kap) ** qq for w, qq in zip(omega, q)], axis=0)))
    assert abs(np.log10(rho) - np.log10(per_mode)) < 1e-6
    assert np.log10(rho) <= S.max_cycle_factor(omega, q, km) + 1e-9
    assert S.max_cycle_factor(omega, q, km) < 0
    # textbook special case with the maximum at the low end only: damped Jacobi (P = 1,
    # omega = 0.8) has spectral radius 1 - 0.8 kappa_min (|1 - 0.8 kappa_max| is smaller)
    rho_j = np.max(np.abs(np.linalg.eigvals(np.eye(N) - 0.8 * J)))
    assert abs(rho_j - (1.0 - 0.8 * km)) < 1e-12
    assert abs(S.max_cycle_factor([0.8], [1], km) - np.log10(rho_j)) < 1e-12


def test_integer_scheme_contracts():
    """Sect. 4.3: after the floor conversion the cycle factor stays below 1 on
    [kappa_m, 2]; a scheme that over-weights the largest omega does not."""
    km = oracle.kappa_min_neumann(300)
    omega, beta, _ = S.solve_optimal(5, km)
    q = S.q_floor(beta)
    assert S.max_cycle_factor(omega, q, km) < 0
    bad = q.copy(); bad[0] = q[0] * 20
    assert S.max_cycle_factor(omega, bad, km) > 0


def test_window_growth_against_brute_force_windows():
    """Pin of the order metric: the largest growth of a contiguous run of steps
    and of a cycle suffix, enumerated window by window (every a < b) at every
    sampled kappa, for a short cycle of a P = 4 scheme in several orders,
    including one that puts the large weights together."""
    km = 1e-3
    omega, beta, _ = S.solve_optimal(4, km)
    q = S.q_floor(beta)
    q = np.minimum(q, 6)
    base = [i for i, c in enumerate(q) for _ in range(int(c))]
    rng = np.random.default_rng(5)
    orders = [base, base[::-1], list(rng.permutation(base)), list(S.order_drift(omega, q, km))]
    samples = 300
    kap = np.geomspace(km, 2.0, samples)
    for order in orders:
        L = np.log10(np.abs(1.0 - np.outer(np.asarray(omega)[np.asarray(order)], kap)))  # M x K
        M = len(order)
        wmax, smax = 0.0, -np.inf
        for a in range(M):
            for b in range(a + 1, M + 1):
                wmax = max(wmax, float(L[a:b].sum(axis=0).max()))
            smax = max(smax, float(L[a:].sum(axis=0).max()))
        window, suffix = S.window_growth(omega, order, km, samples=samples)
        assert abs(window - wmax) < 1e-9 and abs(suffix - smax) < 1e-9, (order, window, wmax, suffix, smax)
