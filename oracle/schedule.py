"""Optimal SRJ parameters, integer conversion and cycle ordering (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check, the CPU-baseline leg of
the benchmark and ``oracle/make_schedules.py`` use this module.

Paper: Adsuara et al., "Scheduled Relaxation Jacobi method: improvements and
applications", arXiv:1511.04292.  Notation follows the paper: P levels, weights
omega_1 > ... > omega_P, fractions beta_i (sum 1), integer repetitions q_i,
M = sum q_i, spectral variable kappa in [kappa_m, kappa_M = 2].

* ``log_gamma``           Eq. Gamma (per-iteration amplification, in logs).
* ``beta_theorem2``       Theorem 2, Eq. betai: beta from omega and the interior
                          maxima kappa_1..kappa_{P-1}.
* ``system``              the reduced system S(omega, kappa) of Sect. 3.5:
                          equal maxima (Eq. equMax) plus the optimality
                          conditions of Eqs. partialbeta / equDifBeta, imposed
                          through Lagrange multipliers (see ``system``).
* ``initial_guess``       Eqs. omegaaprox1 / omegaaprox2 and the kappa_i guess
                          of Sect. 3.5.
* ``solve_optimal``       continuation in P (Sect. 3.3: weights of P+1 levels
                          from the extrapolated extreme weights of P-3..P).
* ``solve_optimal_fine``  any resolution: below kappa_m = 1e-7 the scheme is
                          followed from that bound to kappa_m in extended
                          precision (mpmath, 40 digits; Sect. 3.3 needed 24).
* ``q_floor``             Sect. 4.3: q_i = floor(beta_i / beta_1).
* ``rho``                 Eq. rho.
* ``order_drift``         cycle ordering (Sect. 5.1 asks for the large
                          over-relaxations to be spread over the cycle; the
                          algorithm is this build's reading, see its docstring).
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import optimize

KAPPA_MAX = 2.0


# ---------------------------------------------------------------------------
# Amplification factors
# ---------------------------------------------------------------------------

def log_gamma(kappa, omega, beta):
    """log Gamma(kappa) = sum_i beta_i log|1 - omega_i kappa| (Eq. Gamma)."""
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    omega = np.asarray(omega, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    return np.log(np.abs(1.0 - np.outer(kappa, omega))) @ beta


def log10_cycle_factor(kappa, omega, q):
    """log10 |prod_i G_{omega_i}(kappa)^{q_i}| for one M-cycle (Eq. cycleAmplFact)."""
    kappa = np.atleast_1d(np.asarray(kappa, dtype=np.float64))
    return np.log10(np.abs(1.0 - np.outer(kappa, np.asarray(omega, float)))) @ np.asarray(q, float)


def rho(omega, beta):
    """Convergence performance index rho = sum_i omega_i beta_i (Eq. rho)."""
    return float(np.dot(omega, beta))


def beta_theorem2(omega, kappa_int):
    """Theorem 2 (Eq. betai), with the products over k and l taken separately:

        beta_i = prod_{k=1}^{P-1} (1 - kappa_k omega_i) * prod_{l != i} omega_l / (omega_l - omega_i).
    """
    omega = np.asarray(omega, dtype=np.float64)
    P = len(omega)
    beta = np.empty(P)
    for i in range(P):
        v = 1.0
        for kk in kappa_int:
            v *= 1.0 - kk * omega[i]
        for l in range(P):
            if l != i:
                v *= omega[l] / (omega[l] - omega[i])
        beta[i] = v
    return beta


def interior_maxima(omega, beta):
    """Roots of d log Gamma / d kappa = 0 (Eq. partialG), one in each
    (1/omega_i, 1/omega_{i+1}) (Sect. 3.5)."""
    omega = np.asarray(omega, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    out = []
    for i in range(len(omega) - 1):
        lo, hi = 1.0 / omega[i], 1.0 / omega[i + 1]
        g = lambda k: float(np.sum(beta * omega / (1.0 - k * omega)))
        a, b = lo * (1 + 1e-13), hi * (1 - 1e-13)
        out.append(optimize.brentq(g, a, b, xtol=1e-300, rtol=1e-15, maxiter=500))
    return np.array(out)


# ---------------------------------------------------------------------------
# The system S(omega, kappa)
# ---------------------------------------------------------------------------

def _unpack(x, P):
    """x = (log omega_1..P, t_1..t_{P-1}); kappa_i = 1/omega_i + s(t_i) (1/omega_{i+1} - 1/omega_i)
    with s the logistic function, so each kappa_i stays inside its bracket (Sect. 3.5)."""
    omega = np.exp(x[:P])
    s = 0.5 * (1.0 + np.tanh(0.5 * np.asarray(x[P:], dtype=np.float64)))
    inv = 1.0 / omega
    return omega, inv[:-1] + s * (inv[1:] - inv[:-1])


def _pack(omega, kint):
    inv = 1.0 / np.asarray(omega, dtype=np.float64)
    s = (np.asarray(kint) - inv[:-1]) / (inv[1:] - inv[:-1])
    s = np.clip(s, 1e-12, 1 - 1e-12)
    return np.concatenate([np.log(omega), np.log(s / (1.0 - s))])


def system(x, P, kappa_m):
    """Residuals of the reduced system S(omega, kappa) (Sect. 3.5).

    Unknowns x = (log omega_1..omega_P, t_1..t_{P-1}) with kappa_i placed inside
    (1/omega_i, 1/omega_{i+1}) by t_i (see ``_unpack``); beta follows from
    Theorem 2, so the interior kappa_i are stationary points of Gamma (Eq.
    partialG) by construction.  With kappa_0 = kappa_m and kappa_P = 2:

    * P equations, Eq. equMax: log Gamma(kappa_j) - log Gamma(kappa_0) = 0, j=1..P.
    * P-1 optimality equations.  Eqs. partialbeta / equDifBeta ask that the
      common level of the maxima be stationary in beta when omega moves to keep
      the maxima equal.  This is imposed in its Lagrange-multiplier form: there
      are weights mu_0..mu_P (sum 1) on the active points with
      sum_j mu_j kappa_j / (1 - omega_i kappa_j) = 0 for every i (stationarity
      in omega), and sum_j mu_j (log|1-omega_i kappa_j| - log|1-omega_P kappa_j|)
      = 0 for i = 1..P-1 (stationarity in beta on the simplex).
    """
    omega, kint = _unpack(x, P)
    beta = beta_theorem2(omega, kint)
    kap = np.concatenate([[kappa_m], kint, [KAPPA_MAX]])
    F = log_gamma(kap, omega, beta)
    eq_max = F[1:] - F[0]
    Mm = np.vstack([kap[None, :] / (1.0 - np.outer(omega, kap)), np.ones((1, P + 1))])
    rhs = np.zeros(P + 1)
    rhs[-1] = 1.0
    mu = np.linalg.solve(Mm, rhs)
    a = np.log(np.abs(1.0 - np.outer(omega, kap)))
    eq_opt = (a[:-1, :] - a[-1:, :]) @ mu
    return np.concatenate([eq_max, eq_opt])


def guess_exponents(P):
    """Exponents e of the initial inverse weights omega_1^-1 (omega_1/omega_P)^e,
    Eq. omegaaprox1 (P odd) and Eq. omegaaprox2 (P even), numerators over 2(P-1)."""
    if P == 2:
        return [0.0, 1.0]
    if P % 2 == 1:
        nums = [0] + list(range(1, P - 3, 2)) + [P - 1] + list(range(P + 2, 2 * P - 2, 2)) + [2 * P - 2]
    else:
        nums = [0] + list(range(1, P - 4, 2)) + [P - 2, P] + list(range(P + 3, 2 * P - 2, 2)) + [2 * P - 2]
    assert len(nums) == P
    return [m / (2.0 * (P - 1)) for m in nums]


def initial_guess(P, omega_1, omega_P):
    """Initial unknowns: weights from Eqs. omegaaprox1/2 and
    kappa_i ~ 1/omega_i + (1/omega_{i+1} - 1/omega_i)/3 (Sect. 3.5)."""
    inv = np.array([(1.0 / omega_1) * (omega_1 / omega_P) ** e for e in guess_exponents(P)])
    omega = 1.0 / inv
    kint = np.array([1.0 / omega[i] + (1.0 / omega[i + 1] - 1.0 / omega[i]) / 3.0 for i in range(P - 1)])
    return _pack(omega, kint)


def _accept(sol, P):
    if not np.all(np.isfinite(sol.x)) or np.max(np.abs(sol.fun)) > 1e-10:
        return None
    omega, kint = _unpack(sol.x, P)
    if not np.all(np.diff(omega) < 0) or omega[-1] <= 0.5:
        return None
    for i in range(P - 1):
        if not (1.0 / omega[i] < kint[i] < 1.0 / omega[i + 1]):
            return None
    beta = beta_theorem2(omega, kint)
    if not np.all(beta > 0) or abs(beta.sum() - 1.0) > 1e-9:
        return None
    return omega, beta, kint


def _newton(P, kappa_m, x0):
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        try:
            sol = optimize.root(system, x0, args=(P, kappa_m), method="hybr",
                                options=dict(xtol=1e-15, maxfev=200 * (2 * P)))
        except (np.linalg.LinAlgError, ValueError, FloatingPointError):
            return None
    return _accept(sol, P)


_GRID_R1 = (0.05, 0.1, 0.15, 0.2, 0.3, 0.35, 0.5, 0.7, 0.85, 0.95)
_GRID_WP = (0.98, 0.95, 0.9, 0.85, 0.7, 0.6, 0.55)


class ScheduleError(RuntimeError):
    pass


def solve_optimal(P, kappa_m, return_all=False):
    """Optimal (omega, beta, kappa_int) for P levels at spectral bound kappa_m.

    Levels are solved in turn from 2 to P.  For the next level the guesses of
    omega_1 and omega_P are extrapolated from the last (up to four) solved levels
    (quadratic fits of log omega_1 and of log(omega_P - 1/2) in P, this build's
    reading of the conic fits of Sect. 3.3); the remaining weights follow Eqs.
    omegaaprox1/2.  Levels with fewer than two predecessors, or whose
    extrapolated guess fails, are started from a small grid of (omega_1,
    omega_P) guesses and the lowest level Gamma(kappa_m) among the accepted
    solutions is kept.
    """
    hist = {}
    for p in range(2, P + 1):
        found = None
        if len(hist) >= 2:
            ps = sorted(hist)[-4:]
            deg = min(2, len(ps) - 1)
            c1 = np.polyfit(ps, [math.log(hist[k][0][0]) for k in ps], deg)
            cP = np.polyfit(ps, [math.log(hist[k][0][-1] - 0.5) for k in ps], deg)
            w1 = math.exp(np.polyval(c1, p))
            wP = 0.5 + math.exp(np.polyval(cP, p))
            found = _newton(p, kappa_m, initial_guess(p, w1, wP))
        if found is None:
            best = None
            for r1 in _GRID_R1:
                for wP in _GRID_WP:
                    cand = _newton(p, kappa_m, initial_guess(p, r1 / kappa_m, wP))
                    if cand is None:
                        continue
                    lvl = log_gamma(kappa_m, cand[0], cand[1])[0]
                    if best is None or lvl < best[0] - 1e-13:
                        best = (lvl, cand)
            found = None if best is None else best[1]
        if found is None:
            raise ScheduleError("no optimal SRJ scheme found for P=%d, kappa_m=%.6g" % (p, kappa_m))
        hist[p] = found
    return hist if return_all else hist[P]


# ---------------------------------------------------------------------------
# Large grids: extended precision (Sect. 3.3) and continuation in resolution
# ---------------------------------------------------------------------------

MP_DIGITS = 40          # working precision of the extended-precision stage
KAPPA_DIRECT = 1.0e-7   # below this bound the double-precision solver is not used directly


def system_mp(x, P, kappa_m):
    """``system`` evaluated in mpmath at the current working precision.

    Sect. 3.3 reports that the optimal schemes for large P and fine grids could
    only be computed with extended precision (up to 24 digits); the weights then
    span 1/kappa_m ~ 1e9, and the equations lose that many digits to
    cancellation.  Same unknowns and equations as ``system``."""
    import mpmath as mp
    w = [mp.exp(x[i]) for i in range(P)]
    inv = [1 / v for v in w]
    kint = [inv[i] + (inv[i + 1] - inv[i]) / (1 + mp.exp(-x[P + i])) for i in range(P - 1)]
    beta = []
    for i in range(P):
        v = mp.mpf(1)
        for kk in kint:
            v *= 1 - kk * w[i]
        for l in range(P):
            if l != i:
                v *= w[l] / (w[l] - w[i])
        beta.append(v)
    kap = [mp.mpf(kappa_m)] + kint + [mp.mpf(KAPPA_MAX)]
    a = [[mp.log(abs(1 - w[i] * kap[j])) for j in range(P + 1)] for i in range(P)]
    F = [mp.fsum(beta[i] * a[i][j] for i in range(P)) for j in range(P + 1)]
    eq_max = [F[j] - F[0] for j in range(1, P + 1)]
    Mm = mp.matrix(P + 1, P + 1)
    for i in range(P):
        for j in range(P + 1):
            Mm[i, j] = kap[j] / (1 - w[i] * kap[j])
    for j in range(P + 1):
        Mm[P, j] = 1
    rhs = mp.matrix(P + 1, 1)
    rhs[P] = 1
    mu = mp.lu_solve(Mm, rhs)
    eq_opt = [mp.fsum(mu[j] * (a[i][j] - a[P - 1][j]) for j in range(P + 1)) for i in range(P - 1)]
    return eq_max + eq_opt


def newton_mp(x0, P, kappa_m, tol=1e-28, maxit=25):
    """Newton's method on ``system_mp`` from x0 (central-difference Jacobian,
    step halving until the residual norm decreases).  Returns the solution as
    an mpmath vector, or None."""
    import mpmath as mp
    with mp.workdps(MP_DIGITS):
        x = [mp.mpf(v) for v in x0]
        n = len(x)
        R = system_mp(x, P, kappa_m)
        nr = mp.norm(mp.matrix(R))
        for _ in range(maxit):
            if nr < tol:
                break
            J = mp.matrix(n, n)
            for c in range(n):
                h = mp.mpf(10) ** -15 * max(1, abs(x[c]))
                xp = list(x); xp[c] += h
                xm = list(x); xm[c] -= h
                Rp, Rm = system_mp(xp, P, kappa_m), system_mp(xm, P, kappa_m)
                for r in range(n):
                    J[r, c] = (Rp[r] - Rm[r]) / (2 * h)
            try:
                d = mp.lu_solve(J, mp.matrix(R))
            except ZeroDivisionError:
                return None
            alpha, moved = mp.mpf(1), False
            for _ in range(12):
                xn = [x[i] - alpha * d[i] for i in range(n)]
                Rn = system_mp(xn, P, kappa_m)
                nn = mp.norm(mp.matrix(Rn))
                if nn < nr:
                    x, R, nr, moved = xn, Rn, nn, True
                    break
                alpha /= 2
            if not moved:
                break
        return x if nr < tol else None


def _accept_mp(x, P):
    import mpmath as mp
    with mp.workdps(MP_DIGITS):
        w = [mp.exp(x[i]) for i in range(P)]
        inv = [1 / v for v in w]
        kint = [inv[i] + (inv[i + 1] - inv[i]) / (1 + mp.exp(-x[P + i])) for i in range(P - 1)]
        omega = np.array([float(v) for v in w])
        if not np.all(np.diff(omega) < 0) or omega[-1] <= 0.5:
            return None
        beta = []
        for i in range(P):
            v = mp.mpf(1)
            for kk in kint:
                v *= 1 - kk * w[i]
            for l in range(P):
                if l != i:
                    v *= w[l] / (w[l] - w[i])
            beta.append(v)
        beta = np.array([float(v) for v in beta])
        if not np.all(beta > 0) or abs(beta.sum() - 1.0) > 1e-12:
            return None
        return omega, beta, np.array([float(v) for v in kint])


def follow_resolution(P, kappa_from, sol_from, kappa_to):
    """Follow the optimal P-level scheme from spectral bound kappa_from down to
    kappa_to (a finer grid) in steps of kappa / 2: at each step the unknowns are
    predicted by linear extrapolation in log kappa from the two previous
    solutions and corrected by ``newton_mp``.  The paper computes its tables at
    a sequence of increasing resolutions (Sect. 4.2); this is that sequence
    with the previous resolution's solution as the starting point.  Returns
    (omega, beta, kappa_int) or raises ScheduleError."""
    import mpmath as mp
    omega, _, kint = sol_from
    with mp.workdps(MP_DIGITS):
        x_cur = [mp.mpf(v) for v in _pack(omega, kint)]
        x_prev, k_prev, k_cur = None, None, kappa_from
        ratio = 0.5
        found = None
        while k_cur > kappa_to:
            k_next = max(kappa_to, k_cur * ratio)
            if x_prev is None:
                guess = x_cur
            else:
                a = mp.log(mp.mpf(k_next) / k_cur) / mp.log(mp.mpf(k_cur) / k_prev)
                guess = [x_cur[i] + (x_cur[i] - x_prev[i]) * a for i in range(len(x_cur))]
            x = newton_mp(guess, P, k_next)
            sol = None if x is None else _accept_mp(x, P)
            if sol is None:
                ratio = math.sqrt(ratio)
                if ratio > 0.97:
                    raise ScheduleError("optimal P=%d scheme lost at kappa_m=%.6g" % (P, k_next))
                continue
            x_prev, x_cur, k_prev, k_cur, found = x_cur, x, k_cur, k_next, sol
            ratio = 0.5
    return found


def solve_optimal_fine(P, kappa_m):
    """``solve_optimal`` for any kappa_m: directly when kappa_m >= KAPPA_DIRECT,
    else solved at KAPPA_DIRECT and followed to kappa_m by
    ``follow_resolution`` in extended precision."""
    if kappa_m >= KAPPA_DIRECT:
        return solve_optimal(P, kappa_m)
    return follow_resolution(P, KAPPA_DIRECT, solve_optimal(P, KAPPA_DIRECT), kappa_m)


def polish(P, kappa_m, omega):
    """Newton on S(omega, kappa) from given weights (e.g. a printed table row)."""
    omega = np.asarray(omega, dtype=np.float64)
    kint = np.array([1.0 / omega[i] + (1.0 / omega[i + 1] - 1.0 / omega[i]) / 3.0 for i in range(P - 1)])
    return _newton(P, kappa_m, _pack(omega, kint))


# ---------------------------------------------------------------------------
# Integer repetitions and validation (Sect. 4.3)
# ---------------------------------------------------------------------------

def q_floor(beta):
    """q_i = floor(beta_i / beta_1), so q_1 = 1 (Sect. 4.3)."""
    beta = np.asarray(beta, dtype=np.float64)
    return np.floor(beta / beta[0]).astype(np.int64)


def max_cycle_factor(omega, q, kappa_m, kappa_max=KAPPA_MAX, samples=20001):
    """max over [kappa_m, kappa_max] of log10 |cycle amplification| with integer q.

    Sect. 4.3: Gamma must stay below 1 after the integer conversion, otherwise
    SRJ diverges.  Sampled on a geometric grid plus the interior maxima of the
    integer scheme."""
    omega = np.asarray(omega, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    grid = np.geomspace(kappa_m, kappa_max, samples)
    beta = q / q.sum()
    extra = [k for k in interior_maxima(omega, beta) if kappa_m <= k <= kappa_max]
    kap = np.concatenate([grid, extra])
    return float(np.max(log10_cycle_factor(kap, omega, q)))


# ---------------------------------------------------------------------------
# Cycle ordering
# ---------------------------------------------------------------------------

def _order_drift_once(omega, q, kappa_m, kappa_max, samples):
    """Order of the M weight applications inside one cycle.

    One greedy pass on one sampling grid (see ``order_drift``).  In
    floating point what matters is how far the partial products of the
    amplification factors stray inside the cycle: a rounding error made at one
    step is multiplied by the product of the factors that follow it.  This
    ordering keeps, for every sampled kappa, the running log-product close to
    the straight line from 0 to the full-cycle value: at step s (1-based) it
    applies the weight, among those with repetitions left, that minimises
      max_kappa | sum_{steps <= s} log|1-omega kappa| - (s/M) sum_i q_i log|1-omega_i kappa| |,
    ties going to the lower level index.  kappa is sampled on a geometric grid
    of `samples` points over [kappa_m, kappa_max].  Returns level indices
    (0-based) of length M.
    """
    omega = np.asarray(omega, dtype=np.float64)
    q = [int(v) for v in q]
    P = len(q)
    M = sum(q)
    kap = np.geomspace(kappa_m, kappa_max, samples)
    L = np.log(np.abs(1.0 - np.outer(omega, kap)))          # P x K
    total = (np.asarray(q, float)[:, None] * L).sum(axis=0)
    cur = np.zeros(len(kap))
    left = list(q)
    order = np.empty(M, dtype=np.int64)
    for s in range(M):
        target = total * ((s + 1) / M)
        best_i, best_c = -1, math.inf
        for i in range(P):
            if left[i] == 0:
                continue
            c = float(np.max(np.abs(cur + L[i] - target)))
            if c < best_c:
                best_i, best_c = i, c
        order[s] = best_i
        left[best_i] -= 1
        cur += L[best_i]
    return order


DRIFT_GRIDS = (1000, 2000, 3000, 4000)
TAIL_STEPS = 4


def order_drift(omega, q, kappa_m, kappa_max=KAPPA_MAX, grids=DRIFT_GRIDS, tail=TAIL_STEPS):
    """Order of the M weight applications inside one cycle.

    Sect. 5.1 notes that the largest over-relaxations must be spread over the
    cycle (an even distribution avoids overflow) but gives no algorithm.  In
    floating point what matters is how far the partial products of the
    amplification factors stray inside the cycle: a rounding error made at one
    step is multiplied by the product of the factors that follow it.  The
    greedy pass (``_order_drift_once``) keeps, for every sampled kappa, the
    running log-product close to the straight line from 0 to the full-cycle
    value.  The greedy is sensitive to the sampling grid (on some schedules one
    grid leaves a cluster of large weights late in the cycle), so the pass is
    run on geometric grids of each size in `grids` and the order with the
    smallest worst-window growth (then suffix growth) on a 4001-point grid is
    kept.  The last min(tail, q_P) steps of the cycle use the smallest weight
    omega_P: rounding errors made late in the cycle are amplified most at
    kappa ~ 2, which omega_P damps by |1 - 2 omega_P| per step; the greedy
    orders the other steps.  Returns level indices (0-based) of length M.
    """
    q = [int(v) for v in q]
    P = len(q)
    k = min(int(tail), q[-1]) if P > 1 else 0
    body_q = list(q)
    body_q[-1] -= k
    best = None
    if sum(body_q) > 0:
        for n in grids:
            o = _order_drift_once(omega, body_q, kappa_m, kappa_max, n)
            key = window_growth(omega, o, kappa_m, kappa_max, samples=4001)
            if best is None or key < best[0]:
                best = (key, o)
        body = best[1]
    else:
        body = np.empty(0, dtype=np.int64)
    return np.concatenate([body, np.full(k, P - 1, dtype=np.int64)])


def fp32_cycle_noise(omega, order, kappa_m, kappa_max=KAPPA_MAX, samples=1024):
    """Model of the FP32 rounding noise that one cycle leaves in the residual,
    relative to a white initial residual (used to order the cycle for FP32).

    In the eigenbasis of D^-1 A the correction of a cycle that starts at e = 0
    is, after step k, e_k(kappa) = (1 - prod_{j<=k} (1 - w_j kappa)) / kappa per
    unit of residual.  Rounding at step k adds noise of size eps |e_k| spread
    over all modes; the remaining steps multiply it by the suffix product
    S_k(kappa) = prod_{j>k} (1 - w_j kappa) and the operator maps it into the
    residual with a factor kappa.  Returns
        eps * sqrt( sum_k <e_k^2> <kappa^2 S_k(kappa)^2> ),
    <.> the mean over `samples` evenly spaced kappa in [kappa_m, kappa_max],
    eps = 2^-24 (inf if a product overflows)."""
    w = np.asarray(omega, dtype=np.float64)[np.asarray(order)]
    kap = np.linspace(kappa_m, kappa_max, samples)
    M = len(w)
    back = np.empty(M)
    S = np.ones(samples)
    for k in range(M - 1, -1, -1):
        back[k] = np.mean((kap * S) ** 2)
        S = S * (1.0 - w[k] * kap)
        if not np.all(np.isfinite(S)):
            return math.inf
    Pf = np.ones(samples)
    total = 0.0
    for k in range(M):
        Pf = Pf * (1.0 - w[k] * kap)
        total += np.mean(((1.0 - Pf) / kap) ** 2) * back[k]
        if not math.isfinite(total):
            return math.inf
    return 2.0 ** -24 * math.sqrt(total)


def order_fp32(omega, q, kappa_m, kappa_max=KAPPA_MAX, moves=range(0, 26, 2)):
    """Cycle order for FP32 cycles: the drift order (``order_drift``, tail of 4
    steps of omega_P) with the first m copies of omega_P moved from the body to
    the tail, m chosen to minimise ``fp32_cycle_noise``.  Moving small weights
    from the start of the cycle (where the correction is still small) to the end
    damps the noise made late in the cycle; moving too many unbalances the body
    and the noise explodes, so m is backed off while m + 4 would more than double
    the noise.  Every order of the same weights has the same cycle polynomial
    (Sect. 2): only rounding differs."""
    base = order_drift(omega, q, kappa_m, kappa_max)
    P = len(q)
    if P < 2:
        return base
    small = P - 1
    body = [int(v) for v in base[:-min(TAIL_STEPS, int(q[-1]))]] if q[-1] > 0 else [int(v) for v in base]
    pos = [i for i, v in enumerate(body) if v == small]
    tail0 = len(base) - len(body)

    def cand(m):
        drop = set(pos[:m])
        return np.array([v for i, v in enumerate(body) if i not in drop] + [small] * (tail0 + m), dtype=np.int64)

    ms = [m for m in moves if m <= len(pos)]
    noise = {m: fp32_cycle_noise(omega, cand(m), kappa_m, kappa_max) for m in ms}
    best = min(ms, key=lambda m: noise[m])
    while best > 0 and (best + 4) in noise and noise[best + 4] > 2.0 * noise[best]:
        best -= 2
    return cand(best)


def window_growth(omega, order, kappa_m, kappa_max=KAPPA_MAX, samples=2000):
    """Largest growth (log10) of any contiguous run of steps of one cycle,
    max over kappa of max_{a<=b} |prod_{a<j<=b} (1 - omega_j kappa)|, and the
    largest growth of any cycle suffix.  Both measure how much a rounding error
    can be amplified inside a cycle (Sect. 5.1 overflow remark)."""
    omega = np.asarray(omega, dtype=np.float64)
    kap = np.geomspace(kappa_m, kappa_max, samples)
    L = np.log10(np.abs(1.0 - np.outer(omega, kap)))
    pre = np.vstack([np.zeros(len(kap)), np.cumsum(L[np.asarray(order)], axis=0)])
    window = float(np.max(pre - np.minimum.accumulate(pre, axis=0)))
    suffix = float(np.max(pre[-1][None, :] - pre[:-1]))
    return window, suffix
