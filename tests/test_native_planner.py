"""CPU tests of the library's native schedule planner (srj_schedule_optimal /
srj_schedule_for_grid), against the paper's printed values and, independently,
against the oracle's solver."""
import json
from pathlib import Path

import numpy as np
import pytest

import oracle
import paper_1511_04292_gb300.schedules as sch
from oracle import schedule as S

GOLDEN = json.loads((Path(__file__).parent / "golden" / "paper_schedules.json").read_text())


def test_worked_example_p10_n550():
    """Sect. 5.1: q = {1,1,3,9,21,49,116,268,587,1014}, M = 2069, omega_1..3, rho = 125.85."""
    ex = GOLDEN["worked_example"]
    w, b, _ = sch.optimal(ex["P"], oracle.kappa_min_neumann(ex["N"]))
    q = np.floor(b / b[0]).astype(int)
    assert q.tolist() == ex["q"] and q.sum() == ex["M"]
    assert np.all(np.abs(w[:3] / np.array(ex["omega_leading"]) - 1) < 5e-6)
    assert round(float(np.dot(w, b)), 2) == ex["rho"]


@pytest.mark.parametrize("P,N", [(2, 100), (3, 300), (5, 500), (14, 1024), (15, 256), (14, 4096), (15, 2048)])
def test_printed_rows(P, N):
    """rho of the printed rows (Table 1, P=14 / P=15 tables) to 1.5e-3 and a level
    max Gamma no higher than the printed row's."""
    row = next(r for r in GOLDEN["rows"] if r["P"] == P and r["N"] == N)
    km = oracle.kappa_min_neumann(N)
    w, b, k = sch.optimal(P, km)
    assert abs(np.dot(w, b) / row["rho"] - 1) <= 1.5e-3
    lv = lambda w_, b_: S.log_gamma(np.concatenate([[km], S.interior_maxima(w_, b_ / b_.sum()), [2.0]]),
                                    w_, b_ / b_.sum()).max()
    assert lv(w, b) <= lv(np.array(row["omega"]), np.array(row["beta"])) + 1e-9
    # the returned interior maxima are the stationary points of Gamma (Eq. partialG)
    np.testing.assert_allclose(k, S.interior_maxima(w, b), rtol=1e-8)


@pytest.mark.parametrize("N,P", [(46, 10), (362.75, 12), (2897, 10), (725, 7)])
def test_agrees_with_oracle_solver(N, P):
    km = oracle.kappa_min_neumann(N)
    w, b, _ = sch.optimal(P, km)
    wo, bo, _ = S.solve_optimal(P, km)
    np.testing.assert_allclose(w, wo, rtol=1e-8)
    np.testing.assert_allclose(b, bo, rtol=1e-7)


@pytest.mark.parametrize("ndim,n,P", [(2, 128, 5), (2, 4096, 10), (3, 512, 12), (2, 1024, 8)])
def test_for_grid_matches_packaged_table(ndim, n, P):
    w, q = sch.for_grid([n] * ndim, P)
    row = sch.lookup(ndim, n, P)
    np.testing.assert_allclose(w, row["omega"], rtol=1e-8)
    assert q.tolist() == row["q"].tolist()


def test_single_level_is_the_equioscillating_weight():
    km = 0.01
    w, b, _ = sch.optimal(1, km)
    assert b[0] == 1.0 and abs(w[0] - 2.0 / (km + 2.0)) < 1e-15


LARGE = json.loads((Path(__file__).parent / "golden" / "large_grid_schedules.json").read_text())


def _large_row(n, P):
    return next(r for r in LARGE["rows"] if r["n"] == n and r["P"] == P)


@pytest.mark.parametrize("n,P", [(8192, 10), (16384, 12), (32768, 14), (32768, 15)])
def test_fine_grids_match_the_oracle(n, P):
    """Sect. 3.3: schemes with up to 15 levels for up to 2^15 points per
    dimension.  The native planner (double-double arithmetic below
    kappa_m ~ 1e-7) gives the oracle's 40-digit schemes: omega to 1e-8, q
    exactly, and the integer scheme contracts on the grid (for_grid checks)."""
    row = _large_row(n, P)
    w, q = sch.for_grid((n, n), P)
    np.testing.assert_allclose(w, row["omega"], rtol=1e-8)
    assert q.tolist() == row["q"]


@pytest.mark.parametrize("n,P", [(r["n"], r["P"]) for r in LARGE["rows"]])
def test_fine_grid_schemes_equioscillate(n, P):
    """Pin of the oracle's fine-grid schemes, independent of how they were
    solved: an optimal P-level scheme has P + 1 equal maxima of Gamma on
    [kappa_m, 2] (Sect. 3, Eq. equMax) -- at kappa_m, at the stationary points
    inside each (1/omega_i, 1/omega_{i+1}) and at 2 -- with beta from Theorem 2,
    and no larger value anywhere on a dense sample of the interval."""
    import mpmath as mpm
    row = _large_row(n, P)
    w, b, km = np.array(row["omega"]), np.array(row["beta"]), row["kappa_min"]
    assert abs(b.sum() - 1) < 1e-12 and np.all(np.diff(w) < 0)
    with mpm.workdps(40):
        W = [mpm.mpf(v) for v in w]
        B = [mpm.mpf(v) for v in b]
        lg = lambda k: mpm.fsum(B[i] * mpm.log(abs(1 - W[i] * k)) for i in range(P))
        dlg = lambda k: mpm.fsum(B[i] * W[i] / (1 - W[i] * k) for i in range(P))
        maxima = [lg(mpm.mpf(km)), lg(mpm.mpf(2))]
        for i in range(P - 1):
            lo, hi = 1 / W[i], 1 / W[i + 1]
            k = mpm.findroot(dlg, (lo + (hi - lo) * mpm.mpf("1e-12"), hi - (hi - lo) * mpm.mpf("1e-12")),
                             solver="anderson")
            assert lo < k < hi
            maxima.append(lg(k))
        top = max(maxima)
        assert float(top - min(maxima)) < 1e-9 * abs(float(top)), [float(m) for m in maxima]
    # nothing above the common level between the maxima (dense geometric sample)
    kap = np.geomspace(km, 2.0, 200001)
    vals = np.log(np.abs(1.0 - np.outer(kap, w))) @ b
    assert vals.max() <= float(top) + 1e-9 * abs(float(top))
    # the integer scheme contracts on the grid (Sect. 4.3)
    assert S.max_cycle_factor(w, row["q"], km) < 0


def test_extended_precision_continuation_agrees_with_the_direct_solve():
    """The oracle's two routes to a scheme agree where both apply: solved
    directly in double precision at kappa_m = 2e-7, and followed there in
    40-digit arithmetic from the solution at kappa_m = 8e-7."""
    P = 8
    direct = S.solve_optimal(P, 2e-7)
    followed = S.follow_resolution(P, 8e-7, S.solve_optimal(P, 8e-7), 2e-7)
    np.testing.assert_allclose(followed[0], direct[0], rtol=1e-9)
    np.testing.assert_allclose(followed[1], direct[1], rtol=1e-8)


@pytest.mark.parametrize("P", [0, -3, 33, 1000])
def test_level_count_outside_the_range_is_rejected_with_a_message(P):
    """P outside 1..32 is an argument error, reported before anything is sized
    by P (a negative P must not reach an allocation)."""
    import ctypes
    import paper_1511_04292_gb300 as srj
    L = srj.lib()
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    om = np.empty(64); be = np.empty(64); q = np.empty(64, dtype=np.int32)
    d = (ctypes.c_int64 * 2)(64, 64)
    rc = L.srj_schedule_for_grid(2, d, P, om.ctypes.data_as(dp), q.ctypes.data_as(ip), None)
    assert rc == -1 and b"P must be in 1..32" in L.srj_last_error()
    rc = L.srj_schedule_optimal(P, 1e-3, om.ctypes.data_as(dp), be.ctypes.data_as(dp), None)
    assert rc == -1 and b"P must be in 1..32" in L.srj_last_error()
