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


@pytest.mark.parametrize("P,N", [(2, 100), (3, 300), (5, 500), (14, 1024), (15, 256)])
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
