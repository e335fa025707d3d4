"""Write large_grid_schedules.json: optimal SRJ schemes for fine 2-D Dirichlet
grids (8192^2 .. 32768^2), computed by the oracle only.

Sect. 3.3 of Adsuara et al. (arXiv:1511.04292) gives optimal schemes with up to
P = 15 levels for resolutions up to 2^15 points per dimension; its printed
tables stop at N = 4096 (P = 14) and N = 2048 (P = 15).  For the finer grids
the oracle's solver (``oracle.schedule.solve_optimal_fine``: the direct solve at
kappa_m = 1e-7, followed to each grid's kappa_m in 40-digit arithmetic) supplies
the expected values; the floor rule of Sect. 4.3 gives q.  The tests compare the
library's native planner against these rows and check that every row
equioscillates (the minimax optimality of Sect. 3).

Usage:  python tests/golden/make_large_grid_schedules.py
"""
from __future__ import annotations

import json
import multiprocessing as mp
import sys
import time
from pathlib import Path

HERE = Path(__file__).resolve().parent
sys.path.insert(0, str(HERE.parents[1]))

CASES = [(n, P) for n in (8192, 16384, 32768) for P in (10, 12, 14, 15)]


def one(case):
    import oracle
    from oracle import schedule as S
    n, P = case
    km = oracle.kappa_min_dirichlet((n, n))
    t0 = time.time()
    omega, beta, kint = S.solve_optimal_fine(P, km)
    q = S.q_floor(beta)
    return {"ndim": 2, "n": n, "P": P, "kappa_min": km, "omega": omega.tolist(), "beta": beta.tolist(),
            "kappa_int": kint.tolist(), "q": q.tolist(), "M": int(q.sum()), "seconds": round(time.time() - t0, 1)}


def main():
    with mp.get_context("spawn").Pool(min(len(CASES), 8)) as pool:
        rows = pool.map(one, CASES)
    for r in rows:
        print(r["n"], r["P"], r["M"], r["seconds"], "s")
    out = {"citation": "Optimal SRJ schemes (Sect. 3, floor rule of Sect. 4.3) for n^2 Dirichlet grids, "
                       "kappa_m = 2 sin^2(pi / (2 (n + 1))); written by tests/golden/make_large_grid_schedules.py "
                       "from the oracle's solver (oracle.schedule.solve_optimal_fine).",
           "rows": rows}
    (HERE / "large_grid_schedules.json").write_text(json.dumps(out, indent=1) + "\n")


if __name__ == "__main__":
    main()
