"""Write the SRJ schedule table shipped with the package.

The paper prints optimal parameters only for P = 2..5, 14, 15 (its P = 6..13
tables are not in this copy), and only for Neumann model problems at given N.
The solver in ``oracle/schedule.py`` computes the optimal (omega, beta) of
Sect. 3 directly at the spectral bound kappa_m of each Dirichlet grid (the value
that Eq. effectiveNDirichlet translates into a table row), converts beta to
integer q with the floor rule of Sect. 4.3, checks that the integer scheme
still contracts over [kappa_m, 2], and orders each cycle with
``schedule.order_fp32`` (the drift order with the tail that minimises the
modelled FP32 rounding noise of a cycle).

Usage:  python -m oracle.make_schedules  [output path]
The output is data (weights, repetitions and order); both the CUDA path and the
oracle take it as input.
"""
from __future__ import annotations

import json
import sys
import time
from pathlib import Path

import numpy as np

from oracle import kappa_min_dirichlet, neff_dirichlet
from oracle import schedule as S

# (ndim, interior points per dimension, levels P)
GRIDS = [
    (2, 64, range(5, 11)),
    (2, 128, range(5, 11)),
    (2, 256, range(5, 11)),
    (2, 512, range(5, 11)),
    (2, 1024, range(5, 11)),
    (2, 2048, range(5, 11)),
    (2, 4096, range(5, 13)),
    (3, 128, range(5, 13)),
    (3, 256, range(5, 13)),
    (3, 512, range(5, 13)),
]

DIGITS = "0123456789abcdefghijklmnopqrstuvwxyz"


def encode_order(order):
    """One character per step: the 0-based level index in base 36."""
    return "".join(DIGITS[int(i)] for i in order)


def make_rows(grids=GRIDS, log=print):
    rows = []
    for ndim, n, Ps in grids:
        dims = [n] * ndim
        km = kappa_min_dirichlet(dims)
        t0 = time.time()
        sols = S.solve_optimal(max(Ps), km, return_all=True)
        for P in Ps:
            omega, beta, kint = sols[P]
            q = S.q_floor(beta)
            order = S.order_fp32(omega, q, km)
            gmax = S.max_cycle_factor(omega, q, km)
            window, suffix = S.window_growth(omega, order, km)
            noise = S.fp32_cycle_noise(omega, order, km)
            if not gmax < 0.0:
                raise S.ScheduleError("integer scheme does not contract: P=%d n=%d" % (P, n))
            if not noise < 0.05:
                raise S.ScheduleError("cycle order amplifies FP32 rounding too much: P=%d n=%d" % (P, n))
            rows.append(dict(
                ndim=ndim, n=n, P=P,
                kappa_min=km, n_eff=neff_dirichlet([n + 1] * ndim),
                omega=[float(v) for v in omega], beta=[float(v) for v in beta],
                q=[int(v) for v in q], M=int(q.sum()), rho=S.rho(omega, beta),
                log10_cycle_factor_max=gmax, log10_window_growth=window,
                log10_suffix_growth=suffix, fp32_cycle_noise=noise, order=encode_order(order)))
        log("ndim=%d n=%d P=%s  %.1fs" % (ndim, n, list(Ps), time.time() - t0))
    return rows


def main(argv):
    out = Path(argv[1]) if len(argv) > 1 else (
        Path(__file__).resolve().parent.parent / "paper_1511_04292_gb300" / "schedules.json")
    rows = make_rows()
    doc = dict(
        description=("Optimal SRJ schedules (Adsuara et al., arXiv:1511.04292, Sect. 3) computed at the "
                     "Dirichlet spectral bound kappa_m of n^d grids; q by the floor rule of Sect. 4.3; "
                     "'order' lists the 0-based level index of each step of one M-cycle (base 36)."),
        generator="oracle/make_schedules.py",
        rows=rows)
    out.write_text(json.dumps(doc, indent=1) + "\n")
    print("wrote", out, len(rows), "rows")


if __name__ == "__main__":
    main(sys.argv)
