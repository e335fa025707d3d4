"""SRJ schedule table (weights, repetitions and cycle order per grid).

``schedules.json`` in this package holds optimal SRJ schedules (Sect. 3 of
Adsuara et al., arXiv:1511.04292) computed at the Dirichlet spectral bound of
n^d grids, with the integer repetitions of Sect. 4.3 and a fixed cycle order.
It is input data, like the paper's printed tables.
"""
from __future__ import annotations

import json
from functools import lru_cache
from pathlib import Path

import numpy as np

_PATH = Path(__file__).resolve().parent / "schedules.json"
_DIGITS = "0123456789abcdefghijklmnopqrstuvwxyz"


@lru_cache(maxsize=1)
def _table():
    return json.loads(_PATH.read_text())["rows"]


def decode_order(s):
    return np.array([_DIGITS.index(c) for c in s], dtype=np.int32)


def available():
    return [(r["ndim"], r["n"], r["P"]) for r in _table()]


def lookup(ndim, n, P):
    """Row for an n^ndim grid with P levels: dict with omega, q (int32), order
    (int32, M level indices), beta, rho, kappa_min, n_eff."""
    for r in _table():
        if r["ndim"] == ndim and r["n"] == n and r["P"] == P:
            out = dict(r)
            out["omega"] = np.asarray(r["omega"], dtype=np.float64)
            out["q"] = np.asarray(r["q"], dtype=np.int32)
            out["order"] = decode_order(r["order"])
            return out
    raise KeyError("no schedule for ndim=%d n=%d P=%d (have %s)" % (ndim, n, P, available()))


def optimal(P, kappa_min):
    """Optimal (omega, beta, kappa_int) from the library's native planner (Sect. 3)."""
    import ctypes
    from ._native import check, lib
    om = np.empty(P); be = np.empty(P); ki = np.empty(max(P - 1, 1))
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().srj_schedule_optimal(int(P), float(kappa_min), om.ctypes.data_as(dp), be.ctypes.data_as(dp),
                                     ki.ctypes.data_as(dp)))
    return om, be, ki[:P - 1]


def for_grid(dims, P):
    """(omega, q) for a Dirichlet grid from the native planner (Sect. 3 + Sect. 4.3)."""
    import ctypes
    from ._native import check, lib
    om = np.empty(P); q = np.empty(P, dtype=np.int32); M = ctypes.c_int64()
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    check(lib().srj_schedule_for_grid(len(dims), d, int(P), om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(M)))
    return om, q
