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
