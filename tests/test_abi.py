"""CPU checks of the C ABI: the library loads, exports every symbol that
include/srj.h declares, and its host-only logic (argument checks, spectral
bound, contraction check, cycle order) behaves as specified."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import oracle
import paper_1511_04292_gb300 as srj
from oracle import schedule as S

HEADER = Path(__file__).resolve().parent.parent / "include" / "srj.h"


def declared_functions():
    text = re.sub(r"/\*.*?\*/", "", HEADER.read_text(), flags=re.S)
    return sorted(set(re.findall(r"\b(srj_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = srj.lib()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(srj._native.SIGNATURES), "binding and header disagree"


def test_kappa_min_matches_oracle():
    for dims in [(128, 128), (585 - 1, 280 - 1), (512, 512, 512), (7, 3, 5)]:
        assert abs(srj.kappa_min(dims) / oracle.kappa_min_dirichlet(dims) - 1) < 1e-14


def test_kappa_range_is_the_spectrum_of_the_jacobi_normalised_operator():
    """kappa_min / kappa_max are the extreme eigenvalues of D^-1 A, computed here
    from the dense 5-point (7-point) Dirichlet matrix of small grids."""
    for dims in [(7, 5), (1, 9), (4, 3, 6), (1, 1, 1)]:
        n = int(np.prod(dims))
        d = len(dims)
        A = 2 * d * np.eye(n)
        idx = np.arange(n).reshape(dims[::-1])
        for ax in range(d):
            a = np.take(idx, range(idx.shape[ax] - 1), axis=ax).ravel()
            b = np.take(idx, range(1, idx.shape[ax]), axis=ax).ravel()
            A[a, b] = A[b, a] = -1
        ev = np.linalg.eigvalsh(A / (2 * d))
        lo, hi = srj.kappa_range(dims)
        assert abs(lo - ev[0]) < 1e-13 and abs(hi - ev[-1]) < 1e-13, (dims, lo, hi, ev[0], ev[-1])
        assert lo == srj.kappa_min(dims)


def test_neff_reproduces_the_worked_example():
    """Eq. effectiveNDirichlet, Sect. 5.1: 585 x 280 zones give N_eff = 252.56
    (tests/golden/paper_schedules.json, worked example), and for squares and
    cubes of N zones the large-N form of the same equation,
    sqrt(d/2) / sqrt(sum_i 1/N_i^2) = N / sqrt(2)."""
    import json
    ex = json.loads((Path(__file__).parent / "golden" / "paper_schedules.json").read_text())["worked_example"]
    zones = ex["zones"]
    assert round(srj.neff([z - 1 for z in zones]), 2) == ex["n_eff"]
    assert abs(srj.neff((4095, 4095)) / (4096 / np.sqrt(2)) - 1) < 1e-7
    assert abs(srj.neff((99, 99, 99)) / (100 / np.sqrt(2)) - 1) < 1e-4


def _arr(a, t):
    return np.ascontiguousarray(a, dtype=t)


def test_schedule_check_agrees_with_oracle():
    L = srj.lib()
    for n, P in [(128, 5), (4096, 10), (512, 12)]:
        nd = 3 if (n, P) == (512, 12) else 2
        row = srj.schedules.lookup(nd, n, P)
        w, q = _arr(row["omega"], np.float64), _arr(row["q"], np.int32)
        out = ctypes.c_double()
        srj._native.check(L.srj_schedule_check(P, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                               row["kappa_min"], 2.0, ctypes.byref(out)))
        ref = S.max_cycle_factor(row["omega"], row["q"], row["kappa_min"])
        assert out.value < 0 and abs(out.value - ref) < 1e-6 * max(1.0, abs(ref)), (out.value, ref)


def test_plan_rejects_non_contracting_scheme_before_touching_the_gpu():
    w = _arr([100.0, 0.6], np.float64)
    q = _arr([50, 1], np.int32)  # far too many large steps
    h = ctypes.c_void_p()
    d = (ctypes.c_int64 * 2)(64, 64)
    rc = srj.lib().srj_plan_create(ctypes.byref(h), 2, d, 1 / 65, 2,
                                   w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), None, 0)
    assert rc == -2 and not h.value
    assert b"does not contract" in srj.lib().srj_last_error()


@pytest.mark.parametrize("bad", ["ndim", "dims", "dims_max", "points", "h", "P", "omega", "q", "order", "precision"])
def test_plan_argument_checks(bad):
    w = _arr([2.0, 0.7], np.float64)
    q = _arr([1, 3], np.int32)
    order = _arr([1, 0, 1, 1], np.int32)
    args = dict(ndim=2, dims=(ctypes.c_int64 * 2)(8, 8), h=0.1, P=2, omega=w, q=q, order=order, precision=0)
    if bad == "ndim": args["ndim"] = 4
    if bad == "dims": args["dims"] = (ctypes.c_int64 * 2)(0, 8)
    if bad == "dims_max": args["dims"] = (ctypes.c_int64 * 2)(8, 262141)  # dims[1] <= 262140 (launch grid)
    if bad == "points": args["dims"] = (ctypes.c_int64 * 2)(1 << 20, 1 << 17)  # more than 2^36 points
    if bad == "h": args["h"] = -1.0
    if bad == "P": args["P"] = 0
    if bad == "omega": args["omega"] = _arr([2.0, float("nan")], np.float64)
    if bad == "q": args["q"] = _arr([1, 0], np.int32)
    if bad == "order": args["order"] = _arr([1, 1, 1, 1], np.int32)
    if bad == "precision": args["precision"] = 7
    h = ctypes.c_void_p()
    rc = srj.lib().srj_plan_create(ctypes.byref(h), args["ndim"], args["dims"], args["h"], args["P"],
                                   args["omega"].ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   args["q"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   args["order"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   args["precision"])
    assert rc == -1, (bad, rc)


@pytest.mark.parametrize("n,P", [(128, 5), (4096, 10)])
def test_library_order_keeps_fp32_rounding_low(n, P):
    """The plan's own cycle order (used when none is given) is a valid cycle; its
    modelled FP32 cycle noise is at most that of the plain drift order and below
    the limit mixed plans accept (the oracle's order_fp32 follows the same rule
    in an independent implementation)."""
    row = srj.schedules.lookup(2, n, P)
    w, q = _arr(row["omega"], np.float64), _arr(row["q"], np.int32)
    out = np.empty(int(q.sum()), dtype=np.int32)
    srj._native.check(srj.lib().srj_schedule_order(P, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                   q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                   row["kappa_min"], out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
    assert np.bincount(out, minlength=P).tolist() == q.tolist()
    km = row["kappa_min"]
    nz = S.fp32_cycle_noise(row["omega"], out, km)
    assert nz <= S.fp32_cycle_noise(row["omega"], S.order_drift(row["omega"], row["q"], km), km) * (1 + 1e-9)
    assert nz < 0.05
    assert nz <= S.fp32_cycle_noise(row["omega"], S.order_fp32(row["omega"], row["q"], km), km) * 1.05


def test_packaged_schedules_contract_and_match_their_order():
    """Every packaged row: integer scheme contracts (Sect. 4.3) and its order
    string lists each level exactly q_i times."""
    for nd, n, P in srj.schedules.available():
        row = srj.schedules.lookup(nd, n, P)
        assert row["log10_cycle_factor_max"] < 0
        assert np.bincount(row["order"], minlength=P).tolist() == row["q"].tolist()
        assert abs(row["kappa_min"] - oracle.kappa_min_dirichlet([n] * nd)) < 1e-15


@pytest.mark.parametrize("bad", ["empty", "dims", "dims_max", "h", "P", "omega", "q", "order", "depth", "contraction"])
def test_batch_argument_checks_before_touching_the_gpu(bad):
    """srj_batch_create validates every problem before its first CUDA call:
    bad arguments give SRJ_ERR_INVALID_ARG, a scheme that does not contract on
    its grid SRJ_ERR_BAD_SCHEDULE (no GPU is needed to see either)."""
    ok = dict(dims=(40, 30), h=1 / 41, omega=[2.0, 0.7], q=[1, 3], order=[1, 0, 1, 1])
    probs = [dict(ok), dict(ok, dims=(17, 9))]
    depth = 0
    if bad == "empty": probs = []
    if bad == "dims": probs[1]["dims"] = (0, 9)
    if bad == "dims_max": probs[1]["dims"] = (65537, 9)
    if bad == "h": probs[1]["h"] = float("nan")
    if bad == "P": probs[1]["omega"], probs[1]["q"], probs[1]["order"] = [], [], None
    if bad == "omega": probs[1]["omega"] = [2.0, -0.7]
    if bad == "q": probs[1]["q"] = [1, 0]
    if bad == "order": probs[1]["order"] = [1, 1, 1, 1]
    if bad == "depth": depth = 9
    if bad == "contraction": probs[1]["omega"], probs[1]["q"], probs[1]["order"] = [100.0, 0.6], [50, 1], None
    with pytest.raises(srj.SRJError) as ei:
        srj.Batch(probs, temporal_depth=depth)
    assert ei.value.status == (-2 if bad == "contraction" else -1), (bad, str(ei.value))


def test_tuner_and_self_test_argument_checks_before_touching_the_gpu():
    """srj_batch_tune_depth and srj_selftest_wait_timeout reject bad arguments
    (NULL arrays, an empty or out-of-range depth range, a wait limit outside
    1 us .. 1 s) with SRJ_ERR_INVALID_ARG before any CUDA call."""
    L = srj.lib()
    probs = [dict(dims=(40, 30), h=1 / 41, omega=[2.0, 0.7], q=[1, 3], order=[1, 0, 1, 1])]
    arr, keep, _ = srj.Batch._problem_array(probs)
    dummy = (ctypes.c_void_p * 1)(ctypes.c_void_p(0))
    T = ctypes.c_int()
    for f, u, lo, hi in [(None, dummy, 2, 8), (dummy, dummy, 5, 4), (dummy, dummy, 0, 8), (dummy, dummy, 2, 9)]:
        rc = L.srj_batch_tune_depth(1, arr, f, u, lo, hi, None, ctypes.byref(T), None)
        assert rc == -1, (lo, hi)
    rc = L.srj_batch_tune_depth(1, arr, dummy, dummy, 2, 8, None, None, None)
    assert rc == -1
    for limit in (0, -5, 1000001):
        assert L.srj_selftest_wait_timeout(limit, None) == -1
