"""Host side of the spherical-operator plans (no GPU): the library's coefficient
builder against the oracle's, and argument checking of the C ABI."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1511_04292_gb300 import spherical as sp
from paper_1511_04292_gb300._native import lib


@pytest.mark.parametrize("dims", [(16, 12), (7, 5, 9), (1000, 333), (1, 1), (2, 3, 1)])
def test_library_coefficients_match_the_oracle(dims):
    got = sp.coefficients(dims)
    ref = oracle.spherical_coefficients(dims)
    for a, b in zip(got, ref):
        if b is None:
            assert a is None
            continue
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=1e-14 * np.max(np.abs(b)))


def test_coefficient_helper_rejects_bad_arguments():
    d = (ctypes.c_int64 * 2)(0, 4)
    buf = (ctypes.c_double * 64)()
    assert lib().srj_sph_coefficients(2, d, buf, buf, None) == -1
    d3 = (ctypes.c_int64 * 3)(4, 4, 4)
    assert lib().srj_sph_coefficients(3, d3, buf, buf, None) == -1  # azim required in 3-D
    assert lib().srj_sph_coefficients(4, d3, buf, buf, buf) == -1


def _create(dims, omega, q, order, precision):
    radial, polar, azim = sp.coefficients(dims)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.int32)
    order = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
    d = (ctypes.c_int64 * len(dims))(*dims)
    h = ctypes.c_void_p()
    rc = lib().srj_sph_plan_create(ctypes.byref(h), len(dims), d, radial.ctypes.data_as(dp), polar.ctypes.data_as(dp),
                                   None if azim is None else azim.ctypes.data_as(dp), len(omega),
                                   omega.ctypes.data_as(dp), q.ctypes.data_as(ip),
                                   None if order is None else order.ctypes.data_as(ip), precision)
    assert not h.value
    return rc


@pytest.mark.parametrize("bad", ["precision", "P", "weight", "q", "M", "order_range", "order_count", "contraction"])
def test_plan_rejects_bad_schedules_before_touching_the_gpu(bad):
    """srj_sph_plan_create checks its schedule before any CUDA call: bad
    arguments give SRJ_ERR_INVALID_ARG, a scheme that does not contract on
    [1/omega_max, 2) SRJ_ERR_BAD_SCHEDULE."""
    dims = (16, 12)
    omega, q, order, precision = [2.0, 0.7], [1, 3], [1, 0, 1, 1], 0
    if bad == "precision": precision = 7
    if bad == "P": omega, q, order = [0.5], [1], None
    if bad == "weight": omega = [2.0, 0.0]
    if bad == "q": q = [1, 0]
    if bad == "M": omega, q, order = [1.0], [(1 << 20) + 1], None
    if bad == "order_range": order = [1, 0, 2, 1]
    if bad == "order_count": order = [1, 1, 1, 1]
    if bad == "contraction": omega, q, order = [100.0, 0.6], [50, 1], None
    if bad == "P":
        # P = 0 with the arrays of a valid one-level schedule
        radial, polar, _ = sp.coefficients(dims)
        w = np.array([0.5]); qq = np.array([1], dtype=np.int32)
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
        h = ctypes.c_void_p()
        rc = lib().srj_sph_plan_create(ctypes.byref(h), 2, (ctypes.c_int64 * 2)(*dims), radial.ctypes.data_as(dp),
                                       polar.ctypes.data_as(dp), None, 0, w.ctypes.data_as(dp),
                                       qq.ctypes.data_as(ip), None, 0)
    else:
        rc = _create(dims, omega, q, order, precision)
    assert rc == (-2 if bad == "contraction" else -1), (bad, rc, lib().srj_last_error())
