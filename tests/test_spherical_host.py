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
