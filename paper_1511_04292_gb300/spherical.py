"""SRJ on the spherical-coordinate operators of Sect. 5.2 (native library; FP64, or
FP32 cycles inside FP64 defect correction).

The Poisson equation in (r, theta[, phi]) multiplied by r^2, on cell-centred
grids over r in [0, 1], theta in [0, pi], phi in [0, 2 pi], with the boundary
prescriptions of Sect. 5.2: Dirichlet data at r = 1 (ghost layer), u_0 = u_1 =
u_2 at r = 0, Neumann mirrors in theta, periodic in phi.  Arrays are padded
float64 CUDA tensors of shape (n_theta + 2, n_r + 2) or (n_phi + 2, n_theta + 2,
n_r + 2); r is the fastest axis.  Every step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._native import Stats, check, lib
from . import _dev_ptr, _stream_ptr


def coefficients(dims):
    """(radial[3, n_r+2], polar[3, n_t+2], azim[n_t+2] or None) of the Sect. 5.2
    operator, from the library's host helper."""
    dims = tuple(int(v) for v in dims)
    nr, nt = dims[0], dims[1]
    radial = np.zeros((3, nr + 2))
    polar = np.zeros((3, nt + 2))
    azim = np.zeros(nt + 2) if len(dims) == 3 else None
    d = (ctypes.c_int64 * len(dims))(*dims)
    dp = ctypes.POINTER(ctypes.c_double)
    check(lib().srj_sph_coefficients(len(dims), d, radial.ctypes.data_as(dp), polar.ctypes.data_as(dp),
                                     azim.ctypes.data_as(dp) if azim is not None else None))
    return radial, polar, azim


class SphericalPlan:
    """One spherical grid, its operator coefficients and one SRJ schedule;
    precision "fp64" or "mixed" (FP32 cycles inside FP64 defect correction).
    ``steps`` applies FP64 steps in either precision."""

    def __init__(self, dims, omega, q, order=None, coef=None, precision="fp64"):
        self.dims = tuple(int(v) for v in dims)
        if len(self.dims) not in (2, 3):
            raise ValueError("dims must be (n_r, n_theta) or (n_r, n_theta, n_phi)")
        self.shape = tuple(n + 2 for n in reversed(self.dims))
        radial, polar, azim = coefficients(self.dims) if coef is None else coef
        radial = np.ascontiguousarray(radial, dtype=np.float64)
        polar = np.ascontiguousarray(polar, dtype=np.float64)
        azim = None if azim is None else np.ascontiguousarray(azim, dtype=np.float64)
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.int32)
        ordr = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)
        d = (ctypes.c_int64 * len(self.dims))(*self.dims)
        self._lib = lib()
        self._h = ctypes.c_void_p()
        check(self._lib.srj_sph_plan_create(ctypes.byref(self._h), len(self.dims), d, radial.ctypes.data_as(dp),
                                            polar.ctypes.data_as(dp),
                                            azim.ctypes.data_as(dp) if azim is not None else None, len(omega),
                                            omega.ctypes.data_as(dp), q.ctypes.data_as(ip),
                                            ordr.ctypes.data_as(ip) if ordr is not None else None,
                                            {"fp64": 0, "mixed": 1}[precision]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.srj_sph_plan_destroy(h)
            self._h = None

    def solve(self, b, u, tol, max_cycles, stream=None, check_status=True):
        """SRJ cycles until ||L u - b||_2 / ||L u0 - b||_2 <= tol; u (in place) gets
        its ghost layer and row i = 1 from the prescriptions.  Returns the stats."""
        st = Stats()
        rc = self._lib.srj_sph_solve(self._h, _dev_ptr(b, self.shape, "b"), _dev_ptr(u, self.shape, "u", True),
                                     float(tol), int(max_cycles), _stream_ptr(stream), ctypes.byref(st))
        out = st.as_dict()
        out["status"] = rc
        if check_status:
            check(rc)
        return out

    def steps(self, b, u, first=0, count=1, stream=None):
        check(self._lib.srj_sph_steps(self._h, _dev_ptr(b, self.shape, "b"), _dev_ptr(u, self.shape, "u", True),
                                      int(first), int(count), _stream_ptr(stream)))
        return u

    def residual(self, b, u, r_out=None, stream=None):
        l2 = ctypes.c_double(); linf = ctypes.c_double()
        rp = None if r_out is None else _dev_ptr(r_out, self.shape, "r_out", True)
        check(self._lib.srj_sph_residual(self._h, _dev_ptr(b, self.shape, "b"), _dev_ptr(u, self.shape, "u"), rp,
                                         ctypes.byref(l2), ctypes.byref(linf), _stream_ptr(stream)))
        return l2.value, linf.value

    def set_temporal_depth(self, T):
        """FP32 steps per blocked launch (mixed 2-D plans: 1..8)."""
        check(self._lib.srj_sph_plan_set_temporal_depth(self._h, int(T)))

    def temporal_depth(self):
        out = ctypes.c_int()
        check(self._lib.srj_sph_plan_temporal_depth(self._h, ctypes.byref(out)))
        return out.value

    def finalize(self, u, stream=None):
        check(self._lib.srj_sph_finalize(self._h, _dev_ptr(u, self.shape, "u", True), _stream_ptr(stream)))
        return u
