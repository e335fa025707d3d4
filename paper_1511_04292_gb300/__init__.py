"""GB300-native Scheduled Relaxation Jacobi (SRJ) for Dirichlet Poisson problems.

Method: Adsuara, Cordero-Carrion, Cerda-Duran, Aloy, "Scheduled Relaxation
Jacobi method: improvements and applications", arXiv:1511.04292.

This module is a thin binding over the C ABI of ``include/srj.h``
(``libsrj.so``, hand-written CUDA for sm_103a): it only marshals arguments.
PyTorch provides device memory and streams.  Arrays are float64 CUDA tensors in
the padded layout (nz+2, ny+2, nx+2) / (ny+2, nx+2) whose ghost layer carries
the Dirichlet data.  There is no CPU path: without the native library every
call raises.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import schedules
from ._native import SRJError, Stats, build, check, lib

__all__ = ["Plan", "Batch", "SRJError", "build", "lib", "schedules", "kappa_min", "kappa_range", "neff",
           "schedule_check", "PREC_FP64", "PREC_MIXED", "PREC_FP64_FMA"]

PREC_FP64 = 0
PREC_MIXED = 1
PREC_FP64_FMA = 2
_PREC = {"fp64": PREC_FP64, "mixed": PREC_MIXED, "fp64fma": PREC_FP64_FMA,
         PREC_FP64: PREC_FP64, PREC_MIXED: PREC_MIXED, PREC_FP64_FMA: PREC_FP64_FMA}


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, shape, name, writable=False):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("%s must be a float64 CUDA tensor" % name)
    if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError("%s must be contiguous with shape %s (got %s)" % (name, tuple(shape), tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, shape, name, writable=False):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or (writable and not a.flags.writeable):
            raise TypeError("%s must be a C-contiguous float64 array" % name)
        if tuple(a.shape) != tuple(shape):
            raise ValueError("%s must have shape %s (got %s)" % (name, tuple(shape), tuple(a.shape)))
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if not isinstance(a, torch.Tensor) or a.is_cuda or a.dtype != torch.float64:
        raise TypeError("%s must be a float64 host array (numpy or CPU tensor)" % name)
    if tuple(a.shape) != tuple(shape) or not a.is_contiguous():
        raise ValueError("%s must be contiguous with shape %s (got %s)" % (name, tuple(shape), tuple(a.shape)))
    return ctypes.c_void_p(a.data_ptr())


def kappa_min(dims):
    """Smallest eigenvalue of D^-1 A for a Dirichlet grid (computed by the library)."""
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    out = ctypes.c_double()
    check(lib().srj_kappa_min(len(dims), d, ctypes.byref(out)))
    return out.value


def schedule_check(omega, q, kappa_min, kappa_max=2.0):
    """log10 of the largest cycle amplification |Gamma_cycle| of the integer
    scheme (omega, q) over [kappa_min, kappa_max] (host; < 0 means it contracts)."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    qq = np.ascontiguousarray(q, dtype=np.int32)
    out = ctypes.c_double()
    check(lib().srj_schedule_check(len(om), om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   qq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), float(kappa_min),
                                   float(kappa_max), ctypes.byref(out)))
    return out.value


def kappa_range(dims):
    """(kappa_min, kappa_max): extreme eigenvalues of D^-1 A for a Dirichlet grid."""
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    lo, hi = ctypes.c_double(), ctypes.c_double()
    check(lib().srj_kappa_range(len(dims), d, ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


def neff(dims):
    """Effective Neumann resolution N_eff of a Dirichlet grid (Eq. effectiveNDirichlet)."""
    d = (ctypes.c_int64 * len(dims))(*[int(v) for v in dims])
    out = ctypes.c_double()
    check(lib().srj_neff(len(dims), d, ctypes.byref(out)))
    return out.value


class Plan:
    """An SRJ plan: one grid (dims = (nx, ny[, nz]) interior points, spacing h),
    one schedule (omega_i, q_i[, order]) and one precision: "fp64" (oracle's operation
    order, bit for bit), "fp64fma" (FP64 steps with fused multiply-adds) or "mixed"."""

    def __init__(self, dims, h, omega, q, order=None, precision="fp64"):
        self.dims = tuple(int(v) for v in dims)
        self.ndim = len(self.dims)
        self.h = float(h)
        self.precision = _PREC[precision]
        om = np.ascontiguousarray(omega, dtype=np.float64)
        qq = np.ascontiguousarray(q, dtype=np.int32)
        od = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
        d = (ctypes.c_int64 * self.ndim)(*self.dims)
        handle = ctypes.c_void_p()
        self._lib = lib()
        check(self._lib.srj_plan_create(
            ctypes.byref(handle), self.ndim, d, self.h, len(om),
            om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            qq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            None if od is None else od.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            self.precision))
        self._h = handle
        self.shape = tuple(n + 2 for n in reversed(self.dims))

    @classmethod
    def from_table(cls, dims, P, precision="fp64", h=None):
        """Plan with the packaged schedule for an n^d grid (all dims equal)."""
        n = int(dims[0])
        if any(int(v) != n for v in dims):
            raise ValueError("the packaged table covers n^d grids only")
        row = schedules.lookup(len(dims), n, int(P))
        return cls(dims, 1.0 / (n + 1) if h is None else h, row["omega"], row["q"], row["order"], precision)

    @classmethod
    def auto(cls, dims, P, precision="fp64", h=None):
        """Plan with the optimal P-level schedule for this grid from the library's
        native planner (Sect. 3, floor rule of Sect. 4.3) and its own cycle order."""
        omega, q = schedules.for_grid(dims, P)
        return cls(dims, 1.0 / (max(int(v) for v in dims) + 1) if h is None else h, omega, q, None, precision)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.srj_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        M = ctypes.c_int64(); km = ctypes.c_double(); g = ctypes.c_double()
        check(self._lib.srj_plan_info(self._h, ctypes.byref(M), ctypes.byref(km), ctypes.byref(g)))
        return dict(M=M.value, kappa_min=km.value, log10_cycle_factor_max=g.value)

    def set_temporal_depth(self, T):
        """Steps per blocked FP32 sweep launch (1 = unblocked); 2-D mixed plans only."""
        check(self._lib.srj_plan_set_temporal_depth(self._h, int(T)))

    def temporal_depth(self):
        T = ctypes.c_int()
        check(self._lib.srj_plan_temporal_depth(self._h, ctypes.byref(T)))
        return T.value

    def set_operator(self, sigma=0.0, mask=None, stream=None):
        """A = (2d + sigma) I - neighbours on the active points of mask (uint8 CUDA
        tensor in the padded shape, nonzero = active; None = all interior points)."""
        import torch
        mp = None
        if mask is not None:
            if not isinstance(mask, torch.Tensor) or not mask.is_cuda or mask.dtype != torch.uint8 \
                    or tuple(mask.shape) != self.shape or not mask.is_contiguous():
                raise TypeError("mask must be a contiguous uint8 CUDA tensor of shape %s" % (self.shape,))
            mp = ctypes.c_void_p(mask.data_ptr())
        check(self._lib.srj_plan_set_operator(self._h, float(sigma), mp, _stream_ptr(stream)))

    def set_sweep_variant(self, v):
        """Blocked sweep of 2-D mixed plans: 0 / 2 = one block of 8 / 16 warps per tile;
        1 / 3 = persistent blocks with a bulk-copy prefetch of the next tile;
        4 / 5 = variants 0 / 2 with an L2 prefetch of the next wave's tiles."""
        check(self._lib.srj_plan_set_sweep_variant(self._h, int(v)))

    def sweep_variant(self):
        v = ctypes.c_int()
        check(self._lib.srj_plan_sweep_variant(self._h, ctypes.byref(v)))
        return v.value

    def autotune(self, stream=None):
        """Pick the fastest temporal depth on this plan's grid; returns (T, us per step)."""
        T = ctypes.c_int(); us = ctypes.c_float()
        check(self._lib.srj_plan_autotune(self._h, _stream_ptr(stream), ctypes.byref(T), ctypes.byref(us)))
        return T.value, us.value

    def order(self):
        M = self.info()["M"]
        out = np.empty(M, dtype=np.int32)
        check(self._lib.srj_plan_order(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return out

    def solve(self, f, u, tol, max_cycles, stream=None, raise_on_fail=True):
        """Run SRJ cycles on u (in place) until the relative L2 residual <= tol."""
        st = Stats()
        rc = self._lib.srj_solve(self._h, _dev_ptr(f, self.shape, "f"), _dev_ptr(u, self.shape, "u", True),
                                 float(tol), int(max_cycles), _stream_ptr(stream), ctypes.byref(st))
        out = st.as_dict()
        out["status"] = rc
        if raise_on_fail:
            check(rc)
        return out

    def solve_host(self, f, u, tol, max_cycles, stream=None, raise_on_fail=True):
        """solve() on host arrays (float64, contiguous, padded shape; numpy or CPU
        tensors, pinned for full copy bandwidth): the library copies f and u to
        the device, solves, and copies u back in place."""
        st = Stats()
        rc = self._lib.srj_solve_host(self._h, _host_ptr(f, self.shape, "f"), _host_ptr(u, self.shape, "u", True),
                                      float(tol), int(max_cycles), _stream_ptr(stream), ctypes.byref(st))
        out = st.as_dict()
        out["status"] = rc
        if raise_on_fail:
            check(rc)
        return out

    def steps(self, f, u, first=0, count=1, stream=None):
        """Apply `count` steps of the cycle order from position `first` to u in place."""
        check(self._lib.srj_steps(self._h, _dev_ptr(f, self.shape, "f"), _dev_ptr(u, self.shape, "u", True),
                                  int(first), int(count), _stream_ptr(stream)))
        return u

    def residual(self, f, u, r_out=None, stream=None):
        """(l2, linf) of r = b - A u; fills r_out (padded float64) when given."""
        l2 = ctypes.c_double(); linf = ctypes.c_double()
        rp = None if r_out is None else _dev_ptr(r_out, self.shape, "r_out", True)
        check(self._lib.srj_residual(self._h, _dev_ptr(f, self.shape, "f"), _dev_ptr(u, self.shape, "u"), rp,
                                     ctypes.byref(l2), ctypes.byref(linf), _stream_ptr(stream)))
        return l2.value, linf.value

    def boundary_adjoint(self, lam, grad_g, stream=None):
        """grad_g[ghost] = sum of lam over interior neighbours (dL/dg from dL/db)."""
        check(self._lib.srj_boundary_adjoint(self._h, _dev_ptr(lam, self.shape, "lam"),
                                             _dev_ptr(grad_g, self.shape, "grad_g", True), _stream_ptr(stream)))
        return grad_g


class Batch:
    """Many independent 2-D problems solved together (mixed precision).

    problems: list of dicts with keys dims=(nx, ny), h, omega, q, order (or None).
    """

    @staticmethod
    def _problem_array(problems):
        from ._native import BatchProblem
        keep, shapes = [], []
        arr = (BatchProblem * len(problems))()
        for i, pr in enumerate(problems):
            nx, ny = (int(v) for v in pr["dims"])
            om = np.ascontiguousarray(pr["omega"], dtype=np.float64)
            qq = np.ascontiguousarray(pr["q"], dtype=np.int32)
            od = None if pr.get("order") is None else np.ascontiguousarray(pr["order"], dtype=np.int32)
            keep += [om, qq, od]
            arr[i].nx, arr[i].ny, arr[i].h, arr[i].P = nx, ny, float(pr["h"]), len(om)
            arr[i].omega = om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            arr[i].q = qq.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            arr[i].order = None if od is None else od.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            shapes.append((ny + 2, nx + 2))
        return arr, keep, shapes

    @staticmethod
    def tune_depth(problems, fs, us, tmin=2, tmax=8, stream=None):
        """Temporal depth with the shortest one-cycle batch solve (srj_batch_tune_depth);
        returns (T, ms per cycle).  fs, us are left unchanged."""
        arr, keep, shapes = Batch._problem_array(problems)
        n = len(problems)
        fp = (ctypes.c_void_p * n)(*[_dev_ptr(f, s, "f").value for f, s in zip(fs, shapes)])
        up = (ctypes.c_void_p * n)(*[_dev_ptr(u, s, "u").value for u, s in zip(us, shapes)])
        T = ctypes.c_int(); ms = ctypes.c_double()
        check(lib().srj_batch_tune_depth(n, arr, fp, up, int(tmin), int(tmax), _stream_ptr(stream), ctypes.byref(T),
                                         ctypes.byref(ms)), "srj_batch_last_error")
        return T.value, ms.value

    def __init__(self, problems, temporal_depth=0):
        self._lib = lib()
        arr, self._keep, self.shapes = Batch._problem_array(problems)
        h = ctypes.c_void_p()
        check(self._lib.srj_batch_create(ctypes.byref(h), len(problems), arr, int(temporal_depth)),
              "srj_batch_last_error")
        self._h = h
        self.n = len(problems)

    def info(self):
        pts = ctypes.c_int64(); tiles = ctypes.c_int64(); T = ctypes.c_int(); sm = ctypes.c_int64()
        check(self._lib.srj_batch_info(self._h, ctypes.byref(pts), ctypes.byref(tiles), ctypes.byref(T),
                                       ctypes.byref(sm)), "srj_batch_last_error")
        return dict(points=pts.value, tiles=tiles.value, temporal_depth=T.value, sum_M=sm.value)

    def solve(self, fs, us, tol, max_cycles, stream=None, raise_on_fail=True):
        """fs, us: lists of float64 CUDA tensors (padded layout per problem); us updated in place."""
        if len(fs) != self.n or len(us) != self.n:
            raise ValueError("need one f and one u per problem")
        fp = (ctypes.c_void_p * self.n)(*[_dev_ptr(f, s, "f").value for f, s in zip(fs, self.shapes)])
        up = (ctypes.c_void_p * self.n)(*[_dev_ptr(u, s, "u").value for u, s in zip(us, self.shapes)])
        st = (Stats * self.n)()
        ms = ctypes.c_double()
        rc = self._lib.srj_batch_solve(self._h, fp, up, float(tol), int(max_cycles), _stream_ptr(stream), st,
                                       ctypes.byref(ms))
        if raise_on_fail:
            check(rc, "srj_batch_last_error")
        return [s.as_dict() for s in st], ms.value, rc

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.srj_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
