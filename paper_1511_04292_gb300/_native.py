"""Build and load the native SRJ library (libsrj.so, sm_103a).

The library is compiled in-tree with nvcc into ``_build/`` next to this file.
There is no fallback: if the library cannot be built or loaded, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

_PKG = Path(__file__).resolve().parent
_ROOT = _PKG.parent
_CSRC = _PKG / "csrc"
_BUILD = _PKG / "_build"
LIB_PATH = _BUILD / "libsrj.so"
SOURCES = ["srj_kernels.cu", "srj_tblock.cu", "srj_tblock3.cu", "srj_sph.cu", "srj_plan.cu", "srj_batch.cu", "srj_schedule.cu", "srj_noalloc.cu"]
HEADERS = ["srj_internal.h"]
# host code whose double-double arithmetic relies on explicit roundings: no
# floating-point contraction, so that x86-64 and aarch64 builds agree bit for bit
NO_CONTRACT = {"srj_schedule.cu"}
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = Path(cuda) / "bin" / "nvcc"
    return str(cand) if cand.exists() else "nvcc"


def _stale():
    if not LIB_PATH.exists():
        return True
    t = LIB_PATH.stat().st_mtime
    deps = [_CSRC / s for s in SOURCES + HEADERS] + [_ROOT / "include" / "srj.h"]
    return any(d.stat().st_mtime > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> Path:
    """Compile every translation unit in parallel, then link libsrj.so."""
    if not force and not _stale():
        return LIB_PATH
    _BUILD.mkdir(exist_ok=True)
    common = [_nvcc(), "-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "-I", str(_ROOT / "include")]
    procs = []
    objs = []
    for s in SOURCES:
        obj = _BUILD / (s + ".o")
        objs.append(obj)
        cmd = common + ["-c", str(_CSRC / s), "-o", str(obj)]
        if s in NO_CONTRACT:
            cmd += ["-Xcompiler", "-ffp-contract=off"]
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("nvcc failed: %s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
    tmp = LIB_PATH.with_suffix(".so.tmp%d" % os.getpid())
    link = [_nvcc(), ARCH, "-shared", "-o", str(tmp)] + [str(o) for o in objs]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(link), r.stdout.decode(errors="replace")))
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class SRJError(RuntimeError):
    """A non-zero status from the native library."""

    def __init__(self, status, message):
        super().__init__("SRJ status %d: %s" % (status, message))
        self.status = status


STATUS = {0: "SRJ_OK", -1: "SRJ_ERR_INVALID_ARG", -2: "SRJ_ERR_BAD_SCHEDULE", -3: "SRJ_ERR_NOT_CONVERGED",
          -4: "SRJ_ERR_DIVERGED", -5: "SRJ_ERR_TIMEOUT", -6: "SRJ_ERR_CUDA", -7: "SRJ_ERR_NO_MEMORY"}


class Stats(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int64), ("sweeps", ctypes.c_int64), ("residual_checks", ctypes.c_int64),
                ("r0_l2", ctypes.c_double), ("res_l2", ctypes.c_double), ("res_linf", ctypes.c_double),
                ("rel_res", ctypes.c_double), ("sweep_ms", ctypes.c_double), ("stagnated", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("res_floor", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("h", ctypes.c_double), ("P", ctypes.c_int32),
                ("omega", ctypes.POINTER(ctypes.c_double)), ("q", ctypes.POINTER(ctypes.c_int32)),
                ("order", ctypes.POINTER(ctypes.c_int32))]


# name -> (restype, argtypes)
_VP, _I, _I64, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)
_I32P = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "srj_plan_create": (_I, [ctypes.POINTER(_VP), _I, _I64P, _D, _I, _DP, _I32P, _I32P, _I]),
    "srj_plan_destroy": (_I, [_VP]),
    "srj_plan_info": (_I, [_VP, _I64P, _DP, _DP]),
    "srj_plan_order": (_I, [_VP, _I32P]),
    "srj_plan_set_temporal_depth": (_I, [_VP, _I]),
    "srj_plan_temporal_depth": (_I, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "srj_plan_set_sweep_variant": (_I, [_VP, _I]),
    "srj_plan_set_operator": (_I, [_VP, _D, _VP, _VP]),
    "srj_plan_sweep_variant": (_I, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "srj_plan_autotune": (_I, [_VP, _VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]),
    "srj_solve": (_I, [_VP, _VP, _VP, _D, _I64, _VP, ctypes.POINTER(Stats)]),
    "srj_solve_host": (_I, [_VP, _VP, _VP, _D, _I64, _VP, ctypes.POINTER(Stats)]),
    "srj_steps": (_I, [_VP, _VP, _VP, _I64, _I64, _VP]),
    "srj_residual": (_I, [_VP, _VP, _VP, _VP, _DP, _DP, _VP]),
    "srj_boundary_adjoint": (_I, [_VP, _VP, _VP, _VP]),
    "srj_gradient": (_I, [_VP, _VP, _VP, _VP, _VP, _D, _I64, _VP, ctypes.POINTER(Stats)]),
    "srj_kappa_min": (_I, [_I, _I64P, _DP]),
    "srj_kappa_range": (_I, [_I, _I64P, _DP, _DP]),
    "srj_neff": (_I, [_I, _I64P, _DP]),
    "srj_schedule_check": (_I, [_I, _DP, _I32P, _D, _D, _DP]),
    "srj_schedule_order": (_I, [_I, _DP, _I32P, _D, _I32P]),
    "srj_schedule_optimal": (_I, [_I, _D, _DP, _DP, _DP]),
    "srj_schedule_for_grid": (_I, [_I, _I64P, _I, _DP, _I32P, _I64P]),
    "srj_steps_f32_noalloc": (_I, [_I, _I64P, _D, _I64, _DP, _VP, _VP, _VP]),
    "srj_noalloc_last_error": (ctypes.c_char_p, []),
    "srj_batch_create": (_I, [ctypes.POINTER(_VP), _I, ctypes.POINTER(BatchProblem), _I]),
    "srj_batch_destroy": (_I, [_VP]),
    "srj_batch_info": (_I, [_VP, _I64P, _I64P, ctypes.POINTER(ctypes.c_int), _I64P]),
    "srj_batch_solve": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _D, _I64, _VP,
                             ctypes.POINTER(Stats), _DP]),
    "srj_batch_last_error": (ctypes.c_char_p, []),
    "srj_batch_tune_depth": (_I, [_I, ctypes.POINTER(BatchProblem), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _I, _I,
                                  _VP, ctypes.POINTER(ctypes.c_int), _DP]),
    "srj_sph_coefficients": (_I, [_I, _I64P, _DP, _DP, _DP]),
    "srj_sph_plan_create": (_I, [ctypes.POINTER(_VP), _I, _I64P, _DP, _DP, _DP, _I, _DP, _I32P, _I32P, _I]),
    "srj_sph_plan_destroy": (_I, [_VP]),
    "srj_sph_steps": (_I, [_VP, _VP, _VP, _I64, _I64, _VP]),
    "srj_sph_residual": (_I, [_VP, _VP, _VP, _VP, _DP, _DP, _VP]),
    "srj_sph_solve": (_I, [_VP, _VP, _VP, _D, _I64, _VP, ctypes.POINTER(Stats)]),
    "srj_sph_finalize": (_I, [_VP, _VP, _VP]),
    "srj_sph_plan_set_temporal_depth": (_I, [_VP, _I]),
    "srj_sph_plan_temporal_depth": (_I, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "srj_selftest_wait_timeout": (_I, [_I64, _VP]),
    "srj_last_error": (ctypes.c_char_p, []),
    "srj_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library (built first if needed).  Raises if it cannot be."""
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(str(path))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status, errfn="srj_last_error"):
    if status != 0:
        msg = getattr(lib(), errfn)().decode(errors="replace")
        raise SRJError(status, "%s: %s" % (STATUS.get(status, "?"), msg))
    return status
