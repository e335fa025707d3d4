"""SRJ oracle: slow, obviously correct FP64 CPU reference (TEST INFRASTRUCTURE).

Adsuara, Cordero-Carrion, Cerda-Duran, Aloy, "Scheduled Relaxation Jacobi
method: improvements and applications" (arXiv:1511.04292).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path of
``paper_1511_04292_gb300``; neither imports the other.

Contents
--------
* ``srj_oracle.c`` (loaded through ctypes): the weighted-Jacobi step
  (Sect. 3.1, Eq. 2nd-order_CD, plus the Poisson source of Sect. 5.1), the
  residual and its norms, and the SRJ cycle loop (Sect. 2).
* this module: grid helpers (spectral bounds, Eqs. boundaries /
  boundaries1D3D / effectiveNDirichlet), the expansion of a schedule into its
  ordered weight sequence, and Python entry points around the C code.
* ``srj_oracle_sph.c``: the same step, residual and cycle loop for the
  spherical-coordinate operators of Sect. 5.2 (r^2-scaled Poisson operator,
  u_0 = u_1 = u_2 at r = 0, Neumann in theta, periodic in phi, Dirichlet at
  r = 1), with the coefficient builder ``spherical_coefficients`` below.
* ``schedule.py``: the optimal-parameter solver (Sect. 3) and the integer
  conversion of Sect. 4.3.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "srj_oracle.c"
_SRC_SPH = _HERE / "srj_oracle_sph.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libsrj_oracle.so"
_lib = None

# Return codes of srj_oracle_solve.
CONVERGED, NOT_CONVERGED, DIVERGED, NO_MEMORY = 0, 1, 2, 3


def build(force: bool = False) -> Path:
    """Compile srj_oracle.c and srj_oracle_sph.c with gcc (no FMA contraction, -O2)."""
    _BUILD.mkdir(exist_ok=True)
    newest = max(_SRC.stat().st_mtime, _SRC_SPH.stat().st_mtime)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < newest:
        tmp = _LIB_PATH.with_suffix(".so.tmp%d" % os.getpid())
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=c11", "-o", str(tmp), str(_SRC), str(_SRC_SPH), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB_PATH))
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.c_void_p
        lib.srj_oracle_sweep.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        lib.srj_oracle_sweep.restype = None
        lib.srj_oracle_residual.argtypes = [ctypes.c_int, i64p, ctypes.c_double, dp, dp, dp,
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.srj_oracle_residual.restype = None
        lib.srj_oracle_steps.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_int64, dp,
                                         ctypes.c_int64, ctypes.c_int64, dp, dp, dp]
        lib.srj_oracle_steps.restype = None
        lib.srj_oracle_solve.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_int64, dp, dp, dp,
                                         ctypes.c_double, ctypes.c_int64, i64p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
        lib.srj_oracle_solve.restype = ctypes.c_int
        lib.srj_oracle_sweep_op.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                            dp, dp, dp, dp]
        lib.srj_oracle_sweep_op.restype = None
        lib.srj_oracle_residual_op.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp,
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.srj_oracle_residual_op.restype = None
        lib.srj_oracle_solve_op.argtypes = [ctypes.c_int, i64p, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int64,
                                            dp, dp, dp, ctypes.c_double, ctypes.c_int64, i64p,
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.srj_oracle_solve_op.restype = ctypes.c_int
        lib.srj_oracle_sph_sweep.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.c_double, dp, dp, dp]
        lib.srj_oracle_sph_sweep.restype = None
        lib.srj_oracle_sph_residual.argtypes = [ctypes.c_int, i64p, dp, dp, dp, dp, dp, dp,
                                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.srj_oracle_sph_residual.restype = None
        lib.srj_oracle_sph_finalize.argtypes = [ctypes.c_int, i64p, dp]
        lib.srj_oracle_sph_finalize.restype = None
        lib.srj_oracle_sph_solve.argtypes = [ctypes.c_int, i64p, dp, dp, dp, ctypes.c_int64, dp, dp, dp,
                                             ctypes.c_double, ctypes.c_int64, i64p,
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        lib.srj_oracle_sph_solve.restype = ctypes.c_int
        _lib = lib
    return _lib


# ---------------------------------------------------------------------------
# Grid helpers
# ---------------------------------------------------------------------------

def padded_shape(dims):
    """Padded array shape (slowest first) for interior sizes dims = (nx, ny[, nz])."""
    return tuple(int(n) + 2 for n in reversed(dims))


def _dims3(dims):
    d = [int(v) for v in dims] + [1] * (3 - len(dims))
    return (ctypes.c_int64 * 3)(*d)


def _check(arr, dims, name):
    if arr.dtype != np.float64 or not arr.flags.c_contiguous or arr.shape != padded_shape(dims):
        raise ValueError("%s must be a C-contiguous float64 array of shape %s" % (name, padded_shape(dims)))


def kappa_min_dirichlet(dims):
    """Smallest eigenvalue of the Jacobi-normalised Dirichlet operator D^-1 A.

    Sect. 5.1 gives kappa_m = sin^2(pi/2Nx) + sin^2(pi/2Ny) in 2-D; the d-dim
    normalisation of Eq. boundaries1D3D multiplies the sum by 2/d so that the
    largest eigenvalue stays below 2.  N_i counts zones, N_i = n_i + 1 for n_i
    interior points.
    """
    d = len(dims)
    return (2.0 / d) * sum(math.sin(math.pi / (2.0 * (n + 1))) ** 2 for n in dims)


KAPPA_MAX = 2.0  # Eq. boundaries: kappa_M = 2 for every d and boundary type.


def neff_dirichlet(zones):
    """Effective 2-D Neumann resolution of a Dirichlet grid, Eq. effectiveNDirichlet.

    ``zones`` are the numbers of zones N_i per dimension.
    """
    d = len(zones)
    s = (2.0 / d) * sum(math.sin(math.pi / (2.0 * N)) ** 2 for N in zones)
    return math.pi / (2.0 * math.asin(math.sqrt(s)))


def kappa_min_neumann(N):
    """Eq. boundaries: kappa_m = sin^2(pi / 2N) (2-D Neumann model problem)."""
    return math.sin(math.pi / (2.0 * N)) ** 2


def omega_sequence(omega, order):
    """Ordered weight sequence of one M-cycle: seq[k] = omega[order[k]] (Sect. 2)."""
    omega = np.asarray(omega, dtype=np.float64)
    return np.ascontiguousarray(omega[np.asarray(order, dtype=np.int64)])


# ---------------------------------------------------------------------------
# Entry points around the C oracle
# ---------------------------------------------------------------------------

def sweep(dims, h, omega, f, u):
    """One weighted-Jacobi step; returns the new padded array."""
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    out = np.empty_like(u)
    lib.srj_oracle_sweep(len(dims), _dims3(dims), float(h), float(omega),
                         f.ctypes.data, u.ctypes.data, out.ctypes.data)
    return out


def residual(dims, h, f, u, want_r=False):
    """r = b - A_h u; returns (l2, linf[, r])."""
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    r = np.empty_like(u) if want_r else None
    l2 = ctypes.c_double(); linf = ctypes.c_double()
    lib.srj_oracle_residual(len(dims), _dims3(dims), float(h), f.ctypes.data, u.ctypes.data,
                            r.ctypes.data if want_r else None, ctypes.byref(l2), ctypes.byref(linf))
    return (l2.value, linf.value, r) if want_r else (l2.value, linf.value)


def steps(dims, h, seq, f, u, first=0, count=None):
    """Apply `count` steps of the ordered sequence from position `first`; in place."""
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    seq = np.ascontiguousarray(seq, dtype=np.float64)
    count = len(seq) if count is None else int(count)
    work = np.empty_like(u)
    lib.srj_oracle_steps(len(dims), _dims3(dims), float(h), len(seq), seq.ctypes.data,
                         int(first), count, f.ctypes.data, u.ctypes.data, work.ctypes.data)
    return u


def solve(dims, h, seq, f, u, tol, max_cycles):
    """SRJ cycles until ||r||_2 / ||r_0||_2 <= tol; u is updated in place.

    Returns a dict with status, cycles, sweeps, r0, rel, linf.
    """
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    seq = np.ascontiguousarray(seq, dtype=np.float64)
    cyc = ctypes.c_int64(); r0 = ctypes.c_double(); rel = ctypes.c_double(); linf = ctypes.c_double()
    st = lib.srj_oracle_solve(len(dims), _dims3(dims), float(h), len(seq), seq.ctypes.data,
                              f.ctypes.data, u.ctypes.data, float(tol), int(max_cycles),
                              ctypes.byref(cyc), ctypes.byref(r0), ctypes.byref(rel), ctypes.byref(linf))
    return dict(status=st, cycles=cyc.value, sweeps=cyc.value * len(seq), r0=r0.value,
                rel=rel.value, linf=linf.value)


# ---------------------------------------------------------------------------
# Masked / diagonally shifted operator (Sect. 5.3 test B setting)
# ---------------------------------------------------------------------------

def _mask_ptr(mask, dims):
    if mask is None:
        return None
    if mask.dtype != np.uint8 or not mask.flags.c_contiguous or mask.shape != padded_shape(dims):
        raise ValueError("mask must be a C-contiguous uint8 array of shape %s" % (padded_shape(dims),))
    return mask.ctypes.data


def sweep_op(dims, h, omega, sigma, mask, f, u):
    """One step with A = (2d + sigma) I - neighbours on the active points of mask."""
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    out = np.empty_like(u)
    lib.srj_oracle_sweep_op(len(dims), _dims3(dims), float(h), float(omega), float(sigma), _mask_ptr(mask, dims),
                            f.ctypes.data, u.ctypes.data, out.ctypes.data)
    return out


def residual_op(dims, h, sigma, mask, f, u, want_r=False):
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    r = np.empty_like(u) if want_r else None
    l2 = ctypes.c_double(); linf = ctypes.c_double()
    lib.srj_oracle_residual_op(len(dims), _dims3(dims), float(h), float(sigma), _mask_ptr(mask, dims), f.ctypes.data,
                               u.ctypes.data, r.ctypes.data if want_r else None, ctypes.byref(l2), ctypes.byref(linf))
    return (l2.value, linf.value, r) if want_r else (l2.value, linf.value)


def solve_op(dims, h, sigma, mask, seq, f, u, tol, max_cycles):
    lib = _load()
    _check(f, dims, "f"); _check(u, dims, "u")
    seq = np.ascontiguousarray(seq, dtype=np.float64)
    cyc = ctypes.c_int64(); r0 = ctypes.c_double(); rel = ctypes.c_double()
    st = lib.srj_oracle_solve_op(len(dims), _dims3(dims), float(h), float(sigma), _mask_ptr(mask, dims), len(seq),
                                 seq.ctypes.data, f.ctypes.data, u.ctypes.data, float(tol), int(max_cycles),
                                 ctypes.byref(cyc), ctypes.byref(r0), ctypes.byref(rel))
    return dict(status=st, cycles=cyc.value, r0=r0.value, rel=rel.value)


def shifted_kappa(kappa, ndim, sigma):
    """Eigenvalue of D^-1 A for the shifted operator, from the unshifted one:
    A = (2d + sigma) I - N, N = 2d (1 - kappa) on a sine mode."""
    return (2 * ndim * kappa + sigma) / (2 * ndim + sigma)


# ---------------------------------------------------------------------------
# Spherical-coordinate operators (Sect. 5.2)
# ---------------------------------------------------------------------------

def spherical_coefficients(dims):
    """Separable coefficients of the r^2-scaled spherical Poisson operator (Sect. 5.2).

    dims = (n_r, n_theta[, n_phi]) cell-centred points on r in [0, 1],
    theta in [0, pi], phi in [0, 2 pi]; r_i = (i - 1/2) dr etc.  Second-order
    central differences of r^2 u_rr + 2 r u_r + u_tt + cot(t) u_t
    [+ u_pp / sin^2 t], i.e. the equation of Sect. 5.2 multiplied by r^2:
      cr_m = r (r - dr) / dr^2,  cr_p = r (r + dr) / dr^2,  cr_0 = 2 r^2 / dr^2,
      ct_m = 1/dt^2 - cot(t)/(2 dt),  ct_p = 1/dt^2 + cot(t)/(2 dt),  ct_0 = 2/dt^2,
      cp   = 1 / (sin^2(t) dp^2).
    The radial neighbour coefficients follow the printed difference equation
    (r_i +- dr); the printed matrix entries, with r_i +- 2 dr, would double the
    first-derivative term.  Returns (radial[3, n_r+2], polar[3, n_t+2],
    azim[n_t+2] or None), padded index order.
    """
    nr, nt = int(dims[0]), int(dims[1])
    dr = 1.0 / nr
    dt = math.pi / nt
    radial = np.zeros((3, nr + 2))
    for i in range(nr + 2):
        r = (i - 0.5) * dr
        radial[0, i] = r * (r - dr) / (dr * dr)
        radial[1, i] = r * (r + dr) / (dr * dr)
        radial[2, i] = 2.0 * r * r / (dr * dr)
    polar = np.zeros((3, nt + 2))
    azim = None
    for j in range(1, nt + 1):
        t = (j - 0.5) * dt
        cot = math.cos(t) / math.sin(t)
        polar[0, j] = 1.0 / (dt * dt) - cot / (2.0 * dt)
        polar[1, j] = 1.0 / (dt * dt) + cot / (2.0 * dt)
        polar[2, j] = 2.0 / (dt * dt)
    if len(dims) == 3:
        dp = 2.0 * math.pi / int(dims[2])
        azim = np.zeros(nt + 2)
        for j in range(1, nt + 1):
            sn = math.sin((j - 0.5) * dt)
            azim[j] = 1.0 / (sn * sn * dp * dp)
    return radial, polar, azim


def _coef_ptrs(dims, radial, polar, azim):
    nr, nt = int(dims[0]), int(dims[1])
    radial = np.ascontiguousarray(radial, dtype=np.float64)
    polar = np.ascontiguousarray(polar, dtype=np.float64)
    if radial.shape != (3, nr + 2) or polar.shape != (3, nt + 2):
        raise ValueError("coefficient arrays must have shapes (3, n_r+2) and (3, n_t+2)")
    if len(dims) == 3:
        azim = np.ascontiguousarray(azim, dtype=np.float64)
        if azim.shape != (nt + 2,):
            raise ValueError("azim must have shape (n_t+2,)")
    keep = (radial, polar, azim)
    return keep, radial.ctypes.data, polar.ctypes.data, (azim.ctypes.data if len(dims) == 3 else None)


def sph_sweep(dims, coef, omega, b, u):
    """One weighted-Jacobi step of the spherical operator (srj_oracle_sph.c); returns the new array."""
    lib = _load()
    _check(b, dims, "b"); _check(u, dims, "u")
    keep, pr, pp, pa = _coef_ptrs(dims, *coef)
    out = u.copy()
    lib.srj_oracle_sph_sweep(len(dims), _dims3(dims), pr, pp, pa, float(omega), b.ctypes.data, u.ctypes.data,
                             out.ctypes.data)
    return out


def sph_residual(dims, coef, b, u, want_r=False):
    lib = _load()
    _check(b, dims, "b"); _check(u, dims, "u")
    keep, pr, pp, pa = _coef_ptrs(dims, *coef)
    r = np.empty_like(u) if want_r else None
    l2 = ctypes.c_double(); linf = ctypes.c_double()
    lib.srj_oracle_sph_residual(len(dims), _dims3(dims), pr, pp, pa, b.ctypes.data, u.ctypes.data,
                                r.ctypes.data if want_r else None, ctypes.byref(l2), ctypes.byref(linf))
    return (l2.value, linf.value, r) if want_r else (l2.value, linf.value)


def sph_finalize(dims, u):
    """Ghost layer and row i = 1 from the boundary prescription, in place."""
    lib = _load()
    _check(u, dims, "u")
    lib.srj_oracle_sph_finalize(len(dims), _dims3(dims), u.ctypes.data)
    return u


def sph_solve(dims, coef, seq, b, u, tol, max_cycles):
    """SRJ cycles of seq on the spherical operator until the relative residual <= tol (u in place)."""
    lib = _load()
    _check(b, dims, "b"); _check(u, dims, "u")
    keep, pr, pp, pa = _coef_ptrs(dims, *coef)
    seq = np.ascontiguousarray(seq, dtype=np.float64)
    cyc = ctypes.c_int64(); r0 = ctypes.c_double(); rel = ctypes.c_double()
    st = lib.srj_oracle_sph_solve(len(dims), _dims3(dims), pr, pp, pa, len(seq), seq.ctypes.data, b.ctypes.data,
                                  u.ctypes.data, float(tol), int(max_cycles), ctypes.byref(cyc), ctypes.byref(r0),
                                  ctypes.byref(rel))
    return dict(status=st, cycles=cyc.value, sweeps=cyc.value * len(seq), r0=r0.value, rel=rel.value)
