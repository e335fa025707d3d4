"""Seeded synthetic inputs for the SRJ workloads (shared by tests, bench and oracle).

This module holds input generation only: grids, right-hand sides, boundary data
and initial guesses.  It contains none of the SRJ arithmetic (no sweeps, no
residuals, no schedules), so that the CUDA path and the oracle can both draw
their inputs from it without sharing any of the method.

Grids are uniform on the unit square / cube with n interior points per axis,
spacing h = 1/(n+1) and one ghost layer that holds the Dirichlet data; arrays
are float64 in the padded layout (nz+2, ny+2, nx+2) / (ny+2, nx+2), x fastest.
The problem is -Laplace(u) = f (the paper's Sect. 5.1 example is Laplace(u) =
rhs; only the sign convention differs).
"""
from __future__ import annotations

import math

import numpy as np


def coords(n):
    """Node coordinates x_i = i h, i = 0..n+1 (ghosts at 0 and 1)."""
    return np.arange(n + 2, dtype=np.float64) / (n + 1)


def spacing(n):
    return 1.0 / (n + 1)


def zero_field(dims):
    return np.zeros(tuple(int(v) + 2 for v in reversed(dims)))


# ---------------------------------------------------------------------------
# Workload 1: 2-D manufactured solution, homogeneous Dirichlet
# ---------------------------------------------------------------------------

def manufactured_2d(n):
    """u = sin(pi x) sin(pi y) + 0.1 sin(5 pi x) sin(3 pi y), f = -Laplace(u).

    Returns (f, u_exact, u0) in the padded layout; u0 = 0 (boundary values of u
    are 0)."""
    x = coords(n)
    X, Y = np.meshgrid(x, x, indexing="xy")  # shape (ny+2, nx+2), x fastest
    pi = math.pi
    u = np.sin(pi * X) * np.sin(pi * Y) + 0.1 * np.sin(5 * pi * X) * np.sin(3 * pi * Y)
    f = 2 * pi ** 2 * np.sin(pi * X) * np.sin(pi * Y) + 0.1 * 34 * pi ** 2 * np.sin(5 * pi * X) * np.sin(3 * pi * Y)
    u0 = np.zeros_like(u)
    return np.ascontiguousarray(f), np.ascontiguousarray(u), u0


def exp_xy_2d(nx, ny):
    """Sect. 5.1 example: u = -exp(x y) on the unit square with Dirichlet data from
    u, written for -Laplace(u) = f: f = exp(x y) (x^2 + y^2).  Rectangular grids
    use spacing hx = 1/(nx+1), hy = 1/(ny+1); callers use nx == ny.

    Returns (f, u_exact, u0) with u0 = 0 in the interior and u on the ghosts."""
    x = np.arange(nx + 2) / (nx + 1)
    y = np.arange(ny + 2) / (ny + 1)
    X, Y = np.meshgrid(x, y, indexing="xy")
    u = -np.exp(X * Y)
    f = np.exp(X * Y) * (X ** 2 + Y ** 2)
    u0 = u.copy()
    u0[1:-1, 1:-1] = 0.0
    return f, u, u0


# ---------------------------------------------------------------------------
# Workloads 2, 4, 5: smoothed random fields and polynomial boundary data
# ---------------------------------------------------------------------------

def box_filter_2d(a, width=5):
    """Mean over a width x width window, zero padding outside the array."""
    r = width // 2
    p = np.pad(a, r)
    c = np.cumsum(np.cumsum(p, axis=0), axis=1)
    c = np.pad(c, ((1, 0), (1, 0)))
    n0, n1 = a.shape
    s = c[width:width + n0, width:width + n1] - c[0:n0, width:width + n1] - c[width:width + n0, 0:n1] + c[0:n0, 0:n1]
    return s / (width * width)


def smooth_random_2d(n, seed):
    """f: i.i.d. N(0,1) on the interior, 5x5 box mean; padded layout, ghosts 0."""
    rng = np.random.default_rng(seed)
    f = np.zeros((n + 2, n + 2))
    f[1:-1, 1:-1] = box_filter_2d(rng.standard_normal((n, n)))
    return f


def poly_boundary_2d(n, seed, degree=3):
    """u0: Dirichlet ghosts from a random polynomial sum_{a+b<=degree} c_ab x^a y^b,
    c_ab ~ N(0,1); interior 0."""
    rng = np.random.default_rng(seed)
    x = coords(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    g = np.zeros_like(X)
    for a in range(degree + 1):
        for b in range(degree + 1 - a):
            g += rng.standard_normal() * X ** a * Y ** b
    u0 = g.copy()
    u0[1:-1, 1:-1] = 0.0
    return u0


def random_smooth_problem_2d(n, seed):
    """(f, u0) for the 2-D random smooth workload: seed for f, seed+1 for g."""
    return smooth_random_2d(n, seed), poly_boundary_2d(n, seed + 1)


def random_smooth_problem_2d_device(n, seed, device="cuda"):
    """The 2-D random smooth workload generated on the device, for grids whose
    host generation would take minutes (32768^2: 8.6 GB per array).  f: i.i.d.
    N(0,1) from torch's generator seeded `seed` (so not the numbers of
    smooth_random_2d, the same distribution), 5x5 box mean with zero padding,
    ghosts 0.  u0: the Dirichlet data of poly_boundary_2d(n, seed + 1) (same
    coefficients, same values) on the ghost layer, interior 0.  Returns
    float64 tensors on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    f = torch.zeros((n + 2, n + 2), dtype=torch.float64, device=device)
    z = torch.randn((1, 1, n, n), generator=g, dtype=torch.float64, device=device)
    f[1:-1, 1:-1] = torch.nn.functional.avg_pool2d(z, 5, stride=1, padding=2, count_include_pad=True)[0, 0]
    del z
    rng = np.random.default_rng(seed + 1)
    x = coords(n)
    coef = []
    for a in range(4):
        for b in range(4 - a):
            coef.append((a, b, rng.standard_normal()))
    ring = {"top": (x, np.zeros_like(x)), "bottom": (x, np.ones_like(x)),
            "left": (np.zeros_like(x), x), "right": (np.ones_like(x), x)}
    vals = {}
    for k, (X, Y) in ring.items():
        gv = np.zeros_like(X)
        for a, b, c in coef:
            gv += c * X ** a * Y ** b
        vals[k] = torch.from_numpy(gv).to(device)
    u0 = torch.zeros((n + 2, n + 2), dtype=torch.float64, device=device)
    u0[0, :] = vals["top"]
    u0[-1, :] = vals["bottom"]
    u0[:, 0] = vals["left"]
    u0[:, -1] = vals["right"]
    return f, u0


def smooth_target_2d(n, seed, kmax=4):
    """u_target = sum_{1<=kx,ky<=kmax} a_k sin(kx pi x) sin(ky pi y), a_k ~ N(0,1)/(kx ky)."""
    rng = np.random.default_rng(seed)
    x = coords(n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    t = np.zeros_like(X)
    for kx in range(1, kmax + 1):
        for ky in range(1, kmax + 1):
            t += rng.standard_normal() / (kx * ky) * np.sin(kx * math.pi * X) * np.sin(ky * math.pi * Y)
    return t


# ---------------------------------------------------------------------------
# Workload 3: 3-D Gaussian blobs
# ---------------------------------------------------------------------------

def gaussian_blobs_3d(n, seed, blobs=8, sigma=0.05):
    """f = sum of `blobs` Gaussians exp(-|r-c|^2 / (2 sigma^2)) with amplitudes
    U[-1,1] and centres U[0.2,0.8]^3; padded (nz+2, ny+2, nx+2), ghosts 0.
    Returns (f, u0) with u0 = 0."""
    rng = np.random.default_rng(seed)
    x = coords(n)
    f = np.zeros((n + 2, n + 2, n + 2))
    for _ in range(blobs):
        amp = rng.uniform(-1.0, 1.0)
        c = rng.uniform(0.2, 0.8, size=3)
        gx = np.exp(-(x - c[0]) ** 2 / (2 * sigma ** 2))
        gy = np.exp(-(x - c[1]) ** 2 / (2 * sigma ** 2))
        gz = np.exp(-(x - c[2]) ** 2 / (2 * sigma ** 2))
        f += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    f[0, :, :] = f[-1, :, :] = 0.0
    f[:, 0, :] = f[:, -1, :] = 0.0
    f[:, :, 0] = f[:, :, -1] = 0.0
    return f, np.zeros_like(f)


def random_field(dims, seed, scale=1.0):
    """Plain i.i.d. N(0, scale^2) field in the padded layout (for parity tests)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(tuple(int(v) + 2 for v in reversed(dims)))


# ---------------------------------------------------------------------------
# Spherical test of Sect. 5.2 (axisymmetric r-theta grid)
# ---------------------------------------------------------------------------

def spherical_problem_2d(n, seed, realistic=False):
    """(b, u0) of the Sect. 5.2 test on an n x n (r, theta) cell-centred grid,
    truncated to the l = 0 and l = 2 terms of Eqs. grav:source / grav:sol
    (a_l = 2^-l, k_l the first root of j_l, b_l = c_l from continuity at r = 1).
    b = r^2 s; u0: the analytic solution in the r = 1 ghost layer, zero inside
    (ab initio), or u_analytic (1 + U(-1/2, 1/2) / n) inside (realistic start,
    seeded).  Layout (n + 2, n + 2): theta slowest, r fastest."""
    from scipy.optimize import brentq
    from scipy.special import spherical_jn as jn
    dr, dt = 1.0 / n, math.pi / n
    r = (np.arange(n + 2) - 0.5) * dr
    t = (np.arange(n + 2) - 0.5) * dt
    R, Th = np.meshgrid(r, t)
    P2 = 0.5 * (3 * np.cos(Th) ** 2 - 1)
    k0, k2 = math.pi, brentq(lambda x: jn(2, x), 5.0, 6.5)
    a0, a2 = 1.0, 0.25
    b0 = a0 * k0 * jn(1, k0)
    b2 = -a2 / 5 * (2 * jn(2, k2) - k2 * jn(3, k2))
    Rin = np.where(R <= 1, R, 1.0)
    ua = np.where(R <= 1, (a0 * jn(0, k0 * Rin) + b0) + (a2 * jn(2, k2 * Rin) + b2 * Rin ** 2) * P2,
                  b0 / R + b2 / R ** 3 * P2)
    s = np.where(R <= 1, -a0 * k0 ** 2 * jn(0, k0 * Rin) - a2 * k2 ** 2 * jn(2, k2 * Rin) * P2, 0.0)
    u0 = np.zeros_like(ua)
    if realistic:
        rng = np.random.default_rng(seed)
        u0 = ua * (1.0 + rng.uniform(-0.5, 0.5, ua.shape) / n)
    u0[:, -1] = ua[:, -1]
    return np.ascontiguousarray(R ** 2 * s), np.ascontiguousarray(u0)


# ---------------------------------------------------------------------------
# Workload 4: the batch of independent 2-D problems
# ---------------------------------------------------------------------------

BATCH_SIZES = (64, 128, 256, 512, 1024)
BATCH_LEVELS = (5, 6, 7, 8, 9, 10)


def batch_specs(count=256, seed=4):
    """Per-problem (n, P, seed) for the batched workload: n uniform over
    BATCH_SIZES, P uniform over BATCH_LEVELS."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(BATCH_SIZES, size=count)
    Ps = rng.choice(BATCH_LEVELS, size=count)
    return [(int(n), int(P), 1000 + 2 * i) for i, (n, P) in enumerate(zip(ns, Ps))]
