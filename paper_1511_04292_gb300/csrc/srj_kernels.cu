// SRJ sweep, residual and layout kernels for sm_103a.
//
// Paper: Adsuara et al., "Scheduled Relaxation Jacobi method: improvements and
// applications" (arXiv:1511.04292).  The weighted-Jacobi step is Eq.
// 2nd-order_CD of Sect. 3.1 with the Poisson source of Sect. 5.1; the residual
// is the convergence monitor of Sect. 4.1 taken on b - A u.
//
// A stencil is not a dense contraction: these kernels are bound by HBM
// bandwidth (FP32) or by the FP64 pipe (FP64), not by the tensor cores.
#include "srj_internal.h"

#include <algorithm>
#include <cmath>

namespace srj {

namespace {

constexpr int kThreads = 256;

__host__ __device__ inline int64_t idx64(const Geom& g, int x, int y, int z) {
    return (int64_t)z * g.sy64 + (int64_t)y * g.sx64 + x;
}
__host__ __device__ inline int64_t idx32(const Geom& g, int x, int y, int z) {
    return (int64_t)z * g.plane32 + (int64_t)y * g.p32 + x + 3;
}

// --------------------------------------------------------------------------
// FP64: b = h^2 f
// --------------------------------------------------------------------------
__global__ void k_scale_source(Geom g, double h2, const double* __restrict__ f, double* __restrict__ b) {
    const int64_t n = g.n64;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.sx64);
        const int64_t r = i / g.sx64;
        const int y = (int)(r % (g.ny + 2));
        const int z = (int)(r / (g.ny + 2));
        const bool inner = x >= 1 && x <= g.nx && y >= 1 && y <= g.ny &&
                           (g.nd == 2 || (z >= 1 && z <= g.nz));
        b[i] = inner ? __dmul_rn(h2, f[i]) : 0.0;
    }
}

// --------------------------------------------------------------------------
// FP64 sweep, fixed order, no contraction:
//   s = (((W + E) + S) + N) [+ B) + T];  t = s + b;  d = t - 2d*u;  u' = u + c*d
// --------------------------------------------------------------------------
template <int ND, bool FMA = false>
__global__ void __launch_bounds__(kThreads)
k_sweep_f64(Geom g, const double* __restrict__ uin, double* __restrict__ uout,
            const double* __restrict__ b, double c, double two_d, const unsigned char* __restrict__ mask) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int y = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (x > g.nx || y > g.ny) return;
    const int zlo = (ND == 3) ? 1 : 0;
    const int zhi = (ND == 3) ? g.nz : 0;
    for (int z = zlo + blockIdx.z; z <= zhi; z += gridDim.z) {
        const int64_t p = idx64(g, x, y, z);
        const double uc = uin[p];
        if (mask && !mask[p]) { uout[p] = uc; continue; }
        double s = __dadd_rn(uin[p - 1], uin[p + 1]);
        s = __dadd_rn(s, uin[p - g.sx64]);
        s = __dadd_rn(s, uin[p + g.sx64]);
        if (ND == 3) {
            s = __dadd_rn(s, uin[p - g.sy64]);
            s = __dadd_rn(s, uin[p + g.sy64]);
        }
        const double t = __dadd_rn(s, b[p]);
        if (FMA) {  // 2 fused operations in place of 4
            uout[p] = fma(c, fma(-two_d, uc, t), uc);
        } else {
            const double dd = __dsub_rn(t, __dmul_rn(two_d, uc));
            uout[p] = __dadd_rn(uc, __dmul_rn(c, dd));
        }
    }
}

// --------------------------------------------------------------------------
// Fused residual + norms.  One block per group of rows (grid-stride); each
// thread walks x with stride blockDim.x.  Block partials are reduced by the
// last block to finish (fixed order over blocks, so the result does not depend
// on block scheduling).
// --------------------------------------------------------------------------
__device__ inline void block_reduce(double& ss, double& mx, double* sh_ss, double* sh_mx) {
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh_ss[w] = ss; sh_mx[w] = mx; }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        ss = lane < nw ? sh_ss[lane] : 0.0;
        mx = lane < nw ? sh_mx[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_down_sync(0xffffffffu, ss, o);
            mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        }
    }
}

// Block-wide sum into lane 0 of warp 0.
__device__ inline void block_sum(double& v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
}

template <int ND>
__global__ void __launch_bounds__(kThreads)
k_residual(Geom g, const double* __restrict__ u, const double* __restrict__ src, double h2,
           double* __restrict__ r64, float* __restrict__ r32, double scale, NormScratch ns, double two_d,
           const unsigned char* __restrict__ mask) {
    __shared__ double sh_ss[kThreads / 32], sh_mx[kThreads / 32], sh_fs[kThreads / 32];
    __shared__ bool last;
    double ss = 0.0, mx = 0.0;
    double fs = 0.0;  // sum of a^2, a = |neighbours| + |h2 src| + 2d |u|: scale of the rounding in r
    const int64_t rows = (int64_t)g.ny * (ND == 3 ? g.nz : 1);
    for (int64_t rr = blockIdx.x; rr < rows; rr += gridDim.x) {
        const int y = (int)(rr % g.ny) + 1;
        const int z = (ND == 3) ? (int)(rr / g.ny) + 1 : 0;
        const int64_t base = idx64(g, 0, y, z);
        for (int x = threadIdx.x + 1; x <= g.nx; x += blockDim.x) {
            const int64_t p = base + x;
            if (mask && !mask[p]) {
                if (r32) r32[idx32(g, x, y, z)] = 0.0f;
                continue;
            }
            const double uc = u[p];
            double s = __dadd_rn(u[p - 1], u[p + 1]);
            s = __dadd_rn(s, u[p - g.sx64]);
            s = __dadd_rn(s, u[p + g.sx64]);
            if (ND == 3) {
                s = __dadd_rn(s, u[p - g.sy64]);
                s = __dadd_rn(s, u[p + g.sy64]);
            }
            const double t = __dadd_rn(s, __dmul_rn(h2, src[p]));
            const double r = __dsub_rn(t, __dmul_rn(two_d, uc));
            if (r64) r64[p] = r;
            if (r32) r32[idx32(g, x, y, z)] = (float)(r * scale);
            ss = fma(r, r, ss);
            mx = fmax(mx, fabs(r));
            double a = fabs(u[p - 1]) + fabs(u[p + 1]) + fabs(u[p - g.sx64]) + fabs(u[p + g.sx64]);
            if (ND == 3) a += fabs(u[p - g.sy64]) + fabs(u[p + g.sy64]);
            a += fabs(h2 * src[p]) + two_d * fabs(uc);
            fs = fma(a, a, fs);
        }
    }
    block_reduce(ss, mx, sh_ss, sh_mx);
    block_sum(fs, sh_fs);
    if (threadIdx.x == 0) {
        ns.partials[2 * blockIdx.x] = ss;
        ns.partials[2 * blockIdx.x + 1] = mx;
        ns.partials[2 * kMaxNormBlocks + blockIdx.x] = fs;
        __threadfence();
        const unsigned done = atomicAdd(ns.counter, 1u);
        last = (done == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    ss = 0.0; mx = 0.0; fs = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
        ss += ((volatile double*)ns.partials)[2 * i];
        mx = fmax(mx, ((volatile double*)ns.partials)[2 * i + 1]);
        fs += ((volatile double*)ns.partials)[2 * kMaxNormBlocks + i];
    }
    __syncthreads();  // sh_ss / sh_mx / sh_fs are reused below
    block_reduce(ss, mx, sh_ss, sh_mx);
    block_sum(fs, sh_fs);
    if (threadIdx.x == 0) {
        ns.result[0] = sqrt(ss);
        // fmax drops NaN; a NaN anywhere already makes ss NaN, report it in both
        ns.result[1] = (ss == ss) ? mx : ss;
        // rounding floor of ||r||_2: the unit roundoff times ||a||_2 (each
        // residual entry is a sum of terms of total magnitude a)
        ns.result[2] = 0x1p-53 * sqrt(fs);
        *ns.counter = 0u;
    }
}

// --------------------------------------------------------------------------
// FP32 sweep: one thread per 4 consecutive interior x (one float4), one row
// per thread; 2-D grid over (x quads, y), 3-D loops over z.
// --------------------------------------------------------------------------
template <int ND>
__global__ void __launch_bounds__(kThreads)
k_sweep_f32(Geom g, const float* __restrict__ ein, float* __restrict__ eout,
            const float* __restrict__ r, float c, float two_d, const unsigned char* __restrict__ mask) {
    const int x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);  // 0-based interior x
    const int y = blockIdx.y * blockDim.y + threadIdx.y + 1;
    if (x0 >= g.nx || y > g.ny) return;
    const int zlo = (ND == 3) ? 1 : 0;
    const int zhi = (ND == 3) ? g.nz : 0;
    for (int z = zlo + blockIdx.z; z <= zhi; z += gridDim.z) {
        const int64_t p = idx32(g, x0 + 1, y, z);  // 16-byte aligned
        const float4 cc = *reinterpret_cast<const float4*>(ein + p);
        const float4 up = *reinterpret_cast<const float4*>(ein + p - g.p32);
        const float4 dn = *reinterpret_cast<const float4*>(ein + p + g.p32);
        const float4 rr = *reinterpret_cast<const float4*>(r + p);
        const float lf = ein[p - 1];
        const float rt = ein[p + 4];
        // t = sum of the neighbours + defect.  2-D: ((up + down) + r) + (left + right),
        // the order of the temporally blocked kernels, which form the vertical part
        // before the horizontal neighbours arrive by warp shuffle.  3-D:
        // ((((left + right) + up) + down) + (back + front)) + r, the order of the
        // 3-D blocked kernel.
        float4 t;
        if (ND == 2) {
            t.x = ((up.x + dn.x) + rr.x) + (lf + cc.y);
            t.y = ((up.y + dn.y) + rr.y) + (cc.x + cc.z);
            t.z = ((up.z + dn.z) + rr.z) + (cc.y + cc.w);
            t.w = ((up.w + dn.w) + rr.w) + (cc.z + rt);
        } else {
            const float4 bk = *reinterpret_cast<const float4*>(ein + p - g.plane32);
            const float4 fr = *reinterpret_cast<const float4*>(ein + p + g.plane32);
            t.x = ((((lf + cc.y) + up.x) + dn.x) + (bk.x + fr.x)) + rr.x;
            t.y = ((((cc.x + cc.z) + up.y) + dn.y) + (bk.y + fr.y)) + rr.y;
            t.z = ((((cc.y + cc.w) + up.z) + dn.z) + (bk.z + fr.z)) + rr.z;
            t.w = ((((cc.z + rt) + up.w) + dn.w) + (bk.w + fr.w)) + rr.w;
        }
        float4 o;
        o.x = fmaf(c, fmaf(-two_d, cc.x, t.x), cc.x);
        o.y = fmaf(c, fmaf(-two_d, cc.y, t.y), cc.y);
        o.z = fmaf(c, fmaf(-two_d, cc.z, t.z), cc.z);
        o.w = fmaf(c, fmaf(-two_d, cc.w, t.w), cc.w);
        if (mask) {  // inactive points keep their value
            const int64_t q = idx64(g, x0 + 1, y, z);
            if (!mask[q]) o.x = cc.x;
            if (x0 + 1 < g.nx && !mask[q + 1]) o.y = cc.y;
            if (x0 + 2 < g.nx && !mask[q + 2]) o.z = cc.z;
            if (x0 + 3 < g.nx && !mask[q + 3]) o.w = cc.w;
        }
        if (x0 + 4 <= g.nx) {
            *reinterpret_cast<float4*>(eout + p) = o;
        } else {
            const int v = g.nx - x0;  // 1..3 valid lanes
            eout[p] = o.x;
            if (v > 1) eout[p + 1] = o.y;
            if (v > 2) eout[p + 2] = o.z;
        }
    }
}

// --------------------------------------------------------------------------
// Layout / update kernels (grid-stride over padded points)
// --------------------------------------------------------------------------
__device__ inline bool decode(const Geom& g, int64_t i, int& x, int& y, int& z) {
    x = (int)(i % g.sx64);
    const int64_t r = i / g.sx64;
    y = (int)(r % (g.ny + 2));
    z = (int)(r / (g.ny + 2));
    return x >= 1 && x <= g.nx && y >= 1 && y <= g.ny && (g.nd == 2 || (z >= 1 && z <= g.nz));
}

__global__ void k_update(Geom g, double* __restrict__ u, const float* __restrict__ e, double inv_scale,
                         const unsigned char* __restrict__ mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        if (decode(g, i, x, y, z) && (!mask || mask[i])) u[i] += inv_scale * (double)e[idx32(g, x, y, z)];
    }
}

__global__ void k_to_f32(Geom g, const double* __restrict__ u, float* __restrict__ e) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        decode(g, i, x, y, z);
        e[idx32(g, x, y, z)] = (float)u[i];
    }
}

__global__ void k_source_f32(Geom g, double h2, const double* __restrict__ f, float* __restrict__ r) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        if (decode(g, i, x, y, z)) r[idx32(g, x, y, z)] = (float)(h2 * f[i]);
    }
}

__global__ void k_from_f32(Geom g, const float* __restrict__ e, double* __restrict__ u) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        if (decode(g, i, x, y, z)) u[i] = (double)e[idx32(g, x, y, z)];
    }
}

__global__ void k_boundary_adjoint(Geom g, const double* __restrict__ lam, double* __restrict__ gg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        if (decode(g, i, x, y, z)) { gg[i] = 0.0; continue; }
        double acc = 0.0;
        // interior neighbours of a ghost point: at most one per axis direction
        const int lo[3] = {1, 1, 1};
        const int hi[3] = {g.nx, g.ny, g.nz};
        int c[3] = {x, y, z};
        const int naxes = g.nd;
        for (int ax = 0; ax < naxes; ++ax) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int n[3] = {c[0], c[1], c[2]};
                n[ax] += sgn;
                bool inner = true;
                for (int a = 0; a < naxes; ++a) inner = inner && n[a] >= lo[a] && n[a] <= hi[a];
                if (inner) acc += lam[idx64(g, n[0], n[1], naxes == 3 ? n[2] : 0)];
            }
        }
        gg[i] = acc;
    }
}

__device__ inline double ghost_adjoint(const Geom& g, const double* __restrict__ lam, int x, int y, int z) {
    // interior neighbours of a ghost point: at most one per axis direction
    double acc = 0.0;
    const int c[3] = {x, y, z};
    const int hi[3] = {g.nx, g.ny, g.nz};
    for (int ax = 0; ax < g.nd; ++ax) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            int n[3] = {c[0], c[1], c[2]};
            n[ax] += sgn;
            bool inner = true;
            for (int a = 0; a < g.nd; ++a) inner = inner && n[a] >= 1 && n[a] <= hi[a];
            if (inner) acc += lam[idx64(g, n[0], n[1], g.nd == 3 ? n[2] : 0)];
        }
    }
    return acc;
}

__global__ void k_zero_ghosts(Geom g, double* __restrict__ a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        if (!decode(g, i, x, y, z)) a[i] = 0.0;
    }
}

__global__ void k_adjoint_finish(Geom g, double h2, const double* __restrict__ lam, const double* __restrict__ gu,
                                 double* __restrict__ gf, double* __restrict__ gg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n64; i += (int64_t)gridDim.x * blockDim.x) {
        int x, y, z;
        if (decode(g, i, x, y, z)) {
            gf[i] = h2 * lam[i];
            gg[i] = 0.0;
        } else {
            gf[i] = 0.0;
            gg[i] = ghost_adjoint(g, lam, x, y, z) + gu[i];
        }
    }
}

inline int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

Geom make_geom(int nd, const int64_t* dims) {
    Geom g{};
    g.nd = nd;
    g.nx = (int)dims[0];
    g.ny = (int)dims[1];
    g.nz = nd == 3 ? (int)dims[2] : 1;
    g.sx64 = g.nx + 2;
    g.sy64 = g.sx64 * (g.ny + 2);
    g.n64 = g.sy64 * (nd == 3 ? (g.nz + 2) : 1);
    g.p32 = ((int64_t)g.nx + 8 + 31) / 32 * 32;
    g.plane32 = g.p32 * (g.ny + 2);
    g.n32 = g.plane32 * (nd == 3 ? (g.nz + 2) : 1);
    return g;
}

cudaError_t launch_scale_source(const Geom& g, double h2, const double* f, double* b, cudaStream_t s) {
    k_scale_source<<<grid_for(g.n64), kThreads, 0, s>>>(g, h2, f, b);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f64(const Geom& g, const double* uin, double* uout, const double* b, double c,
                             cudaStream_t s, double two_d, const unsigned char* mask, bool fused) {
    if (two_d == 0.0) two_d = 2.0 * g.nd;
    // Each FP64 update costs the multiprocessor's FP64 pipe (2 instructions per
    // clock), so a small grid is spread over more multiprocessors with blocks
    // of 64 threads instead of 256.
    const int64_t pts = (int64_t)g.nx * g.ny * (g.nd == 3 ? g.nz : 1);
    const dim3 blk = pts < (int64_t{1} << 17) ? dim3(32, 2, 1) : dim3(64, 4, 1);
    dim3 grd((g.nx + blk.x - 1) / blk.x, (g.ny + blk.y - 1) / blk.y,
             g.nd == 3 ? (unsigned)std::min(g.nz, 65535) : 1u);
    if (fused) {
        if (g.nd == 3) k_sweep_f64<3, true><<<grd, blk, 0, s>>>(g, uin, uout, b, c, two_d, mask);
        else           k_sweep_f64<2, true><<<grd, blk, 0, s>>>(g, uin, uout, b, c, two_d, mask);
    } else {
        if (g.nd == 3) k_sweep_f64<3><<<grd, blk, 0, s>>>(g, uin, uout, b, c, two_d, mask);
        else           k_sweep_f64<2><<<grd, blk, 0, s>>>(g, uin, uout, b, c, two_d, mask);
    }
    return cudaGetLastError();
}

cudaError_t launch_residual(const Geom& g, const double* u, const double* src, double h2, double* r64,
                            float* r32, double scale, NormScratch ns, cudaStream_t s, double two_d,
                            const unsigned char* mask) {
    if (two_d == 0.0) two_d = 2.0 * g.nd;
    const int64_t rows = (int64_t)g.ny * (g.nd == 3 ? g.nz : 1);
    const int blocks = (int)std::min<int64_t>(rows, kMaxNormBlocks);
    if (g.nd == 3) k_residual<3><<<blocks, kThreads, 0, s>>>(g, u, src, h2, r64, r32, scale, ns, two_d, mask);
    else           k_residual<2><<<blocks, kThreads, 0, s>>>(g, u, src, h2, r64, r32, scale, ns, two_d, mask);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f32(const Geom& g, const float* ein, float* eout, const float* r, float c,
                             cudaStream_t s, float two_d, const unsigned char* mask) {
    if (two_d == 0.0f) two_d = 2.0f * g.nd;
    const int quads = (g.nx + 3) / 4;
    dim3 blk(64, 4, 1);
    dim3 grd((quads + 63) / 64, (g.ny + 3) / 4, g.nd == 3 ? (unsigned)std::min(g.nz, 65535) : 1u);
    if (g.nd == 3) k_sweep_f32<3><<<grd, blk, 0, s>>>(g, ein, eout, r, c, two_d, mask);
    else           k_sweep_f32<2><<<grd, blk, 0, s>>>(g, ein, eout, r, c, two_d, mask);
    return cudaGetLastError();
}

cudaError_t launch_update(const Geom& g, double* u, const float* e, double inv_scale, cudaStream_t s,
                          const unsigned char* mask) {
    k_update<<<grid_for(g.n64), kThreads, 0, s>>>(g, u, e, inv_scale, mask);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const Geom& g, const double* u, float* e, cudaStream_t s) {
    k_to_f32<<<grid_for(g.n64), kThreads, 0, s>>>(g, u, e);
    return cudaGetLastError();
}

cudaError_t launch_source_f32(const Geom& g, double h2, const double* f, float* r, cudaStream_t s) {
    k_source_f32<<<grid_for(g.n64), kThreads, 0, s>>>(g, h2, f, r);
    return cudaGetLastError();
}

cudaError_t launch_from_f32(const Geom& g, const float* e, double* u, cudaStream_t s) {
    k_from_f32<<<grid_for(g.n64), kThreads, 0, s>>>(g, e, u);
    return cudaGetLastError();
}

cudaError_t launch_zero_ghosts(const Geom& g, double* a, cudaStream_t s) {
    k_zero_ghosts<<<grid_for(g.n64), kThreads, 0, s>>>(g, a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_finish(const Geom& g, double h2, const double* lambda, const double* grad_u,
                                  double* grad_f, double* grad_g, cudaStream_t s) {
    k_adjoint_finish<<<grid_for(g.n64), kThreads, 0, s>>>(g, h2, lambda, grad_u, grad_f, grad_g);
    return cudaGetLastError();
}

cudaError_t launch_boundary_adjoint(const Geom& g, const double* lambda, double* grad_g, cudaStream_t s) {
    k_boundary_adjoint<<<grid_for(g.n64), kThreads, 0, s>>>(g, lambda, grad_g);
    return cudaGetLastError();
}

}  // namespace srj
