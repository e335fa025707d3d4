// SRJ on the spherical-coordinate operators of Sect. 5.2: FP64, or mixed
// precision (FP32 cycles on the defect equation inside FP64 defect correction).
//
// The Poisson equation in (r, theta[, phi]) multiplied by r^2, discretised by
// second-order central differences on cell centres r_i = (i - 1/2) dr,
// theta_j = (j - 1/2) dtheta, phi_k = (k - 1/2) dphi, has separable
// coefficients:
//   (L u)_p = cr_m[i] u(i-1) + cr_p[i] u(i+1) + ct_m[j] u(j-1) + ct_p[j] u(j+1)
//             [+ cp[j] (u(k-1) + u(k+1))] - d_p u_p,
//   d_p = cr_0[i] + ct_0[j] [+ (cp[j] + cp[j])],   L u = b = r^2 s.
// Boundary prescriptions of Sect. 5.2, applied at every step: Dirichlet data in
// the r = 1 ghost layer; u_0 = u_1 = u_2 at r = 0 (row i = 1 copies row 2, and
// row 2 sees u(i-1) = u(i)); Neumann mirrors at theta = 0, pi; periodic phi.
// The weighted-Jacobi step (Sect. 3.1 on this operator, diagonal -d):
//   res = (s - d u_p) - b_p,   u'_p = u_p + omega (res / d),
// each operation rounded once, in this order (the FP64 oracle's order, so the
// two agree bit for bit).  The SRJ cycle is that of the Poisson plans (Sect. 2).
#include "srj_internal.h"

#include <atomic>
#include "../../include/srj.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace srj_sph {
// Device pointers to the separable coefficients (padded index order).
struct Coef {
    const double* cr_m; const double* cr_p; const double* cr_0;
    const double* ct_m; const double* ct_p; const double* ct_0;
    const double* cp;
};
struct Coef32 {
    const float* cr_m; const float* cr_p; const float* cr_0;
    const float* ct_m; const float* ct_p; const float* ct_0;
    const float* cp;
    const float* dd;   // 2-D: d_i = cr_0[i] + ct_0 (ct_0 is the same on every polar row)
    const float* inv;  // 2-D: 1 / d_i
};
}  // namespace srj_sph

namespace {

using srj_sph::Coef;
using srj_sph::Coef32;
constexpr int kResBlocks = 304;   // residual partials (fixed: deterministic reduction order)
constexpr int kResThreads = 256;

// res and d at the active point (i, j, k) of u.
template <int ND>
__device__ __forceinline__ double sph_res(const srj::Geom& g, const Coef& c, const double* __restrict__ b,
                                          const double* __restrict__ u, int i, int j, int k, int64_t p, double* d_out) {
    const double cc = u[p];
    const double um = (i == 2) ? cc : u[p - 1];
    const double up = u[p + 1];
    const double tm = (j == 1) ? cc : u[p - g.sx64];
    const double tp = (j == g.ny) ? cc : u[p + g.sx64];
    double s = __dadd_rn(__dadd_rn(__dmul_rn(c.cr_m[i], um), __dmul_rn(c.cr_p[i], up)),
                         __dadd_rn(__dmul_rn(c.ct_m[j], tm), __dmul_rn(c.ct_p[j], tp)));
    double d = __dadd_rn(c.cr_0[i], c.ct_0[j]);
    if (ND == 3) {
        const double pm = (k == 1) ? u[p + (int64_t)(g.nz - 1) * g.sy64] : u[p - g.sy64];
        const double pp = (k == g.nz) ? u[p - (int64_t)(g.nz - 1) * g.sy64] : u[p + g.sy64];
        s = __dadd_rn(s, __dmul_rn(c.cp[j], __dadd_rn(pm, pp)));
        d = __dadd_rn(d, __dadd_rn(c.cp[j], c.cp[j]));
    }
    *d_out = d;
    return __dsub_rn(__dsub_rn(s, __dmul_rn(d, cc)), b[p]);
}

template <int ND>
__global__ void k_sph_sweep(srj::Geom g, Coef c, double omega, const double* __restrict__ b,
                            const double* __restrict__ uin, double* __restrict__ uout) {
    const int i = 2 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int j = 1 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    if (i > g.nx || j > g.ny) return;
    const int k0 = ND == 3 ? 1 : 0, k1 = ND == 3 ? g.nz : 0;
    for (int k = k0 + (int)blockIdx.z; k <= k1; k += (int)gridDim.z) {
        const int64_t p = (ND == 3 ? (int64_t)k * g.sy64 : 0) + (int64_t)j * g.sx64 + i;
        double d;
        const double res = sph_res<ND>(g, c, b, uin, i, j, k, p, &d);
        const double o = __dadd_rn(uin[p], __dmul_rn(omega, __ddiv_rn(res, d)));
        uout[p] = o;
        if (i == 2) uout[p - 1] = o;  // u_1 = u_2
    }
}

// Per-block partial (sum of res^2, max |res|) over the active points; r (if given) gets res.
template <int ND>
__global__ void k_sph_residual(srj::Geom g, Coef c, const double* __restrict__ b, const double* __restrict__ u,
                               double* __restrict__ r, double* __restrict__ partials) {
    const int64_t na = (int64_t)(g.nx - 1) * g.ny;  // active points per plane
    const int64_t nk = ND == 3 ? g.nz : 1;
    double ss = 0.0, mx = 0.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < na * nk; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kk = t / na, rem = t % na;
        const int j = 1 + (int)(rem / (g.nx - 1));
        const int i = 2 + (int)(rem % (g.nx - 1));
        const int k = ND == 3 ? 1 + (int)kk : 0;
        const int64_t p = (ND == 3 ? (int64_t)k * g.sy64 : 0) + (int64_t)j * g.sx64 + i;
        double d;
        const double res = sph_res<ND>(g, c, b, u, i, j, k, p, &d);
        if (r) r[p] = res;
        ss = __dadd_rn(ss, __dmul_rn(res, res));
        mx = fmax(mx, fabs(res));
    }
    __shared__ double s_ss[kResThreads / 32], s_mx[kResThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ss = __dadd_rn(ss, __shfl_down_sync(0xffffffffu, ss, o));
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { s_ss[w] = ss; s_mx[w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int q = 0; q < kResThreads / 32; ++q) { a = __dadd_rn(a, s_ss[q]); m = fmax(m, s_mx[q]); }
        partials[2 * blockIdx.x] = a;
        partials[2 * blockIdx.x + 1] = m;
    }
}

__global__ void k_sph_norms(const double* __restrict__ partials, int n, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, m = 0.0;
    for (int q = 0; q < n; ++q) { a = __dadd_rn(a, partials[2 * q]); m = fmax(m, partials[2 * q + 1]); }
    out[0] = sqrt(a);
    out[1] = m;
}

// FP32 step on the defect equation L e = r (mixed precision): the same stencil
// and prescriptions; e has homogeneous Dirichlet data at r = 1.  FP32 arrays in
// the pitched layout of the Poisson plans (x stored at column x + 3).  In 2-D
// every operation is rounded explicitly, in the order (fma: one rounding)
//   s = fma(cr_m, um, cr_p up) + fma(ct_m, tm, ct_p tp);  t = fma(-d, e, s) - r;
//   e' = fma(omega * (1/d), t, e),
// which the temporally blocked 2-D kernel repeats bit for bit.
template <int ND>
__global__ void k_sph_sweep_f32(srj::Geom g, Coef32 c, float omega, const float* __restrict__ r,
                                const float* __restrict__ ein, float* __restrict__ eout) {
    const int i = 2 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int j = 1 + (int)(blockIdx.y * blockDim.y + threadIdx.y);
    if (i > g.nx || j > g.ny) return;
    const int k0 = ND == 3 ? 1 : 0, k1 = ND == 3 ? g.nz : 0;
    const float crm = c.cr_m[i], crp = c.cr_p[i], ctm = c.ct_m[j], ctp = c.ct_p[j];
    float d, wd;
    if (ND == 3) {
        d = c.cr_0[i] + c.ct_0[j] + 2.0f * c.cp[j];
        wd = omega / d;
    } else {
        d = c.dd[i];
        wd = __fmul_rn(omega, c.inv[i]);
    }
    for (int k = k0 + (int)blockIdx.z; k <= k1; k += (int)gridDim.z) {
        const int64_t p = (ND == 3 ? (int64_t)k * g.plane32 : 0) + (int64_t)j * g.p32 + i + 3;
        const float cc = ein[p];
        const float um = (i == 2) ? cc : ein[p - 1];
        const float up = ein[p + 1];
        const float tm = (j == 1) ? cc : ein[p - g.p32];
        const float tp = (j == g.ny) ? cc : ein[p + g.p32];
        float o;
        if (ND == 3) {
            float s = (crm * um + crp * up) + (ctm * tm + ctp * tp);
            const float pm = (k == 1) ? ein[p + (int64_t)(g.nz - 1) * g.plane32] : ein[p - g.plane32];
            const float pp = (k == g.nz) ? ein[p - (int64_t)(g.nz - 1) * g.plane32] : ein[p + g.plane32];
            s += c.cp[j] * (pm + pp);
            o = cc + wd * ((s - d * cc) - r[p]);
        } else {
            const float s = __fadd_rn(__fmaf_rn(crm, um, __fmul_rn(crp, up)), __fmaf_rn(ctm, tm, __fmul_rn(ctp, tp)));
            const float t = __fsub_rn(__fmaf_rn(-d, cc, s), r[p]);
            o = __fmaf_rn(wd, t, cc);
        }
        eout[p] = o;
        if (i == 2) eout[p - 1] = o;  // e_1 = e_2
    }
}

// Temporally blocked form of the 2-D FP32 step: T steps per launch on a
// 128 x 64 tile held in registers (one float4 of 4 radial points per lane, a
// band of 8 polar rows per warp, band edges exchanged through shared memory),
// as the Poisson kernel does; after T steps the centre (128 - 2 HX) x (64 - 2T)
// is exact.  Each point is updated with the unblocked kernel's expression in
// its order, including the prescriptions (u_1 = u_2, theta mirrors), so T
// blocked steps give the bits of T single steps.
constexpr int kTbX = 128, kTbY = 64, kTbWarps = 8, kTbBand = 8;
constexpr size_t kTbRsBytes = (size_t)kTbY * 32 * sizeof(float4);  // 32 KB of defect rows

template <int T, bool EDGE>
__device__ __forceinline__ void sph_band(float4 (&e)[kTbBand], const float4* __restrict__ rs, float4* xch,
                                         const float2* ctab, const float (&cs)[8], int lane, int w,
                                         const float (&crm)[4], const float (&crp)[4], const float (&dd)[4],
                                         const float (&inv)[4], const bool (&act)[4], bool has_x1, int Yw,
                                         int ny) {
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
    for (int t = 0; t < T; ++t) {  // not unrolled: one step's live set at a time
        float wd[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) wd[k] = __fmul_rn(cs[t], inv[k]);
        float4* slot = xch + (t & 1) * (2 * kTbWarps * 32);
        slot[(2 * w) * 32 + lane] = e[0];
        slot[(2 * w + 1) * 32 + lane] = e[kTbBand - 1];
        __syncthreads();
        const float4 above = (w > 0) ? slot[(2 * (w - 1) + 1) * 32 + lane] : zero;
        const float4 below = (w + 1 < kTbWarps) ? slot[(2 * (w + 1)) * 32 + lane] : zero;
        float4 upr = above;
#pragma unroll
        for (int i = 0; i < kTbBand; ++i) {
            const float4 cur = e[i];
            const float4 dnr = (i + 1 < kTbBand) ? e[i + 1] : below;
            const float2 ct = ctab[w * kTbBand + i];
            const float lf = __shfl_up_sync(0xffffffffu, cur.w, 1);
            const float rt = __shfl_down_sync(0xffffffffu, cur.x, 1);
            const float cc[4] = {cur.x, cur.y, cur.z, cur.w};
            float lt[4] = {lf, cur.x, cur.y, cur.z};
            const float rg[4] = {cur.y, cur.z, cur.w, rt};
            float tu[4] = {upr.x, upr.y, upr.z, upr.w};
            float td[4] = {dnr.x, dnr.y, dnr.z, dnr.w};
            const float4 rv = rs[(w * kTbBand + i) * 32 + lane];  // this lane's defect row
            const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
            const int y = Yw + i;
            const bool iny = y >= 1 && y <= ny;
            if (EDGE) {
                if (has_x1) lt[1] = cc[1];  // radial point 2 sees u(1) = u(2)
                if (y == 1) { tu[0] = cc[0]; tu[1] = cc[1]; tu[2] = cc[2]; tu[3] = cc[3]; }  // theta mirrors
                if (y == ny) { td[0] = cc[0]; td[1] = cc[1]; td[2] = cc[2]; td[3] = cc[3]; }
            }
            // per point the unblocked kernel's operations in its order; the radial
            // terms (misaligned neighbours) in scalar form, the rest as FP32x2 pairs
            // (every multiply-add is an explicit fma, so nothing is left to contract)
            float hr[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) hr[k] = __fmaf_rn(crm[k], lt[k], __fmul_rn(crp[k], rg[k]));
            const float2 ctm2 = make_float2(ct.x, ct.x), ctp2 = make_float2(ct.y, ct.y);
            float o[4];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int a = 2 * h, b = 2 * h + 1;
                const float2 c2 = make_float2(cc[a], cc[b]);
                const float2 vt = __ffma2_rn(ctm2, make_float2(tu[a], tu[b]),
                                             __fmul2_rn(ctp2, make_float2(td[a], td[b])));
                const float2 sv = __fadd2_rn(make_float2(hr[a], hr[b]), vt);
                const float2 tv = __fadd2_rn(__ffma2_rn(make_float2(-dd[a], -dd[b]), c2, sv),
                                             make_float2(-r4[a], -r4[b]));
                const float2 ov = __ffma2_rn(make_float2(wd[a], wd[b]), tv, c2);
                o[a] = ov.x;
                o[b] = ov.y;
            }
            if (EDGE) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (!(iny && act[k])) o[k] = cc[k];
            }
            if (EDGE && has_x1 && iny && act[1]) o[0] = o[1];  // u_1 = u_2
            upr = cur;
            e[i] = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

template <int T>
__global__ void __launch_bounds__(kTbWarps * 32, 2)
k_sph_tb(srj::Geom g, Coef32 c, srj::TbSteps steps, const float* __restrict__ rin, const float* __restrict__ ein,
         float* __restrict__ eout) {
    constexpr int HX = T <= 4 ? 4 : 8;
    constexpr int TX = kTbX - 2 * HX, TY = kTbY - 2 * T;
    __shared__ float4 xch[2 * 2 * kTbWarps * 32];
    __shared__ float2 ctab[kTbY];
    extern __shared__ float4 rs[];  // [kTbY][32]: the tile's defect rows, each read back by the lane that wrote it
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int X0 = 1 + TX * (int)blockIdx.x - HX, Y0 = 1 + TY * (int)blockIdx.y - T;
    const int Yw = Y0 + w * kTbBand;
    if (threadIdx.x < kTbY) {  // polar coefficients of the tile's rows (read after the first barrier)
        const int y = min(max(Y0 + (int)threadIdx.x, 0), g.ny + 1);
        ctab[threadIdx.x] = make_float2(c.ct_m[y], c.ct_p[y]);
    }
    float crm[4], crp[4], dd[4], inv[4];
    bool act[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int x = X0 + 4 * lane + k;
        const int xc = min(max(x, 0), g.nx + 1);
        crm[k] = c.cr_m[xc]; crp[k] = c.cr_p[xc]; dd[k] = c.dd[xc]; inv[k] = c.inv[xc];
        act[k] = x >= 2 && x <= g.nx;
    }
    const bool has_x1 = X0 + 4 * lane == 1;  // this lane holds radial points 1 and 2
    const int col = X0 + 3 + 4 * lane;        // multiple of 4: each float4 wholly in or out of a row
    const bool colok = col >= 0 && col + 4 <= g.p32;
    float4 e[kTbBand];
#pragma unroll
    for (int i = 0; i < kTbBand; ++i) {
        const int y = Yw + i;
        e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 rv = e[i];
        if (colok && y >= 0 && y <= g.ny + 1) {
            const int64_t off = (int64_t)y * g.p32 + col;
            e[i] = __ldg(reinterpret_cast<const float4*>(ein + off));
            rv = __ldg(reinterpret_cast<const float4*>(rin + off));
        }
        rs[(w * kTbBand + i) * 32 + lane] = rv;
    }
    // no prescription, mask or outside point anywhere in the tile
    const bool interior = X0 >= 3 && X0 + kTbX - 1 <= g.nx && Y0 >= 2 && Y0 + kTbY - 1 <= g.ny - 1;
    if (interior) sph_band<T, false>(e, rs, xch, ctab, steps.c, lane, w, crm, crp, dd, inv, act, has_x1, Yw, g.ny);
    else          sph_band<T, true>(e, rs, xch, ctab, steps.c, lane, w, crm, crp, dd, inv, act, has_x1, Yw, g.ny);
    const int lane_lo = HX / 4, lane_hi = (HX + TX) / 4;
    if (lane < lane_lo || lane >= lane_hi) return;
#pragma unroll
    for (int i = 0; i < kTbBand; ++i) {
        const int row = w * kTbBand + i;
        if (row < T || row >= T + TY) continue;
        const int y = Y0 + row;
        if (y < 1 || y > g.ny) continue;
        const int x = X0 + 4 * lane;
        float* dst = eout + (int64_t)y * g.p32 + x + 3;  // 16-byte aligned
        const float o[4] = {e[i].x, e[i].y, e[i].z, e[i].w};
        if (x >= 1 && x + 3 <= g.nx) {
            *reinterpret_cast<float4*>(dst) = e[i];
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x + k >= 1 && x + k <= g.nx) dst[k] = o[k];
        }
    }
}

// r32 = -(L u - b) * scale at the active points (scale: a power of 2).
template <int ND>
__global__ void k_sph_defect(srj::Geom g, Coef c, const double* __restrict__ b, const double* __restrict__ u,
                             double scale, float* __restrict__ r32) {
    const int64_t na = (int64_t)(g.nx - 1) * g.ny;
    const int64_t nk = ND == 3 ? g.nz : 1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < na * nk; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kk = t / na, rem = t % na;
        const int j = 1 + (int)(rem / (g.nx - 1));
        const int i = 2 + (int)(rem % (g.nx - 1));
        const int k = ND == 3 ? 1 + (int)kk : 0;
        const int64_t p = (ND == 3 ? (int64_t)k * g.sy64 : 0) + (int64_t)j * g.sx64 + i;
        double d;
        r32[(ND == 3 ? (int64_t)k * g.plane32 : 0) + (int64_t)j * g.p32 + i + 3] =
            (float)(-sph_res<ND>(g, c, b, u, i, j, k, p, &d) * scale);
    }
}

// u += e / scale on rows i = 1..n_r (e_1 = e_2 keeps the prescription).
__global__ void k_sph_update(srj::Geom g, double* __restrict__ u, const float* __restrict__ e, double inv_scale) {
    const int64_t n = (int64_t)g.nx * g.ny * (g.nd == 3 ? g.nz : 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int i = 1 + (int)(t % g.nx);
        const int64_t rest = t / g.nx;
        const int j = 1 + (int)(rest % g.ny);
        const int k = g.nd == 3 ? 1 + (int)(rest / g.ny) : 0;
        const int64_t p = (g.nd == 3 ? (int64_t)k * g.sy64 : 0) + (int64_t)j * g.sx64 + i;
        u[p] += inv_scale * (double)e[(g.nd == 3 ? (int64_t)k * g.plane32 : 0) + (int64_t)j * g.p32 + i + 3];
    }
}

// Ghost layer and row i = 1 from the prescriptions (the r = 1 ghost is data).
__global__ void k_sph_fin_r(srj::Geom g, double* __restrict__ u) {  // (j, k): u_1 = u_2, u_0 = u_1
    const int j = 1 + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int k = (g.nd == 3 ? 1 : 0) + (int)blockIdx.y;
    if (j > g.ny) return;
    const int64_t q = (g.nd == 3 ? (int64_t)k * g.sy64 : 0) + (int64_t)j * g.sx64;
    if (g.nx >= 2) u[q + 1] = u[q + 2];
    u[q] = u[q + 1];
}
__global__ void k_sph_fin_t(srj::Geom g, double* __restrict__ u) {  // (i, k): theta mirrors
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int k = (g.nd == 3 ? 1 : 0) + (int)blockIdx.y;
    if (i > g.nx + 1) return;
    const int64_t base = (g.nd == 3 ? (int64_t)k * g.sy64 : 0);
    u[base + i] = u[base + g.sx64 + i];
    u[base + (int64_t)(g.ny + 1) * g.sx64 + i] = u[base + (int64_t)g.ny * g.sx64 + i];
}
__global__ void k_sph_fin_p(srj::Geom g, double* __restrict__ u) {  // (i, j): periodic phi
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= g.sy64) return;
    u[t] = u[(int64_t)g.nz * g.sy64 + t];
    u[(int64_t)(g.nz + 1) * g.sy64 + t] = u[g.sy64 + t];
}

}  // namespace

struct srj_sph_plan {
    int device = 0;
    int nd = 2;
    srj::Geom g{};
    double* coef = nullptr;  // device: radial (3 (nx+2)) | polar (3 (ny+2)) | azim (ny+2)
    srj_sph::Coef c{};
    std::vector<double> seq;  // ordered weights of one M-cycle
    double* ua = nullptr;
    double* ub = nullptr;
    double* bb = nullptr;
    double* partials = nullptr;
    double* norms = nullptr;
    double* host_norms = nullptr;
    int precision = SRJ_PREC_FP64;
    int tdepth = 1;           // mixed 2-D: FP32 steps per blocked launch
    float* coef32 = nullptr;  // mixed: FP32 copy of the coefficients
    srj_sph::Coef32 c32{};
    float* ea = nullptr;      // mixed: FP32 correction (ping-pong) and defect
    float* eb = nullptr;
    float* r32 = nullptr;
    float* e_final = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t cycle = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int sfail(int code, const char* msg) { return srj::set_last_error(code, msg); }

#define SPH_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return sfail(SRJ_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

cudaError_t launch_sweep(const srj_sph_plan* p, double omega, const double* b, const double* uin, double* uout,
                         cudaStream_t s) {
    if (p->g.nx < 2) return cudaSuccess;  // no active point
    dim3 blk(128, 2, 1);
    dim3 grd((unsigned)((p->g.nx - 1 + 127) / 128), (unsigned)((p->g.ny + 1) / 2),
             p->nd == 3 ? (unsigned)std::min(p->g.nz, 64) : 1u);
    if (p->nd == 3) k_sph_sweep<3><<<grd, blk, 0, s>>>(p->g, p->c, omega, b, uin, uout);
    else            k_sph_sweep<2><<<grd, blk, 0, s>>>(p->g, p->c, omega, b, uin, uout);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f32(const srj_sph_plan* p, float omega, const float* ein, float* eout, cudaStream_t s) {
    if (p->g.nx < 2) return cudaSuccess;
    dim3 blk(128, 2, 1);
    dim3 grd((unsigned)((p->g.nx - 1 + 127) / 128), (unsigned)((p->g.ny + 1) / 2),
             p->nd == 3 ? (unsigned)std::min(p->g.nz, 64) : 1u);
    if (p->nd == 3) k_sph_sweep_f32<3><<<grd, blk, 0, s>>>(p->g, p->c32, omega, p->r32, ein, eout);
    else            k_sph_sweep_f32<2><<<grd, blk, 0, s>>>(p->g, p->c32, omega, p->r32, ein, eout);
    return cudaGetLastError();
}

template <int T>
void launch_sph_T(const srj_sph_plan* p, const srj::TbSteps& st, const float* ein, float* eout, cudaStream_t s) {
    constexpr int HX = T <= 4 ? 4 : 8;
    const int TX = kTbX - 2 * HX, TY = kTbY - 2 * T;
    dim3 grd((unsigned)((p->g.nx + TX - 1) / TX), (unsigned)((p->g.ny + TY - 1) / TY), 1);
    k_sph_tb<T><<<grd, kTbWarps * 32, kTbRsBytes, s>>>(p->g, p->c32, st, p->r32, ein, eout);
}

template <int T>
cudaError_t sph_tb_attr() {
    return cudaFuncSetAttribute(k_sph_tb<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTbRsBytes);
}

cudaError_t sph_tb_prepare() {
    // kernel attributes are per device: set them once on each device used
    static std::atomic<bool> done[64] = {};  // idempotent setup; concurrent first calls both set
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    cudaError_t r[7] = {sph_tb_attr<2>(), sph_tb_attr<3>(), sph_tb_attr<4>(), sph_tb_attr<5>(),
                        sph_tb_attr<6>(), sph_tb_attr<7>(), sph_tb_attr<8>()};
    for (cudaError_t x : r) if (x != cudaSuccess) return x;
    done[dev].store(true, std::memory_order_release);
    return cudaSuccess;
}

// n = st.T in 2..8 FP32 steps in one launch (2-D mixed plans).
cudaError_t launch_sweep_f32_tb(const srj_sph_plan* p, const srj::TbSteps& st, const float* ein, float* eout,
                                cudaStream_t s) {
    switch (st.T) {
        case 2: launch_sph_T<2>(p, st, ein, eout, s); break;
        case 3: launch_sph_T<3>(p, st, ein, eout, s); break;
        case 4: launch_sph_T<4>(p, st, ein, eout, s); break;
        case 5: launch_sph_T<5>(p, st, ein, eout, s); break;
        case 6: launch_sph_T<6>(p, st, ein, eout, s); break;
        case 7: launch_sph_T<7>(p, st, ein, eout, s); break;
        case 8: launch_sph_T<8>(p, st, ein, eout, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_defect(const srj_sph_plan* p, double scale, cudaStream_t s) {
    if (p->g.nx < 2) return cudaSuccess;
    if (p->nd == 3) k_sph_defect<3><<<4 * kResBlocks, kResThreads, 0, s>>>(p->g, p->c, p->bb, p->ua, scale, p->r32);
    else            k_sph_defect<2><<<4 * kResBlocks, kResThreads, 0, s>>>(p->g, p->c, p->bb, p->ua, scale, p->r32);
    return cudaGetLastError();
}

cudaError_t launch_residual(const srj_sph_plan* p, const double* b, const double* u, double* r, cudaStream_t s) {
    if (p->g.nx < 2) {
        cudaError_t e = cudaMemsetAsync(p->norms, 0, 2 * sizeof(double), s);
        return e;
    }
    if (p->nd == 3) k_sph_residual<3><<<kResBlocks, kResThreads, 0, s>>>(p->g, p->c, b, u, r, p->partials);
    else            k_sph_residual<2><<<kResBlocks, kResThreads, 0, s>>>(p->g, p->c, b, u, r, p->partials);
    k_sph_norms<<<1, 32, 0, s>>>(p->partials, kResBlocks, p->norms);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const srj_sph_plan* p, double* u, cudaStream_t s) {
    const unsigned nk = p->nd == 3 ? (unsigned)p->g.nz : 1u;
    k_sph_fin_r<<<dim3((unsigned)((p->g.ny + 127) / 128), nk), 128, 0, s>>>(p->g, u);
    k_sph_fin_t<<<dim3((unsigned)((p->g.nx + 2 + 127) / 128), nk), 128, 0, s>>>(p->g, u);
    if (p->nd == 3) k_sph_fin_p<<<(unsigned)((p->g.sy64 + 255) / 256), 256, 0, s>>>(p->g, u);
    return cudaGetLastError();
}

int read_norms(srj_sph_plan* p, cudaStream_t s, double* l2, double* linf) {
    SPH_CUDA(cudaMemcpyAsync(p->host_norms, p->norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    *l2 = p->host_norms[0];
    *linf = p->host_norms[1];
    return SRJ_OK;
}

int check_plan(srj_sph_plan* p) {
    if (!p) return sfail(SRJ_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    SPH_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return sfail(SRJ_ERR_INVALID_ARG, "plan was created on another device");
    return SRJ_OK;
}

void destroy(srj_sph_plan* p) {
    if (!p) return;
    if (p->cycle) cudaGraphExecDestroy(p->cycle);
    if (p->ev0) cudaEventDestroy(p->ev0);
    if (p->ev1) cudaEventDestroy(p->ev1);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaFree(p->coef); cudaFree(p->ua); cudaFree(p->ub); cudaFree(p->bb); cudaFree(p->partials);
    cudaFree(p->norms); cudaFree(p->coef32); cudaFree(p->ea); cudaFree(p->eb); cudaFree(p->r32);
    if (p->host_norms) cudaFreeHost(p->host_norms);
    delete p;
}

// One M-cycle.  FP64: from ua back into ua (an odd M ends with a copy).
// Mixed: e = 0, then the FP32 steps on L e = r32; the result is in e_final.
int capture_cycle(srj_sph_plan* p) {
    cudaGraph_t graph = nullptr;
    SPH_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    const size_t bytes = sizeof(double) * (size_t)p->g.n64;
    if (p->precision == SRJ_PREC_MIXED) {
        const size_t b32 = sizeof(float) * (size_t)p->g.n32;
        err = cudaMemsetAsync(p->ea, 0, b32, p->cap);
        if (err == cudaSuccess) err = cudaMemsetAsync(p->eb, 0, b32, p->cap);
        float *in = p->ea, *out = p->eb;
        const size_t M = p->seq.size();
        for (size_t k = 0; k < M && err == cudaSuccess;) {
            const int n = (int)std::min<size_t>((size_t)p->tdepth, M - k);
            if (n >= 2) {
                srj::TbSteps st{};
                st.T = n;
                for (int t = 0; t < n; ++t) st.c[t] = (float)p->seq[k + t];
                err = launch_sweep_f32_tb(p, st, in, out, p->cap);
            } else {
                err = launch_sweep_f32(p, (float)p->seq[k], in, out, p->cap);
            }
            std::swap(in, out);
            k += (size_t)n;
        }
        p->e_final = in;
    } else {
        for (size_t k = 0; k < p->seq.size() && err == cudaSuccess; ++k) {
            const bool from_a = (k % 2) == 0;
            err = launch_sweep(p, p->seq[k], p->bb, from_a ? p->ua : p->ub, from_a ? p->ub : p->ua, p->cap);
        }
        if (err == cudaSuccess && (p->seq.size() % 2) == 1)
            err = cudaMemcpyAsync(p->ua, p->ub, bytes, cudaMemcpyDeviceToDevice, p->cap);
    }
    cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
    if (err != cudaSuccess) { if (graph) cudaGraphDestroy(graph); SPH_CUDA(err); }
    SPH_CUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&p->cycle, graph, 0);
    cudaGraphDestroy(graph);
    SPH_CUDA(e3);
    return SRJ_OK;
}

int load_inputs(srj_sph_plan* p, const double* b, const double* u, cudaStream_t s) {
    const size_t bytes = sizeof(double) * (size_t)p->g.n64;
    SPH_CUDA(cudaMemcpyAsync(p->bb, b, bytes, cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(cudaMemcpyAsync(p->ua, u, bytes, cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(cudaMemcpyAsync(p->ub, u, bytes, cudaMemcpyDeviceToDevice, s));
    return SRJ_OK;
}

}  // namespace

extern "C" {

int srj_sph_coefficients(int ndim, const int64_t* dims, double* radial, double* polar, double* azim) {
    if ((ndim != 2 && ndim != 3) || !dims || !radial || !polar || (ndim == 3 && !azim))
        return sfail(SRJ_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1 || dims[i] > (int64_t)1 << 20) return sfail(SRJ_ERR_INVALID_ARG, "dims must be in 1..2^20");
    const double pi = 3.14159265358979323846;
    const int64_t nr = dims[0], nt = dims[1];
    const double dr = 1.0 / (double)nr, dt = pi / (double)nt;
    for (int64_t i = 0; i < nr + 2; ++i) {
        const double r = ((double)i - 0.5) * dr;
        radial[i] = r * (r - dr) / (dr * dr);
        radial[(nr + 2) + i] = r * (r + dr) / (dr * dr);
        radial[2 * (nr + 2) + i] = 2.0 * r * r / (dr * dr);
    }
    for (int64_t j = 0; j < nt + 2; ++j) {
        polar[j] = polar[(nt + 2) + j] = polar[2 * (nt + 2) + j] = 0.0;
        if (ndim == 3) azim[j] = 0.0;
        if (j < 1 || j > nt) continue;
        const double t = ((double)j - 0.5) * dt;
        const double cot = std::cos(t) / std::sin(t);
        polar[j] = 1.0 / (dt * dt) - cot / (2.0 * dt);
        polar[(nt + 2) + j] = 1.0 / (dt * dt) + cot / (2.0 * dt);
        polar[2 * (nt + 2) + j] = 2.0 / (dt * dt);
        if (ndim == 3) {
            const double dp = 2.0 * pi / (double)dims[2];
            const double sn = std::sin(t);
            azim[j] = 1.0 / (sn * sn * dp * dp);
        }
    }
    return SRJ_OK;
}

int srj_sph_plan_create(srj_sph_plan_t* out, int ndim, const int64_t* dims, const double* radial,
                        const double* polar, const double* azim, int P, const double* omega, const int32_t* q,
                        const int32_t* order, int precision) {
    if (!out) return sfail(SRJ_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (precision != SRJ_PREC_FP64 && precision != SRJ_PREC_MIXED)
        return sfail(SRJ_ERR_INVALID_ARG, "precision must be SRJ_PREC_FP64 or SRJ_PREC_MIXED");
    if ((ndim != 2 && ndim != 3) || !dims || !radial || !polar || (ndim == 3 && !azim) || !omega || !q)
        return sfail(SRJ_ERR_INVALID_ARG, "bad arguments");
    if (P < 1 || P > 32) return sfail(SRJ_ERR_INVALID_ARG, "P must be in 1..32");
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1 || dims[i] > 65536) return sfail(SRJ_ERR_INVALID_ARG, "dims must be in 1..65536");
    std::vector<double> w(omega, omega + P);
    std::vector<int32_t> qq(q, q + P);
    int64_t M = 0;
    for (int i = 0; i < P; ++i) {
        if (!(std::isfinite(w[i]) && w[i] > 0.0)) return sfail(SRJ_ERR_INVALID_ARG, "weights must be finite and > 0");
        if (qq[i] < 1) return sfail(SRJ_ERR_INVALID_ARG, "repetitions must be >= 1");
        M += qq[i];
    }
    if (M > ((int64_t)1 << 20)) return sfail(SRJ_ERR_INVALID_ARG, "M must be <= 2^20");
    // Contraction of the integer scheme on [1 / max omega, 2): all roots of the
    // cycle polynomial lie in [1 / max omega, 2), below it the polynomial falls
    // monotonically from 1, and the Jacobi-scaled operator has its spectrum in
    // (0, 2): rows weakly diagonally dominant with the boundary prescriptions,
    // strictly in the rows next to the Dirichlet boundary, and irreducible.
    const double wmax = *std::max_element(w.begin(), w.end());
    const double kmax = 2.0 * (1.0 - 1e-12);
    if (!(srj::host_max_cycle_log10_range(w, qq, std::min(1.0 / wmax, 0.5 * kmax), kmax) < 0.0))
        return sfail(SRJ_ERR_BAD_SCHEDULE, "the integer scheme does not contract on [1/omega_max, 2)");
    std::vector<int32_t> ord;
    if (order) {
        ord.assign(order, order + M);
        std::vector<int64_t> cnt(P, 0);
        for (int32_t v : ord) {
            if (v < 0 || v >= P) return sfail(SRJ_ERR_INVALID_ARG, "order entries must be in 0..P-1");
            ++cnt[v];
        }
        for (int i = 0; i < P; ++i)
            if (cnt[i] != qq[i]) return sfail(SRJ_ERR_INVALID_ARG, "order must hold level i exactly q_i times");
    } else {
        ord = srj::host_drift_order(w, qq, 1.0 / wmax);
    }
    auto* p = new srj_sph_plan();
    p->nd = ndim;
    p->precision = precision;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return sfail(SRJ_ERR_CUDA, "no device"); }
    p->g = srj::make_geom(ndim, dims);
    p->seq.resize((size_t)M);
    for (int64_t k = 0; k < M; ++k) p->seq[(size_t)k] = w[(size_t)ord[(size_t)k]];
    const int64_t nr = dims[0], nt = dims[1];
    const size_t ncoef = (size_t)(3 * (nr + 2) + 3 * (nt + 2) + (nt + 2));
    std::vector<double> hc(ncoef, 0.0);
    std::copy(radial, radial + 3 * (nr + 2), hc.begin());
    std::copy(polar, polar + 3 * (nt + 2), hc.begin() + 3 * (nr + 2));
    if (ndim == 3) std::copy(azim, azim + (nt + 2), hc.begin() + 3 * (nr + 2) + 3 * (nt + 2));
    for (double v : hc)
        if (!std::isfinite(v)) { delete p; return sfail(SRJ_ERR_INVALID_ARG, "coefficients must be finite"); }
    const size_t bytes = sizeof(double) * (size_t)p->g.n64;
    if (cudaMalloc(&p->coef, sizeof(double) * ncoef) != cudaSuccess || cudaMalloc(&p->ua, bytes) != cudaSuccess ||
        cudaMalloc(&p->ub, bytes) != cudaSuccess || cudaMalloc(&p->bb, bytes) != cudaSuccess ||
        cudaMalloc(&p->partials, sizeof(double) * 2 * kResBlocks) != cudaSuccess ||
        cudaMalloc(&p->norms, 2 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&p->host_norms, 2 * sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess ||
        cudaMemcpy(p->coef, hc.data(), sizeof(double) * ncoef, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        destroy(p);
        return sfail(SRJ_ERR_CUDA, "plan allocation failed");
    }
    const double* base = p->coef;
    p->c = Coef{base, base + (nr + 2), base + 2 * (nr + 2), base + 3 * (nr + 2), base + 3 * (nr + 2) + (nt + 2),
                base + 3 * (nr + 2) + 2 * (nt + 2), base + 3 * (nr + 2) + 3 * (nt + 2)};
    if (precision == SRJ_PREC_MIXED) {
        std::vector<float> h32(hc.begin(), hc.end());
        // 2-D: per-radius diagonal and its reciprocal in FP32 (the polar diagonal
        // ct_0 = 2 / dtheta^2 is the same on every row)
        const float ct0 = (float)polar[2 * (nt + 2) + 1];
        for (int64_t i = 0; i < nr + 2; ++i) {
            const float d = (float)radial[2 * (nr + 2) + i] + ct0;
            h32.push_back(d);
        }
        for (int64_t i = 0; i < nr + 2; ++i) {
            const float d = h32[ncoef + (size_t)i];
            h32.push_back(d != 0.0f ? 1.0f / d : 0.0f);
        }
        const size_t b32 = sizeof(float) * (size_t)p->g.n32;
        if (cudaMalloc(&p->coef32, sizeof(float) * h32.size()) != cudaSuccess || cudaMalloc(&p->ea, b32) != cudaSuccess ||
            cudaMalloc(&p->eb, b32) != cudaSuccess || cudaMalloc(&p->r32, b32) != cudaSuccess ||
            cudaMemcpy(p->coef32, h32.data(), sizeof(float) * h32.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(p->r32, 0, b32) != cudaSuccess) {
            cudaGetLastError();
            destroy(p);
            return sfail(SRJ_ERR_CUDA, "plan allocation failed");
        }
        const float* b2 = p->coef32;
        p->c32 = Coef32{b2, b2 + (nr + 2), b2 + 2 * (nr + 2), b2 + 3 * (nr + 2), b2 + 3 * (nr + 2) + (nt + 2),
                        b2 + 3 * (nr + 2) + 2 * (nt + 2), b2 + 3 * (nr + 2) + 3 * (nt + 2), b2 + ncoef,
                        b2 + ncoef + (nr + 2)};
        if (ndim == 2 && nr >= 2) {
            if (sph_tb_prepare() != cudaSuccess) {
                cudaGetLastError();
                destroy(p);
                return sfail(SRJ_ERR_CUDA, "set-up of the blocked spherical sweep failed");
            }
            p->tdepth = 8;
        }
    }
    int rc = capture_cycle(p);
    if (rc != SRJ_OK) { destroy(p); return rc; }
    *out = p;
    return SRJ_OK;
}

int srj_sph_plan_destroy(srj_sph_plan_t plan) {
    if (!plan) return SRJ_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    const int pdev = plan->device;
    if (dev != pdev) cudaSetDevice(pdev);
    cudaStreamSynchronize(plan->cap);
    destroy(plan);
    if (dev >= 0 && dev != pdev) cudaSetDevice(dev);
    return SRJ_OK;
}

int srj_sph_steps(srj_sph_plan_t p, const double* b, double* u, int64_t first, int64_t count, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!b || !u || first < 0 || count < 0) return sfail(SRJ_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    rc = load_inputs(p, b, u, s);
    if (rc) return rc;
    const int64_t M = (int64_t)p->seq.size();
    double *in = p->ua, *out = p->ub;
    for (int64_t k = 0; k < count; ++k) {
        SPH_CUDA(launch_sweep(p, p->seq[(size_t)((first + k) % M)], p->bb, in, out, s));
        std::swap(in, out);
    }
    SPH_CUDA(cudaMemcpyAsync(u, in, sizeof(double) * (size_t)p->g.n64, cudaMemcpyDeviceToDevice, s));
    return SRJ_OK;
}

int srj_sph_residual(srj_sph_plan_t p, const double* b, const double* u, double* r_out, double* l2, double* linf,
                     void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!b || !u || !l2 || !linf) return sfail(SRJ_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (r_out) SPH_CUDA(cudaMemsetAsync(r_out, 0, sizeof(double) * (size_t)p->g.n64, s));
    SPH_CUDA(launch_residual(p, b, u, r_out, s));
    return read_norms(p, s, l2, linf);
}

int srj_sph_solve(srj_sph_plan_t p, const double* b, double* u, double tol, int64_t max_cycles, void* stream,
                  srj_stats_t* stats) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!b || !u || !(tol >= 0.0) || max_cycles < 0) return sfail(SRJ_ERR_INVALID_ARG, "bad arguments");
    if (!p->cycle) return sfail(SRJ_ERR_CUDA, "the plan has no cycle graph (a failed re-capture)");
    cudaStream_t s = (cudaStream_t)stream;
    srj_stats_t st{};
    rc = load_inputs(p, b, u, s);
    if (rc) return rc;
    double l2 = 0.0, linf = 0.0;
    SPH_CUDA(launch_residual(p, p->bb, p->ua, nullptr, s));
    rc = read_norms(p, s, &l2, &linf);
    if (rc) return rc;
    st.residual_checks = 1;
    st.r0_l2 = l2;
    int status = SRJ_ERR_NOT_CONVERGED;
    if (l2 == 0.0) status = SRJ_OK;
    else if (!std::isfinite(l2)) status = SRJ_ERR_DIVERGED;
    double best = l2;
    int stall = 0;
    float ms_total = 0.f;
    for (int64_t c = 1; status == SRJ_ERR_NOT_CONVERGED && c <= max_cycles; ++c) {
        double scale = 1.0;
        if (p->precision == SRJ_PREC_MIXED) {
            // defect scaled by a power of 2 so that its largest entry is in [1, 2)
            scale = (linf > 0.0 && std::isfinite(linf)) ? std::ldexp(1.0, -std::ilogb(linf)) : 1.0;
            SPH_CUDA(launch_defect(p, scale, s));
        }
        SPH_CUDA(cudaEventRecord(p->ev0, s));
        SPH_CUDA(cudaGraphLaunch(p->cycle, s));
        SPH_CUDA(cudaEventRecord(p->ev1, s));
        if (p->precision == SRJ_PREC_MIXED) {
            k_sph_update<<<4 * kResBlocks, kResThreads, 0, s>>>(p->g, p->ua, p->e_final, 1.0 / scale);
            SPH_CUDA(cudaGetLastError());
        }
        SPH_CUDA(launch_residual(p, p->bb, p->ua, nullptr, s));
        rc = read_norms(p, s, &l2, &linf);
        if (rc) return rc;
        float ms = 0.f;
        SPH_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        ms_total += ms;
        st.cycles = c;
        st.sweeps = c * (int64_t)p->seq.size();
        st.residual_checks += 1;
        if (!std::isfinite(l2) || l2 > 1e6 * st.r0_l2) { status = SRJ_ERR_DIVERGED; break; }
        if (l2 <= tol * st.r0_l2) { status = SRJ_OK; break; }
        // floating-point floor: the residual has not halved its best value for 4 cycles
        if (l2 < 0.5 * best) { best = l2; stall = 0; }
        else if (++stall >= 4) { st.stagnated = 1; break; }
    }
    SPH_CUDA(launch_finalize(p, p->ua, s));
    SPH_CUDA(cudaMemcpyAsync(u, p->ua, sizeof(double) * (size_t)p->g.n64, cudaMemcpyDeviceToDevice, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    st.res_l2 = l2;
    st.res_linf = linf;
    st.rel_res = st.r0_l2 > 0.0 ? l2 / st.r0_l2 : 0.0;
    st.sweep_ms = ms_total;
    if (stats) *stats = st;
    if (status == SRJ_ERR_NOT_CONVERGED) return sfail(status, "tolerance not reached");
    if (status == SRJ_ERR_DIVERGED) return sfail(status, "residual diverged");
    return SRJ_OK;
}

int srj_sph_plan_set_temporal_depth(srj_sph_plan_t p, int T) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (T < 1 || T > 8) return sfail(SRJ_ERR_INVALID_ARG, "temporal depth must be in 1..8");
    if (T > 1 && !(p->precision == SRJ_PREC_MIXED && p->nd == 2 && p->g.nx >= 2))
        return sfail(SRJ_ERR_INVALID_ARG, "temporal blocking is available for 2-D mixed-precision plans with n_r >= 2");
    p->tdepth = T;
    if (p->cycle) { cudaGraphExecDestroy(p->cycle); p->cycle = nullptr; }
    return capture_cycle(p);
}

int srj_sph_plan_temporal_depth(srj_sph_plan_t p, int* T) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!T) return sfail(SRJ_ERR_INVALID_ARG, "T is NULL");
    *T = p->tdepth;
    return SRJ_OK;
}

int srj_sph_finalize(srj_sph_plan_t p, double* u, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!u) return sfail(SRJ_ERR_INVALID_ARG, "u is NULL");
    SPH_CUDA(launch_finalize(p, u, (cudaStream_t)stream));
    return SRJ_OK;
}

}  // extern "C"
