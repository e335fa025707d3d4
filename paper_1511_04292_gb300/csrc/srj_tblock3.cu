// Temporally blocked FP32 SRJ sweep for 3-D grids (7-point Laplacian): T = 2 or
// 3 consecutive weighted-Jacobi steps (Sect. 3.1 with the Poisson source of
// Sect. 5.1; weights in cycle order, Sect. 2) per HBM round trip.
//
// A block owns a 128 x 32 (x, y) tile, halo included, and streams it through a
// segment of z planes.  Input planes of e and of the FP32 defect r arrive by
// cp.async in shared rings, two planes ahead of use.  At the iteration that
// brings in plane p, stage s = 1..T computes level s on plane p - s from the
// level s-1 planes p-s-1, p-s, p-s+1 (the last one produced by stage s-1 in
// the same iteration); stage T writes the tile's centre (120 x (32 - 2T)) of
// its plane to HBM.  Each thread keeps its own two rows of the level planes it
// still needs in registers; shared memory serves a plane's first read, the
// defect rows and the rows of the neighbouring warps (y neighbours), which
// each stage publishes for the next iteration.  With a halo of 4 columns and T
// rows, every centre point sees only exact values.  Points of the Dirichlet
// ghost layer and outside the grid keep their value, and each update is the
// unblocked kernel's expression in its order, so one launch gives the bits of
// T single-step launches.
//
// The block is persistent (one per SM: the rings take 176 KB for T = 2, 224 KB
// for T = 3) and walks work items (tile, z segment) round robin; a segment
// costs 2T extra plane iterations of pipeline fill, so the launcher picks the
// segment length (about 32 to 128 planes) for which the busiest block walks the
// fewest plane iterations (64 at 512^3 with T = 2, 86 with T = 3).
#include "srj_internal.h"

#include <atomic>

#include <algorithm>

namespace srj {

namespace {

constexpr int kX = 128;                 // tile columns (floats): 32 lanes x float4
constexpr int kWarps = 16;
constexpr int kY = 2 * kWarps;          // tile rows: 2 per warp
constexpr int kHX = 4;                  // x halo: T <= 4 steps rounded up to a float4
constexpr int kTX = kX - 2 * kHX;       // 120 centre columns
constexpr int kZSegMin = 32, kZSegMax = 128;  // output planes per work item (z segment), chosen per grid
constexpr int kPlane = kY * 32;         // float4 per plane tile
template <int T> struct Cfg {
    static constexpr int kD = 2;                     // planes loaded ahead of use (3 measured no faster)
    static constexpr int kERing = kD + 2;            // e planes p-1 .. p+D
    static constexpr int kHY = T;                    // y halo
    static constexpr int kTY = kY - 2 * T;           // centre rows
    static constexpr int kRRing = T + 1 + kD;        // defect planes p-T .. p+D
    static constexpr int kLSlots = 2 * (T - 1);      // levels 1..T-1, two planes each
    static constexpr size_t kSmem = (size_t)(kERing + kRRing + kLSlots) * kPlane * sizeof(float4);
};

__device__ inline void cp_async16(void* smem_dst, const void* gsrc, unsigned src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait_pending() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One 7-point update of 4 consecutive points, in the unblocked kernel's order:
// nb = (((left + right) + up) + down) + (back + front); o = c (nb + r - 6 e) + e.
// Left + right are scalar adds into FP32x2 pairs; the rest is packed.
__device__ __forceinline__ float4 upd7(float4 cc, float4 up, float4 dn, float4 bk, float4 fr, float4 rr, float lf,
                                       float rt, float c) {
    const float2 m6 = make_float2(-6.0f, -6.0f);
    const float2 cv = make_float2(c, c);
    float2 s0 = make_float2(lf + cc.y, cc.x + cc.z);
    float2 s1 = make_float2(cc.y + cc.w, cc.z + rt);
    s0 = __fadd2_rn(s0, make_float2(up.x, up.y));
    s1 = __fadd2_rn(s1, make_float2(up.z, up.w));
    s0 = __fadd2_rn(s0, make_float2(dn.x, dn.y));
    s1 = __fadd2_rn(s1, make_float2(dn.z, dn.w));
    s0 = __fadd2_rn(s0, __fadd2_rn(make_float2(bk.x, bk.y), make_float2(fr.x, fr.y)));
    s1 = __fadd2_rn(s1, __fadd2_rn(make_float2(bk.z, bk.w), make_float2(fr.z, fr.w)));
    s0 = __fadd2_rn(s0, make_float2(rr.x, rr.y));
    s1 = __fadd2_rn(s1, make_float2(rr.z, rr.w));
    const float2 c0 = make_float2(cc.x, cc.y), c1 = make_float2(cc.z, cc.w);
    const float2 o0 = __ffma2_rn(cv, __ffma2_rn(m6, c0, s0), c0);
    const float2 o1 = __ffma2_rn(cv, __ffma2_rn(m6, c1, s1), c1);
    return make_float4(o0.x, o0.y, o1.x, o1.y);
}

// One stage on the two rows (j0, j0 + 1) of this warp: level L+1 of the centre
// plane from this thread's rows of the level-L planes bk / cc / fr, the rows
// above / below from the neighbouring warps, and the defect rows rr.
// keep_plane: the plane is a ghost plane or outside the grid.
__device__ __forceinline__ void stage_rows(const float4 (&bk)[2], const float4 (&cc)[2], const float4 (&fr)[2],
                                           float4 above, float4 below, const float4 (&rr)[2], float c, int lane,
                                           bool keep_plane, const bool (&inx)[4], const bool (&iny)[2],
                                           float4 (&out)[2]) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float4 cur = cc[k];
        const float4 up = k == 0 ? above : cc[0];
        const float4 dn = k == 0 ? cc[1] : below;
        // lanes 0 and 31 receive their own values: those columns are halo
        const float lf = __shfl_up_sync(0xffffffffu, cur.w, 1);
        const float rt = __shfl_down_sync(0xffffffffu, cur.x, 1);
        float4 o = upd7(cur, up, dn, bk[k], fr[k], rr[k], lf, rt, c);
        if (keep_plane || !iny[k]) {
            o = cur;
        } else {
            o.x = inx[0] ? o.x : cur.x;
            o.y = inx[1] ? o.y : cur.y;
            o.z = inx[2] ? o.z : cur.z;
            o.w = inx[3] ? o.w : cur.w;
        }
        out[k] = o;
    }
}

// One work item: the tile whose first column / row has padded coordinates X0 /
// Y0, output planes zs .. ze-1, all T stages.
template <int T>
__device__ __forceinline__ void run_item(const float* __restrict__ ein, const float* __restrict__ rin,
                                         float* __restrict__ eout, const Geom& g, const TbSteps& steps, int X0, int Y0,
                                         int zs, int ze, float4* E, float4* R, float4* L, int lane, int j0, int jup,
                                         int jdn) {
    using C = Cfg<T>;
    constexpr int kERing = C::kERing;
    const int niter = ze - zs + 2 * T;     // planes zs-T .. ze-1+T
    const int col = X0 + 3 + 4 * lane;     // multiple of 4: each float4 wholly in or out of a row
    const bool colok = col >= 0 && col + 4 <= g.p32;
    bool inx[4], iny[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int x = X0 + 4 * lane + q;
        inx[q] = x >= 1 && x <= g.nx;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int y = Y0 + j0 + k;
        iny[k] = y >= 1 && y <= g.ny;
    }
    // plane loads of iteration i (plane zs - T + i): this thread's two rows
    auto issue = [&](int i) {
        if (i < niter) {
            const int p = zs - T + i;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int y = Y0 + j0 + k;
                const bool ok = colok && p >= 0 && p <= g.nz + 1 && y >= 0 && y <= g.ny + 1;
                const int64_t off = ok ? (int64_t)p * g.plane32 + (int64_t)y * g.p32 + col : 0;
                cp_async16(&E[(i % kERing) * kPlane + (j0 + k) * 32 + lane], ein + off, ok ? 16u : 0u);
                cp_async16(&R[(i % C::kRRing) * kPlane + (j0 + k) * 32 + lane], rin + off, ok ? 16u : 0u);
            }
        }
        cp_async_commit();  // possibly empty: keeps one group per iteration
    };
#pragma unroll
    for (int d = 0; d < C::kD; ++d) issue(d);
    // this thread's rows of the planes still needed: lv_bk / lv_cc[s] = level s on planes p-s-2 / p-s-1
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 lv_bk[T][2], lv_cc[T][2];
#pragma unroll
    for (int s = 0; s < T; ++s) {
        lv_bk[s][0] = lv_bk[s][1] = z4;
        lv_cc[s][0] = lv_cc[s][1] = z4;
    }
    // Unrolled by 8: the level planes held per thread rotate with period 2 and
    // the e ring with period 4, so the copies of the rotation become register
    // renaming and those ring offsets constants.  At 512^3 a step took 190.5 us
    // (T = 2) and 185.9 us (T = 3) without unrolling, 163.9 / 154.7 us unrolled
    // by 4, 164.5 / 151.9 us by 8 and 165.6 / 153.9 us by 12.
#pragma unroll 8
    for (int i = 0; i < niter; ++i) {
        cp_async_wait_pending<C::kD - 1>();  // this thread's loads of iteration i have landed
        __syncthreads();    // ... and everyone's; iteration i-1 is fully done
        issue(i + C::kD);   // into slots no longer read
        const int p = zs - T + i;
        float4 fr[2];       // level s-1 on plane p-s+1: the stage's front plane
        const float4* Ep = E + (i % kERing) * kPlane;
        fr[0] = Ep[j0 * 32 + lane];
        fr[1] = Ep[(j0 + 1) * 32 + lane];
#pragma unroll
        for (int s = 1; s <= T; ++s) {
            float4 out[2];
            const bool live = i >= 2 * s;
            if (live) {
                const int q = p - s;  // plane of the level-s result
                // the centre plane's rows of the neighbouring warps, published last iteration
                const float4* Nc = (s == 1) ? E + ((i + kERing - 1) % kERing) * kPlane
                                            : L + ((s - 2) * 2 + ((i + 1) & 1)) * kPlane;
                const float4* Rq = R + ((i + C::kRRing - s) % C::kRRing) * kPlane;
                float4 rr[2];
                rr[0] = Rq[j0 * 32 + lane];
                rr[1] = Rq[(j0 + 1) * 32 + lane];
                stage_rows(lv_bk[s - 1], lv_cc[s - 1], fr, Nc[jup * 32 + lane], Nc[jdn * 32 + lane], rr,
                           steps.c[s - 1], lane, q < 1 || q > g.nz, inx, iny, out);
                if (s < T) {
                    float4* Lw = L + ((s - 1) * 2 + (i & 1)) * kPlane;
                    Lw[j0 * 32 + lane] = out[0];
                    Lw[(j0 + 1) * 32 + lane] = out[1];
                } else if (lane >= kHX / 4 && lane < (kHX + kTX) / 4) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int j = j0 + k;
                        const int y = Y0 + j;
                        if (j < C::kHY || j >= C::kHY + C::kTY || y < 1 || y > g.ny) continue;
                        const int x = X0 + 4 * lane;
                        float* dst = eout + (int64_t)q * g.plane32 + (int64_t)y * g.p32 + x + 3;  // 16-B aligned
                        if (inx[0] && inx[3]) {
                            *reinterpret_cast<float4*>(dst) = out[k];
                        } else {
                            if (inx[0]) dst[0] = out[k].x;
                            if (inx[1]) dst[1] = out[k].y;
                            if (inx[2]) dst[2] = out[k].z;
                            if (inx[3]) dst[3] = out[k].w;
                        }
                    }
                }
            }
            // rotate level s-1: its planes advance by one
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                lv_bk[s - 1][k] = lv_cc[s - 1][k];
                lv_cc[s - 1][k] = fr[k];
                if (s < T && live) fr[k] = out[k];
            }
            if (!live) break;  // later stages start later (uniform over the block)
        }
    }
}

// Persistent blocks walk the work items (tile, z segment of zseg output planes)
// round robin.
template <int T>
__global__ void __launch_bounds__(kWarps * 32, 1)
k_sweep3_f32_tb(const float* __restrict__ ein, const float* __restrict__ rin, float* __restrict__ eout, Geom g,
                TbSteps steps, int tiles_x, int tiles_y, int nseg, int zseg) {
    using C = Cfg<T>;
    extern __shared__ float4 smem[];
    float4* E = smem;                          // [kERing][kPlane]   level-0 e planes
    float4* R = E + C::kERing * kPlane;        // [kRRing][kPlane]   defect planes
    float4* L = R + C::kRRing * kPlane;        // [T-1][2][kPlane]   published level planes
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j0 = 2 * w;                      // this warp's rows of the tile
    const int jup = max(j0 - 1, 0), jdn = min(j0 + 2, kY - 1);  // tile edge: stale halo, never stored
    const int nitems = tiles_x * tiles_y * nseg;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % tiles_x;
        const int by = (item / tiles_x) % tiles_y;
        const int sg = item / (tiles_x * tiles_y);
        const int X0 = 1 + kTX * bx - kHX, Y0 = 1 + C::kTY * by - C::kHY;
        const int zs = 1 + sg * zseg, ze = min(zs + zseg, g.nz + 1);
        run_item<T>(ein, rin, eout, g, steps, X0, Y0, zs, ze, E, R, L, lane, j0, jup, jdn);
        cp_async_wait_all();
        __syncthreads();  // the next item's first loads reuse ring slots
    }
}

}  // namespace

cudaError_t tb3_prepare() {
    // kernel attributes are per device: set them once on each device used
    static std::atomic<bool> done[64] = {};  // idempotent setup; concurrent first calls both set
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sweep3_f32_tb<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg<2>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep3_f32_tb<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<3>::kSmem);
    if (e == cudaSuccess) done[dev].store(true, std::memory_order_release);
    return e;
}

int tb3_max_steps() { return 3; }

cudaError_t launch_sweep3_f32_tb(const Geom& g, const float* ein, const float* rin, float* eout, const TbSteps& steps,
                                 int blocks, cudaStream_t s) {
    if (g.nd != 3 || blocks < 1 || steps.T < 2 || steps.T > 3) return cudaErrorInvalidValue;
    const int T = steps.T;
    const int TY = kY - 2 * T;
    const int tx = (g.nx + kTX - 1) / kTX, ty = (g.ny + TY - 1) / TY;
    // z segments: the count whose busiest block walks the fewest plane iterations,
    // rounds x (segment + 2T warm-up planes), for segments of about 32 to 128 planes
    const int64_t tiles = (int64_t)tx * ty;
    const int ns_lo = std::max(1, (g.nz + kZSegMax - 1) / kZSegMax);
    const int ns_hi = std::max(ns_lo, (g.nz + kZSegMin - 1) / kZSegMin);
    int ns = 1, zseg = g.nz;
    int64_t best = -1;
    for (int n = ns_lo; n <= ns_hi; ++n) {
        const int z = (g.nz + n - 1) / n;         // segments of z planes (the last one may be shorter) ...
        const int nz_seg = (g.nz + z - 1) / z;    // ... and how many of them cover the grid
        const int64_t items = tiles * nz_seg;
        const int64_t grid = std::min<int64_t>(blocks, items);
        const int64_t cost = (items + grid - 1) / grid * (z + 2 * T);
        if (best < 0 || cost < best) { best = cost; ns = nz_seg; zseg = z; }
    }
    const int64_t items = tiles * ns;
    if (items > INT32_MAX) return cudaErrorInvalidValue;
    const unsigned grid = (unsigned)std::min<int64_t>(blocks, items);
    if (T == 2)
        k_sweep3_f32_tb<2><<<grid, kWarps * 32, Cfg<2>::kSmem, s>>>(ein, rin, eout, g, steps, tx, ty, ns, zseg);
    else
        k_sweep3_f32_tb<3><<<grid, kWarps * 32, Cfg<3>::kSmem, s>>>(ein, rin, eout, g, steps, tx, ty, ns, zseg);
    return cudaGetLastError();
}

}  // namespace srj
