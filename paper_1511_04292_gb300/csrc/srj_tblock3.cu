// Temporally blocked FP32 SRJ sweep for 3-D grids (7-point Laplacian): two
// consecutive weighted-Jacobi steps (Sect. 3.1 with the Poisson source of
// Sect. 5.1; weights in cycle order, Sect. 2) per HBM round trip.
//
// A block owns a 128 x 32 (x, y) tile, halo included, and streams it through a
// segment of z planes.  Input planes of e and of the FP32 defect r arrive by
// cp.async in 4-deep shared rings, two planes ahead of use.  At the iteration
// that brings in plane p:
//   stage 1 computes level 1 on plane p-1 from level-0 planes p-2, p-1, p;
//   stage 2 computes level 2 on plane p-2 from level-1 planes p-3, p-2, p-1
//           and writes the tile's centre (120 x 28) of it to HBM.
// Each thread keeps its own two rows of the level-0, level-1 and defect planes
// it still needs in registers; shared memory serves only the first read of a
// plane and the rows of the neighbouring warps (y neighbours).  With a halo of
// 4 columns and 2 rows, every centre point sees only exact level-1 values.  Points of the
// Dirichlet ghost layer and outside the grid keep their value, and each update
// is the unblocked kernel's expression in its order, so one launch gives the
// bits of two single-step launches.
//
// The block is persistent (one per SM: the rings take 160 KB) and walks work
// items (tile, z segment) round robin; a segment of 64 output planes costs 4
// extra plane iterations of pipeline fill.
#include "srj_internal.h"

#include <algorithm>

namespace srj {

namespace {

constexpr int kX = 128;                 // tile columns (floats): 32 lanes x float4
constexpr int kWarps = 16;
constexpr int kY = 2 * kWarps;          // tile rows: 2 per warp
constexpr int kHX = 4, kHY = 2;         // halo: 2 steps, x rounded up to a float4
constexpr int kTX = kX - 2 * kHX;       // 120 centre columns
constexpr int kTY = kY - 2 * kHY;       // 28 centre rows
constexpr int kRing = 4;                // input planes p-1 .. p+2
constexpr int kZSeg = 64;               // output planes per work item
constexpr int kPlane = kY * 32;         // float4 per plane tile
constexpr int kL1 = 2;                  // level-1 planes shared for their y neighbours
constexpr size_t kSmemBytes = (size_t)(2 * kRing + kL1) * kPlane * sizeof(float4);

__device__ inline void cp_async16(void* smem_dst, const void* gsrc, unsigned src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ inline void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
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

__global__ void __launch_bounds__(kWarps * 32, 1)
k_sweep3_f32_tb2(const float* __restrict__ ein, const float* __restrict__ rin, float* __restrict__ eout, Geom g,
                 float c0, float c1, int tiles_x, int tiles_y, int nseg) {
    extern __shared__ float4 smem[];
    float4* E = smem;                      // [kRing][kPlane]  level-0 e planes
    float4* R = E + kRing * kPlane;        // [kRing][kPlane]  defect planes
    float4* L1 = R + kRing * kPlane;       // [kL1][kPlane]    level-1 planes
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j0 = 2 * w;                  // this warp's rows of the tile
    const int nitems = tiles_x * tiles_y * nseg;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        const int bx = item % tiles_x;
        const int by = (item / tiles_x) % tiles_y;
        const int sg = item / (tiles_x * tiles_y);
        const int X0 = 1 + kTX * bx - kHX, Y0 = 1 + kTY * by - kHY;
        const int zs = 1 + sg * kZSeg, ze = min(zs + kZSeg, g.nz + 1);
        const int niter = ze - zs + 4;     // planes zs-2 .. ze+1
        const int col = X0 + 3 + 4 * lane; // multiple of 4: each float4 wholly in or out of a row
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
        // plane loads of iteration i (plane zs - 2 + i): this thread's two rows
        auto issue = [&](int i) {
            if (i < niter) {
                const int p = zs - 2 + i;
                const int slot = i % kRing;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int y = Y0 + j0 + k;
                    const bool ok = colok && p >= 0 && p <= g.nz + 1 && y >= 0 && y <= g.ny + 1;
                    const int64_t off = ok ? (int64_t)p * g.plane32 + (int64_t)y * g.p32 + col : 0;
                    cp_async16(&E[slot * kPlane + (j0 + k) * 32 + lane], ein + off, ok ? 16u : 0u);
                    cp_async16(&R[slot * kPlane + (j0 + k) * 32 + lane], rin + off, ok ? 16u : 0u);
                }
            }
            cp_async_commit();  // possibly empty: keeps one group per iteration
        };
        issue(0);
        issue(1);
        // this thread's rows: level-0 planes p-2, p-1; level-1 planes p-3, p-2; defect plane p-2
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 e_bk[2] = {z4, z4}, e_cc[2] = {z4, z4}, l_bk[2] = {z4, z4}, l_cc[2] = {z4, z4}, r_pv[2] = {z4, z4};
        const int jup = max(j0 - 1, 0), jdn = min(j0 + 2, kY - 1);  // tile edge: stale halo, never stored
        for (int i = 0; i < niter; ++i) {
            cp_async_wait_1();  // this thread's loads of iteration i have landed
            __syncthreads();    // ... and everyone's; iteration i-1 is fully done
            issue(i + 2);       // into the slot of iteration i-2, no longer read
            const float4* Ep = E + (i % kRing) * kPlane;        // plane p
            const float4* Eq = E + ((i + 3) % kRing) * kPlane;  // plane p-1
            const float4* Rq = R + ((i + 3) % kRing) * kPlane;
            float4 e_fr[2], l_fr[2], r_c[2];
            e_fr[0] = Ep[j0 * 32 + lane];
            e_fr[1] = Ep[(j0 + 1) * 32 + lane];
            if (i >= 2) {
                const int q = zs - 3 + i;  // plane of the level-1 result
                r_c[0] = Rq[j0 * 32 + lane];
                r_c[1] = Rq[(j0 + 1) * 32 + lane];
                stage_rows(e_bk, e_cc, e_fr, Eq[jup * 32 + lane], Eq[jdn * 32 + lane], r_c, c0, lane,
                           q < 1 || q > g.nz, inx, iny, l_fr);
                float4* Lw = L1 + (i % kL1) * kPlane;
                Lw[j0 * 32 + lane] = l_fr[0];
                Lw[(j0 + 1) * 32 + lane] = l_fr[1];
            }
            __syncthreads();
            if (i >= 4) {
                const int s = zs - 4 + i;  // plane of the level-2 result, in [zs, ze)
                const float4* Lc = L1 + ((i + 1) % kL1) * kPlane;  // level-1 plane s, from iteration i-1
                float4 o[2];
                stage_rows(l_bk, l_cc, l_fr, Lc[jup * 32 + lane], Lc[jdn * 32 + lane], r_pv, c1, lane, false, inx,
                           iny, o);
                if (lane >= kHX / 4 && lane < (kHX + kTX) / 4) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int j = j0 + k;
                        const int y = Y0 + j;
                        if (j < kHY || j >= kHY + kTY || y < 1 || y > g.ny) continue;
                        const int x = X0 + 4 * lane;
                        float* dst = eout + (int64_t)s * g.plane32 + (int64_t)y * g.p32 + x + 3;  // 16-byte aligned
                        if (inx[0] && inx[3]) {
                            *reinterpret_cast<float4*>(dst) = o[k];
                        } else {
                            if (inx[0]) dst[0] = o[k].x;
                            if (inx[1]) dst[1] = o[k].y;
                            if (inx[2]) dst[2] = o[k].z;
                            if (inx[3]) dst[3] = o[k].w;
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                e_bk[k] = e_cc[k]; e_cc[k] = e_fr[k];
                if (i >= 2) { l_bk[k] = l_cc[k]; l_cc[k] = l_fr[k]; r_pv[k] = r_c[k]; }
            }
        }
        cp_async_wait_all();
        __syncthreads();  // the next item's first loads reuse ring slots 0 and 1
    }
}

}  // namespace

cudaError_t tb3_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_sweep3_f32_tb2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_sweep3_f32_tb2(const Geom& g, const float* ein, const float* rin, float* eout, float c0, float c1,
                                  int blocks, cudaStream_t s) {
    if (g.nd != 3 || blocks < 1) return cudaErrorInvalidValue;
    const int tx = (g.nx + kTX - 1) / kTX, ty = (g.ny + kTY - 1) / kTY, ns = (g.nz + kZSeg - 1) / kZSeg;
    const int items = tx * ty * ns;
    const unsigned grid = (unsigned)std::min(blocks, items);
    k_sweep3_f32_tb2<<<grid, kWarps * 32, kSmemBytes, s>>>(ein, rin, eout, g, c0, c1, tx, ty, ns);
    return cudaGetLastError();
}

}  // namespace srj
