// Temporally blocked FP32 SRJ sweep (2-D, 5-point) for sm_103a.
//
// T consecutive weighted-Jacobi steps (Sect. 3.1, Eq. 2nd-order_CD with the
// Poisson source of Sect. 5.1), each with its own weight of the cycle order
// (Sect. 2), are applied to one tile per HBM round trip: the tile of e and of
// the FP32 defect r is loaded once, the T steps run out of registers (band
// edges exchanged through shared memory), and only the tile's centre is
// written back.
//
// Tile: 128 columns x 64 rows.  One warp spans the 128 columns (a float4 per
// lane), so the left / right neighbours come from warp shuffles; each of the
// 8 warps owns a band of 8 rows, held in registers for all T steps.  After step t the
// values within t cells of the tile edge are stale; with a halo of HX >= T
// columns and T rows the centre (128 - 2 HX) x (64 - 2 T) is exact.  Points
// of the Dirichlet ghost layer and points outside the grid keep their loaded
// value, exactly as in the unblocked sweep, and every update uses the same
// expression, so T blocked steps reproduce T unblocked steps bit for bit.
#include "srj_internal.h"

#include <atomic>

#include <algorithm>

namespace srj {

namespace {

constexpr int kSX = 128;  // tile columns (floats)
constexpr int kSY = 64;   // tile rows
constexpr int kWarps = 8;
constexpr int kBand = kSY / kWarps;

// One warp's band of kBand rows lives in registers for all T steps: e[i]
// (float4, 4 consecutive columns per lane) and the defect rr[i].  Only the
// band's top and bottom rows cross warps, through a double-buffered shared
// slot, so each step costs one barrier and four shared-memory accesses per lane.
// MY: some rows of the tile lie outside 1..ny (iny[] is uniform over the warp);
// MX: some columns lie outside 1..nx.  Those points keep their value.
// cs[t]: weight / 4 of step t.
template <int T, bool MY, bool MX, int W = kWarps>
__device__ __forceinline__ void band_steps(float4 (&e)[kBand], const float4 (&rr)[kBand], float4* xch,
                                           const float (&cs)[8], int lane, int w, const bool (&inx)[4],
                                           const bool (&iny)[kBand]) {
    const float two_d = 4.0f;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float2 m4 = make_float2(-two_d, -two_d);
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const float2 cv = make_float2(cs[t], cs[t]);
        float4* slot = xch + (t & 1) * (2 * W * 32);
        slot[(2 * w) * 32 + lane] = e[0];              // top row of this band
        slot[(2 * w + 1) * 32 + lane] = e[kBand - 1];  // bottom row
        __syncthreads();
        const float4 above = (w > 0) ? slot[(2 * (w - 1) + 1) * 32 + lane] : zero;
        const float4 below = (w + 1 < W) ? slot[(2 * (w + 1)) * 32 + lane] : zero;
        float4 up = above;  // old value of the row above the one being updated
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const float4 cur = e[i];
            const float4 dn = (i + 1 < kBand) ? e[i + 1] : below;
            // Single-step update in FP32x2 form: per component the unblocked
            // sweep's fmaf(c, fmaf(-4, e, t), e) with
            // t = ((up + down) + r) + (left + right), same operations, same
            // order.  The vertical part needs no other lane, so it is formed
            // while the horizontal neighbours travel by shuffle.  The left +
            // right sums are scalar adds whose results land directly in the
            // (x,y) / (z,w) pairs; pairing the misaligned neighbours for a packed
            // add would cost more register moves than the adds it saves.
            float2 v0 = __fadd2_rn(make_float2(up.x, up.y), make_float2(dn.x, dn.y));
            float2 v1 = __fadd2_rn(make_float2(up.z, up.w), make_float2(dn.z, dn.w));
            v0 = __fadd2_rn(v0, make_float2(rr[i].x, rr[i].y));
            v1 = __fadd2_rn(v1, make_float2(rr[i].z, rr[i].w));
            // lanes 0 and 31 receive their own values: those columns lie in the
            // stale halo of the tile, so what they compute is never stored
            const float lf = __shfl_up_sync(0xffffffffu, cur.w, 1);
            const float rt = __shfl_down_sync(0xffffffffu, cur.x, 1);
            const float2 s0 = __fadd2_rn(v0, make_float2(lf + cur.y, cur.x + cur.z));
            const float2 s1 = __fadd2_rn(v1, make_float2(cur.y + cur.w, cur.z + rt));
            const float2 c0 = make_float2(cur.x, cur.y), c1 = make_float2(cur.z, cur.w);
            const float2 o0 = __ffma2_rn(cv, __ffma2_rn(m4, c0, s0), c0);
            const float2 o1 = __ffma2_rn(cv, __ffma2_rn(m4, c1, s1), c1);
            float4 o = make_float4(o0.x, o0.y, o1.x, o1.y);
            if (MX) {
                o.x = inx[0] ? o.x : cur.x;
                o.y = inx[1] ? o.y : cur.y;
                o.z = inx[2] ? o.z : cur.z;
                o.w = inx[3] ? o.w : cur.w;
            }
            if (MY && !iny[i]) o = cur;
            up = cur;
            e[i] = o;
        }
    }
}

// L2 prefetch of the rows of e and of the defect that a warp will load for the
// tile (bx, by): kBand rows of 128 floats from column X0 + 3 (512 bytes, five
// 128-byte lines at most) per array.  Lane (i, part) covers line `part` of row i.
template <int T, int SY>
__device__ __forceinline__ void prefetch_tile_l2(const float* ein, const float* rin, const Geom& g, int bx, int by,
                                                 int lane, int w) {
    constexpr int HX = T <= 4 ? 4 : 8;
    constexpr int TX = kSX - 2 * HX, TY = SY - 2 * T;
    const int X0 = 1 + TX * bx - HX, Y0 = 1 + TY * by - T;
    const int64_t y = (int64_t)Y0 + w * kBand + (lane >> 2);
    const int part = lane & 3;
    const int64_t rows = g.ny + 2;
    if (y < 0 || y >= rows) return;
    const int64_t c = X0 + 3 + part * 32;
    if (c >= g.p32) return;  // every address stays inside row y of the buffer
    const int64_t off = y * g.p32 + (c < 0 ? 0 : c);
    const int64_t off2 = y * g.p32 + X0 + 3 + 127;  // last float of the row segment (fifth line)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ein + off));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(rin + off));
    if (part == 3 && X0 + 3 + 127 < g.p32) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ein + off2));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(rin + off2));
    }
}

// Single grid, T steps per launch.  Block (bx, by) owns the tile whose first
// column / row has padded coordinates X0 = 1 + TX bx - HX, Y0 = 1 + TY by - T;
// interior tiles (the vast majority) load and store without bounds checks.
// PF: after issuing its own loads, each block
// prefetches into L2 the rows of the tile pf_dist blocks further on in launch
// order (the tile that starts on a multiprocessor when a resident block ends),
// so that the next wave's loads are served from L2 while this wave computes.
template <int T, int W, bool PF = false>
__global__ void __launch_bounds__(W * 32, 16 / W)
k_sweep_f32_tb(const float* __restrict__ ein, const float* __restrict__ rin, float* __restrict__ eout, Geom g,
               TbSteps steps, int pf_dist = 0) {
    constexpr int HX = T <= 4 ? 4 : 8;
    constexpr int SY = W * kBand;
    constexpr int TX = kSX - 2 * HX, TY = SY - 2 * T;
    __shared__ float4 xch[2 * 2 * W * 32];  // [slot][warp][top/bottom][lane]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int X0 = 1 + TX * (int)blockIdx.x - HX, Y0 = 1 + TY * (int)blockIdx.y - T;
    const int Yw = Y0 + w * kBand;  // this warp's first row
    const bool xin = X0 >= 1 && X0 + kSX - 1 <= g.nx;
    const bool yin = Y0 >= 1 && Y0 + SY - 1 <= g.ny;
    const int64_t base = (int64_t)Yw * g.p32 + X0 + 3 + 4 * lane;  // this lane's float4 of row Yw
    float4 e[kBand], rr[kBand];
    bool iny[kBand];
    if (xin && yin) {
        const float4* pe = reinterpret_cast<const float4*>(ein + base);
        const float4* pr = reinterpret_cast<const float4*>(rin + base);
        const int64_t stride = g.p32 / 4;  // p32 is a multiple of 32
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            e[i] = __ldg(pe + i * stride);
            rr[i] = __ldg(pr + i * stride);
            iny[i] = true;
        }
    } else {
        // float32 column of padded x is x + 3, a multiple of 4 here: each
        // float4 lies wholly inside or outside the buffer; outside reads as 0
        const int col = X0 + 3 + 4 * lane;
        const bool colok = col >= 0 && col + 4 <= g.p32;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int64_t y = (int64_t)Yw + i;
            e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            rr[i] = e[i];
            if (colok && y >= 0 && y < (int64_t)g.ny + 2) {
                const int64_t off = y * g.p32 + col;
                e[i] = __ldg(reinterpret_cast<const float4*>(ein + off));
                rr[i] = __ldg(reinterpret_cast<const float4*>(rin + off));
            }
            iny[i] = y >= 1 && y <= g.ny;
        }
    }
    if (PF) {
        const int lin = (int)(blockIdx.y * gridDim.x + blockIdx.x) + pf_dist;
        if (lin < (int)(gridDim.x * gridDim.y))
            prefetch_tile_l2<T, SY>(ein, rin, g, lin % (int)gridDim.x, lin / (int)gridDim.x, lane, w);
    }
    bool inx[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = X0 + 4 * lane + j;
        inx[j] = x >= 1 && x <= g.nx;
    }
    if (xin && yin) band_steps<T, false, false, W>(e, rr, xch, steps.c, lane, w, inx, iny);
    else if (xin)   band_steps<T, true, false, W>(e, rr, xch, steps.c, lane, w, inx, iny);
    else if (yin)   band_steps<T, false, true, W>(e, rr, xch, steps.c, lane, w, inx, iny);
    else            band_steps<T, true, true, W>(e, rr, xch, steps.c, lane, w, inx, iny);

    // store the centre: rows T .. T+TY-1, columns HX .. HX+TX-1 of the tile
    const int lane_lo = HX / 4, lane_hi = (HX + TX) / 4;
    if (lane < lane_lo || lane >= lane_hi) return;
    if (xin && yin) {
        float4* po = reinterpret_cast<float4*>(eout + base);
        const int64_t stride = g.p32 / 4;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int row = w * kBand + i;
            if (row >= T && row < T + TY) po[i * stride] = e[i];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kBand; ++i) {
        const int row = w * kBand + i;
        if (row < T || row >= T + TY) continue;
        const int y = Y0 + row;
        if (y < 1 || y > g.ny) continue;
        const int x = X0 + 4 * lane;
        float* dst = eout + (int64_t)y * g.p32 + x + 3;  // 16-byte aligned
        if (inx[0] && inx[3]) {
            *reinterpret_cast<float4*>(dst) = e[i];
        } else {
            if (inx[0]) dst[0] = e[i].x;
            if (inx[1]) dst[1] = e[i].y;
            if (inx[2]) dst[2] = e[i].z;
            if (inx[3]) dst[3] = e[i].w;
        }
    }
}

// ---- bulk-copy prefetch (persistent form) ----------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase `parity` of the barrier to complete, for at most limit_ns
// nanoseconds of wall time.  Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// One-dimensional bulk copy global -> shared (16-byte aligned addresses, size a
// multiple of 16), completing `bytes` transactions on the barrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Persistent form with a bulk-copy prefetch: gridDim.x blocks (W = 8: two per
// SM, W = 16: one) walk the tiles (x fastest).  Warp 0 issues the next tile's
// rows of e and of the defect as one bulk copy per row into a shared staging
// area while the block computes the current tile, so that a tile's loads
// overlap the previous tile's steps instead of following them.  Only the part
// of each row that lies inside the buffer is copied; the rest of the staging
// area keeps stale values, which only ever reach points outside the interior
// (held fixed), exactly like the zeros of the direct-load form, so the stored
// centre is the same bit for bit.
//
// Each wait on the staging barrier is bounded (limit_ns of wall time): when it
// runs out, the block records SRJ_ERR_TIMEOUT in *status, waits once more
// (bounded) for its copies in flight, and returns.  stall != 0 is a self-test
// of that path: the block waits on a barrier phase that nothing completes.
template <int T, int W>
__global__ void __launch_bounds__(W * 32, 16 / W)
k_sweep_f32_tbq(const float* __restrict__ ein, const float* __restrict__ rin, float* __restrict__ eout, Geom g,
                TbSteps steps, int tiles_x, int ntiles, int* __restrict__ status, uint64_t limit_ns, int stall) {
    constexpr int HX = T <= 4 ? 4 : 8;
    constexpr int SY = W * kBand;
    constexpr int TX = kSX - 2 * HX, TY = SY - 2 * T;
    __shared__ float4 xch[2 * 2 * W * 32];
    __shared__ __align__(8) unsigned long long full_bar;
    extern __shared__ __align__(128) float4 stage[];  // [SY][32] rows of e, then [SY][32] rows of the defect
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t bar = smem_addr(&full_bar);
    const uint32_t sbase = smem_addr(stage);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int tile) {  // warp 0 only
        const int bx = tile % tiles_x, by = tile / tiles_x;
        const int X0 = 1 + TX * bx - HX, Y0 = 1 + TY * by - T;
        const int col0 = X0 + 3;  // float32 column of the tile's first point: a multiple of 4
        const int c0 = max(col0, 0), c1 = min(col0 + kSX, (int)g.p32);
        const int y0 = max(Y0, 0), y1 = min(Y0 + SY, g.ny + 2);
        const uint32_t bytes = (uint32_t)(c1 - c0) * 4u;
        if (lane == 0) mbar_arrive_expect_tx(bar, 2u * (uint32_t)(y1 - y0) * bytes);
        __syncwarp();
        const uint32_t dcol = (uint32_t)(c0 - col0) * 4u;
#pragma unroll
        for (int r = lane; r < SY; r += 32) {
            const int y = Y0 + r;
            if (y >= y0 && y < y1) {
                const int64_t off = (int64_t)y * g.p32 + c0;
                bulk_g2s(sbase + (uint32_t)r * 512u + dcol, ein + off, bytes, bar);
                bulk_g2s(sbase + (uint32_t)(SY + r) * 512u + dcol, rin + off, bytes, bar);
            }
        }
    };

    int tile = blockIdx.x;
    if (w == 0 && !stall) issue(tile);
    uint32_t parity = 0;
    for (; tile < ntiles; tile += gridDim.x, parity ^= 1u) {
        const int bx = tile % tiles_x, by = tile / tiles_x;
        const int X0 = 1 + TX * bx - HX, Y0 = 1 + TY * by - T;
        const bool ok = mbar_wait_bounded(bar, parity, limit_ns);
        float4 e[kBand], rr[kBand];
        bool iny[kBand];
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int row = w * kBand + i;
            e[i] = stage[row * 32 + lane];
            rr[i] = stage[(SY + row) * 32 + lane];
            const int y = Y0 + row;
            iny[i] = y >= 1 && y <= g.ny;
        }
        // every thread has read the staging area (and the barrier phase) before
        // warp 0 refills it; the outcome of the waits is uniform over the block
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) {
                atomicExch(status, kStatusTimeout);
                mbar_wait_bounded(bar, parity, limit_ns);  // copies still in flight land first
            }
            return;
        }
        if (w == 0 && tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
        bool inx[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = X0 + 4 * lane + j;
            inx[j] = x >= 1 && x <= g.nx;
        }
        const bool xin = X0 >= 1 && X0 + kSX - 1 <= g.nx;
        const bool yin = Y0 >= 1 && Y0 + SY - 1 <= g.ny;
        if (xin && yin) band_steps<T, false, false, W>(e, rr, xch, steps.c, lane, w, inx, iny);
        else if (xin)   band_steps<T, true, false, W>(e, rr, xch, steps.c, lane, w, inx, iny);
        else if (yin)   band_steps<T, false, true, W>(e, rr, xch, steps.c, lane, w, inx, iny);
        else            band_steps<T, true, true, W>(e, rr, xch, steps.c, lane, w, inx, iny);
        const int lane_lo = HX / 4, lane_hi = (HX + TX) / 4;
        if (lane >= lane_lo && lane < lane_hi) {
            if (xin && yin) {
                float4* po = reinterpret_cast<float4*>(eout + (int64_t)(Y0 + w * kBand) * g.p32 + X0 + 3 + 4 * lane);
                const int64_t stride = g.p32 / 4;
#pragma unroll
                for (int i = 0; i < kBand; ++i) {
                    const int row = w * kBand + i;
                    if (row >= T && row < T + TY) po[i * stride] = e[i];
                }
            } else {
#pragma unroll
                for (int i = 0; i < kBand; ++i) {
                    const int row = w * kBand + i;
                    if (row < T || row >= T + TY) continue;
                    const int y = Y0 + row;
                    if (y < 1 || y > g.ny) continue;
                    float* dst = eout + (int64_t)y * g.p32 + X0 + 3 + 4 * lane;
                    if (inx[0] && inx[3]) {
                        *reinterpret_cast<float4*>(dst) = e[i];
                    } else {
                        if (inx[0]) dst[0] = e[i].x;
                        if (inx[1]) dst[1] = e[i].y;
                        if (inx[2]) dst[2] = e[i].z;
                        if (inx[3]) dst[3] = e[i].w;
                    }
                }
            }
        }
        // the next tile's first exchange must not overwrite a slot a slower
        // warp is still reading in this tile's last step (odd T)
        if (T & 1) __syncthreads();
    }
}

// Batched form: one launch covers the tiles of every problem of a batch; each
// block finds its problem in the tile table and advances it by
// n = min(T, M - k) steps of its own cycle order.  Problems that have finished
// are skipped.  Every tile runs T steps: the record's weights past step n are
// zero, and a step with weight zero returns each point's value unchanged
// (fma(0, y, e) = e for finite y), so the tile holds the same values as after n
// steps.  A runtime step count in the unrolled step loop instead made the
// compiler spill several hundred bytes of registers (-Xptxas -v).
template <int T>
__global__ void __launch_bounds__(kWarps * 32, 2)
k_batch_sweep_tb(const int4* __restrict__ tiles, const BatchArgs* __restrict__ args) {
    constexpr int HX = T <= 4 ? 4 : 8;
    constexpr int TX = kSX - 2 * HX, TY = kSY - 2 * T;
    __shared__ float4 xch[2 * 2 * kWarps * 32];
    const int4 tl = tiles[blockIdx.x];
    const BatchArgs* __restrict__ Ap = args + tl.x;
    struct { const float* ein; float* eout; const float* r32; int64_t p32; int nx, ny, fresh; } A;
    const int n = Ap->n;
    if (n == 0) return;  // problem no longer iterating (uniform over the block)
    A.ein = Ap->ein; A.eout = Ap->eout; A.r32 = Ap->r32; A.p32 = Ap->p32;
    A.nx = Ap->nx; A.ny = Ap->ny; A.fresh = Ap->fresh;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int X0 = 1 + TX * tl.y - HX, Y0 = 1 + TY * tl.z - T;
    const int Yw = Y0 + w * kBand;
    const bool xin = X0 >= 1 && X0 + kSX - 1 <= A.nx;
    const bool yin = Y0 >= 1 && Y0 + kSY - 1 <= A.ny;
    const int64_t base = (int64_t)Yw * A.p32 + X0 + 3 + 4 * lane;
    float4 e[kBand], rr[kBand];
    bool iny[kBand];
    if (xin && yin) {
        const float4* pe = reinterpret_cast<const float4*>(A.ein + base);
        const float4* pr = reinterpret_cast<const float4*>(A.r32 + base);
        const int64_t stride = A.p32 / 4;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!A.fresh) e[i] = __ldg(pe + i * stride);
            rr[i] = __ldg(pr + i * stride);
            iny[i] = true;
        }
    } else {
        const int col = X0 + 3 + 4 * lane;
        const bool colok = col >= 0 && col + 4 <= A.p32;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int64_t y = (int64_t)Yw + i;
            e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            rr[i] = e[i];
            if (colok && y >= 0 && y < (int64_t)A.ny + 2) {
                const int64_t off = y * A.p32 + col;
                if (!A.fresh) e[i] = __ldg(reinterpret_cast<const float4*>(A.ein + off));
                rr[i] = __ldg(reinterpret_cast<const float4*>(A.r32 + off));
            }
            iny[i] = y >= 1 && y <= A.ny;
        }
    }
    bool inx[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = X0 + 4 * lane + j;
        inx[j] = x >= 1 && x <= A.nx;
    }
    if (xin && yin) band_steps<T, false, false>(e, rr, xch, Ap->c, lane, w, inx, iny);
    else if (xin)   band_steps<T, true, false>(e, rr, xch, Ap->c, lane, w, inx, iny);
    else if (yin)   band_steps<T, false, true>(e, rr, xch, Ap->c, lane, w, inx, iny);
    else            band_steps<T, true, true>(e, rr, xch, Ap->c, lane, w, inx, iny);
    const int lane_lo = HX / 4, lane_hi = (HX + TX) / 4;
    if (lane < lane_lo || lane >= lane_hi) return;
    if (xin && yin) {
        float4* po = reinterpret_cast<float4*>(A.eout + base);
        const int64_t stride = A.p32 / 4;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int row = w * kBand + i;
            if (row >= T && row < T + TY) po[i * stride] = e[i];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kBand; ++i) {
        const int row = w * kBand + i;
        if (row < T || row >= T + TY) continue;
        const int y = Y0 + row;
        if (y < 1 || y > A.ny) continue;
        const int x = X0 + 4 * lane;
        float* dst = A.eout + (int64_t)y * A.p32 + x + 3;
        if (inx[0] && inx[3]) {
            *reinterpret_cast<float4*>(dst) = e[i];
        } else {
            if (inx[0]) dst[0] = e[i].x;
            if (inx[1]) dst[1] = e[i].y;
            if (inx[2]) dst[2] = e[i].z;
            if (inx[3]) dst[3] = e[i].w;
        }
    }
}

// Batched sweep over problems grouped by grid size (BatchGroups): a block
// derives its problem, tile and workspaces from the launch parameters, so its
// loads of e and of the defect issue at once, and the problem's record of this
// phase (steps, zero start, weights) is read alongside them.  Reading the
// record first, as k_batch_sweep_tb does, puts a dependent load ahead of every
// tile; on full-grid tiles that cost about a fifth of the sweep time.  The
// input correction is read even at a cycle start (zero start) and then
// replaced by zeros, which is what the tile-list kernel computes.  Like the
// tile-list kernel it always runs T steps, with zero weights past the record's
// step count.
template <int T>
__global__ void __launch_bounds__(kWarps * 32, 2)
k_batch_sweep_grp(const BatchGroups G, float* __restrict__ pool, const BatchArgs* __restrict__ args, int parity) {
    constexpr int HX = T <= 4 ? 4 : 8;
    constexpr int TX = kSX - 2 * HX, TY = kSY - 2 * T;
    __shared__ float4 xch[2 * 2 * kWarps * 32];
    __shared__ float csh[8];
    const int bid = (int)blockIdx.x;
    int g = 0;
#pragma unroll 1
    while (g + 1 < G.ngroups && bid >= G.tile_begin[g + 1]) ++g;
    const int gx = G.gx[g];
    const int local = bid - G.tile_begin[g];
    const int tpp = gx * G.gy[g];
    const int z = local / tpp;
    const int rem = local - z * tpp;
    const int by = rem / gx, bx = rem - by * gx;
    const int nx = G.nx[g], ny = G.ny[g];
    const int64_t p32 = G.p32[g], n32 = G.n32[g];
    const int m = G.member[G.mbase[g] + z];
    float* const wbase = pool + G.off[g] + (int64_t)m * 3 * n32;
    const float* ein = wbase + (parity ? n32 : 0);
    float* eout = wbase + (parity ? 0 : n32);
    const float* rin = wbase + 2 * n32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int X0 = 1 + TX * bx - HX, Y0 = 1 + TY * by - T;
    const int Yw = Y0 + w * kBand;
    const bool xin = X0 >= 1 && X0 + kSX - 1 <= nx;
    const bool yin = Y0 >= 1 && Y0 + kSY - 1 <= ny;
    const int64_t base = (int64_t)Yw * p32 + X0 + 3 + 4 * lane;
    float4 e[kBand], rr[kBand];
    bool iny[kBand];
    if (xin && yin) {
        const float4* pe = reinterpret_cast<const float4*>(ein + base);
        const float4* pr = reinterpret_cast<const float4*>(rin + base);
        const int64_t stride = p32 / 4;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            e[i] = __ldg(pe + i * stride);
            rr[i] = __ldg(pr + i * stride);
            iny[i] = true;
        }
    } else {
        const int col = X0 + 3 + 4 * lane;
        const bool colok = col >= 0 && col + 4 <= p32;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int64_t y = (int64_t)Yw + i;
            e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            rr[i] = e[i];
            if (colok && y >= 0 && y < (int64_t)ny + 2) {
                const int64_t off = y * p32 + col;
                e[i] = __ldg(reinterpret_cast<const float4*>(ein + off));
                rr[i] = __ldg(reinterpret_cast<const float4*>(rin + off));
            }
            iny[i] = y >= 1 && y <= ny;
        }
    }
    const BatchArgs* __restrict__ Ap = args + G.rec[g] + m;
    const int n = Ap->n;
    const int fresh = Ap->fresh;
    if (threadIdx.x < 8) csh[threadIdx.x] = Ap->c[threadIdx.x];
    if (n == 0) return;  // problem no longer iterating (uniform over the block)
    if (fresh) {
#pragma unroll
        for (int i = 0; i < kBand; ++i) e[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    bool inx[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = X0 + 4 * lane + j;
        inx[j] = x >= 1 && x <= nx;
    }
    __syncthreads();  // the weights in csh
    if (xin && yin) {
        band_steps<T, false, false>(e, rr, xch, csh, lane, w, inx, iny);
    } else if (xin) {
        band_steps<T, true, false>(e, rr, xch, csh, lane, w, inx, iny);
    } else if (yin) {
        band_steps<T, false, true>(e, rr, xch, csh, lane, w, inx, iny);
    } else {
        band_steps<T, true, true>(e, rr, xch, csh, lane, w, inx, iny);
    }
    const int lane_lo = HX / 4, lane_hi = (HX + TX) / 4;
    if (lane < lane_lo || lane >= lane_hi) return;
    if (xin && yin) {
        float4* po = reinterpret_cast<float4*>(eout + base);
        const int64_t stride = p32 / 4;
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int row = w * kBand + i;
            if (row >= T && row < T + TY) po[i * stride] = e[i];
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < kBand; ++i) {
        const int row = w * kBand + i;
        if (row < T || row >= T + TY) continue;
        const int y = Y0 + row;
        if (y < 1 || y > ny) continue;
        const int x = X0 + 4 * lane;
        float* dst = eout + (int64_t)y * p32 + x + 3;
        if (inx[0] && inx[3]) {
            *reinterpret_cast<float4*>(dst) = e[i];
        } else {
            if (inx[0]) dst[0] = e[i].x;
            if (inx[1]) dst[1] = e[i].y;
            if (inx[2]) dst[2] = e[i].z;
            if (inx[3]) dst[3] = e[i].w;
        }
    }
}

size_t smem_bytes() { return 0; }

}  // namespace

int tb_max_steps() { return 8; }

template <int W>
constexpr size_t stage_bytes() { return 2 * (size_t)W * kBand * 32 * sizeof(float4); }  // W = 8: 64 KB

template <int T, int W>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_sweep_f32_tbq<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)stage_bytes<W>());
}

template <int T, int W>
void launch_P(unsigned grid, cudaStream_t s, const float* ein, const float* rin, float* eout, const Geom& g,
              const TbSteps& st, int tiles_x, int ntiles, int* status, uint64_t limit_ns, int stall) {
    k_sweep_f32_tbq<T, W><<<grid, W * 32, stage_bytes<W>(), s>>>(ein, rin, eout, g, st, tiles_x, ntiles, status,
                                                                  limit_ns, stall);
}

template <int W>
void launch_PW(int T, unsigned grid, cudaStream_t s, const float* ein, const float* rin, float* eout, const Geom& g,
               const TbSteps& st, int tiles_x, int ntiles, int* status, uint64_t limit_ns, int stall) {
    switch (T) {
        case 2: launch_P<2, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
        case 3: launch_P<3, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
        case 4: launch_P<4, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
        case 5: launch_P<5, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
        case 6: launch_P<6, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
        case 7: launch_P<7, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
        default: launch_P<8, W>(grid, s, ein, rin, eout, g, st, tiles_x, ntiles, status, limit_ns, stall); break;
    }
}

template <int T, int W>
void launch_T(dim3 grd, cudaStream_t s, const float* ein, const float* rin, float* eout, const Geom& g,
              const TbSteps& st, int pf_dist) {
    if (pf_dist > 0) k_sweep_f32_tb<T, W, true><<<grd, W * 32, smem_bytes(), s>>>(ein, rin, eout, g, st, pf_dist);
    else             k_sweep_f32_tb<T, W, false><<<grd, W * 32, smem_bytes(), s>>>(ein, rin, eout, g, st, 0);
}

template <int W>
void launch_W(int T, dim3 grd, cudaStream_t s, const float* ein, const float* rin, float* eout, const Geom& g,
              const TbSteps& st, int pf_dist) {
    switch (T) {
        case 1: launch_T<1, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        case 2: launch_T<2, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        case 3: launch_T<3, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        case 4: launch_T<4, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        case 5: launch_T<5, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        case 6: launch_T<6, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        case 7: launch_T<7, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
        default: launch_T<8, W>(grd, s, ein, rin, eout, g, st, pf_dist); break;
    }
}

template <int T>
void launch_batch_T(unsigned ntiles, cudaStream_t s, const int4* tiles, const BatchArgs* args) {
    k_batch_sweep_tb<T><<<ntiles, kWarps * 32, 0, s>>>(tiles, args);
}

template <int T>
void launch_batch_grp_T(unsigned ntiles, cudaStream_t s, const BatchGroups& G, float* pool, const BatchArgs* args,
                        int parity) {
    k_batch_sweep_grp<T><<<ntiles, kWarps * 32, 0, s>>>(G, pool, args, parity);
}

cudaError_t tb_prepare() {
    // kernel attributes are per device: set them once on each device used
    static std::atomic<bool> done[64] = {};  // idempotent setup; concurrent first calls both set
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    cudaError_t r[14] = {set_attr<2, 8>(),  set_attr<3, 8>(),  set_attr<4, 8>(),  set_attr<5, 8>(),
                         set_attr<6, 8>(),  set_attr<7, 8>(),  set_attr<8, 8>(),  set_attr<2, 16>(),
                         set_attr<3, 16>(), set_attr<4, 16>(), set_attr<5, 16>(), set_attr<6, 16>(),
                         set_attr<7, 16>(), set_attr<8, 16>()};
    for (cudaError_t x : r) if (x != cudaSuccess) e = x;
    if (e == cudaSuccess) done[dev].store(true, std::memory_order_release);
    return e;
}

cudaError_t launch_sweep_f32_tb(const Geom& g, const float* ein, const float* rin, float* eout,
                                const TbSteps& steps, int warps, cudaStream_t s, int pf_dist) {
    if (g.nd != 2 || steps.T < 1 || steps.T > 8 || (warps != 8 && warps != 16) || pf_dist < 0)
        return cudaErrorInvalidValue;
    const int HX = steps.T <= 4 ? 4 : 8;
    const int TX = kSX - 2 * HX, TY = warps * kBand - 2 * steps.T;
    dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, 1);
    if (warps == 16) launch_W<16>(steps.T, grd, s, ein, rin, eout, g, steps, pf_dist);
    else             launch_W<8>(steps.T, grd, s, ein, rin, eout, g, steps, pf_dist);
    return cudaGetLastError();
}

cudaError_t launch_sweep_f32_tbp(const Geom& g, const float* ein, const float* rin, float* eout,
                                 const TbSteps& steps, int warps, int blocks_per_sm, int sms, int* status,
                                 cudaStream_t s, uint64_t limit_ns, int stall) {
    if (g.nd != 2 || steps.T < 2 || steps.T > 8 || (warps != 8 && warps != 16) || sms < 1 || blocks_per_sm < 1 ||
        !status)
        return cudaErrorInvalidValue;
    const int HX = steps.T <= 4 ? 4 : 8;
    const int TX = kSX - 2 * HX, TY = warps * kBand - 2 * steps.T;
    const int tx = (g.nx + TX - 1) / TX, ty = (g.ny + TY - 1) / TY;
    const int ntiles = tx * ty;
    const unsigned grid = (unsigned)std::min(blocks_per_sm * sms, ntiles);
    if (warps == 16) launch_PW<16>(steps.T, grid, s, ein, rin, eout, g, steps, tx, ntiles, status, limit_ns, stall);
    else             launch_PW<8>(steps.T, grid, s, ein, rin, eout, g, steps, tx, ntiles, status, limit_ns, stall);
    return cudaGetLastError();
}

void tb_tile_shape(int T, int* TX, int* TY) {
    const int HX = T <= 4 ? 4 : 8;
    *TX = kSX - 2 * HX;
    *TY = kSY - 2 * T;
}

cudaError_t launch_batch_sweep_grouped(int T, unsigned ntiles, const BatchGroups& G, float* pool,
                                       const BatchArgs* args, int parity, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    if (G.ngroups < 1 || G.ngroups > kMaxBatchGroups || G.tile_begin[G.ngroups] != (int)ntiles)
        return cudaErrorInvalidValue;
    switch (T) {
        case 1: launch_batch_grp_T<1>(ntiles, s, G, pool, args, parity); break;
        case 2: launch_batch_grp_T<2>(ntiles, s, G, pool, args, parity); break;
        case 3: launch_batch_grp_T<3>(ntiles, s, G, pool, args, parity); break;
        case 4: launch_batch_grp_T<4>(ntiles, s, G, pool, args, parity); break;
        case 5: launch_batch_grp_T<5>(ntiles, s, G, pool, args, parity); break;
        case 6: launch_batch_grp_T<6>(ntiles, s, G, pool, args, parity); break;
        case 7: launch_batch_grp_T<7>(ntiles, s, G, pool, args, parity); break;
        default: launch_batch_grp_T<8>(ntiles, s, G, pool, args, parity); break;
    }
    return cudaGetLastError();
}

cudaError_t batch_sweep_set_node(cudaGraphExec_t exec, cudaGraphNode_t node, unsigned ntiles, const BatchGroups* G) {
    if (ntiles == 0) return cudaErrorInvalidValue;
    cudaKernelNodeParams p{};
    cudaError_t e = cudaGraphKernelNodeGetParams(node, &p);
    if (e != cudaSuccess) return e;
    p.gridDim = dim3(ntiles, 1, 1);
    if (!G) return cudaGraphExecKernelNodeSetParams(exec, node, &p);
    // grouped sweep: (const BatchGroups G, float* pool, const BatchArgs* args, int parity)
    void* kp[4] = {const_cast<BatchGroups*>(G), p.kernelParams[1], p.kernelParams[2], p.kernelParams[3]};
    p.kernelParams = kp;
    return cudaGraphExecKernelNodeSetParams(exec, node, &p);
}

cudaError_t launch_batch_sweep_tb(int T, unsigned ntiles, const int4* tiles, const BatchArgs* args, cudaStream_t s) {
    if (ntiles == 0) return cudaSuccess;
    switch (T) {
        case 1: launch_batch_T<1>(ntiles, s, tiles, args); break;
        case 2: launch_batch_T<2>(ntiles, s, tiles, args); break;
        case 3: launch_batch_T<3>(ntiles, s, tiles, args); break;
        case 4: launch_batch_T<4>(ntiles, s, tiles, args); break;
        case 5: launch_batch_T<5>(ntiles, s, tiles, args); break;
        case 6: launch_batch_T<6>(ntiles, s, tiles, args); break;
        case 7: launch_batch_T<7>(ntiles, s, tiles, args); break;
        default: launch_batch_T<8>(ntiles, s, tiles, args); break;
    }
    return cudaGetLastError();
}

}  // namespace srj
