// Temporally blocked FP32 SRJ sweep (2-D, 5-point) for sm_103a.
//
// T consecutive weighted-Jacobi steps (Sect. 3.1, Eq. 2nd-order_CD with the
// Poisson source of Sect. 5.1), each with its own weight of the cycle order
// (Sect. 2), are applied to one tile per HBM round trip: the tile of e and of
// the FP32 defect r is brought into shared memory by two TMA tensor loads
// (cp.async.bulk.tensor, completion on an mbarrier), the T steps run out of
// shared memory and registers, and only the tile's centre is written back.
//
// Tile: 128 columns x 64 rows in shared memory.  One warp spans the 128
// columns (a float4 per lane), so the left / right neighbours come from warp
// shuffles; each of the 8 warps owns a band of 8 rows.  After step t the
// values within t cells of the tile edge are stale; with a halo of HX >= T
// columns and T rows the centre (128 - 2 HX) x (64 - 2 T) is exact.  Points
// of the Dirichlet ghost layer and points outside the grid keep their loaded
// value, exactly as in the unblocked sweep, and every update uses the same
// expression, so T blocked steps reproduce T unblocked steps bit for bit.
#include "srj_internal.h"

#include <cuda.h>

#include <algorithm>

namespace srj {

namespace {

constexpr int kSX = 128;  // tile columns (floats)
constexpr int kSY = 64;   // tile rows
constexpr int kWarps = 8;
constexpr int kBand = kSY / kWarps;
constexpr unsigned kTileBytes = kSX * kSY * sizeof(float);
constexpr unsigned long long kWaitNs = 100000000ull;  // give up on a tile load after 100 ms

__device__ inline uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ inline bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ inline unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ inline float upd(float c, float two_d, float cc, float nb, float rr) {
    return fmaf(c, fmaf(-two_d, cc, nb + rr), cc);
}

template <int T>
__global__ void __launch_bounds__(kWarps * 32, 3)
k_sweep_f32_tb(const __grid_constant__ CUtensorMap map_e, const __grid_constant__ CUtensorMap map_r,
               float* __restrict__ eout, Geom g, TbSteps steps, int* __restrict__ err) {
    constexpr int HX = T <= 4 ? 4 : 8;
    extern __shared__ unsigned char smem_raw[];
    float* A = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float* R = A + kSX * kSY;
    __shared__ __align__(8) uint64_t bar;

    constexpr int TX = kSX - 2 * HX;
    constexpr int TY = kSY - 2 * T;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int X0 = 1 + TX * (int)blockIdx.x - HX;  // padded x of tile column 0
    const int Y0 = 1 + TY * (int)blockIdx.y - T;   // padded y of tile row 0

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, 2 * kTileBytes);
        tma_load_2d(A, &map_e, &bar, X0 + 3, Y0);  // float32 column of padded x is x + 3
        tma_load_2d(R, &map_r, &bar, X0 + 3, Y0);
    }
    bool ready = mbar_try_wait(&bar, 0);
    if (!ready) {
        const unsigned long long t0 = global_ns();
        while (!(ready = mbar_try_wait(&bar, 0)) && global_ns() - t0 < kWaitNs) {
        }
    }
    if (__syncthreads_or(!ready)) {  // the whole block gives up together
        if (threadIdx.x == 0) atomicExch(err, 1);
        return;
    }

    const float two_d = 4.0f;
    bool inx[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int x = X0 + 4 * lane + j;
        inx[j] = x >= 1 && x <= g.nx;
    }
    const float4* A4 = reinterpret_cast<const float4*>(A);
    const float4* R4 = reinterpret_cast<const float4*>(R);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const int r0 = w * kBand;

#pragma unroll
    for (int t = 0; t < T; ++t) {
        const float c = steps.c[t];
        float4 out[kBand];
        float4 up = (r0 > 0) ? A4[(r0 - 1) * 32 + lane] : zero;
        float4 cur = A4[r0 * 32 + lane];
#pragma unroll
        for (int i = 0; i < kBand; ++i) {
            const int row = r0 + i;
            const float4 dn = (row + 1 < kSY) ? A4[(row + 1) * 32 + lane] : zero;
            const float4 rr = R4[row * 32 + lane];
            float lf = __shfl_up_sync(0xffffffffu, cur.w, 1);
            float rt = __shfl_down_sync(0xffffffffu, cur.x, 1);
            if (lane == 0) lf = 0.f;
            if (lane == 31) rt = 0.f;
            const int y = Y0 + row;
            const bool iny = y >= 1 && y <= g.ny;
            float4 o;
            o.x = upd(c, two_d, cur.x, ((lf + cur.y) + up.x) + dn.x, rr.x);
            o.y = upd(c, two_d, cur.y, ((cur.x + cur.z) + up.y) + dn.y, rr.y);
            o.z = upd(c, two_d, cur.z, ((cur.y + cur.w) + up.z) + dn.z, rr.z);
            o.w = upd(c, two_d, cur.w, ((cur.z + rt) + up.w) + dn.w, rr.w);
            o.x = (iny && inx[0]) ? o.x : cur.x;
            o.y = (iny && inx[1]) ? o.y : cur.y;
            o.z = (iny && inx[2]) ? o.z : cur.z;
            o.w = (iny && inx[3]) ? o.w : cur.w;
            out[i] = o;
            up = cur;
            cur = dn;
        }
        if (t + 1 < T) {
            __syncthreads();  // every warp has read the old values
#pragma unroll
            for (int i = 0; i < kBand; ++i) reinterpret_cast<float4*>(A)[(r0 + i) * 32 + lane] = out[i];
            __syncthreads();
        } else {
            const int lane_lo = HX / 4, lane_hi = (HX + TX) / 4;  // centre columns
            if (lane < lane_lo || lane >= lane_hi) return;
#pragma unroll
            for (int i = 0; i < kBand; ++i) {
                const int row = r0 + i;
                if (row < T || row >= T + TY) continue;
                const int y = Y0 + row;
                if (y < 1 || y > g.ny) continue;
                const int x = X0 + 4 * lane;
                float* dst = eout + (int64_t)y * g.p32 + x + 3;  // 16-byte aligned
                if (inx[0] && inx[3]) {
                    *reinterpret_cast<float4*>(dst) = out[i];
                } else {
                    if (inx[0]) dst[0] = out[i].x;
                    if (inx[1]) dst[1] = out[i].y;
                    if (inx[2]) dst[2] = out[i].z;
                    if (inx[3]) dst[3] = out[i].w;
                }
            }
        }
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

size_t smem_bytes() { return 2 * (size_t)kTileBytes + 128; }

}  // namespace

int tb_max_steps() { return 8; }

cudaError_t make_tile_map(const Geom& g, const float* base, TileMap* out) {
    static_assert(sizeof(TileMap) >= sizeof(CUtensorMap), "TileMap too small");
    EncodeTiled enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const int64_t rows = (int64_t)(g.ny + 2) * (g.nd == 3 ? (g.nz + 2) : 1);
    cuuint64_t dims[2] = {(cuuint64_t)g.p32, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)g.p32 * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kSX, (cuuint32_t)kSY};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(out->bytes), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                     const_cast<float*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int T>
cudaError_t set_attr() {
    return cudaFuncSetAttribute(k_sweep_f32_tb<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
}

template <int T>
void launch_T(dim3 grd, cudaStream_t s, const CUtensorMap& me, const CUtensorMap& mr, float* eout, const Geom& g,
              const TbSteps& st, int* err) {
    k_sweep_f32_tb<T><<<grd, kWarps * 32, smem_bytes(), s>>>(me, mr, eout, g, st, err);
}

cudaError_t tb_prepare() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    cudaError_t r[8] = {set_attr<1>(), set_attr<2>(), set_attr<3>(), set_attr<4>(),
                        set_attr<5>(), set_attr<6>(), set_attr<7>(), set_attr<8>()};
    for (cudaError_t x : r) if (x != cudaSuccess) e = x;
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_sweep_f32_tb(const Geom& g, const TileMap& map_in, const TileMap& map_r, float* eout,
                                const TbSteps& steps, int* err, cudaStream_t s) {
    if (g.nd != 2 || steps.T < 1 || steps.T > 8) return cudaErrorInvalidValue;
    const CUtensorMap& me = *reinterpret_cast<const CUtensorMap*>(map_in.bytes);
    const CUtensorMap& mr = *reinterpret_cast<const CUtensorMap*>(map_r.bytes);
    const int HX = steps.T <= 4 ? 4 : 8;
    const int TX = kSX - 2 * HX, TY = kSY - 2 * steps.T;
    dim3 grd((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, 1);
    switch (steps.T) {
        case 1: launch_T<1>(grd, s, me, mr, eout, g, steps, err); break;
        case 2: launch_T<2>(grd, s, me, mr, eout, g, steps, err); break;
        case 3: launch_T<3>(grd, s, me, mr, eout, g, steps, err); break;
        case 4: launch_T<4>(grd, s, me, mr, eout, g, steps, err); break;
        case 5: launch_T<5>(grd, s, me, mr, eout, g, steps, err); break;
        case 6: launch_T<6>(grd, s, me, mr, eout, g, steps, err); break;
        case 7: launch_T<7>(grd, s, me, mr, eout, g, steps, err); break;
        default: launch_T<8>(grd, s, me, mr, eout, g, steps, err); break;
    }
    return cudaGetLastError();
}

}  // namespace srj
