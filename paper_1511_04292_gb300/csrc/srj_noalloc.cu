// Allocation-free variant of the FP32 sweep entry point (srj_steps_f32_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a few
// sweeps: code that owns all device memory through its own fixed pool and
// forbids foreign cudaMalloc calls, and latency-critical loops where cudaMalloc /
// cudaFree would synchronise the device.  For them this entry point keeps the
// FP32 sweep's work buffers (two iterates and the FP32 source) in one
// file-scope device array of fixed size instead of a plan's cudaMalloc'd
// workspaces.
//
// The array is part of the library image: every GPU that loads the library
// holds it (kNoAllocBytes) until the process exits.  Its device address is
// looked up with cudaGetSymbolAddress on the first call made in a device's
// CUDA context, and again on the first call after that context has been
// replaced (cudaDeviceReset and a new context on the same device); that lookup
// allocates nothing.  All calls share the array and it keeps the last call's
// contents, so each call clears the parts it uses; calls whose GPU work
// overlaps (on different streams, or from different host threads) race on it.
#include "srj_internal.h"
#include "../../include/srj.h"

#include <cmath>
#include <cstdio>
#include <mutex>

namespace {

// 3 work buffers of kNoAllocFloats floats each (pitched FP32 layout).
constexpr int64_t kNoAllocFloats = int64_t(1) << 20;  // 4 MiB per buffer
constexpr int64_t kNoAllocBytes = 3 * kNoAllocFloats * 4;

static __device__ __align__(256) float g_noalloc_scratch[3 * kNoAllocFloats];
static_assert(sizeof(g_noalloc_scratch) == kNoAllocBytes, "scratch size");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // id of the context the address belongs to

// Unique id of the calling thread's current CUDA context (driver entry points
// cuCtxGetCurrent / cuCtxGetId, found through the runtime; no link to libcuda).
// Returns false when the driver does not provide them.
bool current_context_id(unsigned long long* id) {
    typedef int (*get_current_t)(void**);
    typedef int (*get_id_t)(void*, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<get_current_t>(f1);
            get_id = reinterpret_cast<get_id_t>(f2);
        }
        looked_up = true;
    }
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

thread_local char g_noalloc_err[256];

int noalloc_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
    if (e != cudaSuccess) std::snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s: %s", msg, cudaGetErrorString(e));
    else std::snprintf(g_noalloc_err, sizeof g_noalloc_err, "%s", msg);
    return code;
}

// Device address of the static array for the current device (set-up on first use).
int scratch_for_current_device(float** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "cudaGetDevice failed", e);
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SRJ_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long ctx = 0;  // no current context yet: look the address up (which creates it)
    const bool have_ctx = current_context_id(&ctx);
    if (!g_scratch_addr[dev] || !have_ctx || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return noalloc_fail(SRJ_ERR_CUDA, "cudaGetSymbolAddress(scratch) failed", e);
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = have_ctx ? ctx : 0;
    }
    *out = static_cast<float*>(g_scratch_addr[dev]);
    return SRJ_OK;
}

}  // namespace

extern "C" const char* srj_noalloc_last_error(void) { return g_noalloc_err; }

extern "C" int srj_steps_f32_noalloc(int ndim, const int64_t* dims, double h, int64_t count,
                                     const double* omega_seq, const double* f, double* u, void* stream) {
    g_noalloc_err[0] = '\0';
    if (ndim != 2 && ndim != 3) return noalloc_fail(SRJ_ERR_INVALID_ARG, "ndim must be 2 or 3");
    if (!dims || !f || !u || count < 0 || (count > 0 && !omega_seq))
        return noalloc_fail(SRJ_ERR_INVALID_ARG, "NULL argument or negative count");
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1 || dims[i] > 65535) return noalloc_fail(SRJ_ERR_INVALID_ARG, "dims must be in 1..65535");
    if (!(h > 0.0) || !std::isfinite(h)) return noalloc_fail(SRJ_ERR_INVALID_ARG, "h must be finite and > 0");
    for (int64_t k = 0; k < count; ++k)
        if (!(omega_seq[k] > 0.0) || !std::isfinite(omega_seq[k]))
            return noalloc_fail(SRJ_ERR_INVALID_ARG, "weights must be finite and > 0");
    const srj::Geom g = srj::make_geom(ndim, dims);
    if (g.n32 > kNoAllocFloats) {
        std::snprintf(g_noalloc_err, sizeof g_noalloc_err,
                      "grid needs %lld floats per work buffer; the static scratch holds %lld "
                      "(about 1M padded points: e.g. 1016^2 or 96^3)",
                      (long long)g.n32, (long long)kNoAllocFloats);
        return SRJ_ERR_INVALID_ARG;
    }
    float* base = nullptr;
    int rc = scratch_for_current_device(&base);
    if (rc) return rc;
    float* ea = base;
    float* eb = base + kNoAllocFloats;
    float* r32 = base + 2 * kNoAllocFloats;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double h2 = h * h;
    const size_t by = sizeof(float) * (size_t)g.n32;
    cudaError_t e;
    // the previous call's contents are still there: clear what is read before written
    if ((e = cudaMemsetAsync(ea, 0, by, s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "memset", e);
    if ((e = cudaMemsetAsync(eb, 0, by, s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "memset", e);
    if ((e = cudaMemsetAsync(r32, 0, by, s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "memset", e);
    if ((e = srj::launch_to_f32(g, u, ea, s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "to_f32", e);
    if ((e = srj::launch_to_f32(g, u, eb, s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "to_f32", e);
    if ((e = srj::launch_source_f32(g, h2, f, r32, s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "source_f32", e);
    for (int64_t k = 0; k < count; ++k) {
        const bool from_a = (k % 2) == 0;
        const float c = (float)(omega_seq[k] / (double)(2 * ndim));
        if ((e = srj::launch_sweep_f32(g, from_a ? ea : eb, from_a ? eb : ea, r32, c, s)) != cudaSuccess)
            return noalloc_fail(SRJ_ERR_CUDA, "sweep_f32", e);
    }
    if ((e = srj::launch_from_f32(g, (count % 2) ? eb : ea, u, s)) != cudaSuccess)
        return noalloc_fail(SRJ_ERR_CUDA, "from_f32", e);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return noalloc_fail(SRJ_ERR_CUDA, "stream sync", e);
    return SRJ_OK;
}
