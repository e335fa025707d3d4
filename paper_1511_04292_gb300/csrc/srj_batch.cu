// Batched SRJ: many independent 2-D Dirichlet Poisson problems of different
// sizes, each with its own schedule (Sect. 2: weights omega_i repeated q_i
// times per M-cycle), solved together in mixed precision (FP32 cycles on the
// defect equation inside FP64 correction, as in srj_solve).
//
// Work is organised in phases.  One phase is four launches:
//   1. step (one thread per problem): the cycle-end test of the previous phase
//      (norms, convergence test of the Sect. 4.1 monitor on b - A u, restart of
//      the next cycle from e = 0), the problem's sweep record for this phase,
//      and its state after the sweep (k += n with n = min(T, M - k), buffers
//      swapped, cycle end flagged);
//   2. blocked FP32 sweep over the tiles of every active problem;
//   3. FP64 update u += e / s for the problems whose cycle ended;
//   4. FP64 residual r = b - A u for them (written as FP32 r * s, with L2 / max
//      partial sums per row block).
// Launches 3 and 4 walk the row blocks that launch 1 listed as due in this
// phase, from a fixed grid of a few blocks per SM, so that a phase in which no
// cycle ends costs them next to nothing.
// Kernel boundaries order the phases (no device-side waits); every launch reads
// the per-problem state from device memory, so one CUDA graph of G phases (and
// a closing cycle-end test) is captured and replayed until no problem is
// active.  Every active problem swaps its buffers in every phase and all start
// together, so with G even a problem's buffer index is the phase's parity in
// the graph, a launch parameter of the grouped sweep.
#include "srj_internal.h"
#include "../../include/srj.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

namespace {

thread_local std::string g_batch_err;

int bfail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_batch_err = buf;
    return code;
}

#define SRJ_BCUDA(call)                                                                              \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess)                                                                       \
            return bfail(SRJ_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                                  \
    } while (0)

constexpr int kRowsPerBlock = 16;
constexpr int kThreads = 256;
constexpr int kPhasesPerGraph = 16;

enum { kFinInit0 = 0, kFinInit1 = 1, kFinCycle = 2 };

// The step record of problem p for the coming phase (0 steps when inactive),
// then its state after that phase's sweep.  Weights past the record's n steps
// are zero: the sweep runs T steps on every tile, and a zero-weight step leaves
// each point's value as it is.
__device__ __forceinline__ void prepare_and_advance(const srj::BatchProb& P, srj::BatchState& s, const float* cw,
                                                    srj::BatchArgs* args, int T) {
    srj::BatchArgs a;
    a.n = s.active ? min(T, P.M - s.k) : 0;
    a.ein = s.cur ? P.eb : P.ea;
    a.eout = s.cur ? P.ea : P.eb;
    a.r32 = P.r32;
    a.p32 = P.p32;
    a.nx = P.nx;
    a.ny = P.ny;
    a.fresh = s.fresh;
#pragma unroll
    for (int t = 0; t < 8; ++t) a.c[t] = (t < a.n) ? cw[P.c_off + s.k + t] : 0.f;
    args[P.rec] = a;
    if (!s.active) return;
    s.k += a.n;
    s.cur ^= 1;
    s.fresh = 0;
    if (s.k == P.M) s.cycle_end = 1;
}

// L2^2 and max of the residual from the problem's row-block partials (in row order).
__device__ __forceinline__ void sum_partials(const srj::BatchProb& P, const double* partials, double& a, double& m) {
    a = 0.0;
    m = 0.0;
    for (int b = P.rb_begin; b < P.rb_end; ++b) {
        a += partials[2 * b];
        m = fmax(m, partials[2 * b + 1]);
    }
}

// Cycle-end test (Sect. 4.1 monitor on b - A u at the end of a cycle):
// converged, diverged, out of cycles, stagnated at the floating-point floor, or
// the next cycle starts from e = 0.
__device__ __forceinline__ void finish_cycle(const srj::BatchProb& P, srj::BatchState& s, const double* partials,
                                             double tol, int max_cycles) {
    double a, m;
    sum_partials(P, partials, a, m);
    const double l2 = sqrt(a);
    s.l2 = l2;
    s.linf = (a == a) ? m : a;
    s.cycles += 1;
    s.cycle_end = 0;
    if (!isfinite(l2) || l2 > 1e6 * s.r0) { s.status = SRJ_ERR_DIVERGED; s.active = 0; }
    else if (l2 / s.r0 <= tol) { s.status = SRJ_OK; s.active = 0; }
    else if (s.cycles >= max_cycles) { s.status = SRJ_ERR_NOT_CONVERGED; s.active = 0; }
    else if (!(l2 < 0.5 * s.best) && ++s.stall >= 4) {  // floating-point floor reached
        s.status = SRJ_ERR_NOT_CONVERGED; s.stagnated = 1; s.active = 0;
    } else {
        if (l2 < 0.5 * s.best) { s.best = l2; s.stall = 0; }
        s.k = 0; s.fresh = 1;
    }
}

// due / ndue: per phase parity, the row blocks of the problems whose cycle ends
// with this phase's sweep (in no particular order; each row block's results go
// to its own slots) and their number.  The update and the residual of the phase
// walk that list; the step of the next phase, of the other parity, clears this
// phase's count only after both have run.
__global__ void k_batch_step(const srj::BatchProb* __restrict__ probs, srj::BatchState* __restrict__ st,
                             const double* __restrict__ partials, const float* __restrict__ cw,
                             srj::BatchArgs* __restrict__ args, int nprob, int T, double tol, int max_cycles,
                             int* __restrict__ due, int* __restrict__ ndue, int nrowblocks, int parity) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) ndue[parity ^ 1] = 0;  // the next phase's list starts empty
    if (p >= nprob) return;
    srj::BatchState s = st[p];
    const srj::BatchProb P = probs[p];
    if (s.active && s.cycle_end) finish_cycle(P, s, partials, tol, max_cycles);
    prepare_and_advance(P, s, cw, args, T);
    st[p] = s;
    if (s.active && s.cycle_end) {
        const int nrb = P.rb_end - P.rb_begin;
        int* d = due + (size_t)parity * nrowblocks + atomicAdd(&ndue[parity], nrb);
        for (int r = 0; r < nrb; ++r) d[r] = P.rb_begin + r;
    }
}

// u += inv_scale * e on the rows of row block id, when its problem is at a cycle end.
__device__ __forceinline__ void update_rowblock(const srj::BatchProb* __restrict__ probs,
                                                const srj::BatchState* __restrict__ st,
                                                const int2* __restrict__ rowblocks, int id) {
    const int2 rb = rowblocks[id];
    const srj::BatchState s = st[rb.x];
    if (!s.active || !s.cycle_end) return;
    const srj::BatchProb P = probs[rb.x];
    const float* e = s.cur ? P.eb : P.ea;
    const int y1 = min(rb.y + kRowsPerBlock - 1, P.ny);
    const int64_t sx = P.nx + 2;
    for (int y = rb.y; y <= y1; ++y)
        for (int x = threadIdx.x + 1; x <= P.nx; x += blockDim.x)
            P.u[(int64_t)y * sx + x] += s.inv_scale * (double)e[(int64_t)y * P.p32 + x + 3];
}

// Row blocks due[parity][0 .. ndue[parity]) (grid-stride), or row block
// blockIdx.x when ndue is NULL.
__global__ void k_batch_update(const srj::BatchProb* __restrict__ probs, const srj::BatchState* __restrict__ st,
                               const int2* __restrict__ rowblocks, const int* __restrict__ due,
                               const int* __restrict__ ndue, int nrowblocks, int parity) {
    if (!ndue) { update_rowblock(probs, st, rowblocks, (int)blockIdx.x); return; }
    const int n = ndue[parity];
    const int* d = due + (size_t)parity * nrowblocks;
    for (int j = blockIdx.x; j < n; j += gridDim.x) update_rowblock(probs, st, rowblocks, d[j]);
}

// r = (h^2 f + sum nbrs u) - 4 u in the oracle's operation order on row block
// id; optional FP32 defect r * scale; the block's L2 / max partials in the row
// block's slot.  `all`: every active problem (initial residual), otherwise only
// problems at a cycle end.  Uniform over the block.
__device__ __forceinline__ void residual_rowblock(const srj::BatchProb* __restrict__ probs,
                                                  const srj::BatchState* __restrict__ st,
                                                  const int2* __restrict__ rowblocks, int id,
                                                  double* __restrict__ partials, int write_r32, int all,
                                                  double* sh_ss, double* sh_mx) {
    const int2 rb = rowblocks[id];
    const srj::BatchState s = st[rb.x];
    if (!(s.active && (all || s.cycle_end))) return;
    double ss = 0.0, mx = 0.0;
    const srj::BatchProb P = probs[rb.x];
    const int y1 = min(rb.y + kRowsPerBlock - 1, P.ny);
    const int64_t sx = P.nx + 2;
    for (int y = rb.y; y <= y1; ++y) {
        for (int x = threadIdx.x + 1; x <= P.nx; x += blockDim.x) {
            const int64_t q = (int64_t)y * sx + x;
            const double uc = P.u[q];
            double sm = __dadd_rn(P.u[q - 1], P.u[q + 1]);
            sm = __dadd_rn(sm, P.u[q - sx]);
            sm = __dadd_rn(sm, P.u[q + sx]);
            const double t = __dadd_rn(sm, __dmul_rn(P.h2, P.f[q]));
            const double r = __dsub_rn(t, __dmul_rn(4.0, uc));
            if (write_r32) P.r32[(int64_t)y * P.p32 + x + 3] = (float)(r * s.scale);
            ss = fma(r, r, ss);
            mx = fmax(mx, fabs(r));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh_ss[w] = ss; sh_mx[w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, m = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += sh_ss[i]; m = fmax(m, sh_mx[i]); }
        partials[2 * id] = a;
        partials[2 * id + 1] = (a == a) ? m : a;
    }
    __syncthreads();  // sh_ss / sh_mx are reused by the block's next row block
}

// Row blocks due[parity][0 .. ndue[parity]) (grid-stride), or row block
// blockIdx.x when ndue is NULL.
__global__ void k_batch_residual(const srj::BatchProb* __restrict__ probs, const srj::BatchState* __restrict__ st,
                                 const int2* __restrict__ rowblocks, const int* __restrict__ due,
                                 const int* __restrict__ ndue, int nrowblocks, int parity,
                                 double* __restrict__ partials, int write_r32, int all) {
    __shared__ double sh_ss[kThreads / 32], sh_mx[kThreads / 32];
    if (!ndue) {
        residual_rowblock(probs, st, rowblocks, (int)blockIdx.x, partials, write_r32, all, sh_ss, sh_mx);
        return;
    }
    const int n = ndue[parity];
    const int* d = due + (size_t)parity * nrowblocks;
    for (int j = blockIdx.x; j < n; j += gridDim.x)
        residual_rowblock(probs, st, rowblocks, d[j], partials, write_r32, all, sh_ss, sh_mx);
}

__global__ void k_batch_finalize(const srj::BatchProb* __restrict__ probs, srj::BatchState* __restrict__ st,
                                 const double* __restrict__ partials, int nprob, int mode, double tol,
                                 int max_cycles) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nprob) return;
    srj::BatchState s = st[p];
    if (!s.active) return;
    if (mode == kFinInit1) { s.cycle_end = 0; s.fresh = 1; s.k = 0; st[p] = s; return; }
    if (mode == kFinCycle) {
        if (!s.cycle_end) return;
        finish_cycle(probs[p], s, partials, tol, max_cycles);
        st[p] = s;
        return;
    }
    double a, m;  // kFinInit0: the initial residual
    sum_partials(probs[p], partials, a, m);
    const double l2 = sqrt(a);
    s.l2 = l2;
    s.linf = (a == a) ? m : a;
    s.r0 = l2;
    s.best = l2;
    s.stall = 0;
    if (!isfinite(l2)) { s.status = SRJ_ERR_DIVERGED; s.active = 0; }
    else if (l2 == 0.0 || !(tol < 1.0)) { s.status = SRJ_OK; s.active = 0; }
    else {
        int ex = 0;
        frexp(s.linf, &ex);
        s.scale = ldexp(1.0, -ex);
        s.inv_scale = ldexp(1.0, ex);
    }
    st[p] = s;
}

// Number of problems still iterating, and their flags.
__global__ void k_batch_count(const srj::BatchState* __restrict__ st, int nprob, int* __restrict__ out,
                              unsigned char* __restrict__ flags) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    int c = 0;
    for (int p = threadIdx.x; p < nprob; p += blockDim.x) {
        const int a = st[p].active ? 1 : 0;
        flags[p] = (unsigned char)a;
        c += a;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) *out = cnt;
}

}  // namespace

struct srj_batch {
    int device = 0;
    int nprob = 0;
    int T = 8;
    std::vector<srj::BatchProb> probs;   // host copy (f / u filled per solve)
    std::vector<int> M;
    int64_t total_points = 0;
    int ntiles = 0, nrowblocks = 0;
    bool grouped = false;       // at most kMaxBatchGroups grid sizes: grouped sweep
    srj::BatchGroups groups{};  // every problem launched
    std::vector<int> gid, gz;   // group and group-local index of each problem
    std::vector<int4> tiles;    // tile list (problem, tile x, tile y) of every problem
    std::vector<int> tile_begin;  // first tile of each problem in `tiles`
    std::vector<unsigned char> launched;  // problems the graph's sweep launches cover
    cudaGraph_t graph = nullptr;          // kept: its nodes are re-targeted between launches
    std::vector<cudaGraphNode_t> sweep_nodes;
    int* d_due = nullptr;                 // 2 x nrowblocks: row blocks due per phase parity
    int* d_ndue = nullptr;                // 2 counts
    int rowblock_grid = 1;                // blocks of the graph's update / residual launches
    unsigned char* d_flags = nullptr;
    unsigned char* h_flags = nullptr;
    srj::BatchProb* d_probs = nullptr;
    srj::BatchState* d_state = nullptr;
    int4* d_tiles = nullptr;
    srj::BatchArgs* d_args = nullptr;
    int2* d_rowblocks = nullptr;
    float* d_cw = nullptr;
    float* d_pool = nullptr;  // all FP32 workspaces
    double* d_partials = nullptr;
    int* d_count = nullptr;
    int* h_count = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t phases = nullptr;
    double graph_tol = -1.0;
    int graph_max_cycles = -1;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    ~srj_batch() {
        if (phases) cudaGraphExecDestroy(phases);
        if (graph) cudaGraphDestroy(graph);
        cudaFree(d_due); cudaFree(d_ndue); cudaFree(d_flags);
        if (h_flags) cudaFreeHost(h_flags);
        if (cap) cudaStreamDestroy(cap);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        cudaFree(d_probs); cudaFree(d_state); cudaFree(d_tiles); cudaFree(d_rowblocks); cudaFree(d_args);
        cudaFree(d_cw); cudaFree(d_pool); cudaFree(d_partials); cudaFree(d_count);
        if (h_count) cudaFreeHost(h_count);
    }
};

namespace {

// The node a capture has just added (the only dependency of what comes next).
cudaError_t last_node(cudaStream_t s, cudaGraphNode_t* out) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    if (st != cudaStreamCaptureStatusActive || nd != 1) return cudaErrorStreamCaptureInvalidated;
    *out = deps[0];
    return cudaSuccess;
}

cudaError_t issue_phase(srj_batch* b, cudaStream_t s, double tol, int max_cycles, int parity) {
    const int pb = (b->nprob + kThreads - 1) / kThreads;
    k_batch_step<<<pb, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_partials, b->d_cw, b->d_args, b->nprob, b->T,
                                         tol, max_cycles, b->d_due, b->d_ndue, b->nrowblocks, parity);
    cudaError_t e = b->grouped
                        ? srj::launch_batch_sweep_grouped(b->T, (unsigned)b->ntiles, b->groups, b->d_pool, b->d_args,
                                                          parity, s)
                        : srj::launch_batch_sweep_tb(b->T, (unsigned)b->ntiles, b->d_tiles, b->d_args, s);
    cudaGraphNode_t n;
    if (e == cudaSuccess) e = last_node(s, &n);
    if (e != cudaSuccess) return e;
    b->sweep_nodes.push_back(n);
    k_batch_update<<<b->rowblock_grid, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_rowblocks, b->d_due, b->d_ndue,
                                                         b->nrowblocks, parity);
    k_batch_residual<<<b->rowblock_grid, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_rowblocks, b->d_due,
                                                           b->d_ndue, b->nrowblocks, parity, b->d_partials, 1, 0);
    return cudaGetLastError();
}

// Point the graph's sweep launches at the problems flagged in `want` (those
// still iterating at the start of the next graph launch).  Problems that finish
// during a launch keep their blocks until the next one; those blocks see no
// steps and leave early.  (Update and residual walk the phase's due list.)
int retarget(srj_batch* b, const unsigned char* want, cudaStream_t s) {
    if (b->launched.size() == (size_t)b->nprob && std::equal(b->launched.begin(), b->launched.end(), want)) return SRJ_OK;
    unsigned ntiles = 0;
    srj::BatchGroups G = b->groups;
    std::vector<int4> tl;
    if (b->grouped) {
        std::vector<std::vector<int>> mem(G.ngroups);
        for (int p = 0; p < b->nprob; ++p)
            if (want[p]) mem[b->gid[p]].push_back(b->gz[p]);
        int mb = 0, tb = 0;
        for (int g = 0; g < G.ngroups; ++g) {
            G.mbase[g] = mb;
            G.tile_begin[g] = tb;
            for (int m : mem[g]) G.member[mb++] = (uint16_t)m;
            tb += (int)mem[g].size() * G.gx[g] * G.gy[g];
        }
        G.tile_begin[G.ngroups] = tb;
        ntiles = (unsigned)tb;
    } else {
        for (int p = 0; p < b->nprob; ++p)
            if (want[p]) tl.insert(tl.end(), b->tiles.begin() + b->tile_begin[p], b->tiles.begin() + b->tile_begin[p + 1]);
        ntiles = (unsigned)tl.size();
    }
    if (ntiles == 0) return SRJ_OK;  // nothing left to launch: the solve loop ends
    if (!b->grouped)
        SRJ_BCUDA(cudaMemcpyAsync(b->d_tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice, s));
    for (cudaGraphNode_t n : b->sweep_nodes)
        SRJ_BCUDA(srj::batch_sweep_set_node(b->phases, n, ntiles, b->grouped ? &G : nullptr));
    b->launched.assign(want, want + b->nprob);
    return SRJ_OK;
}

int capture_phases(srj_batch* b, double tol, int max_cycles, cudaStream_t s) {
    if (b->phases) { cudaGraphExecDestroy(b->phases); b->phases = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    b->sweep_nodes.clear();
    b->launched.clear();
    // the captured sweeps cover every problem: full tile list
    SRJ_BCUDA(cudaMemcpyAsync(b->d_tiles, b->tiles.data(), sizeof(int4) * b->tiles.size(), cudaMemcpyHostToDevice, s));
    cudaGraph_t graph = nullptr;
    SRJ_BCUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    static_assert(kPhasesPerGraph % 2 == 0, "buffer parity must repeat from one graph launch to the next");
    for (int i = 0; i < kPhasesPerGraph && err == cudaSuccess; ++i) err = issue_phase(b, b->cap, tol, max_cycles, i & 1);
    if (err == cudaSuccess) {  // cycle-end test of the last phase, so that the state is final between launches
        const int pb = (b->nprob + kThreads - 1) / kThreads;
        k_batch_finalize<<<pb, kThreads, 0, b->cap>>>(b->d_probs, b->d_state, b->d_partials, b->nprob, kFinCycle, tol,
                                                      max_cycles);
        err = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (err != cudaSuccess) { if (graph) cudaGraphDestroy(graph); b->sweep_nodes.clear(); SRJ_BCUDA(err); }
    SRJ_BCUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&b->phases, graph, 0);
    if (e3 != cudaSuccess) { cudaGraphDestroy(graph); b->sweep_nodes.clear(); SRJ_BCUDA(e3); }
    b->graph = graph;
    b->launched.assign(b->nprob, 1);
    b->graph_tol = tol;
    b->graph_max_cycles = max_cycles;
    return SRJ_OK;
}

}  // namespace

extern "C" {

const char* srj_batch_last_error(void) { return g_batch_err.c_str(); }

int srj_batch_create(srj_batch_t* out, int nprob, const srj_batch_problem_t* pr, int temporal_depth) {
    if (!out) return bfail(SRJ_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || nprob > (1 << 20) || !pr) return bfail(SRJ_ERR_INVALID_ARG, "need 1..2^20 problems");
    if (temporal_depth == 0) temporal_depth = 8;
    if (temporal_depth < 1 || temporal_depth > srj::tb_max_steps())
        return bfail(SRJ_ERR_INVALID_ARG, "temporal depth must be in 1..%d", srj::tb_max_steps());
    srj_batch* b = new (std::nothrow) srj_batch();
    if (!b) return bfail(SRJ_ERR_NO_MEMORY, "host allocation failed");
    auto bail = [&](int code) { delete b; return code; };
    b->nprob = nprob;
    b->T = temporal_depth;
    int TX = 0, TY = 0;
    srj::tb_tile_shape(b->T, &TX, &TY);

    // Grid sizes: with at most kMaxBatchGroups distinct ones the pool is laid out
    // group by group and the grouped sweep is used (BatchGroups).
    std::vector<int> gid(nprob, 0), gz(nprob, 0);
    std::vector<std::pair<int64_t, int64_t>> gdims;
    std::vector<int> gcount;
    {
        std::map<std::pair<int64_t, int64_t>, int> seen;
        bool dims_ok = true;
        for (int p = 0; p < nprob; ++p) {
            const std::pair<int64_t, int64_t> d(pr[p].nx, pr[p].ny);
            if (d.first < 1 || d.second < 1 || d.first > 65536 || d.second > 65536) dims_ok = false;
            auto it = seen.find(d);
            int g = 0;
            if (it == seen.end()) {
                g = (int)gdims.size();
                seen.emplace(d, g);
                gdims.push_back(d);
                gcount.push_back(0);
            } else {
                g = it->second;
            }
            gid[p] = g;
            gz[p] = gcount[g]++;
        }
        b->grouped = dims_ok && gdims.size() <= (size_t)srj::kMaxBatchGroups && nprob <= srj::kMaxGroupedProblems;
    }
    const int ngroups = (int)gdims.size();
    std::vector<size_t> goff, gn32;
    std::vector<int> grec;
    size_t grouped_floats = 0;
    if (b->grouped) {
        int racc = 0;
        for (int g = 0; g < ngroups; ++g) {
            const int64_t dims[2] = {gdims[g].first, gdims[g].second};
            gn32.push_back((size_t)((srj::make_geom(2, dims).n32 + 63) / 64 * 64));
            goff.push_back(grouped_floats);
            grouped_floats += (size_t)gcount[g] * 3 * gn32[g];
            grec.push_back(racc);
            racc += gcount[g];
        }
    }

    std::vector<float> cw;
    std::vector<int4> tiles;
    std::vector<int2> rowblocks;
    std::vector<size_t> pool_off;
    size_t pool_floats = 0;
    b->probs.resize(nprob);
    for (int p = 0; p < nprob; ++p) {
        const srj_batch_problem_t& q = pr[p];
        if (q.nx < 1 || q.ny < 1 || q.nx > 65536 || q.ny > 65536)
            return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: dims out of range", p));
        if (!(q.h > 0.0) || !std::isfinite(q.h)) return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: bad h", p));
        if (q.P < 1 || q.P > 32 || !q.omega || !q.q) return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: bad schedule", p));
        std::vector<double> w(q.omega, q.omega + q.P);
        std::vector<int32_t> qq(q.q, q.q + q.P);
        int64_t M = 0;
        for (int i = 0; i < q.P; ++i) {
            if (!(w[i] > 0.0) || !std::isfinite(w[i]) || qq[i] < 1)
                return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: bad weight or repetition", p));
            M += qq[i];
        }
        if (M > (1 << 20)) return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: M too large", p));
        const int64_t dims[2] = {q.nx, q.ny};
        const double g = srj::host_max_cycle_log10(w, qq, 2, dims);
        if (!(g < 0.0)) return bail(bfail(SRJ_ERR_BAD_SCHEDULE, "problem %d: integer scheme does not contract (%.3g)", p, g));
        std::vector<int32_t> order;
        if (q.order) {
            order.assign(q.order, q.order + M);
            std::vector<int64_t> cnt(q.P, 0);
            for (int32_t v : order) {
                if (v < 0 || v >= q.P) return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: order out of range", p));
                cnt[v]++;
            }
            for (int i = 0; i < q.P; ++i)
                if (cnt[i] != qq[i]) return bail(bfail(SRJ_ERR_INVALID_ARG, "problem %d: order does not match q", p));
        } else {
            order = srj::host_drift_order(w, qq, srj::host_kappa_min(2, dims));
        }
        srj::BatchProb& P = b->probs[p];
        const srj::Geom geo = srj::make_geom(2, dims);
        P.nx = (int)q.nx;
        P.ny = (int)q.ny;
        P.p32 = geo.p32;
        P.h2 = q.h * q.h;
        P.M = (int)M;
        P.c_off = (int)cw.size();
        for (int32_t v : order) cw.push_back((float)(w[v] / 4.0));
        const size_t n32 = (size_t)((geo.n32 + 63) / 64 * 64);
        if (b->grouped) {
            pool_off.push_back(goff[gid[p]] + (size_t)gz[p] * 3 * gn32[gid[p]]);
            P.rec = grec[gid[p]] + gz[p];
        } else {
            pool_off.push_back(pool_floats);
            pool_floats += 3 * n32;
            P.rec = p;
        }
        b->M.push_back((int)M);
        b->total_points += q.nx * q.ny;
        const int gx = (int)((q.nx + TX - 1) / TX), gy = (int)((q.ny + TY - 1) / TY);
        b->tile_begin.push_back((int)tiles.size());
        for (int by = 0; by < gy; ++by)
            for (int bx = 0; bx < gx; ++bx) tiles.push_back(make_int4(p, bx, by, 0));
        P.rb_begin = (int)rowblocks.size();
        for (int y = 1; y <= q.ny; y += kRowsPerBlock) rowblocks.push_back(make_int2(p, y));
        P.rb_end = (int)rowblocks.size();
        if (cw.size() > (size_t)1 << 30) return bail(bfail(SRJ_ERR_INVALID_ARG, "weight table too large"));
    }
    if (tiles.size() > (size_t)INT32_MAX || rowblocks.size() > (size_t)INT32_MAX)
        return bail(bfail(SRJ_ERR_INVALID_ARG, "too many tiles"));
    b->tile_begin.push_back((int)tiles.size());
    b->tiles = tiles;
    b->gid = gid;
    b->gz = gz;
    b->ntiles = (int)tiles.size();
    b->nrowblocks = (int)rowblocks.size();
    if (b->grouped) {
        pool_floats = grouped_floats;
        srj::BatchGroups& G = b->groups;
        G.ngroups = ngroups;
        int64_t tb = 0;
        for (int g = 0; g < ngroups; ++g) {
            const int64_t dims[2] = {gdims[g].first, gdims[g].second};
            const srj::Geom geo = srj::make_geom(2, dims);
            G.tile_begin[g] = (int)tb;
            G.gx[g] = (int)((dims[0] + TX - 1) / TX);
            G.gy[g] = (int)((dims[1] + TY - 1) / TY);
            tb += (int64_t)gcount[g] * G.gx[g] * G.gy[g];
            G.nx[g] = (int)dims[0];
            G.ny[g] = (int)dims[1];
            G.rec[g] = grec[g];
            G.p32[g] = geo.p32;
            G.n32[g] = (int64_t)gn32[g];
            G.off[g] = (int64_t)goff[g];
        }
        G.tile_begin[ngroups] = (int)tb;
        int mb = 0;
        for (int g = 0; g < ngroups; ++g) {
            G.mbase[g] = mb;
            for (int m = 0; m < gcount[g]; ++m) G.member[mb++] = (uint16_t)m;
        }
        if (tb != b->ntiles) return bail(bfail(SRJ_ERR_INVALID_ARG, "internal: grouped tile count %lld != %d", (long long)tb, b->ntiles));
    }
    if (cudaGetDevice(&b->device) != cudaSuccess) return bail(bfail(SRJ_ERR_CUDA, "no CUDA device"));
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess || sms < 1) sms = 1;
        b->rowblock_grid = std::max(1, std::min(b->nrowblocks, 4 * sms));
    }
    auto alloc = [](void** ptr, size_t by) { return cudaMalloc(ptr, by) == cudaSuccess; };
    bool ok = alloc((void**)&b->d_pool, sizeof(float) * pool_floats) &&
              alloc((void**)&b->d_probs, sizeof(srj::BatchProb) * nprob) &&
              alloc((void**)&b->d_state, sizeof(srj::BatchState) * nprob) &&
              alloc((void**)&b->d_tiles, sizeof(int4) * tiles.size()) &&
              alloc((void**)&b->d_args, sizeof(srj::BatchArgs) * (size_t)nprob) &&
              alloc((void**)&b->d_rowblocks, sizeof(int2) * rowblocks.size()) &&
              alloc((void**)&b->d_cw, sizeof(float) * cw.size()) &&
              alloc((void**)&b->d_partials, sizeof(double) * 2 * rowblocks.size()) &&
              alloc((void**)&b->d_count, sizeof(int)) &&
              alloc((void**)&b->d_due, sizeof(int) * 2 * rowblocks.size()) &&
              alloc((void**)&b->d_ndue, sizeof(int) * 2) &&
              alloc((void**)&b->d_flags, (size_t)nprob);
    if (!ok) { cudaGetLastError(); return bail(bfail(SRJ_ERR_NO_MEMORY, "device allocation failed")); }
    for (int p = 0; p < nprob; ++p) {
        const int64_t dims[2] = {pr[p].nx, pr[p].ny};
        const size_t n32 = (size_t)((srj::make_geom(2, dims).n32 + 63) / 64 * 64);
        b->probs[p].ea = b->d_pool + pool_off[p];
        b->probs[p].eb = b->probs[p].ea + n32;
        b->probs[p].r32 = b->probs[p].eb + n32;
        b->probs[p].f = nullptr;
        b->probs[p].u = nullptr;
    }
    if (cudaMemset(b->d_pool, 0, sizeof(float) * pool_floats) != cudaSuccess ||
        cudaMemcpy(b->d_tiles, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_rowblocks, rowblocks.data(), sizeof(int2) * rowblocks.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_cw, cw.data(), sizeof(float) * cw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_count, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&b->h_flags, (size_t)nprob) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess ||
        srj::tb_prepare() != cudaSuccess) {
        cudaGetLastError();
        return bail(bfail(SRJ_ERR_CUDA, "batch set-up failed"));
    }
    *out = b;
    return SRJ_OK;
}

int srj_batch_tune_depth(int nprob, const srj_batch_problem_t* pr, const double* const* f, const double* const* u,
                         int tmin, int tmax, void* stream, int* best_T, double* best_ms_per_cycle) {
    if (!f || !u || !best_T) return bfail(SRJ_ERR_INVALID_ARG, "NULL argument");
    if (tmin < 1 || tmax > srj::tb_max_steps() || tmin > tmax)
        return bfail(SRJ_ERR_INVALID_ARG, "depth range must lie in 1..%d", srj::tb_max_steps());
    if (nprob < 1 || !pr) return bfail(SRJ_ERR_INVALID_ARG, "need at least one problem");
    cudaStream_t s = (cudaStream_t)stream;
    // the trial solves overwrite their iterates: run them on copies of u
    std::vector<double*> uc((size_t)nprob, nullptr);
    auto free_all = [&] { for (double* x : uc) cudaFree(x); };
    for (int p = 0; p < nprob; ++p) {
        if (!f[p] || !u[p]) { free_all(); return bfail(SRJ_ERR_INVALID_ARG, "problem %d: NULL array", p); }
        const size_t by = sizeof(double) * (size_t)(pr[p].nx + 2) * (size_t)(pr[p].ny + 2);
        if (cudaMalloc((void**)&uc[p], by) != cudaSuccess) {
            cudaGetLastError();
            free_all();
            return bfail(SRJ_ERR_NO_MEMORY, "copies of the iterates");
        }
    }
    int bestT = 0;
    double best = INFINITY;
    for (int T = tmax; T >= tmin; --T) {
        srj_batch_t b = nullptr;
        int rc = srj_batch_create(&b, nprob, pr, T);
        if (rc) { free_all(); return rc; }
        double ms = INFINITY;
        for (int rep = 0; rep < 2 && rc == SRJ_OK; ++rep) {  // the first solve captures the phase graph
            for (int p = 0; p < nprob; ++p) {
                const size_t by = sizeof(double) * (size_t)(pr[p].nx + 2) * (size_t)(pr[p].ny + 2);
                if (cudaMemcpyAsync(uc[p], u[p], by, cudaMemcpyDeviceToDevice, s) != cudaSuccess) rc = SRJ_ERR_CUDA;
            }
            double dms = 0.0;
            if (rc == SRJ_OK) {
                // one cycle of every problem (tol 0): every phase of the longest cycle runs once
                rc = srj_batch_solve(b, f, uc.data(), 0.0, 1, stream, nullptr, &dms);
                if (rc == SRJ_ERR_NOT_CONVERGED) rc = SRJ_OK;
            }
            if (rep == 1) ms = dms;
        }
        srj_batch_destroy(b);
        if (rc) { free_all(); return rc; }
        if (ms < best) { best = ms; bestT = T; }
    }
    free_all();
    *best_T = bestT;
    if (best_ms_per_cycle) *best_ms_per_cycle = best;
    return SRJ_OK;
}

int srj_batch_destroy(srj_batch_t b) {
    if (!b) return SRJ_OK;
    cudaDeviceSynchronize();
    delete b;
    return SRJ_OK;
}

int srj_batch_info(srj_batch_t b, int64_t* total_points, int64_t* tiles, int* temporal_depth, int64_t* sum_M) {
    if (!b) return bfail(SRJ_ERR_INVALID_ARG, "batch is NULL");
    if (total_points) *total_points = b->total_points;
    if (tiles) *tiles = b->ntiles;
    if (temporal_depth) *temporal_depth = b->T;
    if (sum_M) { int64_t s = 0; for (int m : b->M) s += m; *sum_M = s; }
    return SRJ_OK;
}

int srj_batch_solve(srj_batch_t b, const double* const* f, double* const* u, double tol, int64_t max_cycles,
                    void* stream, srj_stats_t* stats, double* device_ms) {
    if (!b || !f || !u) return bfail(SRJ_ERR_INVALID_ARG, "NULL argument");
    if (!(tol >= 0.0) || max_cycles < 0 || max_cycles > (1 << 30))
        return bfail(SRJ_ERR_INVALID_ARG, "tol must be >= 0 and max_cycles in 0..2^30");
    int dev = -1;
    SRJ_BCUDA(cudaGetDevice(&dev));
    if (dev != b->device) return bfail(SRJ_ERR_INVALID_ARG, "batch was created on device %d", b->device);
    cudaStream_t s = (cudaStream_t)stream;
    for (int p = 0; p < b->nprob; ++p) {
        if (!f[p] || !u[p]) return bfail(SRJ_ERR_INVALID_ARG, "problem %d: NULL array", p);
        b->probs[p].f = f[p];
        b->probs[p].u = u[p];
    }
    std::vector<srj::BatchState> st(b->nprob);
    for (auto& x : st) {
        std::memset(&x, 0, sizeof x);
        x.active = 1;
        x.cycle_end = 1;
        x.fresh = 1;
        x.scale = x.inv_scale = 1.0;
    }
    SRJ_BCUDA(cudaMemcpyAsync(b->d_probs, b->probs.data(), sizeof(srj::BatchProb) * b->nprob, cudaMemcpyHostToDevice, s));
    SRJ_BCUDA(cudaMemcpyAsync(b->d_state, st.data(), sizeof(srj::BatchState) * b->nprob, cudaMemcpyHostToDevice, s));
    const int pb = (b->nprob + kThreads - 1) / kThreads;
    const int mc = (int)std::max<int64_t>(max_cycles, 1);
    // initial residual (norms, then the scaled FP32 defect)
    k_batch_residual<<<b->nrowblocks, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_rowblocks, nullptr, nullptr,
                                                        b->nrowblocks, 0, b->d_partials, 0, 1);
    k_batch_finalize<<<pb, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_partials, b->nprob, kFinInit0, tol, mc);
    k_batch_residual<<<b->nrowblocks, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_rowblocks, nullptr, nullptr,
                                                        b->nrowblocks, 0, b->d_partials, 1, 1);
    k_batch_finalize<<<pb, kThreads, 0, s>>>(b->d_probs, b->d_state, b->d_partials, b->nprob, kFinInit1, tol, mc);
    SRJ_BCUDA(cudaGetLastError());
    if (b->graph_tol != tol || b->graph_max_cycles != mc || !b->phases) {
        int rc = capture_phases(b, tol, mc, s);
        if (rc) return rc;
    } else {
        const std::vector<unsigned char> all(b->nprob, 1);
        int rc = retarget(b, all.data(), s);  // a previous solve may have left fewer problems launched
        if (rc) return rc;
    }
    // Each phase advances every active problem by at least one step, so
    // sum_p M_p * max_cycles phases bound the loop.
    int64_t max_phases = 0;
    for (int m : b->M) max_phases = std::max<int64_t>(max_phases, (int64_t)m);
    max_phases = max_phases * mc + kPhasesPerGraph;
    SRJ_BCUDA(cudaMemsetAsync(b->d_ndue, 0, 2 * sizeof(int), s));  // both due lists start empty
    SRJ_BCUDA(cudaEventRecord(b->ev0, s));
    int64_t phases = 0;
    if (max_cycles > 0) {
        for (;;) {
            SRJ_BCUDA(cudaGraphLaunch(b->phases, s));
            phases += kPhasesPerGraph;
            k_batch_count<<<1, kThreads, 0, s>>>(b->d_state, b->nprob, b->d_count, b->d_flags);
            SRJ_BCUDA(cudaMemcpyAsync(b->h_count, b->d_count, sizeof(int), cudaMemcpyDeviceToHost, s));
            SRJ_BCUDA(cudaMemcpyAsync(b->h_flags, b->d_flags, (size_t)b->nprob, cudaMemcpyDeviceToHost, s));
            SRJ_BCUDA(cudaStreamSynchronize(s));
            if (*b->h_count == 0 || phases >= max_phases) break;
            int rc = retarget(b, b->h_flags, s);  // drop the problems that have finished
            if (rc) return rc;
        }
    }
    SRJ_BCUDA(cudaEventRecord(b->ev1, s));
    SRJ_BCUDA(cudaMemcpyAsync(st.data(), b->d_state, sizeof(srj::BatchState) * b->nprob, cudaMemcpyDeviceToHost, s));
    SRJ_BCUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    SRJ_BCUDA(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    if (device_ms) *device_ms = ms;
    int status = SRJ_OK;
    for (int p = 0; p < b->nprob; ++p) {
        const srj::BatchState& x = st[p];
        int ps = x.active ? SRJ_ERR_NOT_CONVERGED : x.status;
        if (max_cycles == 0 && x.active) ps = (x.r0 == 0.0) ? SRJ_OK : SRJ_ERR_NOT_CONVERGED;
        if (stats) {
            srj_stats_t& o = stats[p];
            o.cycles = x.cycles;
            o.sweeps = (int64_t)x.cycles * b->M[p];
            o.residual_checks = 1 + x.cycles;
            o.r0_l2 = x.r0;
            o.res_l2 = x.l2;
            o.res_linf = x.linf;
            o.rel_res = x.r0 > 0 ? x.l2 / x.r0 : 0.0;
            o.sweep_ms = ms;
            o.stagnated = x.stagnated;
            o.reserved = 0;
        }
        if (ps != SRJ_OK && status == SRJ_OK) status = ps;
    }
    if (status != SRJ_OK) bfail(status, "not every problem converged");
    return status;
}

}  // extern "C"
