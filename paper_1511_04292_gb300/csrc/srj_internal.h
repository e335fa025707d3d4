// Internal declarations shared by the SRJ kernels and the host runtime.
// Not part of the public ABI (see include/srj.h).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace srj {

// Geometry of one grid: interior sizes, padded float64 layout (the ABI layout)
// and the pitched float32 layout used by the mixed-precision workspaces.
//
// float32 layout: rows of `p32` floats (a multiple of 32, i.e. 128-byte rows);
// padded coordinate x (0..nx+1) of a row is stored at column x + 3, so that
// the first interior point (x = 1) sits at column 4, 16-byte aligned, and
// float4 loads of interior points are aligned.  Rows y = 0..ny+1, planes
// z = 0..nz+1 (3-D) follow each other densely.
struct Geom {
    int nd;
    int nx, ny, nz;        // interior points (nz = 1 in 2-D)
    int64_t sx64, sy64;    // float64 strides: row = nx+2, plane = (nx+2)(ny+2)
    int64_t n64;           // float64 padded element count
    int64_t p32, plane32;  // float32 row pitch (floats) and plane size
    int64_t n32;           // float32 element count
};

Geom make_geom(int nd, const int64_t* dims);

// Reduction scratch for the fused residual norms: per-block partial sums and
// maxima, a completion counter and the final norms.
struct NormScratch {
    double* partials;      // 3 * kMaxNormBlocks doubles: (sum r^2, max |r|) pairs, then sums of a^2
    unsigned int* counter; // zero between launches
    double* result;        // [0] = ||r||_2, [1] = max |r|, [2] = rounding floor of ||r||_2
};
constexpr int kMaxNormBlocks = 1216;  // 8 blocks per SM on 152 SMs

// ---- launchers (all asynchronous on `s`) ----------------------------------

// b = h2 * f on the interior (float64 padded layout; ghosts of b set to 0).
cudaError_t launch_scale_source(const Geom& g, double h2, const double* f, double* b, cudaStream_t s);

// One FP64 weighted-Jacobi step, fixed operation order, no FMA (fused: the
// update as fma(c, fma(-2d, u, t), u), t = neighbour sum + b).
//   uout = uin + c * ((sum nbrs(uin) + b) - 2d uin)    (interior only)
// two_d: the diagonal 2d + sigma of a shifted operator (0 = plain 2d); mask:
// padded uint8 array, 0 = point held fixed (NULL = all interior points active).
cudaError_t launch_sweep_f64(const Geom& g, const double* uin, double* uout, const double* b,
                             double c, cudaStream_t s, double two_d = 0.0, const unsigned char* mask = nullptr, bool fused = false);

// Fused residual r = (h2 * src + sum nbrs(u)) - 2d u on the interior, with L2 /
// max norms reduced into ns.result.  Optional outputs: r64 (padded float64,
// interior only), r32 (pitched float32, value r * scale).
cudaError_t launch_residual(const Geom& g, const double* u, const double* src, double h2,
                            double* r64, float* r32, double scale, NormScratch ns, cudaStream_t s,
                            double two_d = 0.0, const unsigned char* mask = nullptr);

// One FP32 weighted-Jacobi step on the pitched float32 layout:
//   eout = ein + c * ((sum nbrs(ein) + r) - 2d ein)    (interior only)
cudaError_t launch_sweep_f32(const Geom& g, const float* ein, float* eout, const float* r,
                             float c, cudaStream_t s, float two_d = 0.0f, const unsigned char* mask = nullptr);

// u (float64 padded, interior) += inv_scale * e (float32 pitched).
cudaError_t launch_update(const Geom& g, double* u, const float* e, double inv_scale, cudaStream_t s,
                          const unsigned char* mask = nullptr);

// Layout conversions used by srj_steps on mixed plans.
cudaError_t launch_to_f32(const Geom& g, const double* u, float* e, cudaStream_t s);          // all points
cudaError_t launch_source_f32(const Geom& g, double h2, const double* f, float* r, cudaStream_t s);  // interior
cudaError_t launch_from_f32(const Geom& g, const float* e, double* u, cudaStream_t s);        // interior

// ---- temporally blocked FP32 sweep (2-D) ----------------------------------

// Weights of up to 8 consecutive steps: c[t] = omega / 2d for step t < T.
struct TbSteps {
    int T;
    float c[8];
};

int tb_max_steps();
cudaError_t tb_prepare();  // kernel attributes (dynamic shared memory)
// T = steps.T consecutive FP32 steps in one launch: reads ein and the defect
// rin (pitched float32), writes the interior of eout (eout != ein).
// warps: 8 (128 x 64 tiles) or 16 (128 x 128 tiles).  pf_dist > 0: each block
// also prefetches into L2 the tile pf_dist blocks further on in launch order.
cudaError_t launch_sweep_f32_tb(const Geom& g, const float* ein, const float* rin, float* eout,
                                const TbSteps& steps, int warps, cudaStream_t s, int pf_dist = 0);
// Persistent variant (steps.T >= 2): blocks_per_sm * sms blocks of `warps`
// warps (8: 128 x 64 tiles, two blocks per SM; 16: 128 x 128 tiles, one block
// per SM) walk the tiles, prefetching the next tile's rows by bulk copies
// while computing the current one.  Same results bit for bit.  Each wait on a
// prefetch is bounded by limit_ns of wall time; a wait that runs out sets
// *status = kStatusTimeout (device memory) and ends its block.  stall != 0
// launches the bounded-wait self-test (no copy is issued; every wait runs out).
constexpr int kStatusTimeout = 1;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
cudaError_t launch_sweep_f32_tbp(const Geom& g, const float* ein, const float* rin, float* eout,
                                 const TbSteps& steps, int warps, int blocks_per_sm, int sms, int* status,
                                 cudaStream_t s, uint64_t limit_ns = kWaitLimitNs, int stall = 0);

// 3-D: steps.T = 2 or 3 consecutive FP32 steps in one launch, by persistent
// blocks (at most `blocks`, one per SM) streaming z segments of 128 x 32 tiles.
// Same bits as steps.T single steps.
cudaError_t tb3_prepare();  // kernel attributes (dynamic shared memory)
int tb3_max_steps();
cudaError_t launch_sweep3_f32_tb(const Geom& g, const float* ein, const float* rin, float* eout, const TbSteps& steps,
                                 int blocks, cudaStream_t s);

// ---- batched solver (independent 2-D problems, mixed precision) -----------

// Static per-problem data, in device memory.
struct BatchProb {
    int nx, ny;            // interior points
    int64_t p32;           // float32 row pitch
    double h2;             // h^2
    int M;                 // steps per cycle
    int c_off;             // offset of the problem's weights in the weight table
    float *ea, *eb, *r32;  // pitched float32 workspaces (ghosts 0)
    const double* f;       // caller's arrays (set per solve)
    double* u;
    int rb_begin, rb_end;  // range of the problem's row blocks (residual partials)
    int rec;               // index of the problem's sweep record (BatchArgs)
};

// Dynamic per-problem state, in device memory.
struct BatchState {
    int k;          // position in the cycle
    int cur;        // 0: current correction in ea, 1: in eb
    int fresh;      // correction is identically 0 (start of a cycle)
    int active;     // still iterating
    int cycle_end;  // a cycle has just completed (update / residual due)
    int cycles;     // completed cycles
    int status;     // SRJ_OK / NOT_CONVERGED / DIVERGED when inactive
    int stall;      // cycles since the residual last halved its best value
    double best;    // smallest residual norm so far
    double scale, inv_scale;  // power-of-two scaling of the FP32 defect
    double r0, l2, linf;
    int stagnated, pad2;
};

// What one sweep phase needs of a problem, written at the start of the phase.
// The tile-list sweep reads every field; the grouped sweep (BatchGroups) takes
// the workspaces from its launch parameters and reads n, fresh and c.
struct BatchArgs {
    const float* ein;      // current correction
    float* eout;           // next correction
    const float* r32;      // FP32 defect
    int64_t p32;           // float32 row pitch
    int nx, ny;            // interior points
    int n;                 // steps in this phase (0: inactive)
    int fresh;             // ein is identically 0
    float c[8];            // weight / 4 of each step; 0 past step n (identity steps)
};

// Problems of one grid size form a group; a group's FP32 workspaces follow each
// other in the pool at a fixed stride (ea, eb, r32 of n32 floats each per
// problem) and its problems have consecutive record indices.  A sweep block
// then finds its problem, tile and workspaces from these launch parameters
// alone, without a memory read ahead of its tile loads.
// Only the problems still iterating are launched: member[] lists, per group,
// the group-local indices of the launched problems (the z-th launched problem
// of group g is member[mbase[g] + z]).
constexpr int kMaxBatchGroups = 16;
constexpr int kMaxGroupedProblems = 1024;
struct BatchGroups {
    int ngroups;
    int tile_begin[kMaxBatchGroups + 1];  // first block of each group in launch order
    int gx[kMaxBatchGroups], gy[kMaxBatchGroups];  // tiles per problem in x / y
    int nx[kMaxBatchGroups], ny[kMaxBatchGroups];  // interior points
    int rec[kMaxBatchGroups];                      // record index of the group's first problem
    int mbase[kMaxBatchGroups];                    // first entry of the group in member[]
    int64_t p32[kMaxBatchGroups];                  // float32 row pitch
    int64_t n32[kMaxBatchGroups];                  // floats per workspace
    int64_t off[kMaxBatchGroups];                  // pool offset of the group's first problem
    uint16_t member[kMaxGroupedProblems];
};

void tb_tile_shape(int T, int* TX, int* TY);
cudaError_t launch_batch_sweep_tb(int T, unsigned ntiles, const int4* tiles, const BatchArgs* args, cudaStream_t s);
// parity: the phase's position in its graph modulo 2, which is every active
// problem's buffer index (0: input in ea, output in eb; 1: the reverse).
cudaError_t launch_batch_sweep_grouped(int T, unsigned ntiles, const BatchGroups& G, float* pool,
                                       const BatchArgs* args, int parity, cudaStream_t s);
// Relaunch shape of a captured batch sweep node (either kind): ntiles blocks
// and, for the grouped sweep, the launched problems in G.
cudaError_t batch_sweep_set_node(cudaGraphExec_t exec, cudaGraphNode_t node, unsigned ntiles, const BatchGroups* G);

// Host-side schedule helpers shared by the plan and the batch (srj_plan.cu).
std::vector<int32_t> host_drift_order(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin);
double host_max_cycle_log10(const std::vector<double>& w, const std::vector<int32_t>& q, int nd, const int64_t* dims);
double host_kappa_min(int nd, const int64_t* dims);
// log10 of max |Gamma(kappa)| over [kmin, kmax] for the integer scheme (omega, q).
double host_max_cycle_log10_range(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin,
                                  double kmax);
// Record the message returned by srj_last_error; returns code.
int set_last_error(int code, const char* msg);

// Set the ghost layer of a padded float64 grid to 0.
cudaError_t launch_zero_ghosts(const Geom& g, double* a, cudaStream_t s);
// grad_f = h2 * lambda (interior; ghosts 0); grad_g = B^T lambda + grad_u on the
// ghost layer (interior 0).
cudaError_t launch_adjoint_finish(const Geom& g, double h2, const double* lambda, const double* grad_u,
                                  double* grad_f, double* grad_g, cudaStream_t s);

// grad_g[ghost q] = sum of lambda over the interior neighbours of q; interior 0.
cudaError_t launch_boundary_adjoint(const Geom& g, const double* lambda, double* grad_g, cudaStream_t s);

}  // namespace srj
