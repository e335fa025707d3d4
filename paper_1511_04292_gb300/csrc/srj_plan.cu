// Host runtime and C ABI of the SRJ library (see include/srj.h).
//
// A plan holds one grid, one SRJ schedule (Sect. 2: weights omega_i repeated
// q_i times per M-cycle) in a fixed order, its device workspaces and CUDA
// graphs of one M-cycle of sweeps.  srj_solve replays the cycle graph and
// checks the residual at every cycle end (Sect. 4.1 monitor, on b - A u).
//
// Mixed precision: each cycle runs on the defect equation A e = r in FP32
// with e = 0 at the start and on the boundary, r = b - A u evaluated in FP64;
// u += e in FP64 afterwards.  For a fixed cycle this is the same linear map as
// applying the cycle to u directly (the cycle polynomial acts on the error),
// so the convergence per cycle is that of the FP64 iteration up to FP32
// rounding of the correction.
#include "srj_internal.h"
#include "../../include/srj.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define SRJ_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(SRJ_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                 \
    } while (0)

constexpr int kMaxLevels = 32;
constexpr int64_t kMaxM = int64_t(1) << 20;
constexpr double kMaxFP32CycleNoise = 0.05;  // modelled FP32 rounding left by one cycle (fp32_cycle_noise)
// A solve whose residual stops halving within this factor of the rounding floor
// of the FP64 residual (unit roundoff x ||sum of |terms|||_2) ends at once.
// Solves run to stagnation end at 0.3 - 1.4 times the estimate (FP64 and mixed,
// 256^2 and 2048^2).
constexpr double kFloorFactor = 8.0;
constexpr int kCheckSamples = 20001;

// Largest eigenvalue of D^-1 A on the Dirichlet grid: (2/d) sum_i cos^2(pi / 2(n_i+1)) < 2.
double kappa_max_of(int nd, const int64_t* dims) {
    const double pi = 3.14159265358979323846;
    double s = 0.0;
    for (int i = 0; i < nd; ++i) {
        const double t = std::cos(pi / (2.0 * (double)(dims[i] + 1)));
        s += t * t;
    }
    return (2.0 / nd) * s;
}

double kappa_min_of(int nd, const int64_t* dims) {
    const double pi = 3.14159265358979323846;
    double s = 0.0;
    for (int i = 0; i < nd; ++i) {
        const double t = std::sin(pi / (2.0 * (double)(dims[i] + 1)));
        s += t * t;
    }
    return (2.0 / nd) * s;
}

// log10 |cycle amplification| at kappa: sum_i q_i log10 |1 - omega_i kappa|.
double cycle_log10(const std::vector<double>& w, const std::vector<int32_t>& q, double k) {
    double s = 0.0;
    for (size_t i = 0; i < w.size(); ++i) s += q[i] * std::log10(std::fabs(1.0 - w[i] * k));
    return s;
}

// Largest log10 cycle factor on [kmin, kmax]: dense geometric sampling, then a
// golden-section refinement around every sampled local maximum.
double max_cycle_log10(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin, double kmax) {
    const int n = kCheckSamples;
    std::vector<double> ks(n), vs(n);
    const double lr = std::log(kmax / kmin);
    for (int i = 0; i < n; ++i) {
        ks[i] = kmin * std::exp(lr * i / (n - 1));
        vs[i] = cycle_log10(w, q, ks[i]);
    }
    ks[n - 1] = kmax;
    vs[n - 1] = cycle_log10(w, q, kmax);
    double best = -INFINITY;
    for (int i = 0; i < n; ++i) {
        const bool lmax = (i == 0 || vs[i] >= vs[i - 1]) && (i == n - 1 || vs[i] >= vs[i + 1]);
        if (!lmax) { best = std::max(best, vs[i]); continue; }
        double a = ks[std::max(i - 1, 0)], b = ks[std::min(i + 1, n - 1)];
        const double gr = 0.6180339887498949;
        double c = b - gr * (b - a), d = a + gr * (b - a);
        double fc = cycle_log10(w, q, c), fd = cycle_log10(w, q, d);
        for (int it = 0; it < 80; ++it) {
            if (fc > fd) { b = d; d = c; fd = fc; c = b - gr * (b - a); fc = cycle_log10(w, q, c); }
            else         { a = c; c = d; fc = fd; d = a + gr * (b - a); fd = cycle_log10(w, q, d); }
        }
        best = std::max({best, vs[i], fc, fd});
    }
    return best;
}

// Cycle order that keeps, at every sampled kappa, the running log-product of
// the amplification factors close to its straight line from 0 to the full
// cycle value (a rounding error made at one step is multiplied by the factors
// of the steps after it, so large excursions cost accuracy; Sect. 5.1 asks for
// the large over-relaxations to be spread over the cycle).  Greedy: at step s
// take the level with repetitions left that minimises the largest deviation.
std::vector<int32_t> drift_order_once(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin,
                                      int K) {
    const int P = (int)w.size();
    int64_t M = 0;
    for (int v : q) M += v;
    std::vector<double> L((size_t)P * K), total(K, 0.0), cur(K, 0.0);
    const double lr = std::log(2.0 / kmin);
    for (int j = 0; j < K; ++j) {
        const double k = kmin * std::exp(lr * j / (K - 1));
        for (int i = 0; i < P; ++i) {
            L[(size_t)i * K + j] = std::log(std::fabs(1.0 - w[i] * k));
            total[j] += q[i] * L[(size_t)i * K + j];
        }
    }
    std::vector<int32_t> left(q), order((size_t)M);
    for (int64_t s = 0; s < M; ++s) {
        const double frac = (double)(s + 1) / (double)M;
        int best = -1;
        double bestc = INFINITY;
        for (int i = 0; i < P; ++i) {
            if (left[i] == 0) continue;
            double c = 0.0;
            const double* Li = &L[(size_t)i * K];
            // a level whose deviation already reaches the best one cannot win: stop early
            for (int j = 0; j < K && c < bestc; ++j) c = std::max(c, std::fabs(cur[j] + Li[j] - frac * total[j]));
            if (c < bestc) { bestc = c; best = i; }
        }
        order[(size_t)s] = best;
        left[best] -= 1;
        const double* Lb = &L[(size_t)best * K];
        for (int j = 0; j < K; ++j) cur[j] += Lb[j];
    }
    return order;
}

}  // namespace



// Largest log10 growth of a contiguous run of steps (window) and of a cycle
// suffix, max over a geometric kappa grid on [kmin, 2].
void order_growth(const std::vector<double>& w, const std::vector<int32_t>& order, double kmin, int K,
                  double* window, double* suffix) {
    const int P = (int)w.size();
    std::vector<double> L((size_t)P * K);
    const double lr = std::log(2.0 / kmin);
    for (int j = 0; j < K; ++j) {
        const double k = kmin * std::exp(lr * j / (K - 1));
        for (int i = 0; i < P; ++i) L[(size_t)i * K + j] = std::log10(std::fabs(1.0 - w[i] * k));
    }
    std::vector<double> pre(K, 0.0), lo(K, 0.0), mx_pre(K, 0.0);
    double wmax = 0.0;
    for (int32_t lev : order) {
        const double* Li = &L[(size_t)lev * K];
        for (int j = 0; j < K; ++j) {
            pre[j] += Li[j];
            wmax = std::max(wmax, pre[j] - lo[j]);
            lo[j] = std::min(lo[j], pre[j]);
            mx_pre[j] = std::max(mx_pre[j], pre[j]);
        }
    }
    // suffix from step a = total - prefix(a); max over a of (total - min prefix)
    std::vector<double> minpre(K, 0.0), run(K, 0.0);
    double smax = -INFINITY;
    for (size_t s = 0; s < order.size(); ++s) {
        const double* Li = &L[(size_t)order[s] * K];
        for (int j = 0; j < K; ++j) {
            smax = std::max(smax, pre[j] - run[j]);  // suffix starting at step s
            run[j] += Li[j];
        }
    }
    *window = wmax;
    *suffix = smax;
}

// The greedy pass depends on its sampling grid; run it on a few grids and keep
// the order with the smallest worst-window growth (then suffix growth).  The
// cycle ends with min(4, q_P) steps of the smallest weight: rounding made late
// in a cycle is amplified most near kappa = 2, which omega_P damps by
// |1 - 2 omega_P| per step.  The greedy orders the other steps.
std::vector<int32_t> drift_order(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin) {
    const int P = (int)w.size();
    const int tail = P > 1 ? std::min(4, q[P - 1]) : 0;
    std::vector<int32_t> body_q(q);
    body_q[P - 1] -= tail;
    std::vector<int32_t> best;
    int64_t body_M = 0;
    for (int v : body_q) body_M += v;
    if (body_M > 0) {
        // the four greedy passes are independent: one host thread each
        const int grids[4] = {1000, 2000, 3000, 4000};
        std::vector<int32_t> o[4];
        double wg[4], sg[4];
        std::vector<std::thread> th;
        for (int g = 0; g < 4; ++g)
            th.emplace_back([&, g] {
                o[g] = drift_order_once(w, body_q, kmin, grids[g]);
                order_growth(w, o[g], kmin, 4001, &wg[g], &sg[g]);
            });
        for (auto& t : th) t.join();
        double bw = INFINITY, bs = INFINITY;
        for (int g = 0; g < 4; ++g)
            if (wg[g] < bw || (wg[g] == bw && sg[g] < bs)) { bw = wg[g]; bs = sg[g]; best = o[g]; }
    }
    for (int t = 0; t < tail; ++t) best.push_back(P - 1);
    return best;
}

// Model of the FP32 rounding noise one cycle leaves in the residual, relative
// to a white initial residual.  In the eigenbasis of D^-1 A the correction of a
// cycle started at e = 0 is e_k(kappa) = (1 - prod_{j<=k}(1 - w_j kappa)) / kappa
// after step k; rounding adds eps |e_k| over all modes, the later steps multiply
// it by S_k(kappa) = prod_{j>k}(1 - w_j kappa), the operator by kappa:
//   noise = eps sqrt( sum_k <e_k^2> <kappa^2 S_k^2> ),  <.> = mean over kappa.
double fp32_cycle_noise(const std::vector<double>& omega, const std::vector<int32_t>& order, double kmin,
                        double kmax = 2.0, int samples = 1024) {
    const size_t M = order.size();
    std::vector<double> kap(samples), S(samples, 1.0), Pf(samples, 1.0), back(M);
    for (int j = 0; j < samples; ++j) kap[j] = kmin + (kmax - kmin) * j / (samples - 1);
    for (size_t k = M; k-- > 0;) {
        const double w = omega[(size_t)order[k]];
        double m = 0.0;
        for (int j = 0; j < samples; ++j) {
            const double v = kap[j] * S[j];
            m += v * v;
            S[j] *= 1.0 - w * kap[j];
        }
        back[k] = m / samples;
        if (!std::isfinite(back[k]) || !std::isfinite(S[0]) || !std::isfinite(S[samples - 1])) return INFINITY;
    }
    double total = 0.0;
    for (size_t k = 0; k < M; ++k) {
        const double w = omega[(size_t)order[k]];
        double m = 0.0;
        for (int j = 0; j < samples; ++j) {
            Pf[j] *= 1.0 - w * kap[j];
            const double e = (1.0 - Pf[j]) / kap[j];
            m += e * e;
        }
        total += (m / samples) * back[k];
        if (!std::isfinite(total)) return INFINITY;
    }
    return std::ldexp(std::sqrt(total), -24);
}

// Cycle order for FP32 cycles: the drift order with the first m copies of the
// smallest weight moved from the body to the tail, m in 0, 2, ..., 24 chosen to
// minimise fp32_cycle_noise and backed off while m + 4 would more than double
// it.  Small weights moved from the start of the cycle (where the correction is
// still small) to the end damp the rounding made late in the cycle; moving too
// many unbalances the body.  The cycle polynomial does not depend on the order.
std::vector<int32_t> fp32_order(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin) {
    std::vector<int32_t> base = drift_order(w, q, kmin);
    const int P = (int)w.size();
    if (P < 2) return base;
    const int small = P - 1;
    const size_t tail0 = (size_t)std::min(4, q[P - 1]);
    std::vector<int32_t> body(base.begin(), base.end() - (long)tail0);
    std::vector<size_t> pos;
    for (size_t i = 0; i < body.size(); ++i)
        if (body[i] == small) pos.push_back(i);
    auto cand = [&](int m) {
        std::vector<int32_t> o;
        o.reserve(base.size());
        size_t next = 0;
        for (size_t i = 0; i < body.size(); ++i) {
            if (next < (size_t)m && i == pos[next]) { ++next; continue; }
            o.push_back(body[i]);
        }
        for (size_t t = 0; t < tail0 + (size_t)m; ++t) o.push_back(small);
        return o;
    };
    // the candidates' noise models are independent: one host thread each
    std::vector<int> ms;
    for (int m = 0; m <= 24 && (size_t)m <= pos.size(); m += 2) ms.push_back(m);
    std::vector<double> noise(ms.size());
    {
        std::vector<std::thread> th;
        for (size_t c = 0; c < ms.size(); ++c)
            th.emplace_back([&, c] { noise[c] = fp32_cycle_noise(w, cand(ms[c]), kmin); });
        for (auto& t : th) t.join();
    }
    int best = 0;
    for (size_t c = 0; c < ms.size(); ++c)
        if (noise[c] < noise[(size_t)best / 2]) best = ms[c];
    while (best > 0 && (size_t)(best + 4) / 2 < noise.size() && noise[(size_t)(best + 4) / 2] > 2.0 * noise[(size_t)best / 2])
        best -= 2;
    return cand(best);
}

namespace srj {
std::vector<int32_t> host_drift_order(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin) {
    return fp32_order(w, q, kmin);
}
double host_max_cycle_log10(const std::vector<double>& w, const std::vector<int32_t>& q, int nd,
                            const int64_t* dims) {
    const double kmin = kappa_min_of(nd, dims), kmax = kappa_max_of(nd, dims);
    return kmin < kmax ? max_cycle_log10(w, q, kmin, kmax) : cycle_log10(w, q, kmin);
}
double host_kappa_min(int nd, const int64_t* dims) { return kappa_min_of(nd, dims); }
double host_max_cycle_log10_range(const std::vector<double>& w, const std::vector<int32_t>& q, double kmin,
                                  double kmax) {
    return max_cycle_log10(w, q, kmin, kmax);
}
int set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace srj

struct srj_plan {
    int device = 0;
    srj::Geom g{};
    int64_t dims[3] = {1, 1, 1};
    double h = 0, h2 = 0;
    int precision = SRJ_PREC_FP64;
    bool fused64 = false;  // SRJ_PREC_FP64_FMA: FP64 steps with fused multiply-adds
    std::vector<double> omega;
    std::vector<int32_t> q, order;
    int64_t M = 0;
    std::vector<double> c64;  // omega_k / 2d per step, in cycle order
    double kappa_min = 0, kappa_max = 2, gmax = 0;

    // FP64 workspaces: two iterates and b = h^2 f
    double *ua = nullptr, *ub = nullptr, *b = nullptr;
    // mixed workspaces: two FP32 corrections and the FP32 defect
    float *ea = nullptr, *eb = nullptr, *r32 = nullptr;
    srj::NormScratch ns{};
    int* kstatus = nullptr;  // device status word of the prefetching sweep: ns.result[3]
    double* host_norms = nullptr;  // pinned: l2, linf, rounding floor, then the device status word (int)

    // temporally blocked FP32 sweeps (2-D mixed plans): depth and tensor maps
    int tdepth = 1;
    double sigma = 0.0;              // diagonal shift: A = (2d + sigma) I - neighbours
    double diag64 = 0.0;             // 2d + sigma
    unsigned char* mask = nullptr;   // plan-owned copy of the activity mask (NULL: all active)
    // blocked sweep: 0 = one block of 8 warps per 128 x 64 tile; 1 = persistent blocks of 8 warps (two per SM)
    // with bulk-copy prefetch; 2 = one block of 16 warps per 128 x 128 tile; 3 = persistent blocks of 16 warps
    // (one per SM) with bulk-copy prefetch; 4 / 5 = variants 0 / 2 with an L2 prefetch of the next wave's tiles
    int variant = 0;
    int sm_count = 152;
    float* e_final = nullptr;  // buffer holding the correction after one cycle
    double *host_f = nullptr, *host_u = nullptr;  // device staging of srj_solve_host (allocated on first use)

    cudaStream_t cap = nullptr;             // private stream used for graph capture
    cudaGraphExec_t cycle_exec[2] = {nullptr, nullptr};  // start buffer a / b
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;            // brackets of each cycle graph

    ~srj_plan() {
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        for (auto& ge : cycle_exec) if (ge) cudaGraphExecDestroy(ge);
        if (cap) cudaStreamDestroy(cap);
        cudaFree(ua); cudaFree(ub); cudaFree(b);
        cudaFree(ea); cudaFree(eb); cudaFree(r32);
        cudaFree(ns.partials); cudaFree(ns.counter); cudaFree(ns.result);
        cudaFree(mask);
        cudaFree(host_f); cudaFree(host_u);
        if (host_norms) cudaFreeHost(host_norms);
    }
};

namespace {

// Issue `count` FP32 steps of the cycle order from position `first`, starting
// from buffer ea; returns the buffer that holds the result in *final.
cudaError_t issue_f32_steps(srj_plan* p, int64_t first, int64_t count, cudaStream_t s, float** final) {
    const int64_t M = p->M;
    float* in = p->ea;
    float* out = p->eb;
    cudaError_t err = cudaSuccess;
    const int T = p->tdepth;
    for (int64_t k = 0; k < count && err == cudaSuccess;) {
        const int n = (int)std::min<int64_t>(T, count - k);
        if (T == 1 || n == 1) {
            err = srj::launch_sweep_f32(p->g, in, out, p->r32, (float)p->c64[(size_t)((first + k) % M)], s, (float)p->diag64, p->mask);
        } else if (p->g.nd == 3) {  // 3-D: 2 or 3 steps per launch, z-streamed tiles
            srj::TbSteps st{};
            st.T = n;
            for (int t = 0; t < n; ++t) st.c[t] = (float)p->c64[(size_t)((first + k + t) % M)];
            err = srj::launch_sweep3_f32_tb(p->g, in, p->r32, out, st, p->sm_count, s);
        } else {
            srj::TbSteps st{};
            st.T = n;
            for (int t = 0; t < n; ++t) st.c[t] = (float)p->c64[(size_t)((first + k + t) % M)];
            const int v = p->variant;
            const int warps = (v == 2 || v == 3 || v == 5) ? 16 : 8;
            err = (v == 1 || v == 3) ? srj::launch_sweep_f32_tbp(p->g, in, p->r32, out, st, warps, 16 / warps,
                                                                 p->sm_count, p->kstatus, s)
                                     : srj::launch_sweep_f32_tb(p->g, in, p->r32, out, st, warps, s,
                                                                v >= 4 ? (16 / warps) * p->sm_count : 0);
        }
        std::swap(in, out);
        k += n;
    }
    *final = in;
    return err;
}

// Capture one M-cycle of sweeps starting from buffer `start` (0 = a, 1 = b).
int capture_cycle(srj_plan* p, int start) {
    cudaGraph_t graph = nullptr;
    SRJ_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    if (p->precision == SRJ_PREC_FP64) {
        for (int64_t k = 0; k < p->M && err == cudaSuccess; ++k) {
            const bool from_a = ((k + start) % 2) == 0;
            err = srj::launch_sweep_f64(p->g, from_a ? p->ua : p->ub, from_a ? p->ub : p->ua, p->b,
                                        p->c64[(size_t)k], p->cap, p->diag64, p->mask, p->fused64);
        }
    } else {
        err = cudaMemsetAsync(p->ea, 0, sizeof(float) * (size_t)p->g.n32, p->cap);
        if (err == cudaSuccess) err = issue_f32_steps(p, 0, p->M, p->cap, &p->e_final);
    }
    cudaError_t e2 = cudaStreamEndCapture(p->cap, &graph);
    if (err != cudaSuccess) { if (graph) cudaGraphDestroy(graph); SRJ_CUDA(err); }
    SRJ_CUDA(e2);
    cudaError_t e3 = cudaGraphInstantiate(&p->cycle_exec[start], graph, 0);
    cudaGraphDestroy(graph);
    SRJ_CUDA(e3);
    return SRJ_OK;
}

int check_plan(srj_plan_t p) {
    if (!p) return fail(SRJ_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    SRJ_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return fail(SRJ_ERR_INVALID_ARG, "plan was created on device %d, current is %d", p->device, dev);
    return SRJ_OK;
}

// The device status word of the prefetching sweep (0, or kStatusTimeout when a
// bounded wait ran out); reset to 0 when it is reported.
int take_kstatus(srj_plan* p, int word, cudaStream_t s) {
    if (word == 0) return SRJ_OK;
    SRJ_CUDA(cudaMemsetAsync(p->kstatus, 0, sizeof(int), s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    return fail(SRJ_ERR_TIMEOUT, "a bounded wait of the prefetching sweep ran out (%d); the results are incomplete", word);
}

int read_norms(srj_plan* p, cudaStream_t s, double* l2, double* linf) {
    SRJ_CUDA(cudaMemcpyAsync(p->host_norms, p->ns.result, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    *l2 = p->host_norms[0];
    *linf = p->host_norms[1];
    int word = 0;
    std::memcpy(&word, p->host_norms + 3, sizeof(int));
    return take_kstatus(p, word, s);
}

// Read the device status word alone (after work that leaves no norms).
int read_kstatus(srj_plan* p, cudaStream_t s) {
    int* h = reinterpret_cast<int*>(p->host_norms + 3);
    SRJ_CUDA(cudaMemcpyAsync(h, p->kstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    return take_kstatus(p, *h, s);
}

// Re-capture the cycle graphs (after a change of the temporal depth).
int recapture(srj_plan* p) {
    for (auto& ge : p->cycle_exec)
        if (ge) { cudaGraphExecDestroy(ge); ge = nullptr; }
    int rc = capture_cycle(p, 0);
    if (rc == SRJ_OK && p->precision == SRJ_PREC_FP64 && (p->M % 2) == 1) rc = capture_cycle(p, 1);
    return rc;
}

int set_depth(srj_plan* p, int T) {
    if (T < 1 || T > srj::tb_max_steps()) return fail(SRJ_ERR_INVALID_ARG, "temporal depth must be in 1..%d", srj::tb_max_steps());
    if (T > 1 && p->precision != SRJ_PREC_MIXED)
        return fail(SRJ_ERR_INVALID_ARG, "temporal blocking is available for mixed-precision plans");
    if (T > srj::tb3_max_steps() && p->g.nd == 3)
        return fail(SRJ_ERR_INVALID_ARG, "3-D plans take temporal depth 1..%d", srj::tb3_max_steps());
    if (T > 1 && (p->mask || p->sigma != 0.0))
        return fail(SRJ_ERR_INVALID_ARG, "temporal blocking implements the plain operator (no mask, no shift)");
    p->tdepth = T;
    return recapture(p);
}

}  // namespace

extern "C" {

const char* srj_last_error(void) { return g_last_error.c_str(); }

const char* srj_version(void) { return "srj-gb300 0.1 (sm_103a)"; }

int srj_kappa_min(int ndim, const int64_t* dims, double* kappa_min) {
    if ((ndim != 2 && ndim != 3) || !dims || !kappa_min) return fail(SRJ_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < ndim; ++i) if (dims[i] < 1) return fail(SRJ_ERR_INVALID_ARG, "dims must be >= 1");
    *kappa_min = kappa_min_of(ndim, dims);
    return SRJ_OK;
}

int srj_kappa_range(int ndim, const int64_t* dims, double* kappa_min, double* kappa_max) {
    if ((ndim != 2 && ndim != 3) || !dims) return fail(SRJ_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < ndim; ++i) if (dims[i] < 1) return fail(SRJ_ERR_INVALID_ARG, "dims must be >= 1");
    if (kappa_min) *kappa_min = kappa_min_of(ndim, dims);
    if (kappa_max) *kappa_max = kappa_max_of(ndim, dims);
    return SRJ_OK;
}

int srj_neff(int ndim, const int64_t* dims, double* n_eff) {
    if ((ndim != 2 && ndim != 3) || !dims || !n_eff) return fail(SRJ_ERR_INVALID_ARG, "bad arguments");
    for (int i = 0; i < ndim; ++i) if (dims[i] < 1) return fail(SRJ_ERR_INVALID_ARG, "dims must be >= 1");
    // Eq. effectiveNDirichlet with N_i = n_i + 1 zones; the sum is kappa_min
    *n_eff = M_PI / (2.0 * std::asin(std::sqrt(kappa_min_of(ndim, dims))));
    return SRJ_OK;
}

static int check_levels(int P, const double* omega, const int32_t* q, int64_t* M) {
    if (P < 1 || P > kMaxLevels) return fail(SRJ_ERR_INVALID_ARG, "P must be in 1..%d", kMaxLevels);
    if (!omega || !q) return fail(SRJ_ERR_INVALID_ARG, "omega and q must be non-NULL");
    *M = 0;
    for (int i = 0; i < P; ++i) {
        if (!(omega[i] > 0.0) || !std::isfinite(omega[i])) return fail(SRJ_ERR_INVALID_ARG, "omega[%d] must be finite and > 0", i);
        if (q[i] < 1) return fail(SRJ_ERR_INVALID_ARG, "q[%d] must be >= 1", i);
        *M += q[i];
    }
    if (*M > kMaxM) return fail(SRJ_ERR_INVALID_ARG, "M = %lld exceeds %lld", (long long)*M, (long long)kMaxM);
    return SRJ_OK;
}

int srj_schedule_check(int P, const double* omega, const int32_t* q, double kappa_min, double kappa_max,
                       double* log10_max) {
    int64_t M = 0;
    int rc = check_levels(P, omega, q, &M);
    if (rc) return rc;
    if (!log10_max || !(kappa_min > 0.0) || !(kappa_min < kappa_max) || !(kappa_max <= 2.0))
        return fail(SRJ_ERR_INVALID_ARG, "need 0 < kappa_min < kappa_max <= 2 and an output pointer");
    *log10_max = max_cycle_log10(std::vector<double>(omega, omega + P), std::vector<int32_t>(q, q + P), kappa_min,
                                 kappa_max);
    return SRJ_OK;
}

int srj_schedule_order(int P, const double* omega, const int32_t* q, double kappa_min, int32_t* order_out) {
    int64_t M = 0;
    int rc = check_levels(P, omega, q, &M);
    if (rc) return rc;
    if (!order_out || !(kappa_min > 0.0) || !(kappa_min < 2.0)) return fail(SRJ_ERR_INVALID_ARG, "bad kappa_min or output");
    std::vector<int32_t> o = fp32_order(std::vector<double>(omega, omega + P), std::vector<int32_t>(q, q + P), kappa_min);
    std::memcpy(order_out, o.data(), sizeof(int32_t) * o.size());
    return SRJ_OK;
}

int srj_plan_create(srj_plan_t* out, int ndim, const int64_t* dims, double h, int P, const double* omega,
                    const int32_t* q, const int32_t* order, int precision) {
    if (!out) return fail(SRJ_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(SRJ_ERR_INVALID_ARG, "ndim must be 2 or 3 (got %d)", ndim);
    if (!dims || !omega || !q) return fail(SRJ_ERR_INVALID_ARG, "dims, omega and q must be non-NULL");
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1 || dims[i] > (int64_t(1) << 30))
            return fail(SRJ_ERR_INVALID_ARG, "dims[%d] = %lld out of range", i, (long long)dims[i]);
    if (!(h > 0.0) || !std::isfinite(h)) return fail(SRJ_ERR_INVALID_ARG, "h must be finite and > 0");
    if (precision != SRJ_PREC_FP64 && precision != SRJ_PREC_MIXED && precision != SRJ_PREC_FP64_FMA)
        return fail(SRJ_ERR_INVALID_ARG, "unknown precision %d", precision);
    const bool fused64 = precision == SRJ_PREC_FP64_FMA;
    if (fused64) precision = SRJ_PREC_FP64;
    int64_t M = 0;
    if (int rc0 = check_levels(P, omega, q, &M)) return rc0;
    if (dims[1] > 262140) return fail(SRJ_ERR_INVALID_ARG, "dims[1] must be <= 262140 (launch grid limit)");
    const int64_t pts = dims[0] * dims[1] * (ndim == 3 ? dims[2] : 1);
    if (pts > (int64_t(1) << 36)) return fail(SRJ_ERR_INVALID_ARG, "grid too large");

    srj_plan* p = new (std::nothrow) srj_plan();
    if (!p) return fail(SRJ_ERR_NO_MEMORY, "host allocation failed");
    auto bail = [&](int code) { delete p; return code; };

    p->omega.assign(omega, omega + P);
    p->q.assign(q, q + P);
    p->M = M;
    p->precision = precision;
    p->fused64 = fused64;
    p->h = h;
    p->h2 = h * h;
    for (int i = 0; i < ndim; ++i) p->dims[i] = dims[i];
    p->g = srj::make_geom(ndim, dims);
    p->kappa_min = kappa_min_of(ndim, dims);
    p->kappa_max = kappa_max_of(ndim, dims);

    p->gmax = p->kappa_min < p->kappa_max ? max_cycle_log10(p->omega, p->q, p->kappa_min, p->kappa_max)
                                          : cycle_log10(p->omega, p->q, p->kappa_min);
    if (!(p->gmax < 0.0))
        return bail(fail(SRJ_ERR_BAD_SCHEDULE,
                         "integer scheme does not contract on [kappa_min=%.6g, kappa_max=%.6g]: max log10 cycle factor %.4g",
                         p->kappa_min, p->kappa_max, p->gmax));

    if (order) {
        std::vector<int64_t> cnt(P, 0);
        for (int64_t k = 0; k < M; ++k) {
            if (order[k] < 0 || order[k] >= P) return bail(fail(SRJ_ERR_INVALID_ARG, "order[%lld] out of range", (long long)k));
            cnt[order[k]]++;
        }
        for (int i = 0; i < P; ++i)
            if (cnt[i] != q[i]) return bail(fail(SRJ_ERR_INVALID_ARG, "order uses level %d %lld times, q=%d", i, (long long)cnt[i], q[i]));
        p->order.assign(order, order + M);
    } else {
        p->order = fp32_order(p->omega, p->q, p->kappa_min);
    }
    if (precision == SRJ_PREC_MIXED) {
        const double nz = fp32_cycle_noise(p->omega, p->order, p->kappa_min);
        if (!(nz < kMaxFP32CycleNoise))
            return bail(fail(SRJ_ERR_BAD_SCHEDULE,
                             "cycle order amplifies FP32 rounding too much (modelled cycle noise %.3g, limit %.3g); "
                             "use another order or FP64", nz, kMaxFP32CycleNoise));
    }
    p->diag64 = (double)(2 * ndim);
    p->c64.resize((size_t)M);
    for (int64_t k = 0; k < M; ++k) p->c64[(size_t)k] = p->omega[p->order[(size_t)k]] / p->diag64;

    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(fail(SRJ_ERR_CUDA, "no CUDA device"));
    auto alloc = [&](void** ptr, size_t bytes) -> bool { return cudaMalloc(ptr, bytes) == cudaSuccess; };
    bool ok = true;
    if (precision == SRJ_PREC_FP64) {
        const size_t by = sizeof(double) * (size_t)p->g.n64;
        ok = alloc((void**)&p->ua, by) && alloc((void**)&p->ub, by) && alloc((void**)&p->b, by);
    } else {
        const size_t by = sizeof(float) * (size_t)p->g.n32;
        ok = alloc((void**)&p->ea, by) && alloc((void**)&p->eb, by) && alloc((void**)&p->r32, by);
        if (ok) ok = cudaMemset(p->ea, 0, by) == cudaSuccess && cudaMemset(p->eb, 0, by) == cudaSuccess &&
                     cudaMemset(p->r32, 0, by) == cudaSuccess;
    }
    ok = ok && alloc((void**)&p->ns.partials, sizeof(double) * 3 * srj::kMaxNormBlocks) &&
         alloc((void**)&p->ns.counter, sizeof(unsigned)) && alloc((void**)&p->ns.result, 4 * sizeof(double));
    if (!ok) { cudaGetLastError(); return bail(fail(SRJ_ERR_NO_MEMORY, "device allocation failed")); }
    if (ok) p->kstatus = reinterpret_cast<int*>(p->ns.result + 3);
    if (cudaMemset(p->ns.counter, 0, sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(p->ns.result, 0, 4 * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&p->host_norms, 4 * sizeof(double)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(SRJ_ERR_CUDA, "plan setup failed"));
    }
    if (precision == SRJ_PREC_MIXED) {
        if (srj::tb_prepare() != cudaSuccess || srj::tb3_prepare() != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(SRJ_ERR_CUDA, "set-up of the blocked sweep failed"));
        }
        p->tdepth = ndim == 2 ? 8 : 2;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) == cudaSuccess && sms > 0)
            p->sm_count = sms;
    }
    int rc = recapture(p);
    if (rc != SRJ_OK) return bail(rc);
    if (cudaStreamSynchronize(p->cap) != cudaSuccess) return bail(fail(SRJ_ERR_CUDA, "plan setup sync failed"));
    *out = p;
    return SRJ_OK;
}

int srj_plan_destroy(srj_plan_t plan) {
    if (!plan) return SRJ_OK;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->device) cudaSetDevice(plan->device);
    cudaDeviceSynchronize();
    delete plan;
    if (dev >= 0 && dev != plan->device) cudaSetDevice(dev);
    return SRJ_OK;
}

int srj_plan_set_temporal_depth(srj_plan_t plan, int T) {
    int rc = check_plan(plan);
    if (rc) return rc;
    return set_depth(plan, T);
}

int srj_plan_set_operator(srj_plan_t p, double sigma, const unsigned char* mask, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    const int nd = p->g.nd;
    const double diag = (double)(2 * nd) + sigma;
    if (!std::isfinite(sigma) || !(diag > 0.0)) return fail(SRJ_ERR_INVALID_ARG, "need 2d + sigma > 0");
    // spectrum of D^-1 A for the shifted operator; a mask selects a principal
    // submatrix, whose eigenvalues lie in the same range (Cauchy interlacing)
    const double km = ((double)(2 * nd) * p->kappa_min + sigma) / diag;
    const double kx = ((double)(2 * nd) * p->kappa_max + sigma) / diag;
    if (!(km > 0.0)) return fail(SRJ_ERR_BAD_SCHEDULE, "shifted operator is not positive definite on this grid");
    const double gmax = km < kx ? max_cycle_log10(p->omega, p->q, km, kx) : cycle_log10(p->omega, p->q, km);
    if (!(gmax < 0.0))
        return fail(SRJ_ERR_BAD_SCHEDULE, "integer scheme does not contract on the shifted spectrum [%.6g, %.6g]", km, kx);
    cudaStream_t s = (cudaStream_t)stream;
    if (mask) {
        if (!p->mask) SRJ_CUDA(cudaMalloc((void**)&p->mask, (size_t)p->g.n64));
        SRJ_CUDA(cudaMemcpyAsync(p->mask, mask, (size_t)p->g.n64, cudaMemcpyDeviceToDevice, s));
        SRJ_CUDA(cudaStreamSynchronize(s));
    } else if (p->mask) {
        SRJ_CUDA(cudaFree(p->mask));
        p->mask = nullptr;
    }
    p->sigma = sigma;
    p->diag64 = diag;
    p->gmax = gmax;
    for (int64_t k = 0; k < p->M; ++k) p->c64[(size_t)k] = p->omega[p->order[(size_t)k]] / diag;
    // the blocked kernels implement the plain operator only
    if (p->mask || sigma != 0.0) p->tdepth = 1;
    return recapture(p);
}

int srj_plan_set_sweep_variant(srj_plan_t plan, int v) {
    int rc = check_plan(plan);
    if (rc) return rc;
    if (v < 0 || v > 5) return fail(SRJ_ERR_INVALID_ARG, "sweep variant must be in 0..5");
    plan->variant = v;
    return recapture(plan);
}

int srj_selftest_wait_timeout(int64_t limit_us, void* stream) {
    if (limit_us < 1 || limit_us > 1000000) return fail(SRJ_ERR_INVALID_ARG, "limit_us must be in 1..1e6");
    const int64_t dims[2] = {64, 64};
    const srj::Geom g = srj::make_geom(2, dims);
    cudaStream_t s = (cudaStream_t)stream;
    SRJ_CUDA(srj::tb_prepare());
    float* buf = nullptr;
    const size_t by = sizeof(float) * (size_t)g.n32;
    SRJ_CUDA(cudaMalloc((void**)&buf, 3 * by + 256));
    int* status = reinterpret_cast<int*>(reinterpret_cast<char*>(buf) + 3 * by);
    int host_status = 0;
    srj::TbSteps st{};
    st.T = 2;
    st.c[0] = st.c[1] = 0.25f;
    cudaError_t e = cudaMemsetAsync(buf, 0, 3 * by + 256, s);
    if (e == cudaSuccess)
        e = srj::launch_sweep_f32_tbp(g, buf, buf + g.n32, buf + 2 * g.n32, st, 8, 2, 4, status, s,
                                      (uint64_t)limit_us * 1000ull, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    SRJ_CUDA(e);
    if (host_status == srj::kStatusTimeout)
        return fail(SRJ_ERR_TIMEOUT, "bounded waits ran out after %lld us and were reported (self-test passed)",
                    (long long)limit_us);
    return fail(SRJ_OK, "no bounded wait ran out (status word %d)", host_status);
}

int srj_plan_sweep_variant(srj_plan_t plan, int* v) {
    if (!plan || !v) return fail(SRJ_ERR_INVALID_ARG, "NULL argument");
    *v = plan->variant;
    return SRJ_OK;
}

int srj_plan_temporal_depth(srj_plan_t plan, int* T) {
    if (!plan || !T) return fail(SRJ_ERR_INVALID_ARG, "NULL argument");
    *T = plan->tdepth;
    return SRJ_OK;
}

int srj_plan_autotune(srj_plan_t p, void* stream, int* best_T, float* best_us_per_step) {
    int rc = check_plan(p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // candidates (T, variant): the unblocked sweep, then the blocked variants for T = 2..8 (2-D) or T = 2, 3 (3-D)
    int candT[43], candV[43];
    for (int i = 0; i < 8; ++i) { candT[i] = i + 1; candV[i] = 0; }
    for (int v = 1, i = 8; v <= 5; ++v)
        for (int T = 2; T <= 8; ++T, ++i) { candT[i] = T; candV[i] = v; }
    int ncand = (p->precision == SRJ_PREC_MIXED && !p->mask && p->sigma == 0.0) ? (p->g.nd == 2 ? 43 : 3) : 1;
    int bestV = p->variant;
    const int64_t steps = std::min<int64_t>(std::max<int64_t>(p->M, 24), 840);  // 840 = lcm(1..8)
    float best = INFINITY;
    int bestT = p->tdepth;
    for (int ci = 0; ci < ncand; ++ci) {
        p->tdepth = candT[ci];
        p->variant = candV[ci];
        float* fin = nullptr;
        float ms_best = INFINITY;
        for (int rep = 0; rep < 3; ++rep) {
            SRJ_CUDA(cudaEventRecord(p->ev0, s));
            if (p->precision == SRJ_PREC_MIXED) {
                SRJ_CUDA(issue_f32_steps(p, 0, steps, s, &fin));
            } else {
                for (int64_t k = 0; k < steps; ++k) {
                    const bool a = (k % 2) == 0;
                    SRJ_CUDA(srj::launch_sweep_f64(p->g, a ? p->ua : p->ub, a ? p->ub : p->ua, p->b,
                                                   p->c64[(size_t)(k % p->M)], s, p->diag64, p->mask, p->fused64));
                }
            }
            SRJ_CUDA(cudaEventRecord(p->ev1, s));
            SRJ_CUDA(cudaEventSynchronize(p->ev1));
            float ms = 0.f;
            SRJ_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
            ms_best = std::min(ms_best, ms);
        }
        if (ms_best < best) { best = ms_best; bestT = candT[ci]; bestV = candV[ci]; }
    }
    p->variant = bestV;
    if ((rc = read_kstatus(p, s))) return rc;
    if (best_T) *best_T = bestT;
    if (best_us_per_step) *best_us_per_step = best * 1000.f / (float)steps;
    return set_depth(p, bestT);
}

int srj_plan_info(srj_plan_t plan, int64_t* M, double* kappa_min, double* gmax) {
    if (!plan) return fail(SRJ_ERR_INVALID_ARG, "plan is NULL");
    if (M) *M = plan->M;
    if (kappa_min) *kappa_min = plan->kappa_min;
    if (gmax) *gmax = plan->gmax;
    return SRJ_OK;
}

int srj_plan_order(srj_plan_t plan, int32_t* out) {
    if (!plan || !out) return fail(SRJ_ERR_INVALID_ARG, "NULL argument");
    std::memcpy(out, plan->order.data(), sizeof(int32_t) * (size_t)plan->M);
    return SRJ_OK;
}

int srj_residual(srj_plan_t p, const double* f, const double* u, double* r_out, double* l2, double* linf,
                 void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!f || !u) return fail(SRJ_ERR_INVALID_ARG, "f and u must be non-NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (r_out) SRJ_CUDA(cudaMemsetAsync(r_out, 0, sizeof(double) * (size_t)p->g.n64, s));
    SRJ_CUDA(srj::launch_residual(p->g, u, f, p->h2, r_out, nullptr, 1.0, p->ns, s, p->diag64, p->mask));
    double a, bb;
    rc = read_norms(p, s, &a, &bb);
    if (rc) return rc;
    if (l2) *l2 = a;
    if (linf) *linf = bb;
    return SRJ_OK;
}

int srj_steps(srj_plan_t p, const double* f, double* u, int64_t first, int64_t count, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!f || !u || count < 0) return fail(SRJ_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t M = p->M;
    first = ((first % M) + M) % M;
    if (p->precision == SRJ_PREC_FP64) {
        const size_t by = sizeof(double) * (size_t)p->g.n64;
        SRJ_CUDA(cudaMemcpyAsync(p->ua, u, by, cudaMemcpyDeviceToDevice, s));
        SRJ_CUDA(cudaMemcpyAsync(p->ub, u, by, cudaMemcpyDeviceToDevice, s));
        SRJ_CUDA(srj::launch_scale_source(p->g, p->h2, f, p->b, s));
        for (int64_t k = 0; k < count; ++k) {
            const bool from_a = (k % 2) == 0;
            SRJ_CUDA(srj::launch_sweep_f64(p->g, from_a ? p->ua : p->ub, from_a ? p->ub : p->ua, p->b,
                                           p->c64[(size_t)((first + k) % M)], s, p->diag64, p->mask, p->fused64));
        }
        SRJ_CUDA(cudaMemcpyAsync(u, (count % 2) ? p->ub : p->ua, by, cudaMemcpyDeviceToDevice, s));
    } else {
        SRJ_CUDA(srj::launch_to_f32(p->g, u, p->ea, s));
        SRJ_CUDA(srj::launch_to_f32(p->g, u, p->eb, s));
        SRJ_CUDA(cudaMemsetAsync(p->r32, 0, sizeof(float) * (size_t)p->g.n32, s));
        SRJ_CUDA(srj::launch_source_f32(p->g, p->h2, f, p->r32, s));
        float* fin = nullptr;
        SRJ_CUDA(issue_f32_steps(p, first, count, s, &fin));
        SRJ_CUDA(srj::launch_from_f32(p->g, fin, u, s));
    }
    return read_kstatus(p, s);
}

static int solve_impl(srj_plan_t p, const double* f, double h2, double* u, double tol, int64_t max_cycles,
                      void* stream, srj_stats_t* stats);

int srj_solve(srj_plan_t p, const double* f, double* u, double tol, int64_t max_cycles, void* stream,
              srj_stats_t* stats) {
    int rc = check_plan(p);
    if (rc) return rc;
    return solve_impl(p, f, p->h2, u, tol, max_cycles, stream, stats);
}

int srj_solve_host(srj_plan_t p, const double* f, double* u, double tol, int64_t max_cycles, void* stream,
                   srj_stats_t* stats) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!f || !u) return fail(SRJ_ERR_INVALID_ARG, "f and u must be non-NULL");
    const size_t by64 = sizeof(double) * (size_t)p->g.n64;
    if (!p->host_f) {
        if (cudaMalloc(&p->host_f, by64) != cudaSuccess || cudaMalloc(&p->host_u, by64) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(p->host_f);
            cudaFree(p->host_u);
            p->host_f = p->host_u = nullptr;
            return fail(SRJ_ERR_NO_MEMORY, "device staging buffers for host arrays");
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    SRJ_CUDA(cudaMemcpyAsync(p->host_f, f, by64, cudaMemcpyHostToDevice, s));
    SRJ_CUDA(cudaMemcpyAsync(p->host_u, u, by64, cudaMemcpyHostToDevice, s));
    rc = solve_impl(p, p->host_f, p->h2, p->host_u, tol, max_cycles, stream, stats);
    if (rc != SRJ_OK && rc != SRJ_ERR_NOT_CONVERGED && rc != SRJ_ERR_DIVERGED) return rc;
    SRJ_CUDA(cudaMemcpyAsync(u, p->host_u, by64, cudaMemcpyDeviceToHost, s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    return rc;
}

int srj_gradient(srj_plan_t p, const double* grad_u, double* lambda, double* grad_f, double* grad_g, double tol,
                 int64_t max_cycles, void* stream, srj_stats_t* stats) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!grad_u || !lambda || !grad_f || !grad_g) return fail(SRJ_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    // A is symmetric: lambda solves A lambda = dL/du (interior) with zero ghosts;
    // the right-hand side is passed as the source with h^2 replaced by 1.
    SRJ_CUDA(srj::launch_zero_ghosts(p->g, lambda, s));
    rc = solve_impl(p, grad_u, 1.0, lambda, tol, max_cycles, stream, stats);
    if (rc != SRJ_OK && rc != SRJ_ERR_NOT_CONVERGED) return rc;
    SRJ_CUDA(srj::launch_adjoint_finish(p->g, p->h2, lambda, grad_u, grad_f, grad_g, s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    return rc;
}

static int solve_impl(srj_plan_t p, const double* f, double h2, double* u, double tol, int64_t max_cycles,
                      void* stream, srj_stats_t* stats) {
    int rc = SRJ_OK;
    if (!f || !u) return fail(SRJ_ERR_INVALID_ARG, "f and u must be non-NULL");
    if (!(tol >= 0.0) || max_cycles < 0) return fail(SRJ_ERR_INVALID_ARG, "tol must be >= 0 and max_cycles >= 0");
    if (!p->cycle_exec[0] || (p->precision == SRJ_PREC_FP64 && (p->M % 2) == 1 && !p->cycle_exec[1]))
        return fail(SRJ_ERR_CUDA, "the plan has no cycle graph (a failed re-capture)");
    cudaStream_t s = (cudaStream_t)stream;
    srj_stats_t st{};
    const size_t by64 = sizeof(double) * (size_t)p->g.n64;
    double l2 = 0, linf = 0;
    int cur = 0;  // FP64: which buffer holds the iterate (0 = ua, 1 = ub)
    double scale = 1.0;

    if (p->precision == SRJ_PREC_FP64) {
        SRJ_CUDA(cudaMemcpyAsync(p->ua, u, by64, cudaMemcpyDeviceToDevice, s));
        SRJ_CUDA(cudaMemcpyAsync(p->ub, u, by64, cudaMemcpyDeviceToDevice, s));
        SRJ_CUDA(srj::launch_scale_source(p->g, h2, f, p->b, s));
        SRJ_CUDA(srj::launch_residual(p->g, p->ua, p->b, 1.0, nullptr, nullptr, 1.0, p->ns, s, p->diag64, p->mask));
    } else {
        const size_t by32 = sizeof(float) * (size_t)p->g.n32;
        SRJ_CUDA(cudaMemsetAsync(p->eb, 0, by32, s));  // ghosts of the corrections are 0
        SRJ_CUDA(srj::launch_residual(p->g, u, f, h2, nullptr, nullptr, 1.0, p->ns, s, p->diag64, p->mask));
    }
    if ((rc = read_norms(p, s, &l2, &linf))) return rc;
    st.residual_checks = 1;
    st.r0_l2 = l2;
    st.res_l2 = l2;
    st.res_linf = linf;
    st.rel_res = l2 > 0 ? 1.0 : 0.0;
    int status = SRJ_OK;
    if (!std::isfinite(l2)) status = fail(SRJ_ERR_DIVERGED, "initial residual is not finite");
    else if (l2 > 0.0 && !(1.0 <= tol)) {
        status = SRJ_ERR_NOT_CONVERGED;
        if (p->precision == SRJ_PREC_MIXED) {
            // FP32 defect scaled by a power of two so that its largest entry is ~1
            int ex = 0;
            std::frexp(linf, &ex);
            scale = std::ldexp(1.0, -ex);
            SRJ_CUDA(srj::launch_residual(p->g, u, f, h2, nullptr, p->r32, scale, p->ns, s, p->diag64, p->mask));
        }
        double best = st.r0_l2;
        int stall = 0;
        for (int64_t c = 0; c < max_cycles; ++c) {
            SRJ_CUDA(cudaEventRecord(p->ev0, s));
            if (p->precision == SRJ_PREC_FP64) {
                SRJ_CUDA(cudaGraphLaunch(p->cycle_exec[p->M % 2 ? cur : 0], s));
                SRJ_CUDA(cudaEventRecord(p->ev1, s));
                if (p->M % 2) cur ^= 1;
                SRJ_CUDA(srj::launch_residual(p->g, cur ? p->ub : p->ua, p->b, 1.0, nullptr, nullptr, 1.0, p->ns, s, p->diag64, p->mask));
            } else {
                SRJ_CUDA(cudaGraphLaunch(p->cycle_exec[0], s));
                SRJ_CUDA(cudaEventRecord(p->ev1, s));
                SRJ_CUDA(srj::launch_update(p->g, u, p->e_final, 1.0 / scale, s, p->mask));
                SRJ_CUDA(srj::launch_residual(p->g, u, f, h2, nullptr, p->r32, scale, p->ns, s, p->diag64, p->mask));
            }
            if ((rc = read_norms(p, s, &l2, &linf))) return rc;
            float ms = 0.f;
            SRJ_CUDA(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
            st.sweep_ms += ms;
            st.cycles = c + 1;
            st.sweeps = st.cycles * p->M;
            st.residual_checks += 1;
            st.res_l2 = l2;
            st.res_linf = linf;
            st.rel_res = l2 / st.r0_l2;
            if (!std::isfinite(l2) || l2 > 1e6 * st.r0_l2) {
                status = fail(SRJ_ERR_DIVERGED, "residual diverged at cycle %lld (rel %.3g)", (long long)(c + 1), st.rel_res);
                break;
            }
            if (st.rel_res <= tol) { status = SRJ_OK; break; }
            st.res_floor = p->host_norms[2];
            const bool halved = l2 < 0.5 * best;
            if (!halved && l2 <= kFloorFactor * st.res_floor) {
                // within a small factor of the rounding floor of the FP64 residual, and no
                // longer halving: further cycles cannot reach tol
                st.stagnated = 1;
                status = fail(SRJ_ERR_NOT_CONVERGED,
                              "residual reached the FP64 rounding floor at rel %.3g after %lld cycles (floor %.3g, tol %.3g)",
                              st.rel_res, (long long)(c + 1), st.res_floor / st.r0_l2, tol);
                break;
            }
            if (halved) { best = l2; stall = 0; }
            else if (++stall >= 4) {
                st.stagnated = 1;
                status = fail(SRJ_ERR_NOT_CONVERGED, "residual stagnated at rel %.3g after %lld cycles (tol %.3g)",
                              st.rel_res, (long long)(c + 1), tol);
                break;
            }
        }
        if (status == SRJ_ERR_NOT_CONVERGED && !st.stagnated)
            fail(SRJ_ERR_NOT_CONVERGED, "not converged after %lld cycles (rel %.3g)", (long long)max_cycles, st.rel_res);
    }
    if (p->precision == SRJ_PREC_FP64 && st.cycles > 0)
        SRJ_CUDA(cudaMemcpyAsync(u, cur ? p->ub : p->ua, by64, cudaMemcpyDeviceToDevice, s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    if (stats) *stats = st;
    return status;
}

int srj_boundary_adjoint(srj_plan_t p, const double* lambda, double* grad_g, void* stream) {
    int rc = check_plan(p);
    if (rc) return rc;
    if (!lambda || !grad_g) return fail(SRJ_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    SRJ_CUDA(srj::launch_boundary_adjoint(p->g, lambda, grad_g, s));
    SRJ_CUDA(cudaStreamSynchronize(s));
    return SRJ_OK;
}

}  // extern "C"
