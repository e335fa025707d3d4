// Native optimal-schedule planner (host code): optimal SRJ weights omega and
// fractions beta for P levels at a spectral bound kappa_min (Sect. 3 of
// Adsuara et al., arXiv:1511.04292), integer repetitions by the floor rule of
// Sect. 4.3.
//
// Unknowns x = (log omega_1..omega_P, t_1..t_{P-1}); each interior maximum
// kappa_i is placed inside (1/omega_i, 1/omega_{i+1}) by the logistic of t_i
// (Sect. 3.5 bracket).  beta follows from Theorem 2 (Eq. betai), which makes
// the kappa_i stationary points of Gamma (Eq. partialG).  The 2P-1 equations:
//   * equal maxima (Eq. equMax): log Gamma(kappa_j) - log Gamma(kappa_0), j = 1..P,
//     with kappa_0 = kappa_min and kappa_P = 2;
//   * optimality (Eqs. partialbeta / equDifBeta) in Lagrange-multiplier form:
//     weights mu_0..mu_P (sum 1) with sum_j mu_j kappa_j / (1 - omega_i kappa_j) = 0
//     for every i, and sum_j mu_j (log|1 - omega_i kappa_j| - log|1 - omega_P kappa_j|) = 0
//     for i = 1..P-1.
// Solved by Levenberg-Marquardt (finite-difference Jacobian, LU with partial
// pivoting, adaptive damping), level by level from P = 2
// with the initial guesses of Sect. 3.3 (Eqs. omegaaprox1 / omegaaprox2 for
// the inner weights, extrapolated extreme weights from the solved levels).
#include "srj_internal.h"
#include "../../include/srj.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

constexpr double kKappaMax = 2.0;

struct Sol {
    std::vector<double> omega, beta, kint;
    double tmean = -4.0;  // mean logistic position of the interior maxima
};

double logistic(double t) { return 0.5 * (1.0 + std::tanh(0.5 * t)); }

void unpack(const std::vector<double>& x, int P, std::vector<double>& w, std::vector<double>& k) {
    w.resize(P);
    k.resize(P - 1);
    for (int i = 0; i < P; ++i) w[i] = std::exp(x[i]);
    for (int i = 0; i < P - 1; ++i) {
        const double a = 1.0 / w[i], b = 1.0 / w[i + 1];
        k[i] = a + logistic(x[P + i]) * (b - a);
    }
}

std::vector<double> beta_thm2(const std::vector<double>& w, const std::vector<double>& k) {
    const int P = (int)w.size();
    std::vector<double> b(P);
    for (int i = 0; i < P; ++i) {
        double v = 1.0;
        for (double kk : k) v *= 1.0 - kk * w[i];
        for (int l = 0; l < P; ++l)
            if (l != i) v *= w[l] / (w[l] - w[i]);
        b[i] = v;
    }
    return b;
}

// Solve A y = rhs (n x n, row-major) in place by Gaussian elimination with
// partial pivoting.  Returns false when singular.
bool lu_solve(std::vector<double>& A, std::vector<double>& rhs, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (!(std::fabs(A[piv * n + c]) > 0.0) || !std::isfinite(A[piv * n + c])) return false;
        if (piv != c) {
            for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
            std::swap(rhs[c], rhs[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double s = rhs[c];
        for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * rhs[j];
        rhs[c] = s / A[c * n + c];
    }
    return true;
}

double log_gamma(double kap, const std::vector<double>& w, const std::vector<double>& b) {
    double s = 0.0;
    for (size_t i = 0; i < w.size(); ++i) s += b[i] * std::log(std::fabs(1.0 - w[i] * kap));
    return s;
}

bool residual(const std::vector<double>& x, int P, double km, std::vector<double>& R) {
    std::vector<double> w, k;
    unpack(x, P, w, k);
    const std::vector<double> b = beta_thm2(w, k);
    std::vector<double> kap(P + 1);
    kap[0] = km;
    for (int i = 0; i < P - 1; ++i) kap[i + 1] = k[i];
    kap[P] = kKappaMax;
    R.assign(2 * P - 1, 0.0);
    const double F0 = log_gamma(kap[0], w, b);
    for (int j = 1; j <= P; ++j) R[j - 1] = log_gamma(kap[j], w, b) - F0;
    // multipliers: rows i < P: kappa_j / (1 - omega_i kappa_j); last row: ones
    const int n = P + 1;
    std::vector<double> M((size_t)n * n), rhs(n, 0.0);
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < n; ++j) M[i * n + j] = kap[j] / (1.0 - w[i] * kap[j]);
    for (int j = 0; j < n; ++j) M[P * n + j] = 1.0;
    rhs[P] = 1.0;
    if (!lu_solve(M, rhs, n)) return false;
    for (int i = 0; i < P - 1; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j)
            s += rhs[j] * (std::log(std::fabs(1.0 - w[i] * kap[j])) - std::log(std::fabs(1.0 - w[P - 1] * kap[j])));
        R[P + i] = s;
    }
    for (double r : R)
        if (!std::isfinite(r)) return false;
    return true;
}

double norm2(const std::vector<double>& v) {
    double s = 0.0;
    for (double x : v) s += x * x;
    return std::sqrt(s);
}

// Levenberg-Marquardt on R(x) = 0: (J^T J + lambda diag(J^T J)) d = J^T R with the
// damping lambda adapted to the success of each step (finite-difference J).
bool newton(std::vector<double>& x, int P, double km) {
    const int n = 2 * P - 1;
    std::vector<double> R, Rp, Rm, J((size_t)n * n);
    if (!residual(x, P, km, R)) return false;
    double nr = norm2(R);
    double lambda = 1e-3;
    for (int it = 0; it < 400 && nr >= 1e-13; ++it) {
        for (int c = 0; c < n; ++c) {
            const double hstep = 1e-7 * std::max(1.0, std::fabs(x[c]));
            std::vector<double> xp = x, xm = x;
            xp[c] += hstep;
            xm[c] -= hstep;
            if (!residual(xp, P, km, Rp) || !residual(xm, P, km, Rm)) return false;
            for (int r = 0; r < n; ++r) J[r * n + c] = (Rp[r] - Rm[r]) / (2.0 * hstep);
        }
        std::vector<double> JtJ((size_t)n * n, 0.0), JtR(n, 0.0);
        for (int i = 0; i < n; ++i) {
            for (int r = 0; r < n; ++r) JtR[i] += J[r * n + i] * R[r];
            for (int j = 0; j < n; ++j) {
                double sacc = 0.0;
                for (int r = 0; r < n; ++r) sacc += J[r * n + i] * J[r * n + j];
                JtJ[i * n + j] = sacc;
            }
        }
        bool moved = false;
        for (int tries = 0; tries < 40; ++tries) {
            std::vector<double> A = JtJ, d = JtR;
            for (int i = 0; i < n; ++i) A[i * n + i] += lambda * std::max(JtJ[i * n + i], 1e-300);
            if (lu_solve(A, d, n)) {
                std::vector<double> xn = x, Rn;
                for (int c = 0; c < n; ++c) xn[c] -= d[c];
                if (residual(xn, P, km, Rn)) {
                    const double nn = norm2(Rn);
                    if (nn < nr) {
                        x = xn;
                        R = Rn;
                        nr = nn;
                        lambda = std::max(lambda / 3.0, 1e-12);
                        moved = true;
                        break;
                    }
                }
            }
            lambda *= 4.0;
            if (lambda > 1e12) break;
        }
        if (!moved) break;
    }
    return nr < 1e-10;
}

std::vector<double> guess_exponents(int P) {
    std::vector<int> nums;
    if (P == 2) return {0.0, 1.0};
    nums.push_back(0);
    if (P % 2 == 1) {
        for (int m = 1; m < P - 3; m += 2) nums.push_back(m);
        nums.push_back(P - 1);
        for (int m = P + 2; m < 2 * P - 2; m += 2) nums.push_back(m);
    } else {
        for (int m = 1; m < P - 4; m += 2) nums.push_back(m);
        nums.push_back(P - 2);
        nums.push_back(P);
        for (int m = P + 3; m < 2 * P - 2; m += 2) nums.push_back(m);
    }
    nums.push_back(2 * P - 2);
    std::vector<double> e;
    for (int m : nums) e.push_back(m / (2.0 * (P - 1)));
    return e;
}

// Weights from Eqs. omegaaprox1 / omegaaprox2; each interior maximum at
// logistic position t0 of its bracket (1/omega_i, 1/omega_{i+1}).  The paper's
// guess kappa_i ~ 1/omega_i + (1/omega_{i+1} - 1/omega_i)/3 is t0 = log(1/2);
// converged maxima sit much closer to 1/omega_i (t ~ -3 .. -8), and
// Levenberg-Marquardt converges far more often from t0 ~ -4.
std::vector<double> initial_guess(int P, double w1, double wP, double t0) {
    const std::vector<double> e = guess_exponents(P);
    std::vector<double> w(P), x(2 * P - 1);
    for (int i = 0; i < P; ++i) w[i] = 1.0 / ((1.0 / w1) * std::pow(w1 / wP, e[i]));
    for (int i = 0; i < P; ++i) x[i] = std::log(w[i]);
    for (int i = 0; i < P - 1; ++i) x[P + i] = t0;
    return x;
}

bool accept(const std::vector<double>& x, int P, Sol* out) {
    std::vector<double> w, k;
    unpack(x, P, w, k);
    for (int i = 0; i + 1 < P; ++i)
        if (!(w[i] > w[i + 1])) return false;
    if (!(w[P - 1] > 0.5)) return false;
    const std::vector<double> b = beta_thm2(w, k);
    double s = 0.0;
    for (double v : b) {
        if (!(v > 0.0)) return false;
        s += v;
    }
    if (std::fabs(s - 1.0) > 1e-9) return false;
    out->omega = w;
    out->beta = b;
    out->kint = k;
    double tm = 0.0;
    for (int i = 0; i < P - 1; ++i) tm += x[P + i];
    out->tmean = tm / (P - 1);
    return true;
}

// quadratic (or lower) least-squares fit of y(P) over the given points, evaluated at P0
double poly_extrapolate(const std::vector<double>& Ps, const std::vector<double>& ys, double P0) {
    const int m = (int)Ps.size();
    const int deg = std::min(2, m - 1);
    const int n = deg + 1;
    std::vector<double> A((size_t)n * n, 0.0), r(n, 0.0);
    for (int k = 0; k < m; ++k) {
        double pw[3] = {1.0, Ps[k], Ps[k] * Ps[k]};
        for (int i = 0; i < n; ++i) {
            r[i] += pw[i] * ys[k];
            for (int j = 0; j < n; ++j) A[i * n + j] += pw[i] * pw[j];
        }
    }
    if (!lu_solve(A, r, n)) return ys.back();
    double v = 0.0, pw = 1.0;
    for (int i = 0; i < n; ++i, pw *= P0) v += r[i] * pw;
    return v;
}

}  // namespace

extern "C" int srj_schedule_optimal(int P, double kappa_min, double* omega, double* beta, double* kappa_int) {
    if (P < 1 || P > 32 || !omega || !beta) return SRJ_ERR_INVALID_ARG;
    if (!(kappa_min > 0.0) || !(kappa_min < 1.0)) return SRJ_ERR_INVALID_ARG;
    if (P == 1) {  // one level: the best single weight equalises kappa_min and 2
        omega[0] = 2.0 / (kappa_min + kKappaMax);
        beta[0] = 1.0;
        return SRJ_OK;
    }
    std::vector<Sol> hist;  // hist[p - 2] = solution for p levels
    const double r1s[10] = {0.05, 0.1, 0.15, 0.2, 0.3, 0.35, 0.5, 0.7, 0.85, 0.95};
    const double wps[7] = {0.98, 0.95, 0.9, 0.85, 0.7, 0.6, 0.55};
    for (int p = 2; p <= P; ++p) {
        Sol found;
        bool ok = false;
        if (hist.size() >= 2) {
            std::vector<double> Ps, l1, lP;
            for (size_t h = hist.size() >= 4 ? hist.size() - 4 : 0; h < hist.size(); ++h) {
                Ps.push_back((double)(h + 2));
                l1.push_back(std::log(hist[h].omega.front()));
                lP.push_back(std::log(hist[h].omega.back() - 0.5));
            }
            const double w1 = std::exp(poly_extrapolate(Ps, l1, p));
            const double wP = 0.5 + std::exp(poly_extrapolate(Ps, lP, p));
            for (double t0 : {hist.back().tmean, -4.0, std::log(0.5)}) {
                std::vector<double> x = initial_guess(p, w1, wP, t0);
                if (newton(x, p, kappa_min) && accept(x, p, &found)) { ok = true; break; }
            }
        }
        if (!ok) {
            double best = INFINITY;
            for (double t0 : {-4.0, -2.0, -6.0}) {
                for (double r1 : r1s)
                    for (double wP : wps) {
                        std::vector<double> x = initial_guess(p, r1 / kappa_min, wP, t0);
                        Sol s;
                        if (newton(x, p, kappa_min) && accept(x, p, &s)) {
                            const double lvl = log_gamma(kappa_min, s.omega, s.beta);
                            if (lvl < best - 1e-13) { best = lvl; found = s; ok = true; }
                        }
                    }
                if (ok) break;
            }
        }
        if (!ok) return SRJ_ERR_BAD_SCHEDULE;
        hist.push_back(found);
    }
    const Sol& s = hist.back();
    for (int i = 0; i < P; ++i) { omega[i] = s.omega[i]; beta[i] = s.beta[i]; }
    if (kappa_int)
        for (int i = 0; i < P - 1; ++i) kappa_int[i] = s.kint[i];
    return SRJ_OK;
}

extern "C" int srj_schedule_for_grid(int ndim, const int64_t* dims, int P, double* omega, int32_t* q,
                                     int64_t* M_out) {
    if ((ndim != 2 && ndim != 3) || !dims || !omega || !q) return SRJ_ERR_INVALID_ARG;
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1) return SRJ_ERR_INVALID_ARG;
    const double km = srj::host_kappa_min(ndim, dims);
    if (!(km < 1.0)) return SRJ_ERR_INVALID_ARG;  // tiny grids: use plain Jacobi
    std::vector<double> b(P);
    int rc = srj_schedule_optimal(P, km, omega, b.data(), nullptr);
    if (rc) return rc;
    int64_t M = 0;
    for (int i = 0; i < P; ++i) {
        q[i] = (int32_t)std::floor(b[i] / b[0]);  // Sect. 4.3
        if (q[i] < 1) q[i] = 1;
        M += q[i];
    }
    std::vector<double> w(omega, omega + P);
    std::vector<int32_t> qq(q, q + P);
    if (!(srj::host_max_cycle_log10(w, qq, ndim, dims) < 0.0)) return SRJ_ERR_BAD_SCHEDULE;
    if (M_out) *M_out = M;
    return SRJ_OK;
}
