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
//
// Precision (Sect. 3.3 needed 24 digits for the largest grids): near the
// solution the Jacobian's condition number grows like the weights' spread
// omega_1 / omega_P ~ 1 / kappa_min, and the normal equations square it, so in
// double arithmetic the iteration stalls near a solution for kappa_min below
// ~1e-7 (grids beyond ~7000^2).  Each start therefore runs Levenberg-Marquardt
// in double until it stalls, then again from that point in double-double
// arithmetic (about 32 significant digits), in which the system is evaluated,
// differentiated and solved, until the residual is below 1e-22.  The
// double-double format is Dekker's (1971): a value is an unevaluated sum hi + lo
// of two doubles with |lo| <= ulp(hi) / 2; sums use Knuth's error-free two-sum,
// products the exact fma residual, and exp / log are computed from their Taylor
// series after argument reduction (exp) or by one Newton step on exp (log).
// Every operation is written out with explicit roundings (the file is compiled
// without floating-point contraction), so x86-64 and aarch64 hosts give the same
// bits.
#include "srj_internal.h"
#include "../../include/srj.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

namespace {

constexpr double kKappaMax = 2.0;

// ---- double-double arithmetic ----------------------------------------------

struct dd {
    double hi, lo;
    dd() : hi(0.0), lo(0.0) {}
    dd(double h) : hi(h), lo(0.0) {}  // NOLINT: implicit on purpose (mixed expressions)
    dd(double h, double l) : hi(h), lo(l) {}
};

inline dd two_sum(double a, double b) {
    const double s = a + b;
    const double bb = s - a;
    return dd(s, (a - (s - bb)) + (b - bb));
}
inline dd quick_two_sum(double a, double b) {  // |a| >= |b|
    const double s = a + b;
    return dd(s, b - (s - a));
}
inline dd two_prod(double a, double b) {
    const double p = a * b;
    return dd(p, std::fma(a, b, -p));
}
inline dd operator+(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    const dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    const double c1 = a.hi * b.lo;
    const double c2 = a.lo * b.hi;
    p.lo += c1;
    p.lo += c2;
    return quick_two_sum(p.hi, p.lo);
}
inline dd operator/(dd a, dd b) {
    const double q1 = a.hi / b.hi;
    dd r = a - b * dd(q1);
    const double q2 = r.hi / b.hi;
    r = r - b * dd(q2);
    const double q3 = r.hi / b.hi;
    return quick_two_sum(q1, q2) + dd(q3);
}
inline dd& operator+=(dd& a, dd b) { return a = a + b; }
inline dd& operator-=(dd& a, dd b) { return a = a - b; }
inline dd& operator*=(dd& a, dd b) { return a = a * b; }
inline bool operator<(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline bool operator>(dd a, dd b) { return b < a; }
inline dd ldexp_dd(dd a, int k) { return dd(std::ldexp(a.hi, k), std::ldexp(a.lo, k)); }

const dd kLn2(0.6931471805599453, 2.3190468138462996e-17);

// exp(a) = 2^k exp(r), r = a - k ln 2; exp(r) - 1 from the Taylor series of
// exp(r / 1024) - 1, squared back ten times in the form (1 + s)^2 - 1 = 2 s + s^2.
dd dd_exp(dd a) {
    if (a.hi > 709.0) return dd(INFINITY);
    if (a.hi < -745.0) return dd(0.0);
    const double k = std::floor(a.hi / kLn2.hi + 0.5);
    const dd r = ldexp_dd(a - kLn2 * dd(k), -10);
    dd s = r, t = r;
    for (int n = 2; n <= 14; ++n) {
        t = t * r / dd((double)n);
        s += t;
        if (std::fabs(t.hi) < 1e-36 * std::fabs(s.hi)) break;
    }
    for (int i = 0; i < 10; ++i) s = ldexp_dd(s, 1) + s * s;
    return ldexp_dd(s + dd(1.0), (int)k);
}
// log(a), a > 0: one Newton step x + a exp(-x) - 1 from the double logarithm.
dd dd_log(dd a) {
    if (!(a.hi > 0.0)) return dd(a.hi == 0.0 ? -INFINITY : NAN);
    const dd x(std::log(a.hi));
    return x + (a * dd_exp(-x) - dd(1.0));
}

// scalar interface of the solver, for double and for dd
inline double r_exp(double x) { return std::exp(x); }
inline double r_log(double x) { return std::log(x); }
inline double r_abs(double x) { return std::fabs(x); }
inline double to_d(double x) { return x; }
inline dd r_exp(dd x) { return dd_exp(x); }
inline dd r_log(dd x) { return dd_log(x); }
inline dd r_abs(dd x) { return x.hi < 0.0 ? -x : x; }
inline double to_d(dd x) { return x.hi + x.lo; }

template <class R> struct Prec;
template <> struct Prec<double> {
    static constexpr double fd_step = 1e-7;   // central differences, relative step
    static constexpr double stop = 1e-13;     // residual norm at which the iteration stops
    static constexpr double success = 1e-10;  // residual norm that counts as a solution
    static constexpr int max_iter = 400;
    static constexpr double lambda_min = 1e-12;  // smallest damping
    static constexpr bool newton_first = false;  // try the undamped step J d = R first
};
template <> struct Prec<dd> {
    static constexpr double fd_step = 1e-12;
    static constexpr double stop = 1e-26;
    static constexpr double success = 1e-22;
    static constexpr int max_iter = 20;
    static constexpr double lambda_min = 1e-30;
    static constexpr bool newton_first = true;
};

// ---- the system S(omega, kappa) -----------------------------------------------

struct Sol {
    std::vector<double> omega, beta, kint;
    std::vector<dd> x;    // the unknowns (log omega, t) of the solution
    double tmean = -4.0;  // mean logistic position of the interior maxima
};

// logistic s(t) = 1 / (1 + e^-t), accurate for t of either sign
template <class R>
R logistic(R t) { return R(1.0) / (R(1.0) + r_exp(-t)); }

template <class R>
void unpack(const std::vector<R>& x, int P, std::vector<R>& w, std::vector<R>& k) {
    w.resize(P);
    k.resize(P - 1);
    for (int i = 0; i < P; ++i) w[i] = r_exp(x[i]);
    for (int i = 0; i < P - 1; ++i) {
        const R a = R(1.0) / w[i], b = R(1.0) / w[i + 1];
        k[i] = a + logistic(x[P + i]) * (b - a);
    }
}

template <class R>
std::vector<R> beta_thm2(const std::vector<R>& w, const std::vector<R>& k) {
    const int P = (int)w.size();
    std::vector<R> b(P);
    for (int i = 0; i < P; ++i) {
        R v(1.0);
        for (const R& kk : k) v *= R(1.0) - kk * w[i];
        for (int l = 0; l < P; ++l)
            if (l != i) v *= w[l] / (w[l] - w[i]);
        b[i] = v;
    }
    return b;
}

// Solve A y = rhs (n x n, row-major) in place by Gaussian elimination with
// partial pivoting.  Returns false when singular.
template <class R>
bool lu_solve(std::vector<R>& A, std::vector<R>& rhs, int n) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (r_abs(A[r * n + c]) > r_abs(A[piv * n + c])) piv = r;
        const double pv = to_d(A[piv * n + c]);
        if (!(std::fabs(pv) > 0.0) || !std::isfinite(pv)) return false;
        if (piv != c) {
            for (int j = 0; j < n; ++j) std::swap(A[c * n + j], A[piv * n + j]);
            std::swap(rhs[c], rhs[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const R f = A[r * n + c] / A[c * n + c];
            if (to_d(f) == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            rhs[r] -= f * rhs[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        R s = rhs[c];
        for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * rhs[j];
        rhs[c] = s / A[c * n + c];
    }
    return true;
}

template <class R>
R log_gamma(R kap, const std::vector<R>& w, const std::vector<R>& b) {
    R s(0.0);
    for (size_t i = 0; i < w.size(); ++i) s += b[i] * r_log(r_abs(R(1.0) - w[i] * kap));
    return s;
}

template <class R>
bool residual(const std::vector<R>& x, int P, double km, std::vector<R>& Rv) {
    std::vector<R> w, k;
    unpack(x, P, w, k);
    const std::vector<R> b = beta_thm2(w, k);
    std::vector<R> kap(P + 1);
    kap[0] = R(km);
    for (int i = 0; i < P - 1; ++i) kap[i + 1] = k[i];
    kap[P] = R(kKappaMax);
    // L[i][j] = log|1 - omega_i kappa_j|
    const int n = P + 1;
    std::vector<R> L((size_t)P * n);
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < n; ++j) L[(size_t)i * n + j] = r_log(r_abs(R(1.0) - w[i] * kap[j]));
    Rv.assign(2 * P - 1, R(0.0));
    std::vector<R> F(n, R(0.0));
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < P; ++i) F[j] += b[i] * L[(size_t)i * n + j];
    for (int j = 1; j <= P; ++j) Rv[j - 1] = F[j] - F[0];
    // multipliers: rows i < P: kappa_j / (1 - omega_i kappa_j); last row: ones
    std::vector<R> M((size_t)n * n), rhs(n, R(0.0));
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < n; ++j) M[i * n + j] = kap[j] / (R(1.0) - w[i] * kap[j]);
    for (int j = 0; j < n; ++j) M[P * n + j] = R(1.0);
    rhs[P] = R(1.0);
    if (!lu_solve(M, rhs, n)) return false;
    for (int i = 0; i < P - 1; ++i) {
        R s(0.0);
        for (int j = 0; j < n; ++j) s += rhs[j] * (L[(size_t)i * n + j] - L[(size_t)(P - 1) * n + j]);
        Rv[P + i] = s;
    }
    for (const R& r : Rv)
        if (!std::isfinite(to_d(r))) return false;
    return true;
}

template <class R>
double norm2(const std::vector<R>& v) {
    double s = 0.0;
    for (const R& x : v) s += to_d(x) * to_d(x);
    return std::sqrt(s);
}

// Levenberg-Marquardt on R(x) = 0: (J^T J + lambda diag(J^T J)) d = J^T R with the
// damping lambda adapted to the success of each step (finite-difference J).
// Returns the final residual norm (infinity when the system could not be evaluated).
template <class R>
double newton(std::vector<R>& x, int P, double km) {
    const int n = 2 * P - 1;
    std::vector<R> Rv, Rp, Rm, J((size_t)n * n);
    if (!residual(x, P, km, Rv)) return INFINITY;
    double nr = norm2(Rv);
    double lambda = 1e-3;
    for (int it = 0; it < Prec<R>::max_iter && nr >= Prec<R>::stop; ++it) {
        for (int c = 0; c < n; ++c) {
            const R hstep(Prec<R>::fd_step * std::max(1.0, std::fabs(to_d(x[c]))));
            std::vector<R> xp = x, xm = x;
            xp[c] += hstep;
            xm[c] -= hstep;
            if (!residual(xp, P, km, Rp) || !residual(xm, P, km, Rm)) return INFINITY;
            for (int r = 0; r < n; ++r) J[r * n + c] = (Rp[r] - Rm[r]) / (hstep + hstep);
        }
        std::vector<R> JtJ((size_t)n * n, R(0.0)), JtR(n, R(0.0));
        for (int i = 0; i < n; ++i) {
            for (int r = 0; r < n; ++r) JtR[i] += J[r * n + i] * Rv[r];
            for (int j = 0; j < n; ++j) {
                R sacc(0.0);
                for (int r = 0; r < n; ++r) sacc += J[r * n + i] * J[r * n + j];
                JtJ[i * n + j] = sacc;
            }
        }
        bool moved = false;
        if (Prec<R>::newton_first) {
            // Newton step on the square system, halved until the residual decreases
            std::vector<R> A = J, d = Rv;
            if (lu_solve(A, d, n)) {
                R alpha(1.0);
                for (int h = 0; h < 8 && !moved; ++h, alpha *= R(0.5)) {
                    std::vector<R> xn = x, Rn;
                    for (int c = 0; c < n; ++c) xn[c] -= alpha * d[c];
                    if (residual(xn, P, km, Rn)) {
                        const double nn = norm2(Rn);
                        if (nn < nr) { x = xn; Rv = Rn; nr = nn; moved = true; }
                    }
                }
            }
            if (moved) continue;
        }
        for (int tries = 0; tries < 40; ++tries) {
            std::vector<R> A = JtJ, d = JtR;
            for (int i = 0; i < n; ++i) {
                const double dg = std::max(to_d(JtJ[i * n + i]), 1e-300);
                A[i * n + i] += R(lambda * dg);
            }
            if (lu_solve(A, d, n)) {
                std::vector<R> xn = x, Rn;
                for (int c = 0; c < n; ++c) xn[c] -= d[c];
                if (residual(xn, P, km, Rn)) {
                    const double nn = norm2(Rn);
                    if (nn < nr) {
                        x = xn;
                        Rv = Rn;
                        nr = nn;
                        lambda = std::max(lambda / 3.0, Prec<R>::lambda_min);
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
    return nr;
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

// A converged double-double solution: weights decreasing, omega_P > 1/2, beta > 0
// with unit sum.
bool accept(const std::vector<dd>& x, int P, Sol* out) {
    std::vector<dd> w, k;
    unpack(x, P, w, k);
    for (int i = 0; i + 1 < P; ++i)
        if (!(w[i] > w[i + 1])) return false;
    if (!(to_d(w[P - 1]) > 0.5)) return false;
    const std::vector<dd> b = beta_thm2(w, k);
    dd s(0.0);
    for (const dd& v : b) {
        if (!(to_d(v) > 0.0)) return false;
        s += v;
    }
    if (std::fabs(to_d(s) - 1.0) > 1e-9) return false;
    out->omega.resize(P);
    out->beta.resize(P);
    out->kint.resize(P - 1);
    for (int i = 0; i < P; ++i) { out->omega[i] = to_d(w[i]); out->beta[i] = to_d(b[i]); }
    for (int i = 0; i < P - 1; ++i) out->kint[i] = to_d(k[i]);
    out->x = x;
    double tm = 0.0;
    for (int i = 0; i < P - 1; ++i) tm += to_d(x[P + i]);
    out->tmean = tm / (P - 1);
    return true;
}

// Double-double stage of a start (see solve_from).
bool polish_dd(const std::vector<double>& x, int p, double km, Sol* out) {
    std::vector<dd> xd(x.begin(), x.end());
    if (!(newton(xd, p, km) < Prec<dd>::success)) return false;
    return accept(xd, p, out);
}

// One start: Levenberg-Marquardt in double until it stalls, then in
// double-double from there.  Starts that end far from any solution in double
// (residual above 1e-3) are dropped before the double-double stage.
bool solve_from(const std::vector<double>& x0, int p, double km, Sol* out) {
    std::vector<double> x = x0;
    if (!(newton(x, p, km) < 1e-3)) return false;
    return polish_dd(x, p, km, out);
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


// Level by level from 2 to P at kappa_min (Sect. 3.3 continuation in P).
// Returns 0 or the level that could not be solved.
int solve_levels(int P, double kappa_min, Sol* out) {
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
            for (double t0 : {hist.back().tmean, -4.0, std::log(0.5)})
                if (solve_from(initial_guess(p, w1, wP, t0), p, kappa_min, &found)) { ok = true; break; }
        }
        // A grid of starts: each runs in double; the ones that end near a solution
        // are polished in double-double in the order of their level max Gamma, and
        // the first that converges (the lowest level among the solutions) is kept.
        for (double t0 : {-4.0, -2.0, -6.0}) {
            if (ok) break;
            std::vector<std::pair<double, std::vector<double>>> cand;
            for (double r1 : r1s)
                for (double wP : wps) {
                    std::vector<double> x = initial_guess(p, r1 / kappa_min, wP, t0);
                    if (!(newton(x, p, kappa_min) < 1e-3)) continue;
                    std::vector<double> w, k;
                    unpack(x, p, w, k);
                    bool mono = w[p - 1] > 0.5;
                    for (int i = 0; i + 1 < p; ++i) mono = mono && w[i] > w[i + 1];
                    if (!mono) continue;
                    const double lvl = log_gamma(kappa_min, w, beta_thm2(w, k));
                    if (std::isfinite(lvl)) cand.emplace_back(lvl, x);
                }
            std::sort(cand.begin(), cand.end(),
                      [](const std::pair<double, std::vector<double>>& a,
                         const std::pair<double, std::vector<double>>& b) { return a.first < b.first; });
            for (const auto& c : cand)
                if (polish_dd(c.second, p, kappa_min, &found)) { ok = true; break; }
        }
        if (!ok) return p;
        hist.push_back(found);
    }
    *out = hist.back();
    return 0;
}

// Below this spectral bound the level-by-level search is started at the bound
// itself no more: the P-level solution is found at kKappaDirect and followed
// down to kappa_min in steps of kappa / 2 (Newton in double-double from the
// linear extrapolation of the unknowns in log kappa).
constexpr double kKappaDirect = 1.2e-7;

bool follow_kappa(int P, double k_from, const Sol& s_from, double k_to, Sol* out) {
    std::vector<dd> x_prev, x_cur = s_from.x;
    double k_prev = 0.0, k_cur = k_from;
    double ratio = 0.5;
    while (k_cur > k_to) {
        const double k_next = std::max(k_to, k_cur * ratio);
        std::vector<dd> x = x_cur;
        if (!x_prev.empty()) {
            const double a = std::log(k_next / k_cur) / std::log(k_cur / k_prev);
            for (size_t i = 0; i < x.size(); ++i) x[i] = x_cur[i] + (x_cur[i] - x_prev[i]) * dd(a);
        }
        Sol s;
        if (newton(x, P, k_next) < Prec<dd>::success && accept(x, P, &s)) {
            x_prev = x_cur;
            x_cur = x;
            k_prev = k_cur;
            k_cur = k_next;
            *out = s;
            ratio = 0.5;  // back to the full step after a success
        } else {
            ratio = std::sqrt(ratio);  // shorter step
            if (ratio > 0.97) return false;
        }
    }
    return true;
}

}  // namespace

extern "C" int srj_schedule_optimal(int P, double kappa_min, double* omega, double* beta, double* kappa_int) {
    if (P < 1 || P > 32) return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_optimal: P must be in 1..32");
    if (!omega || !beta) return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_optimal: NULL output");
    if (!(kappa_min > 0.0) || !(kappa_min < 1.0))
        return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_optimal: kappa_min must lie in (0, 1)");
    if (P == 1) {  // one level: the best single weight equalises kappa_min and 2
        omega[0] = 2.0 / (kappa_min + kKappaMax);
        beta[0] = 1.0;
        return SRJ_OK;
    }
    Sol s;
    const double k0 = std::max(kappa_min, kKappaDirect);
    const int bad = solve_levels(P, k0, &s);
    char msg[240];
    if (bad) {
        std::snprintf(msg, sizeof msg,
                      "srj_schedule_optimal: no solution of the optimality system found for %d levels "
                      "(level %d of %d) at kappa_min = %.6g",
                      bad, bad, P, k0);
        return srj::set_last_error(SRJ_ERR_BAD_SCHEDULE, msg);
    }
    if (kappa_min < k0) {
        Sol t;
        if (!follow_kappa(P, k0, s, kappa_min, &t)) {
            std::snprintf(msg, sizeof msg,
                          "srj_schedule_optimal: the %d-level solution at kappa_min = %.6g could not be followed "
                          "down to kappa_min = %.6g",
                          P, k0, kappa_min);
            return srj::set_last_error(SRJ_ERR_BAD_SCHEDULE, msg);
        }
        s = t;
    }
    for (int i = 0; i < P; ++i) { omega[i] = s.omega[i]; beta[i] = s.beta[i]; }
    if (kappa_int)
        for (int i = 0; i < P - 1; ++i) kappa_int[i] = s.kint[i];
    return SRJ_OK;
}

extern "C" int srj_schedule_for_grid(int ndim, const int64_t* dims, int P, double* omega, int32_t* q,
                                     int64_t* M_out) {
    if ((ndim != 2 && ndim != 3) || !dims || !omega || !q)
        return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_for_grid: bad ndim or NULL argument");
    if (P < 1 || P > 32) return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_for_grid: P must be in 1..32");
    for (int i = 0; i < ndim; ++i)
        if (dims[i] < 1) return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_for_grid: dims must be >= 1");
    const double km = srj::host_kappa_min(ndim, dims);
    if (!(km < 1.0))  // tiny grids: use plain Jacobi
        return srj::set_last_error(SRJ_ERR_INVALID_ARG, "srj_schedule_for_grid: grid too small (kappa_min >= 1)");
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
    if (!(srj::host_max_cycle_log10(w, qq, ndim, dims) < 0.0))
        return srj::set_last_error(SRJ_ERR_BAD_SCHEDULE,
                                   "srj_schedule_for_grid: the integer scheme (floor rule) does not contract on the grid");
    if (M_out) *M_out = M;
    return SRJ_OK;
}
