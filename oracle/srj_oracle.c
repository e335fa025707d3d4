/*
 * SRJ oracle: plain, single-threaded FP64 reference of the Scheduled Relaxation
 * Jacobi hot path (Adsuara et al., "Scheduled Relaxation Jacobi method:
 * improvements and applications", arXiv:1511.04292).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header or constant with the CUDA
 * path.  Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so
 * every operation below rounds exactly once, in the order written).
 *
 * Grid layout (both 2-D and 3-D): a dense row-major array of the interior
 * points plus one ghost layer on every side, x fastest:
 *   2-D: index(x, y)    = y * (nx + 2) + x,                 x in [0, nx+1], y in [0, ny+1]
 *   3-D: index(x, y, z) = (z * (ny + 2) + y) * (nx + 2) + x
 * Interior points are x = 1..nx etc.  The ghost layer of u holds the Dirichlet
 * boundary values g and is never modified.  f has the same padded shape; its
 * ghost layer is ignored.
 *
 * Discrete problem (Sect. 5.1, written for -Laplace(u) = f so that A is SPD):
 *   (A_h u)_p = 2d u_p - sum_{nbrs q} u_q,   b_p = h^2 f_p  (+ ghost neighbours),
 * so that A_h u = b, with d the number of dimensions and h the mesh spacing.
 *
 * One weighted-Jacobi step with weight omega (Eq. 2nd-order_CD of Sect. 3.1,
 * with the Poisson source term added as in Sect. 5.1):
 *   u'_p = u_p + (omega / 2d) * (h^2 f_p + sum_{nbrs} u_q - 2d u_p).
 * The arithmetic order is fixed and written out below:
 *   s  = (((u_W + u_E) + u_S) + u_N) [+ u_B) + u_T]
 *   t  = s + (h*h) * f_p
 *   dd = t - (2d) * u_p
 *   u' = u_p + (omega / (2d)) * dd
 *
 * SRJ M-cycle (Sect. 2): apply the weights of one cycle, omega_1 q_1 times, ...,
 * omega_P q_P times, in a given order; repeat cycles.  Convergence is tested at
 * cycle ends on the relative L2 norm of the residual r = b - A_h u.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>

static int64_t padded_count(int ndim, const int64_t n[3])
{
    int64_t c = (n[0] + 2) * (n[1] + 2);
    if (ndim == 3) c *= (n[2] + 2);
    return c;
}

/* Residual r_p = (h^2 f_p + sum nbrs u) - 2d u_p at one interior point, in the
 * same operation order as the sweep (so that a sweep is u + c * residual). */
static double point_defect(int ndim, const int64_t n[3], double h2, const double *f,
                           const double *u, int64_t p)
{
    const int64_t sx = 1, sy = n[0] + 2, sz = (n[0] + 2) * (n[1] + 2);
    double s = u[p - sx] + u[p + sx];
    s = s + u[p - sy];
    s = s + u[p + sy];
    if (ndim == 3) {
        s = s + u[p - sz];
        s = s + u[p + sz];
    }
    double hf = h2 * f[p];
    double t = s + hf;
    double two_d = (double)(2 * ndim);
    double du = two_d * u[p];
    return t - du;
}

/* One weighted-Jacobi step (Eq. 2nd-order_CD + source).  u_in and u_out must not
 * alias.  The ghost layer of u_out is copied from u_in. */
void srj_oracle_sweep(int ndim, const int64_t n[3], double h, double omega,
                      const double *f, const double *u_in, double *u_out)
{
    const int64_t nz = (ndim == 3) ? n[2] : 1;
    const int64_t sy = n[0] + 2, sz = (n[0] + 2) * (n[1] + 2);
    const double h2 = h * h;
    const double c = omega / (double)(2 * ndim);
    memcpy(u_out, u_in, sizeof(double) * (size_t)padded_count(ndim, n));
    for (int64_t z = 0; z < nz; ++z) {
        const int64_t zoff = (ndim == 3) ? (z + 1) * sz : 0;
        for (int64_t y = 1; y <= n[1]; ++y) {
            for (int64_t x = 1; x <= n[0]; ++x) {
                const int64_t p = zoff + y * sy + x;
                double dd = point_defect(ndim, n, h2, f, u_in, p);
                double cd = c * dd;
                u_out[p] = u_in[p] + cd;
            }
        }
    }
}

/* Residual r = b - A_h u on the interior (Sect. 5.1), its L2 and max norms.
 * r (padded layout, ghost layer set to 0) may be NULL. */
void srj_oracle_residual(int ndim, const int64_t n[3], double h, const double *f,
                         const double *u, double *r, double *l2, double *linf)
{
    const int64_t nz = (ndim == 3) ? n[2] : 1;
    const int64_t sy = n[0] + 2, sz = (n[0] + 2) * (n[1] + 2);
    const double h2 = h * h;
    double ss = 0.0, mx = 0.0;
    if (r) memset(r, 0, sizeof(double) * (size_t)padded_count(ndim, n));
    for (int64_t z = 0; z < nz; ++z) {
        const int64_t zoff = (ndim == 3) ? (z + 1) * sz : 0;
        for (int64_t y = 1; y <= n[1]; ++y) {
            for (int64_t x = 1; x <= n[0]; ++x) {
                const int64_t p = zoff + y * sy + x;
                double rp = point_defect(ndim, n, h2, f, u, p);
                if (r) r[p] = rp;
                ss += rp * rp;
                double a = fabs(rp);
                if (a > mx || isnan(a)) mx = a;
            }
        }
    }
    *l2 = sqrt(ss);
    *linf = mx;
}

/* Apply `count` consecutive steps of the ordered weight sequence seq[0..M-1],
 * starting at position `first` (wrapping around the cycle).  The result is left
 * in u (work is a scratch array of the same size). */
void srj_oracle_steps(int ndim, const int64_t n[3], double h, int64_t M, const double *seq,
                      int64_t first, int64_t count, const double *f, double *u, double *work)
{
    const size_t bytes = sizeof(double) * (size_t)padded_count(ndim, n);
    double *a = u, *b = work;
    for (int64_t k = 0; k < count; ++k) {
        srj_oracle_sweep(ndim, n, h, seq[(first + k) % M], f, a, b);
        double *t = a; a = b; b = t;
    }
    if (a != u) memcpy(u, a, bytes);
}

/* SRJ solve (Sect. 2 cycles; Sect. 4.1 convergence monitor, here on the relative
 * L2 residual).  Returns 0 converged, 1 not converged within max_cycles,
 * 2 diverged (non-finite residual), 3 out of memory. */
int srj_oracle_solve(int ndim, const int64_t n[3], double h, int64_t M, const double *seq,
                     const double *f, double *u, double tol, int64_t max_cycles,
                     int64_t *cycles_out, double *r0_out, double *rel_out, double *linf_out)
{
    double l2, linf;
    srj_oracle_residual(ndim, n, h, f, u, NULL, &l2, &linf);
    const double r0 = l2;
    *r0_out = r0;
    *cycles_out = 0;
    *rel_out = (r0 > 0.0) ? 1.0 : 0.0;
    *linf_out = linf;
    if (r0 == 0.0) return 0;
    if (!isfinite(r0)) return 2;
    double *work = (double *)malloc(sizeof(double) * (size_t)padded_count(ndim, n));
    if (!work) return 3;
    int status = 1;
    for (int64_t c = 1; c <= max_cycles; ++c) {
        srj_oracle_steps(ndim, n, h, M, seq, 0, M, f, u, work);
        srj_oracle_residual(ndim, n, h, f, u, NULL, &l2, &linf);
        *cycles_out = c;
        *rel_out = l2 / r0;
        *linf_out = linf;
        if (!isfinite(l2)) { status = 2; break; }
        if (l2 / r0 <= tol) { status = 0; break; }
    }
    free(work);
    return status;
}

/* ------------------------------------------------------------------------
 * Masked, diagonally shifted operator (the Grad-Shafranov test B setting of
 * Sect. 5.3: the iteration is applied only inside a region given by a mask,
 * points outside keep their values; Eq. GS_linear adds a term proportional to
 * the unknown, a shift of the diagonal).  Cartesian form:
 *   (A u)_p = (2d + sigma) u_p - sum_{nbrs} u_q   on active points p,
 * sigma = -C^2 h^2 for Laplace(u) + C^2 u = rhs, +k^2 h^2 for a screened Poisson
 * operator.  mask: 1 = active (updated), 0 = held fixed; NULL = every interior
 * point active.  With sigma = 0 and mask = NULL these reduce exactly to
 * srj_oracle_sweep / srj_oracle_residual (same operations in the same order).
 * ------------------------------------------------------------------------ */
static double point_defect_op(int ndim, const int64_t n[3], double h2, double diag, const double *f,
                              const double *u, int64_t p)
{
    const int64_t sx = 1, sy = n[0] + 2, sz = (n[0] + 2) * (n[1] + 2);
    double s = u[p - sx] + u[p + sx];
    s = s + u[p - sy];
    s = s + u[p + sy];
    if (ndim == 3) {
        s = s + u[p - sz];
        s = s + u[p + sz];
    }
    double hf = h2 * f[p];
    double t = s + hf;
    double du = diag * u[p];
    return t - du;
}

void srj_oracle_sweep_op(int ndim, const int64_t n[3], double h, double omega, double sigma,
                         const unsigned char *mask, const double *f, const double *u_in, double *u_out)
{
    const int64_t nz = (ndim == 3) ? n[2] : 1;
    const int64_t sy = n[0] + 2, sz = (n[0] + 2) * (n[1] + 2);
    const double h2 = h * h;
    const double diag = (double)(2 * ndim) + sigma;
    const double c = omega / diag;
    memcpy(u_out, u_in, sizeof(double) * (size_t)padded_count(ndim, n));
    for (int64_t z = 0; z < nz; ++z) {
        const int64_t zoff = (ndim == 3) ? (z + 1) * sz : 0;
        for (int64_t y = 1; y <= n[1]; ++y) {
            for (int64_t x = 1; x <= n[0]; ++x) {
                const int64_t p = zoff + y * sy + x;
                if (mask && !mask[p]) continue;
                double dd = point_defect_op(ndim, n, h2, diag, f, u_in, p);
                double cd = c * dd;
                u_out[p] = u_in[p] + cd;
            }
        }
    }
}

void srj_oracle_residual_op(int ndim, const int64_t n[3], double h, double sigma, const unsigned char *mask,
                            const double *f, const double *u, double *r, double *l2, double *linf)
{
    const int64_t nz = (ndim == 3) ? n[2] : 1;
    const int64_t sy = n[0] + 2, sz = (n[0] + 2) * (n[1] + 2);
    const double h2 = h * h;
    const double diag = (double)(2 * ndim) + sigma;
    double ss = 0.0, mx = 0.0;
    if (r) memset(r, 0, sizeof(double) * (size_t)padded_count(ndim, n));
    for (int64_t z = 0; z < nz; ++z) {
        const int64_t zoff = (ndim == 3) ? (z + 1) * sz : 0;
        for (int64_t y = 1; y <= n[1]; ++y) {
            for (int64_t x = 1; x <= n[0]; ++x) {
                const int64_t p = zoff + y * sy + x;
                if (mask && !mask[p]) continue;
                double rp = point_defect_op(ndim, n, h2, diag, f, u, p);
                if (r) r[p] = rp;
                ss += rp * rp;
                double a = fabs(rp);
                if (a > mx || isnan(a)) mx = a;
            }
        }
    }
    *l2 = sqrt(ss);
    *linf = mx;
}

/* SRJ cycles with the masked / shifted operator; same contract as srj_oracle_solve. */
int srj_oracle_solve_op(int ndim, const int64_t n[3], double h, double sigma, const unsigned char *mask, int64_t M,
                        const double *seq, const double *f, double *u, double tol, int64_t max_cycles,
                        int64_t *cycles_out, double *r0_out, double *rel_out)
{
    double l2, linf;
    srj_oracle_residual_op(ndim, n, h, sigma, mask, f, u, NULL, &l2, &linf);
    const double r0 = l2;
    *r0_out = r0;
    *cycles_out = 0;
    *rel_out = (r0 > 0.0) ? 1.0 : 0.0;
    if (r0 == 0.0) return 0;
    if (!isfinite(r0)) return 2;
    const size_t bytes = sizeof(double) * (size_t)padded_count(ndim, n);
    double *work = (double *)malloc(bytes);
    if (!work) return 3;
    int status = 1;
    for (int64_t c = 1; c <= max_cycles; ++c) {
        double *a = u, *b = work;
        for (int64_t k = 0; k < M; ++k) {
            srj_oracle_sweep_op(ndim, n, h, seq[k], sigma, mask, f, a, b);
            double *t = a; a = b; b = t;
        }
        if (a != u) memcpy(u, a, bytes);
        srj_oracle_residual_op(ndim, n, h, sigma, mask, f, u, NULL, &l2, &linf);
        *cycles_out = c;
        *rel_out = l2 / r0;
        if (!isfinite(l2)) { status = 2; break; }
        if (l2 / r0 <= tol) { status = 0; break; }
    }
    free(work);
    return status;
}
