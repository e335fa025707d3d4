/*
 * SRJ oracle, spherical-coordinate operators (Sect. 5.2 of Adsuara et al.,
 * arXiv:1511.04292): plain single-threaded FP64 reference.
 *
 * TEST INFRASTRUCTURE ONLY, like srj_oracle.c: nothing in the product links or
 * calls it, and it shares no code with the CUDA path.  Built together with
 * srj_oracle.c (gcc -O2 -ffp-contract=off), so each operation rounds once, in
 * the order written.
 *
 * Grid: n[0] radial points (x, fastest), n[1] polar points (y) and, in 3-D,
 * n[2] azimuthal points (z), with one ghost layer on every side, in the padded
 * layout of srj_oracle.c.  Cell centres r_i = (i - 1/2) dr, theta_j = (j - 1/2)
 * dtheta, phi_k = (k - 1/2) dphi.
 *
 * Operator: the Poisson operator in spherical coordinates multiplied by r^2
 * (Sect. 5.2), second-order central differences, written with separable
 * coefficients:
 *   (L u)_p = cr_m[i] u(i-1) + cr_p[i] u(i+1) + ct_m[j] u(j-1) + ct_p[j] u(j+1)
 *             [+ cp[j] (u(k-1) + u(k+1))]  -  d_p u_p,
 *   d_p     = cr_0[i] + ct_0[j]  [+ (cp[j] + cp[j])],
 * and the system L u = b with b = r^2 s.  Boundary conditions (Sect. 5.2):
 *   r = 1 (ghost i = n_r + 1): Dirichlet data, held fixed in the ghost layer;
 *   r = 0: u_0 = u_1 = u_2, imposed at every iteration: the row i = 1 is not
 *          iterated, it copies row 2; row 2 sees u(i-1) = u(i);
 *   theta = 0, pi: homogeneous Neumann, mirror ghosts u(j=0) = u(1),
 *          u(n_t+1) = u(n_t);
 *   phi: periodic, u(k=0) = u(n_p), u(n_p+1) = u(1).
 * The iterated unknowns ("active points") are i = 2..n_r, all j, k.
 *
 * One weighted-Jacobi step with weight omega (Sect. 3.1 applied to this
 * operator; its diagonal is -d_p):
 *   s  = (cr_m um + cr_p up) + (ct_m tm + ct_p tp)   [+ cp (pm + pp)]
 *   t  = s - d u_p;   res = t - b_p;   u'_p = u_p + omega * (res / d)
 * with the neighbour values after the boundary substitutions above.  The
 * residual of the system at an active point is res.
 *
 * Coefficient arrays (inputs): radial[3 * (n_r + 2)] = cr_m | cr_p | cr_0,
 * polar[3 * (n_t + 2)] = ct_m | ct_p | ct_0, azim[n_t + 2] = cp (3-D only),
 * each indexed by its padded index.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

static int64_t sph_count(int ndim, const int64_t n[3])
{
    int64_t c = (n[0] + 2) * (n[1] + 2);
    if (ndim == 3) c *= (n[2] + 2);
    return c;
}

/* res at the active point (i, j, k) of u, and the point's d. */
static double sph_point(int ndim, const int64_t n[3], const double *radial, const double *polar,
                        const double *azim, const double *b, const double *u, int64_t i, int64_t j, int64_t k,
                        double *d_out)
{
    const int64_t sx = n[0] + 2, sy = (n[0] + 2) * (n[1] + 2);
    const int64_t nr = n[0], nt = n[1];
    const int64_t p = (ndim == 3 ? k * sy : 0) + j * sx + i;
    const double c = u[p];
    const double um = (i == 2) ? c : u[p - 1];
    const double up = u[p + 1];
    const double tm = (j == 1) ? c : u[p - sx];
    const double tp = (j == nt) ? c : u[p + sx];
    const double *cr_m = radial, *cr_p = radial + (nr + 2), *cr_0 = radial + 2 * (nr + 2);
    const double *ct_m = polar, *ct_p = polar + (nt + 2), *ct_0 = polar + 2 * (nt + 2);
    double s = (cr_m[i] * um + cr_p[i] * up) + (ct_m[j] * tm + ct_p[j] * tp);
    double d = cr_0[i] + ct_0[j];
    if (ndim == 3) {
        const int64_t np = n[2];
        const double pm = (k == 1) ? u[p + (np - 1) * sy] : u[p - sy];
        const double pp = (k == np) ? u[p - (np - 1) * sy] : u[p + sy];
        s = s + azim[j] * (pm + pp);
        d = d + (azim[j] + azim[j]);
    }
    const double t = s - d * c;
    *d_out = d;
    return t - b[p];
}

/* One Jacobi step uin -> uout (active points, then the row i = 1 := row 2). */
void srj_oracle_sph_sweep(int ndim, const int64_t n[3], const double *radial, const double *polar,
                          const double *azim, double omega, const double *b, const double *uin, double *uout)
{
    const int64_t sx = n[0] + 2, sy = (n[0] + 2) * (n[1] + 2);
    const int64_t kz = (ndim == 3) ? n[2] : 1;
    for (int64_t k = (ndim == 3 ? 1 : 0); k < (ndim == 3 ? kz + 1 : 1); ++k)
        for (int64_t j = 1; j <= n[1]; ++j) {
            for (int64_t i = 2; i <= n[0]; ++i) {
                double d;
                const double res = sph_point(ndim, n, radial, polar, azim, b, uin, i, j, k, &d);
                const int64_t p = (ndim == 3 ? k * sy : 0) + j * sx + i;
                uout[p] = uin[p] + omega * (res / d);
            }
            const int64_t q = (ndim == 3 ? k * sy : 0) + j * sx;
            if (n[0] >= 2) uout[q + 1] = uout[q + 2];
            else uout[q + 1] = uin[q + 1];  /* n_r = 1: no active point */
        }
}

/* res at the active points (into r when r != NULL; other points 0); L2 and max norms. */
void srj_oracle_sph_residual(int ndim, const int64_t n[3], const double *radial, const double *polar,
                             const double *azim, const double *b, const double *u, double *r, double *l2,
                             double *linf)
{
    const int64_t sx = n[0] + 2, sy = (n[0] + 2) * (n[1] + 2);
    if (r) memset(r, 0, sizeof(double) * (size_t)sph_count(ndim, n));
    double ss = 0.0, mx = 0.0;
    const int64_t kz = (ndim == 3) ? n[2] : 1;
    for (int64_t k = (ndim == 3 ? 1 : 0); k < (ndim == 3 ? kz + 1 : 1); ++k)
        for (int64_t j = 1; j <= n[1]; ++j)
            for (int64_t i = 2; i <= n[0]; ++i) {
                double d;
                const double res = sph_point(ndim, n, radial, polar, azim, b, u, i, j, k, &d);
                if (r) r[(ndim == 3 ? k * sy : 0) + j * sx + i] = res;
                ss += res * res;
                if (fabs(res) > mx) mx = fabs(res);
            }
    *l2 = sqrt(ss);
    *linf = mx;
}

/* Ghost layer and row i = 1 from the boundary prescription (the r = 1 ghost is data). */
void srj_oracle_sph_finalize(int ndim, const int64_t n[3], double *u)
{
    const int64_t sx = n[0] + 2, sy = (n[0] + 2) * (n[1] + 2);
    const int64_t nr = n[0], nt = n[1];
    const int64_t k0 = (ndim == 3) ? 1 : 0, k1 = (ndim == 3) ? n[2] : 0;
    for (int64_t k = k0; k <= k1; ++k) {
        const int64_t base = (ndim == 3 ? k * sy : 0);
        for (int64_t j = 1; j <= nt; ++j) {
            const int64_t q = base + j * sx;
            if (nr >= 2) u[q + 1] = u[q + 2];
            u[q] = u[q + 1];
        }
        for (int64_t i = 0; i <= nr + 1; ++i) {
            u[base + i] = u[base + sx + i];
            u[base + (nt + 1) * sx + i] = u[base + nt * sx + i];
        }
    }
    if (ndim == 3) {
        const int64_t np = n[2];
        for (int64_t j = 0; j <= nt + 1; ++j)
            for (int64_t i = 0; i <= nr + 1; ++i) {
                u[j * sx + i] = u[np * sy + j * sx + i];
                u[(np + 1) * sy + j * sx + i] = u[sy + j * sx + i];
            }
    }
}

/* SRJ cycles of the M-step sequence seq until ||res||_2 / ||res_0||_2 <= tol;
 * then finalize.  Returns 0 converged, 1 not converged, 2 diverged, 3 no memory. */
int srj_oracle_sph_solve(int ndim, const int64_t n[3], const double *radial, const double *polar,
                         const double *azim, int64_t M, const double *seq, const double *b, double *u, double tol,
                         int64_t max_cycles, int64_t *cycles_out, double *r0_out, double *rel_out)
{
    double l2, linf;
    srj_oracle_sph_residual(ndim, n, radial, polar, azim, b, u, NULL, &l2, &linf);
    const double r0 = l2;
    *r0_out = r0;
    *cycles_out = 0;
    *rel_out = (r0 > 0.0) ? 1.0 : 0.0;
    int status = 1;
    if (r0 == 0.0) status = 0;
    else if (!isfinite(r0)) status = 2;
    else {
        const size_t bytes = sizeof(double) * (size_t)sph_count(ndim, n);
        double *work = (double *)malloc(bytes);
        if (!work) return 3;
        memcpy(work, u, bytes);
        for (int64_t c = 1; c <= max_cycles; ++c) {
            double *a = u, *w = work;
            for (int64_t s = 0; s < M; ++s) {
                srj_oracle_sph_sweep(ndim, n, radial, polar, azim, seq[s], b, a, w);
                double *t = a; a = w; w = t;
            }
            if (a != u) memcpy(u, a, bytes);
            srj_oracle_sph_residual(ndim, n, radial, polar, azim, b, u, NULL, &l2, &linf);
            *cycles_out = c;
            *rel_out = l2 / r0;
            if (!isfinite(l2)) { status = 2; break; }
            if (l2 / r0 <= tol) { status = 0; break; }
        }
        free(work);
    }
    srj_oracle_sph_finalize(ndim, n, u);
    return status;
}
