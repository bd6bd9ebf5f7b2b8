/*
 * FP64 CPU oracle for parallel-beam filtered back-projection and for the
 * TV-penalised least-squares reconstruction solved by ISTA/FISTA.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the benchmark's CPU-baseline leg load this file; the library never does,
 * and it shares no code, header, table or helper with the CUDA path.
 *
 * Everything is plain loops in double precision, written from the paper's
 * definitions (PyHST2, Mirone et al.):
 *   - dark subtraction and flat division of the raw radiographies (Sec. 2.3),
 *     followed by -ln for absorption tomography (abstract, Sec. 2.1);
 *   - "default filtered backprojection" (Sec. 2.3): Ram-Lak ramp filter along
 *     detector rows, then back-projection with linear interpolation of the
 *     filtered sinogram at t = (x-cx) cos(th) + (y-cy) sin(th) + axis(th)
 *     (per-projection axis position and angle, Sec. 2.1);
 *   - the forward projector, defined as the exact transpose of the
 *     unweighted back-projector (Sec. 2.3, last paragraph; Eq. 1);
 *   - isotropic total variation (Eq. 2) and its proximal map by Chambolle's
 *     dual fixed point (the paper cites Chambolle 2004 for isotropic TV);
 *   - ISTA / FISTA (Sec. 3.1, after Eq. 3) on 1/2 ||y - P x||^2 + beta TV(x)
 *     (Eq. 3), with the energy of Eq. 3 recorded at every iteration;
 *   - the overlapping-patch functional (Sec. 3.2.1, Eqs. 4-8), its gradient
 *     (Eq. 9) computed with the steps of Algorithm 1, and ISTA/FISTA with L1
 *     shrinkage on the patch coefficients.
 * Readings where the paper is silent (filter form, interpolation at the
 * detector edge, clamping of non-positive counts, TV step tau, start of the
 * dual field) are stated beside each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------------
 * Flat/dark normalisation (Sec. 2.3): r = (I - D) / (F - D), p = -ln r.
 * Reading: where F - D <= 0 the pixel carries no beam and p = 0; otherwise
 * r is clamped below at 1e-6 (p <= 13.8) so that zero or negative counts
 * stay finite.  r > 1 is kept (p < 0).  One slice: I is [n_rows][n_bins]
 * (one detector row per projection), F and D are [n_bins].
 * ------------------------------------------------------------------- */
void orc_normalise(const double *I, const double *F, const double *D,
                   int64_t n_rows, int64_t n_bins, double *p)
{
    for (int64_t r = 0; r < n_rows; r++)
        for (int64_t b = 0; b < n_bins; b++) {
            double den = F[b] - D[b];
            double v;
            if (den <= 0.0) {
                v = 0.0;
            } else {
                double ratio = (I[r * n_bins + b] - D[b]) / den;
                if (ratio < 1e-6) ratio = 1e-6;
                v = -log(ratio);
            }
            p[r * n_bins + b] = v;
        }
}

/* Ram-Lak kernel in the spatial domain, unit bin spacing (Kak & Slaney form):
 * h(0) = 1/4, h(n odd) = -1/(pi^2 n^2), h(n even, n != 0) = 0.            */
static double ramlak(int64_t n)
{
    if (n == 0) return 0.25;
    if (n % 2 == 0) return 0.0;
    return -1.0 / (M_PI * M_PI * (double)n * (double)n);
}

/* ---------------------------------------------------------------------
 * Ramp filter (Sec. 2.3, filtered back-projection; the paper does not name
 * the filter).  Reading: Ram-Lak, applied as the linear convolution of each
 * row with h, keeping the n_bins outputs aligned with the input bins:
 *   q[m] = sum_{k=0}^{n_bins-1} h(m - k) p[k].
 * This equals the circular convolution of the row zero-padded to any length
 * P >= 2 n_bins with h periodised on [-P/2, P/2).
 * ------------------------------------------------------------------- */
void orc_ramlak_filter(const double *p, int64_t n_rows, int64_t n_bins, double *q)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n_rows; r++)
        for (int64_t m = 0; m < n_bins; m++) {
            double acc = 0.0;
            for (int64_t k = 0; k < n_bins; k++)
                acc += ramlak(m - k) * p[r * n_bins + k];
            q[r * n_bins + m] = acc;
        }
}

/* Other ramp filters (the C boundary's Shepp-Logan and Hann options), as spatial
 * kernels of unit bin spacing applied by the same linear convolution:
 *   kind 1, Shepp-Logan (Kak & Slaney): h(n) = -2 / (pi^2 (4 n^2 - 1));
 *   kind 2, Hann: the Ram-Lak kernel smoothed by (1/4, 1/2, 1/4),
 *           h(n) = h_RL(n)/2 + (h_RL(n-1) + h_RL(n+1))/4.
 * kind 0 is Ram-Lak. */
static double filter_kernel(int kind, int64_t n)
{
    switch (kind) {
    case 1: return -2.0 / (M_PI * M_PI * (4.0 * (double)n * (double)n - 1.0));
    case 2: return 0.5 * ramlak(n) + 0.25 * (ramlak(n - 1) + ramlak(n + 1));
    default: return ramlak(n);
    }
}

void orc_filter(const double *p, int64_t n_rows, int64_t n_bins, int kind, double *q)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n_rows; r++)
        for (int64_t m = 0; m < n_bins; m++) {
            double acc = 0.0;
            for (int64_t k = 0; k < n_bins; k++)
                acc += filter_kernel(kind, m - k) * p[r * n_bins + k];
            q[r * n_bins + m] = acc;
        }
}

/* Detector coordinate of pixel (row i, column j) at angle index a. */
static double coord(int64_t i, int64_t j, double cth, double sth, double axis,
                    double cx, double cy)
{
    return ((double)j - cx) * cth + ((double)i - cy) * sth + axis;
}

/* ---------------------------------------------------------------------
 * Back-projection (Sec. 2.3): img[i][j] = weight * sum_a L(q_a, t_a(i,j)),
 * L(q, t) = (1 - f) q[i0] + f q[i0 + 1], i0 = floor(t), f = t - i0, and
 * q[k] = 0 for k outside [0, n_bins) (reading of the texture fetch: exact
 * linear interpolation, zero outside the detector).  For FBP,
 * weight = pi / (n_angles * pixel_size).
 * ------------------------------------------------------------------- */
void orc_backproject(const double *q, int64_t n_angles, int64_t n_bins,
                     const double *angles, const double *axis,
                     int64_t nx, int64_t ny, double cx, double cy,
                     double weight, double *img)
{
    double *cs = (double *)malloc(sizeof(double) * 2 * (n_angles > 0 ? n_angles : 1));
    for (int64_t a = 0; a < n_angles; a++) {
        cs[2 * a] = cos(angles[a]);
        cs[2 * a + 1] = sin(angles[a]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ny; i++)
        for (int64_t j = 0; j < nx; j++) {
            double acc = 0.0;
            for (int64_t a = 0; a < n_angles; a++) {
                double t = coord(i, j, cs[2 * a], cs[2 * a + 1], axis[a], cx, cy);
                double fl = floor(t);
                double f = t - fl;
                int64_t i0 = (int64_t)fl;
                const double *row = q + a * n_bins;
                double v0 = (i0 >= 0 && i0 < n_bins) ? row[i0] : 0.0;
                double v1 = (i0 + 1 >= 0 && i0 + 1 < n_bins) ? row[i0 + 1] : 0.0;
                acc += (1.0 - f) * v0 + f * v1;
            }
            img[i * nx + j] = weight * acc;
        }
    free(cs);
}

/* Back-projection at selected pixels only (rows ii[k], columns jj[k]); the
 * same definition as orc_backproject, for spot checks of large images. */
void orc_backproject_at(const double *q, int64_t n_angles, int64_t n_bins,
                        const double *angles, const double *axis,
                        const int64_t *ii, const int64_t *jj, int64_t n_points,
                        double cx, double cy, double weight, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n_points; k++) {
        double acc = 0.0;
        for (int64_t a = 0; a < n_angles; a++) {
            double t = coord(ii[k], jj[k], cos(angles[a]), sin(angles[a]), axis[a], cx, cy);
            double fl = floor(t);
            double f = t - fl;
            int64_t i0 = (int64_t)fl;
            const double *row = q + a * n_bins;
            double v0 = (i0 >= 0 && i0 < n_bins) ? row[i0] : 0.0;
            double v1 = (i0 + 1 >= 0 && i0 + 1 < n_bins) ? row[i0 + 1] : 0.0;
            acc += (1.0 - f) * v0 + f * v1;
        }
        out[k] = weight * acc;
    }
}

/* ---------------------------------------------------------------------
 * Forward projection: the exact transpose of the unweighted back-projector,
 * scaled by `scale` (the pixel size, so that the result approximates line
 * integrals in physical units):
 *   sino[a][b] = scale * sum_{i,j} img[i][j] * max(0, 1 - |t_a(i,j) - b|).
 * Written as the scatter of each pixel into the two bins floor(t) and
 * floor(t)+1 with weights 1-f and f, which are the only b where the hat
 * function is non-zero.
 * ------------------------------------------------------------------- */
void orc_project(const double *img, int64_t n_angles, int64_t n_bins,
                 const double *angles, const double *axis,
                 int64_t nx, int64_t ny, double cx, double cy,
                 double scale, double *sino)
{
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n_angles; a++) {
        double *row = sino + a * n_bins;
        for (int64_t b = 0; b < n_bins; b++) row[b] = 0.0;
        double cth = cos(angles[a]), sth = sin(angles[a]);
        for (int64_t i = 0; i < ny; i++)
            for (int64_t j = 0; j < nx; j++) {
                double t = coord(i, j, cth, sth, axis[a], cx, cy);
                double fl = floor(t);
                double f = t - fl;
                int64_t i0 = (int64_t)fl;
                double v = img[i * nx + j];
                if (i0 >= 0 && i0 < n_bins) row[i0] += (1.0 - f) * v;
                if (i0 + 1 >= 0 && i0 + 1 < n_bins) row[i0 + 1] += f * v;
            }
        for (int64_t b = 0; b < n_bins; b++) row[b] *= scale;
    }
}

/* ---------------------------------------------------------------------
 * Discrete gradient and divergence for Eq. 2 (isotropic TV, Chambolle 2004):
 * forward differences with Neumann boundary,
 *   g1[i][j] = x[i+1][j] - x[i][j]  (0 on the last row),
 *   g2[i][j] = x[i][j+1] - x[i][j]  (0 on the last column),
 * and div = -grad^T.
 * ------------------------------------------------------------------- */
void orc_grad(const double *x, int64_t ny, int64_t nx, double *g1, double *g2)
{
    for (int64_t i = 0; i < ny; i++)
        for (int64_t j = 0; j < nx; j++) {
            double v = x[i * nx + j];
            g1[i * nx + j] = (i + 1 < ny) ? x[(i + 1) * nx + j] - v : 0.0;
            g2[i * nx + j] = (j + 1 < nx) ? x[i * nx + j + 1] - v : 0.0;
        }
}

void orc_div(const double *p1, const double *p2, int64_t ny, int64_t nx, double *d)
{
    for (int64_t i = 0; i < ny; i++)
        for (int64_t j = 0; j < nx; j++) {
            double a = (i + 1 < ny) ? p1[i * nx + j] : 0.0;
            if (i > 0) a -= p1[(i - 1) * nx + j];
            double b = (j + 1 < nx) ? p2[i * nx + j] : 0.0;
            if (j > 0) b -= p2[i * nx + j - 1];
            d[i * nx + j] = a + b;
        }
}

/* Eq. 2: TV(x) = sum over pixels of sqrt((d1 x)^2 + (d2 x)^2). */
double orc_tv(const double *x, int64_t ny, int64_t nx)
{
    double tv = 0.0;
    for (int64_t i = 0; i < ny; i++)
        for (int64_t j = 0; j < nx; j++) {
            double v = x[i * nx + j];
            double a = (i + 1 < ny) ? x[(i + 1) * nx + j] - v : 0.0;
            double b = (j + 1 < nx) ? x[i * nx + j + 1] - v : 0.0;
            tv += sqrt(a * a + b * b);
        }
    return tv;
}

/* ---------------------------------------------------------------------
 * Proximal map of lam * TV (Eq. 2) by Chambolle's dual fixed point:
 *   g = div p^n - z / lam
 *   p^{n+1} = (p^n + tau grad g) / (1 + tau |grad g|)   (pixelwise norm)
 * for n_inner steps, then x = z - lam div p.  p1, p2 carry the dual field in
 * (start; zeros for a cold start) and out.  Reading: tau = 1/8 unless given;
 * lam <= 0 (beta = 0) is the identity.
 * ------------------------------------------------------------------- */
void orc_tv_prox(const double *z, int64_t ny, int64_t nx, double lam, double tau,
                 int64_t n_inner, double *p1, double *p2, double *x)
{
    int64_t n = ny * nx;
    if (lam <= 0.0) {                 /* no penalty: the prox is the identity */
        memcpy(x, z, sizeof(double) * n);
        return;
    }
    double *g = (double *)malloc(sizeof(double) * n);
    double *g1 = (double *)malloc(sizeof(double) * n);
    double *g2 = (double *)malloc(sizeof(double) * n);
    for (int64_t it = 0; it < n_inner; it++) {
        orc_div(p1, p2, ny, nx, g);
        for (int64_t k = 0; k < n; k++) g[k] -= z[k] / lam;
        orc_grad(g, ny, nx, g1, g2);
        for (int64_t k = 0; k < n; k++) {
            double nrm = sqrt(g1[k] * g1[k] + g2[k] * g2[k]);
            double den = 1.0 + tau * nrm;
            p1[k] = (p1[k] + tau * g1[k]) / den;
            p2[k] = (p2[k] + tau * g2[k]) / den;
        }
    }
    orc_div(p1, p2, ny, nx, g);
    for (int64_t k = 0; k < n; k++) x[k] = z[k] - lam * g[k];
    free(g); free(g1); free(g2);
}

/* ROF duality gap of (x = z - lam div p, p):
 *   primal 1/2||x - z||^2 + lam TV(x)  minus  dual 1/2||z||^2 - 1/2||z - lam div p||^2. */
double orc_rof_gap(const double *z, int64_t ny, int64_t nx, double lam,
                   const double *p1, const double *p2)
{
    int64_t n = ny * nx;
    double *d = (double *)malloc(sizeof(double) * n);
    double *x = (double *)malloc(sizeof(double) * n);
    orc_div(p1, p2, ny, nx, d);
    double fid = 0.0, zz = 0.0, xx = 0.0;
    for (int64_t k = 0; k < n; k++) {
        x[k] = z[k] - lam * d[k];
        fid += (x[k] - z[k]) * (x[k] - z[k]);
        zz += z[k] * z[k];
        xx += x[k] * x[k];
    }
    double primal = 0.5 * fid + lam * orc_tv(x, ny, nx);
    double dual = 0.5 * zz - 0.5 * xx;
    free(d); free(x);
    return primal - dual;
}

/* Geometry of one slice, as the solver needs it. */
typedef struct {
    int64_t n_angles, n_bins, nx, ny;
    const double *angles, *axis;
    double cx, cy, pixel_size;
} orc_geom;

static void P_apply(const orc_geom *g, const double *x, double *y)
{
    orc_project(x, g->n_angles, g->n_bins, g->angles, g->axis, g->nx, g->ny,
                g->cx, g->cy, g->pixel_size, y);
}

static void PT_apply(const orc_geom *g, const double *y, double *x)
{
    orc_backproject(y, g->n_angles, g->n_bins, g->angles, g->axis, g->nx, g->ny,
                    g->cx, g->cy, g->pixel_size, x);
}

/* Energy of Eq. 3: 1/2 ||y - P x||^2 + beta TV(x). */
double orc_energy(const orc_geom *g, const double *sino, const double *x, double beta)
{
    int64_t m = g->n_angles * g->n_bins;
    double *r = (double *)malloc(sizeof(double) * m);
    P_apply(g, x, r);
    double s = 0.0;
    for (int64_t k = 0; k < m; k++) s += (sino[k] - r[k]) * (sino[k] - r[k]);
    free(r);
    return 0.5 * s + beta * orc_tv(x, g->ny, g->nx);
}

/* ---------------------------------------------------------------------
 * Largest eigenvalue of P^T P by power iteration from the caller's start
 * vector v (seeded; overwritten with the last normalised iterate):
 *   w = P^T P v, v = w / ||w||;  returns <v, P^T P v> / <v, v> for the final v.
 * ------------------------------------------------------------------- */
double orc_power_iteration(const orc_geom *g, double *v, int64_t n_it)
{
    int64_t n = g->nx * g->ny, m = g->n_angles * g->n_bins;
    double *w = (double *)malloc(sizeof(double) * n);
    double *y = (double *)malloc(sizeof(double) * m);
    double nv = 0.0;
    for (int64_t k = 0; k < n; k++) nv += v[k] * v[k];
    nv = sqrt(nv);
    for (int64_t k = 0; k < n; k++) v[k] /= nv;
    for (int64_t it = 0; it < n_it; it++) {
        P_apply(g, v, y);
        PT_apply(g, y, w);
        double nw = 0.0;
        for (int64_t k = 0; k < n; k++) nw += w[k] * w[k];
        nw = sqrt(nw);
        for (int64_t k = 0; k < n; k++) v[k] = w[k] / nw;
    }
    P_apply(g, v, y);
    double ray = 0.0;
    for (int64_t k = 0; k < m; k++) ray += y[k] * y[k];     /* <v, P^T P v> = ||P v||^2 */
    free(w); free(y);
    return ray;
}

/* ---------------------------------------------------------------------
 * ISTA / FISTA (Sec. 3.1, Eq. 3) with constant step 1/L:
 *   x_k = prox_{(beta/L) TV}( y_k - (1/L) P^T (P y_k - sino) )
 *   FISTA: t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2,
 *          y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1});
 *   ISTA:  y_{k+1} = x_k.
 * Start y_1 = x_0 = x (input), t_1 = 1.  The TV prox runs n_inner Chambolle
 * steps from a zero dual field at every outer iteration (reading: cold start).
 * energy[k] = Eq. 3 at x_{k+1} (k = 0 .. n_iter-1).  x is overwritten with
 * the last iterate.
 * ------------------------------------------------------------------- */
/* as orc_fista; z_last (or NULL) receives the prox input z of the last
 * iteration, y - (1/L) P^T (P y - sino), and gap (or NULL) [n_iter] the ROF
 * duality gap of each iteration's prox (orc_rof_gap of its z and final dual
 * field; 0 when beta = 0, where the prox is the identity) */
void orc_fista_z(const orc_geom *g, const double *sino, double beta, double L,
                 int64_t n_iter, int64_t n_inner, double tau, int fista,
                 double *x, double *energy, double *gap, double *z_last, int warm_dual)
{
    int64_t n = g->nx * g->ny, m = g->n_angles * g->n_bins;
    double *y = (double *)malloc(sizeof(double) * n);
    double *xprev = (double *)malloc(sizeof(double) * n);
    double *z = (double *)malloc(sizeof(double) * n);
    double *grad = (double *)malloc(sizeof(double) * n);
    double *p1 = (double *)malloc(sizeof(double) * n);
    double *p2 = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * m);
    memcpy(y, x, sizeof(double) * n);
    memcpy(xprev, x, sizeof(double) * n);
    double t = 1.0;
    for (int64_t k = 0; k < n_iter; k++) {
        P_apply(g, y, r);
        for (int64_t q = 0; q < m; q++) r[q] -= sino[q];
        PT_apply(g, r, grad);
        for (int64_t q = 0; q < n; q++) z[q] = y[q] - grad[q] / L;
        /* the dual field starts at zero (the reading: a cold start), or with
         * warm_dual at the previous iteration's final dual field */
        if (k == 0 || !warm_dual) {
            memset(p1, 0, sizeof(double) * n);
            memset(p2, 0, sizeof(double) * n);
        }
        orc_tv_prox(z, g->ny, g->nx, beta / L, tau, n_inner, p1, p2, x);
        if (gap) gap[k] = beta > 0.0 ? orc_rof_gap(z, g->ny, g->nx, beta / L, p1, p2) : 0.0;
        double tn = fista ? 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)) : 1.0;
        double w = fista ? (t - 1.0) / tn : 0.0;
        for (int64_t q = 0; q < n; q++) {
            y[q] = x[q] + w * (x[q] - xprev[q]);
            xprev[q] = x[q];
        }
        t = tn;
        if (energy) energy[k] = orc_energy(g, sino, x, beta);
    }
    if (z_last) memcpy(z_last, z, sizeof(double) * n);
    free(y); free(xprev); free(z); free(grad); free(p1); free(p2); free(r);
}

void orc_fista(const orc_geom *g, const double *sino, double beta, double L,
               int64_t n_iter, int64_t n_inner, double tau, int fista,
               double *x, double *energy)
{
    orc_fista_z(g, sino, beta, L, n_iter, n_inner, tau, fista, x, energy, NULL, NULL, 0);
}

/* ---------------------------------------------------------------------
 * beta-selection estimators (Sec. 4, Eqs. 10-11).
 * Cosine of the angle between two images: <a, b> / (||a|| ||b||)
 * (NaN when either norm is zero).
 * ------------------------------------------------------------------- */
double orc_cosine(const double *a, const double *b, int64_t n)
{
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (int64_t k = 0; k < n; k++) {
        ab += a[k] * b[k];
        aa += a[k] * a[k];
        bb += b[k] * b[k];
    }
    if (aa == 0.0 || bb == 0.0) return NAN;
    return ab / (sqrt(aa) * sqrt(bb));
}

/* Decoherence estimator (Eq. 11): E = Cos(I(beta) - I(0+), I(beta)). */
double orc_ecohe(const double *I_beta, const double *I_0, int64_t n)
{
    double *d = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int64_t k = 0; k < n; k++) d[k] = I_beta[k] - I_0[k];
    double c = orc_cosine(d, I_beta, n);
    free(d);
    return c;
}

/* ---------------------------------------------------------------------
 * Preprocessing variants (Sec. 2.3), on a raw stack I [na][nz][nb]
 * (projection-major) in the paper's order: dark/flat correction with flats
 * interpolated in time, hot-spot median filter, -ln, ring filter.
 *
 * Flat field: projection a uses F = (1 - w) flats[f0] + w flats[f0 + 1],
 * f0 = floor(pos[a]), w = pos[a] - f0 (pos clamped to [0, nf - 1]; flats are
 * [nf][nz][nb]); r = (I - D) / (F - D), r = 1 where F - D <= 0.
 * ------------------------------------------------------------------- */
void orc_flatfield(const double *I, const double *flats, int64_t nf, const double *pos, const double *D,
                   int64_t na, int64_t nz, int64_t nb, double *r)
{
    for (int64_t a = 0; a < na; a++) {
        double ps = nf > 1 ? pos[a] : 0.0;
        if (ps < 0.0) ps = 0.0;
        if (ps > (double)(nf - 1)) ps = (double)(nf - 1);
        int64_t f0 = (int64_t)floor(ps);
        if (f0 > nf - 2) f0 = nf > 1 ? nf - 2 : 0;
        double w = ps - (double)f0;
        for (int64_t z = 0; z < nz; z++)
            for (int64_t b = 0; b < nb; b++) {
                int64_t k = z * nb + b;
                double F = flats[f0 * nz * nb + k];
                if (nf > 1) F = (1.0 - w) * F + w * flats[(f0 + 1) * nz * nb + k];
                double den = F - D[k];
                r[(a * nz + z) * nb + b] = den > 0.0 ? (I[(a * nz + z) * nb + b] - D[k]) / den : 1.0;
            }
    }
}

static int cmp_double(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

/* Hot-spot filter: in each projection, a pixel whose neighbours' median (the
 * up to 8 pixels around it in the (z, b) plane that exist; for an even count
 * the mean of the two middle values) is smaller than the pixel by more than
 * `threshold` takes that median.  Neighbours are read from the input. */
void orc_hotspot(const double *r, int64_t na, int64_t nz, int64_t nb, double threshold, double *out)
{
    for (int64_t a = 0; a < na; a++)
        for (int64_t z = 0; z < nz; z++)
            for (int64_t b = 0; b < nb; b++) {
                double v[8];
                int n = 0;
                for (int dz = -1; dz <= 1; dz++)
                    for (int db = -1; db <= 1; db++) {
                        if (dz == 0 && db == 0) continue;
                        int64_t zz = z + dz, bb = b + db;
                        if (zz < 0 || zz >= nz || bb < 0 || bb >= nb) continue;
                        v[n++] = r[(a * nz + zz) * nb + bb];
                    }
                double x = r[(a * nz + z) * nb + b];
                double med = x;
                if (n > 0) {
                    qsort(v, n, sizeof(double), cmp_double);
                    med = (n % 2) ? v[n / 2] : 0.5 * (v[n / 2 - 1] + v[n / 2]);
                }
                out[(a * nz + z) * nb + b] = (med < x - threshold) ? med : x;
            }
}

/* p = -ln(max(r, 1e-6)) (absorption; same clamp as orc_normalise). */
void orc_log(const double *r, int64_t n, double *p)
{
    for (int64_t k = 0; k < n; k++) p[k] = -log(r[k] < 1e-6 ? 1e-6 : r[k]);
}

/* Ring filter on one sinogram p [na][nb] (in place): s(b) = mean over angles,
 * m(b) = mean of s over [b - h, b + h] inside [0, nb) with h = (window-1)/2,
 * and p(a, b) -= s(b) - m(b) (the high-pass part of the angular mean). */
void orc_ring(double *p, int64_t na, int64_t nb, int64_t window)
{
    double *sm = (double *)calloc(nb > 0 ? nb : 1, sizeof(double));
    double *hp = (double *)calloc(nb > 0 ? nb : 1, sizeof(double));
    int64_t h = (window - 1) / 2;
    for (int64_t b = 0; b < nb; b++) {
        double acc = 0.0;
        for (int64_t a = 0; a < na; a++) acc += p[a * nb + b];
        sm[b] = acc / (double)na;
    }
    for (int64_t b = 0; b < nb; b++) {
        double acc = 0.0;
        int64_t cnt = 0;
        for (int64_t c = b - h; c <= b + h; c++)
            if (c >= 0 && c < nb) {
                acc += sm[c];
                cnt++;
            }
        hp[b] = sm[b] - acc / (double)cnt;
    }
    for (int64_t a = 0; a < na; a++)
        for (int64_t b = 0; b < nb; b++) p[a * nb + b] -= hp[b];
    free(sm);
    free(hp);
}

/* ---------------------------------------------------------------------
 * Overlapping-patch functional (Sec. 3.2.1, Eqs. 4-9; Algorithm 1).
 *
 * Patches of m x m pixels sit on a grid: along an axis of n pixels the k-th
 * patch starts at min(k * stride, n - m), k = 0 .. K-1, K = ceil((n - m) /
 * stride) + 1, so they cover the image (Eq. 4).  The core of a pixel (Eqs.
 * 5-6) is the patch whose centre start + (m-1)/2 is nearest in L1; on a
 * product grid that is the nearest centre along each axis (ties: the lower
 * index).  Patches P [N][m*m] (row-major inside the patch, N = Kr * Kc,
 * patch index kr * Kc + kc) come from the coefficients W [N][Nc] and the
 * dictionary D [Nc][m*m] as P = W D; the image takes each pixel from its core
 * patch (Eq. 7).  f(W) = ||y - Pi x||^2 + rho sum_p sum_{i in p} (x_i - P_pi)^2
 * (Eq. 8), F = f + beta ||W||_1.  Pi is the projector (scaled by the pixel
 * size) or the identity (denoising).
 * ------------------------------------------------------------------- */
typedef struct {
    int64_t ny, nx, m, stride, kr, kc;
} orc_patchgrid;

static int64_t pg_count(int64_t n, int64_t m, int64_t stride)
{
    return (n - m + stride - 1) / stride + 1;
}

static int64_t pg_start(int64_t k, int64_t n, int64_t m, int64_t stride)
{
    int64_t r = k * stride;
    return r > n - m ? n - m : r;
}

static int64_t pg_core(int64_t i, int64_t n, int64_t m, int64_t stride, int64_t K)
{
    int64_t best = 0;
    double bd = 1e300;
    for (int64_t k = 0; k < K; k++) {
        double d = fabs((double)i - ((double)pg_start(k, n, m, stride) + 0.5 * (double)(m - 1)));
        if (d < bd) {
            bd = d;
            best = k;
        }
    }
    return best;
}

void orc_patch_grid(int64_t ny, int64_t nx, int64_t m, int64_t stride, int64_t *kr, int64_t *kc)
{
    *kr = pg_count(ny, m, stride);
    *kc = pg_count(nx, m, stride);
}

/* orthonormal 2-D DCT-II basis of m x m patches: D [m*m][m*m], row u*m+v */
void orc_dct_dictionary(int64_t m, double *D)
{
    for (int64_t u = 0; u < m; u++)
        for (int64_t v = 0; v < m; v++)
            for (int64_t a = 0; a < m; a++)
                for (int64_t b = 0; b < m; b++) {
                    double au = u ? sqrt(2.0 / m) : sqrt(1.0 / m);
                    double av = v ? sqrt(2.0 / m) : sqrt(1.0 / m);
                    D[(u * m + v) * m * m + a * m + b] =
                        au * av * cos(M_PI * (2 * a + 1) * u / (2.0 * m)) * cos(M_PI * (2 * b + 1) * v / (2.0 * m));
                }
}

/* C = A B with A [r][k], B [k][c] */
static void matmul(const double *A, const double *B, int64_t r, int64_t k, int64_t c, double *C)
{
    for (int64_t i = 0; i < r; i++)
        for (int64_t j = 0; j < c; j++) {
            double acc = 0.0;
            for (int64_t t = 0; t < k; t++) acc += A[i * k + t] * B[t * c + j];
            C[i * c + j] = acc;
        }
}

/* Eq. 7: x_j = P[core(j)][j - r_core(j)] */
void orc_patch_assemble(const double *P, int64_t ny, int64_t nx, int64_t m, int64_t stride, double *X)
{
    int64_t kr = pg_count(ny, m, stride), kc = pg_count(nx, m, stride);
    for (int64_t i = 0; i < ny; i++) {
        int64_t pr = pg_core(i, ny, m, stride, kr), ri = pg_start(pr, ny, m, stride);
        for (int64_t j = 0; j < nx; j++) {
            int64_t pc = pg_core(j, nx, m, stride, kc), rj = pg_start(pc, nx, m, stride);
            X[i * nx + j] = P[(pr * kc + pc) * m * m + (i - ri) * m + (j - rj)];
        }
    }
}

/* S_j = sum of the patches covering j, Nv_j = their number (Algorithm 1) */
void orc_patch_sum(const double *P, int64_t ny, int64_t nx, int64_t m, int64_t stride, double *S, double *Nv)
{
    int64_t kr = pg_count(ny, m, stride), kc = pg_count(nx, m, stride);
    for (int64_t k = 0; k < ny * nx; k++) S[k] = Nv[k] = 0.0;
    for (int64_t a = 0; a < kr; a++)
        for (int64_t b = 0; b < kc; b++) {
            int64_t ri = pg_start(a, ny, m, stride), rj = pg_start(b, nx, m, stride);
            for (int64_t u = 0; u < m; u++)
                for (int64_t v = 0; v < m; v++) {
                    S[(ri + u) * nx + rj + v] += P[(a * kc + b) * m * m + u * m + v];
                    Nv[(ri + u) * nx + rj + v] += 1.0;
                }
        }
}

typedef struct {
    int64_t ny, nx, m, stride, nc;
    const double *D;        /* [nc][m*m] */
    double rho;
    int denoise;            /* 1: Pi = identity */
    const orc_geom *g;      /* projector geometry when denoise == 0 */
} orc_patchprob;

static void pi_apply(const orc_patchprob *q, const double *x, double *y)
{
    if (q->denoise) memcpy(y, x, sizeof(double) * q->ny * q->nx);
    else P_apply(q->g, x, y);
}

static void pit_apply(const orc_patchprob *q, const double *y, double *x)
{
    if (q->denoise) memcpy(x, y, sizeof(double) * q->ny * q->nx);
    else PT_apply(q->g, y, x);
}

static int64_t data_size(const orc_patchprob *q)
{
    return q->denoise ? q->ny * q->nx : q->g->n_angles * q->g->n_bins;
}

/* f(W) of Eq. 8 (the smooth part) */
double orc_patch_f(const orc_patchprob *q, const double *W, const double *y)
{
    int64_t kr = pg_count(q->ny, q->m, q->stride), kc = pg_count(q->nx, q->m, q->stride), N = kr * kc;
    int64_t mm = q->m * q->m, n = q->ny * q->nx, md = data_size(q);
    double *P = (double *)malloc(sizeof(double) * N * mm);
    double *X = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * md);
    matmul(W, q->D, N, q->nc, mm, P);
    orc_patch_assemble(P, q->ny, q->nx, q->m, q->stride, X);
    pi_apply(q, X, r);
    double f = 0.0;
    for (int64_t k = 0; k < md; k++) f += (y[k] - r[k]) * (y[k] - r[k]);
    double pen = 0.0;
    for (int64_t a = 0; a < kr; a++)
        for (int64_t b = 0; b < kc; b++) {
            int64_t ri = pg_start(a, q->ny, q->m, q->stride), rj = pg_start(b, q->nx, q->m, q->stride);
            for (int64_t u = 0; u < q->m; u++)
                for (int64_t v = 0; v < q->m; v++) {
                    double d = X[(ri + u) * q->nx + rj + v] - P[(a * kc + b) * mm + u * q->m + v];
                    pen += d * d;
                }
        }
    free(P); free(X); free(r);
    return f + q->rho * pen;
}

/* Gradient of f (Eq. 9), computed with Algorithm 1's steps:
 *   P = W D; X from the cores; R = Pi^T (Pi X - y); S, Nv;
 *   P'_pi = [core(r_p + i) = p] (R + rho (Nv X - S))_{r_p+i} + rho (P_pi - X_{r_p+i});
 *   G = 2 P' D^T.
 * Reading: R carries the sign of Eq. 9 (Pi^T (Pi x - y)); Algorithm 1 prints
 * Bp(data - Fp(X)), the opposite sign, which is not the gradient of Eq. 8. */
void orc_patch_gradient(const orc_patchprob *q, const double *W, const double *y, double *G)
{
    int64_t kr = pg_count(q->ny, q->m, q->stride), kc = pg_count(q->nx, q->m, q->stride), N = kr * kc;
    int64_t mm = q->m * q->m, n = q->ny * q->nx, md = data_size(q);
    double *P = (double *)malloc(sizeof(double) * N * mm);
    double *Pp = (double *)malloc(sizeof(double) * N * mm);
    double *X = (double *)malloc(sizeof(double) * n);
    double *R = (double *)malloc(sizeof(double) * n);
    double *S = (double *)malloc(sizeof(double) * n);
    double *Nv = (double *)malloc(sizeof(double) * n);
    double *r = (double *)malloc(sizeof(double) * md);
    double *DT = (double *)malloc(sizeof(double) * mm * q->nc);
    matmul(W, q->D, N, q->nc, mm, P);
    orc_patch_assemble(P, q->ny, q->nx, q->m, q->stride, X);
    pi_apply(q, X, r);
    for (int64_t k = 0; k < md; k++) r[k] -= y[k];
    pit_apply(q, r, R);
    orc_patch_sum(P, q->ny, q->nx, q->m, q->stride, S, Nv);
    for (int64_t a = 0; a < kr; a++)
        for (int64_t b = 0; b < kc; b++) {
            int64_t p = a * kc + b;
            int64_t ri = pg_start(a, q->ny, q->m, q->stride), rj = pg_start(b, q->nx, q->m, q->stride);
            for (int64_t u = 0; u < q->m; u++)
                for (int64_t v = 0; v < q->m; v++) {
                    int64_t j = (ri + u) * q->nx + rj + v;
                    double val = q->rho * (P[p * mm + u * q->m + v] - X[j]);
                    int64_t cr = pg_core(ri + u, q->ny, q->m, q->stride, kr);
                    int64_t cc = pg_core(rj + v, q->nx, q->m, q->stride, kc);
                    if (cr == a && cc == b) val += R[j] + q->rho * (Nv[j] * X[j] - S[j]);
                    Pp[p * mm + u * q->m + v] = val;
                }
        }
    for (int64_t t = 0; t < q->nc; t++)
        for (int64_t k = 0; k < mm; k++) DT[k * q->nc + t] = q->D[t * mm + k];
    matmul(Pp, DT, N, mm, q->nc, G);
    for (int64_t k = 0; k < N * q->nc; k++) G[k] *= 2.0;
    free(P); free(Pp); free(X); free(R); free(S); free(Nv); free(r); free(DT);
}

/* ISTA/FISTA on F(W) = f(W) + beta ||W||_1 (Sec. 3.2.2): a gradient step of
 * length 1/L, then the L1 shrinkage sign(v) max(|v| - beta/L, 0); FISTA
 * momentum as in orc_fista.  W in: start, out: last iterate; energy[k] = F at
 * iterate k; X receives the image of the last iterate. */
void orc_patch_fista(const orc_patchprob *q, const double *y, double beta, double L, int64_t n_iter, int fista,
                     double *W, double *energy, double *X)
{
    int64_t kr = pg_count(q->ny, q->m, q->stride), kc = pg_count(q->nx, q->m, q->stride);
    int64_t nw = kr * kc * q->nc;
    double *Y = (double *)malloc(sizeof(double) * nw);
    double *Wp = (double *)malloc(sizeof(double) * nw);
    double *G = (double *)malloc(sizeof(double) * nw);
    memcpy(Y, W, sizeof(double) * nw);
    memcpy(Wp, W, sizeof(double) * nw);
    double t = 1.0;
    for (int64_t k = 0; k < n_iter; k++) {
        orc_patch_gradient(q, Y, y, G);
        for (int64_t e = 0; e < nw; e++) {
            double v = Y[e] - G[e] / L;
            double a = fabs(v) - beta / L;
            W[e] = a > 0.0 ? (v > 0.0 ? a : -a) : 0.0;
        }
        double tn = fista ? 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)) : 1.0;
        double w = fista ? (t - 1.0) / tn : 0.0;
        for (int64_t e = 0; e < nw; e++) {
            Y[e] = W[e] + w * (W[e] - Wp[e]);
            Wp[e] = W[e];
        }
        t = tn;
        if (energy) {
            double l1 = 0.0;
            for (int64_t e = 0; e < nw; e++) l1 += fabs(W[e]);
            energy[k] = orc_patch_f(q, W, y) + beta * l1;
        }
    }
    if (X) {
        int64_t mm = q->m * q->m, N = kr * kc;
        double *P = (double *)malloc(sizeof(double) * N * mm);
        matmul(W, q->D, N, q->nc, mm, P);
        orc_patch_assemble(P, q->ny, q->nx, q->m, q->stride, X);
        free(P);
    }
    free(Y); free(Wp); free(G);
}
