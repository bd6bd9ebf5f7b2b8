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
 *     (Eq. 3), with the energy of Eq. 3 recorded at every iteration.
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
void orc_fista(const orc_geom *g, const double *sino, double beta, double L,
               int64_t n_iter, int64_t n_inner, double tau, int fista,
               double *x, double *energy)
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
        memset(p1, 0, sizeof(double) * n);
        memset(p2, 0, sizeof(double) * n);
        orc_tv_prox(z, g->ny, g->nx, beta / L, tau, n_inner, p1, p2, x);
        double tn = fista ? 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t)) : 1.0;
        double w = fista ? (t - 1.0) / tn : 0.0;
        for (int64_t q = 0; q < n; q++) {
            y[q] = x[q] + w * (x[q] - xprev[q]);
            xprev[q] = x[q];
        }
        t = tn;
        if (energy) energy[k] = orc_energy(g, sino, x, beta);
    }
    free(y); free(xprev); free(z); free(grad); free(p1); free(p2); free(r);
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
