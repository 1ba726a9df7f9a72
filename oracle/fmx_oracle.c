/*
 * fmx_oracle.c -- plain, slow, FP64 CPU oracle for the averaged-Yee Maxwell step
 * of Lu et al., "An O(N) Maxwell solver with improved numerical dispersion
 * properties" (arXiv:1907.13088).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this code.  It shares nothing with the CUDA
 * path: no header, no helper, no coefficient generator.
 *
 * Every operator is applied to a whole periodic array with the paper's own
 * definitions, in the order the paper states them:
 *   D_x f = (f_{k+1/2} - f_{k-1/2})/dx, alpha_x f = (f_{k+1} + 4 f_k + f_{k-1})/6
 *        (Sec. 2, operator definitions), written as alpha_x = 1 + Dbar_xx/6,
 *        which is the same operator;
 *   Faraday update, Eqs. faraday_x..z;
 *   auxiliary-field source, Eqs. ampere_aux_x..z (Sec. 2.2.1);
 *   matrix A, Eqs. matrixA_1st..matrixA_last;
 *   fixed-point iteration, Algorithm 1;
 *   E^{n+1} = E^n + Delta E (Sec. 2.2.1, text after Eq. matrixA_last).
 * Reduced dimensions follow Sec. 2.2.2/2.2.3: an inactive axis has D -> 0 and
 * alpha -> 1, so every term that holds it is dropped.
 *
 * Storage: each component is a dense nx*ny*nz array, x fastest.  Index (i,j,k)
 * of a component sits at the physical position of the Yee variable list of
 * Sec. 2: Ex (i+1/2, j, k), Ey (i, j+1/2, k), Ez (i, j, k+1/2),
 * Bx (i, j+1/2, k+1/2), By (i+1/2, j, k+1/2), Bz (i+1/2, j+1/2, k); j like E.
 * Boundaries are periodic.  E is at t = n dt and B at t = (n+1/2) dt.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "fmx_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Sets the number of OpenMP threads the loops use (n <= 0 leaves it) and
 * returns the number in effect; 1 when built without OpenMP. */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* coefficients                                                               */
/* ------------------------------------------------------------------------- */

static double round_f32(double v) { return (double)(float)v; }

/* dt_CFL of Eq. dt_cfl_3d (and its 2D/1D forms): (sum over active axes of
 * 1/d_i^2)^(-1/2) / c. */
double orc_dt_cfl(const orc_params *p)
{
    double s = 0.0;
    for (int a = 0; a < p->dims; ++a) s += 1.0 / (p->d[a] * p->d[a]);
    return 1.0 / (p->c * sqrt(s));
}

/* The scalar factors that multiply a field anywhere in the step.  Each is
 * computed in binary64 in the order written; with coef_f32 set each is then
 * rounded once to binary32 (the values a binary32 field advance multiplies
 * by).  sigma_i = (c dt/d_i)^2 and sigma_ij = c^2 dt^2/(d_i d_j) are the
 * ratios that appear in Eqs. matrixA_1st..matrixA_last. */
void orc_coefficients(const orc_params *p, double co[ORC_NCOEF])
{
    const double cdt = p->c * p->dt;
    double k[3], s[3];
    for (int a = 0; a < 3; ++a) { k[a] = cdt / p->d[a]; s[a] = k[a] * k[a]; }
    co[ORC_KX] = k[0];
    co[ORC_KY] = k[1];
    co[ORC_KZ] = k[2];
    co[ORC_Q] = (4.0 * M_PI) * p->dt;
    if (p->lumped) {
        /* lumping the averaging operators (alpha -> 1) recovers Yee: A = 0 */
        for (int c = ORC_C6; c < ORC_NCOEF; ++c) co[c] = 0.0;
    } else {
        co[ORC_C6] = 1.0 / 6.0;
        co[ORC_AX] = (s[0] - 1.0) / 6.0;
        co[ORC_AY] = (s[1] - 1.0) / 6.0;
        co[ORC_AZ] = (s[2] - 1.0) / 6.0;
        co[ORC_AYZ] = (s[1] + s[2] - 1.0) / 36.0;
        co[ORC_AZX] = (s[2] + s[0] - 1.0) / 36.0;
        co[ORC_AXY] = (s[0] + s[1] - 1.0) / 36.0;
        co[ORC_BYZ] = -(k[1] * k[2]) / 6.0;
        co[ORC_BZX] = -(k[2] * k[0]) / 6.0;
        co[ORC_BXY] = -(k[0] * k[1]) / 6.0;
    }
    if (p->coef_f32)
        for (int c = 0; c < ORC_NCOEF; ++c) co[c] = round_f32(co[c]);
}

/* ------------------------------------------------------------------------- */
/* elementary periodic operators on one component array                     */
/* ------------------------------------------------------------------------- */

typedef struct {
    long n[3];
    long ncell;
    int active[3];
} shape_t;

static shape_t shape_of(const orc_params *p)
{
    shape_t s;
    for (int a = 0; a < 3; ++a) {
        s.n[a] = p->n[a];
        s.active[a] = a < p->dims;
    }
    s.ncell = s.n[0] * s.n[1] * s.n[2];
    return s;
}

static long wrapi(long i, long n) { i %= n; return i < 0 ? i + n : i; }

/* value of f at the cell shifted by `off` along axis a (periodic) */
static inline double at(const shape_t *s, const double *f, long i, long j, long k, int a, long off)
{
    long ii = i, jj = j, kk = k;
    if (a == 0) ii = wrapi(i + off, s->n[0]);
    if (a == 1) jj = wrapi(j + off, s->n[1]);
    if (a == 2) kk = wrapi(k + off, s->n[2]);
    return f[(kk * s->n[1] + jj) * s->n[0] + ii];
}

/* out = Dbar_a f (Eq. defining Dbar: difference of the two values half a cell
 * either side).  `fwd` = 1 when f sits on integer positions along a (result
 * at +1/2, same index): f[i+1] - f[i].  `fwd` = 0 when f sits on half-integer
 * positions (result on the integer position, same index): f[i] - f[i-1].
 * An inactive axis gives zero (D -> 0). */
static void dbar(const shape_t *s, const double *f, double *out, int a, int fwd)
{
    if (!s->active[a]) { memset(out, 0, sizeof(double) * s->ncell); return; }
#pragma omp parallel for collapse(2) schedule(static)
    for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
            for (long i = 0; i < s->n[0]; ++i) {
                double v = fwd ? at(s, f, i, j, k, a, 1) - at(s, f, i, j, k, a, 0)
                               : at(s, f, i, j, k, a, 0) - at(s, f, i, j, k, a, -1);
                out[(k * s->n[1] + j) * s->n[0] + i] = v;
            }
}

/* out = Dbar_aa f = f[i+1] - 2 f[i] + f[i-1] (zero on an inactive axis) */
static void dbar2(const shape_t *s, const double *f, double *out, int a)
{
    if (!s->active[a]) { memset(out, 0, sizeof(double) * s->ncell); return; }
#pragma omp parallel for collapse(2) schedule(static)
    for (long k = 0; k < s->n[2]; ++k)
        for (long j = 0; j < s->n[1]; ++j)
            for (long i = 0; i < s->n[0]; ++i)
                out[(k * s->n[1] + j) * s->n[0] + i] =
                    at(s, f, i, j, k, a, 1) - 2.0 * at(s, f, i, j, k, a, 0) + at(s, f, i, j, k, a, -1);
}

/* y = y + w * x */
static void axpy(const shape_t *s, double w, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (long c = 0; c < s->ncell; ++c) y[c] += w * x[c];
}

/* out = alpha_a f = f + c6 * Dbar_aa f; identity on an inactive axis */
static void alpha(const shape_t *s, double c6, const double *f, double *out, double *tmp, int a)
{
    memcpy(out, f, sizeof(double) * s->ncell);
    if (!s->active[a]) return;
    dbar2(s, f, tmp, a);
    axpy(s, c6, tmp, out);
}

static double *alloc_cells(const shape_t *s) { return (double *)calloc((size_t)s->ncell, sizeof(double)); }

/* ------------------------------------------------------------------------- */
/* low-pass filter                                                            */
/* ------------------------------------------------------------------------- */

/* One pass of the binomial (1/4, 1/2, 1/4) low-pass along every active axis,
 * repeated `passes` times, in place.  The paper asks for "low pass filtering"
 * of the current (Sec. 4.2, Sec. 5) without fixing the stencil; this reading
 * takes the binomial filter, the same on every component. */
void orc_filter(const orc_params *p, double *f, int ncomp, int passes)
{
    shape_t s = shape_of(p);
    double *t = alloc_cells(&s);
    for (int q = 0; q < ncomp; ++q) {
        double *g = f + (size_t)q * s.ncell;
        for (int pass = 0; pass < passes; ++pass)
            for (int a = 0; a < 3; ++a) {
                if (!s.active[a]) continue;
#pragma omp parallel for collapse(2) schedule(static)
                for (long k = 0; k < s.n[2]; ++k)
                    for (long j = 0; j < s.n[1]; ++j)
                        for (long i = 0; i < s.n[0]; ++i)
                            t[(k * s.n[1] + j) * s.n[0] + i] =
                                0.25 * at(&s, g, i, j, k, a, -1) + 0.5 * at(&s, g, i, j, k, a, 0) +
                                0.25 * at(&s, g, i, j, k, a, 1);
                memcpy(g, t, sizeof(double) * s.ncell);
            }
    }
    free(t);
}

/* ------------------------------------------------------------------------- */
/* auxiliary-field source, Eqs. ampere_aux_x..z                               */
/* ------------------------------------------------------------------------- */

/* dEp = c dt curl(alpha B) - 4 pi dt j, i.e. the change of the auxiliary field
 * E' over one step: (1/c) D_t E'_x = D_y(alpha_z B_z) - D_z(alpha_y B_y)
 * - (4 pi / c) j_x and cyclic.  B sits on half-integer positions along every
 * axis it is differentiated along, so each Dbar here is the backward form.
 * j may be NULL (vacuum). */
void orc_source(const orc_params *p, const double *B, const double *J, double *dEp)
{
    shape_t s = shape_of(p);
    double co[ORC_NCOEF];
    orc_coefficients(p, co);
    const long n = s.ncell;
    const double *Bx = B, *By = B + n, *Bz = B + 2 * n;
    double *ab = alloc_cells(&s), *d = alloc_cells(&s), *t = alloc_cells(&s);
    double *ex = dEp, *ey = dEp + n, *ez = dEp + 2 * n;
    memset(dEp, 0, sizeof(double) * 3 * n);

    /* x: k_y Dbar_y(alpha_z Bz) - k_z Dbar_z(alpha_y By) */
    alpha(&s, co[ORC_C6], Bz, ab, t, 2); dbar(&s, ab, d, 1, 0); axpy(&s, co[ORC_KY], d, ex);
    alpha(&s, co[ORC_C6], By, ab, t, 1); dbar(&s, ab, d, 2, 0); axpy(&s, -co[ORC_KZ], d, ex);
    /* y: k_z Dbar_z(alpha_x Bx) - k_x Dbar_x(alpha_z Bz) */
    alpha(&s, co[ORC_C6], Bx, ab, t, 0); dbar(&s, ab, d, 2, 0); axpy(&s, co[ORC_KZ], d, ey);
    alpha(&s, co[ORC_C6], Bz, ab, t, 2); dbar(&s, ab, d, 0, 0); axpy(&s, -co[ORC_KX], d, ey);
    /* z: k_x Dbar_x(alpha_y By) - k_y Dbar_y(alpha_x Bx) */
    alpha(&s, co[ORC_C6], By, ab, t, 1); dbar(&s, ab, d, 0, 0); axpy(&s, co[ORC_KX], d, ez);
    alpha(&s, co[ORC_C6], Bx, ab, t, 0); dbar(&s, ab, d, 1, 0); axpy(&s, -co[ORC_KY], d, ez);

    if (J)
        for (int c = 0; c < 3; ++c) axpy(&s, -co[ORC_Q], J + (size_t)c * n, dEp + (size_t)c * n);
    free(ab); free(d); free(t);
}

/* ------------------------------------------------------------------------- */
/* matrix A, Eqs. matrixA_1st..matrixA_last                                   */
/* ------------------------------------------------------------------------- */

/* Adds coefficient * Dbar_i(fwd) Dbar_j(bwd) (f + c6 Dbar_kk f) to out: the
 * off-diagonal element A_ij acting on E_j at the position of E_i.  E_j sits
 * on a half-integer position along j (backward difference brings it to the
 * integer position), and the result must sit on a half-integer position along
 * i (forward difference). */
static void add_cross(const shape_t *s, double coef, double c6, const double *f, double *out, int ai,
                      int aj, int ak, double *t1, double *t2)
{
    if (!s->active[ai] || !s->active[aj]) return;
    memcpy(t1, f, sizeof(double) * s->ncell);
    if (s->active[ak]) { dbar2(s, f, t2, ak); axpy(s, c6, t2, t1); } /* (1 + Dbar_kk/6) f */
    dbar(s, t1, t2, aj, 0);
    dbar(s, t2, t1, ai, 1);
    axpy(s, coef, t1, out);
}

/* Adds the diagonal element A_ii f = a_j Dbar_jj f + a_k Dbar_kk f
 * + a_jk Dbar_jjkk f to out (j, k the two other axes). */
static void add_diag(const shape_t *s, double aj_, double ak_, double ajk, const double *f, double *out,
                     int aj, int ak, double *t1, double *t2)
{
    if (s->active[aj]) { dbar2(s, f, t1, aj); axpy(s, aj_, t1, out); }
    if (s->active[ak]) { dbar2(s, f, t1, ak); axpy(s, ak_, t1, out); }
    if (s->active[aj] && s->active[ak]) {
        dbar2(s, f, t1, aj);
        dbar2(s, t1, t2, ak);
        axpy(s, ajk, t2, out);
    }
}

/* out = A . in for the three components of Delta E */
void orc_apply_A(const orc_params *p, const double *in, double *out)
{
    shape_t s = shape_of(p);
    double co[ORC_NCOEF];
    orc_coefficients(p, co);
    const long n = s.ncell;
    const double *x = in, *y = in + n, *z = in + 2 * n;
    double *ox = out, *oy = out + n, *oz = out + 2 * n;
    double *t1 = alloc_cells(&s), *t2 = alloc_cells(&s);
    memset(out, 0, sizeof(double) * 3 * n);
    const double c6 = co[ORC_C6];
    /* A_xx, A_xy, A_xz */
    add_diag(&s, co[ORC_AY], co[ORC_AZ], co[ORC_AYZ], x, ox, 1, 2, t1, t2);
    add_cross(&s, co[ORC_BXY], c6, y, ox, 0, 1, 2, t1, t2);
    add_cross(&s, co[ORC_BZX], c6, z, ox, 0, 2, 1, t1, t2);
    /* A_yx, A_yy, A_yz */
    add_cross(&s, co[ORC_BXY], c6, x, oy, 1, 0, 2, t1, t2);
    add_diag(&s, co[ORC_AZ], co[ORC_AX], co[ORC_AZX], y, oy, 2, 0, t1, t2);
    add_cross(&s, co[ORC_BYZ], c6, z, oy, 1, 2, 0, t1, t2);
    /* A_zx, A_zy, A_zz */
    add_cross(&s, co[ORC_BZX], c6, x, oz, 2, 0, 1, t1, t2);
    add_cross(&s, co[ORC_BYZ], c6, y, oz, 2, 1, 0, t1, t2);
    add_diag(&s, co[ORC_AX], co[ORC_AY], co[ORC_AXY], z, oz, 0, 1, t1, t2);
    free(t1); free(t2);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1                                                                */
/* ------------------------------------------------------------------------- */

static double sumsq(long n, const double *a)
{
    double s = 0.0;
    for (long c = 0; c < n; ++c) s += a[c] * a[c];
    return s;
}

/* Solves (1 - A) dE = dEp by Algorithm 1: dE_(0) = dEp, dE_(s+1) = dEp
 * + A dE_(s).  Fixed mode applies A exactly m times.  Residual mode (the
 * alternative the paper weighs in Sec. 2.2.1) stops after the first sweep
 * whose update satisfies ||dE_(s+1) - dE_(s)||_2 <= tol ||dEp||_2 (L2 over
 * all three components); dEp = 0 needs no sweep; no convergence within m_max
 * sweeps returns ORC_ENOCONV.  *sweeps and *resid report what happened. */
/* Chebyshev acceleration of the solve (1 - A) x = dE' (the textbook
 * three-term recurrence of Chebyshev semi-iteration for a symmetric matrix
 * whose spectrum lies in [al, be]; here M = 1 - A, al = 1 - cheb_hi,
 * be = 1 - cheb_lo).  x_0 = dE' as in Algorithm 1; every sweep applies A once:
 *   r_k = dE' - x_k + A x_k,  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) r_k,
 *   x_{k+1} = x_k + d_k,  rho_0 = delta / theta, rho_k = 1 / (2 theta / delta - rho_{k-1}),
 * with theta = (be + al)/2, delta = (be - al)/2 and d_0 = r_0 / theta.  The
 * stop rule of residual mode is the same as for Algorithm 1: ||d_k|| <= tol
 * ||dE'||. */
static int solve_chebyshev(const orc_params *p, const double *dEp, double *x, int *sweeps, double *resid)
{
    shape_t s = shape_of(p);
    const long n3 = 3 * s.ncell;
    double *Ax = (double *)calloc((size_t)n3, sizeof(double));
    double *d = (double *)calloc((size_t)n3, sizeof(double));
    memcpy(x, dEp, sizeof(double) * n3);
    const double al = 1.0 - p->cheb_hi, be = 1.0 - p->cheb_lo;
    const double theta = 0.5 * (be + al), delta = 0.5 * (be - al);
    const double sig = theta / delta;
    double rho = 1.0 / sig;
    const double nrm = sqrt(sumsq(n3, dEp));
    const int cap = p->residual ? p->m_max : p->m;
    int rc = (p->residual && nrm > 0.0) ? ORC_ENOCONV : ORC_OK;
    int done = 0;
    double r = 0.0;
    for (int k = 0; k < cap && !(p->residual && nrm == 0.0); ++k) {
        orc_apply_A(p, x, Ax);
        double c1, c2;
        if (k == 0) {
            c1 = 0.0;
            c2 = 1.0 / theta;
        } else {
            const double rho_new = 1.0 / (2.0 * sig - rho);
            c1 = rho_new * rho;
            c2 = 2.0 * rho_new / delta;
            rho = rho_new;
        }
        double dd = 0.0;
        for (long c = 0; c < n3; ++c) {
            const double rk = dEp[c] - x[c] + Ax[c];
            d[c] = c1 * d[c] + c2 * rk;
            x[c] += d[c];
            dd += d[c] * d[c];
        }
        ++done;
        if (p->residual) {
            r = sqrt(dd) / nrm;
            if (r <= p->tol) { rc = ORC_OK; break; }
        }
    }
    free(Ax);
    free(d);
    if (sweeps) *sweeps = done;
    if (resid) *resid = r;
    return rc;
}

int orc_solve(const orc_params *p, const double *dEp, double *dE, int *sweeps, double *resid)
{
    if (p->cheb) return solve_chebyshev(p, dEp, dE, sweeps, resid);
    shape_t s = shape_of(p);
    const long n3 = 3 * s.ncell;
    double *Ad = (double *)calloc((size_t)n3, sizeof(double));
    memcpy(dE, dEp, sizeof(double) * n3);
    int rc = ORC_OK;
    int done = 0;
    double r = 0.0;
    if (!p->residual) {
        for (int it = 0; it < p->m; ++it) {
            orc_apply_A(p, dE, Ad);
            for (long c = 0; c < n3; ++c) dE[c] = dEp[c] + Ad[c];
            ++done;
        }
    } else {
        double nrm = sqrt(sumsq(n3, dEp));
        if (nrm > 0.0) {
            rc = ORC_ENOCONV;
            while (done < p->m_max) {
                orc_apply_A(p, dE, Ad);
                double dd = 0.0;
                for (long c = 0; c < n3; ++c) {
                    double v = dEp[c] + Ad[c];
                    dd += (v - dE[c]) * (v - dE[c]);
                    dE[c] = v;
                }
                ++done;
                r = sqrt(dd) / nrm;
                if (r <= p->tol) { rc = ORC_OK; break; }
            }
        }
    }
    free(Ad);
    if (sweeps) *sweeps = done;
    if (resid) *resid = r;
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Faraday update, Eqs. faraday_x..z                                          */
/* ------------------------------------------------------------------------- */

/* B <- B - c dt curl E.  E sits on integer positions along every axis it is
 * differentiated along, so each Dbar here is the forward form. */
void orc_faraday(const orc_params *p, const double *E, double *B)
{
    shape_t s = shape_of(p);
    double co[ORC_NCOEF];
    orc_coefficients(p, co);
    const long n = s.ncell;
    const double *Ex = E, *Ey = E + n, *Ez = E + 2 * n;
    double *Bx = B, *By = B + n, *Bz = B + 2 * n;
    double *d = alloc_cells(&s);
    /* (1/c) D_t Bx = -[D_y Ez - D_z Ey] */
    dbar(&s, Ez, d, 1, 1); axpy(&s, -co[ORC_KY], d, Bx);
    dbar(&s, Ey, d, 2, 1); axpy(&s, co[ORC_KZ], d, Bx);
    /* (1/c) D_t By = -[D_z Ex - D_x Ez] */
    dbar(&s, Ex, d, 2, 1); axpy(&s, -co[ORC_KZ], d, By);
    dbar(&s, Ez, d, 0, 1); axpy(&s, co[ORC_KX], d, By);
    /* (1/c) D_t Bz = -[D_x Ey - D_y Ex] */
    dbar(&s, Ey, d, 0, 1); axpy(&s, -co[ORC_KX], d, Bz);
    dbar(&s, Ex, d, 1, 1); axpy(&s, co[ORC_KY], d, Bz);
    free(d);
}

/* ------------------------------------------------------------------------- */
/* one full step                                                              */
/* ------------------------------------------------------------------------- */

/* Advances (E^n, B^{n+1/2}) by nsteps steps with the current J (static over
 * the steps; NULL for vacuum).  Order per step: filter the current (target
 * CURRENT), source dEp, Algorithm 1, E update, Faraday update, filter the
 * fields (target FIELDS).  Arrays are [3][ncell]. */
int orc_step(const orc_params *p, double *E, double *B, const double *J, int nsteps, orc_stats *st)
{
    shape_t s = shape_of(p);
    const long n3 = 3 * s.ncell;
    double *jf = NULL;
    if (J) {
        jf = (double *)malloc(sizeof(double) * n3);
        memcpy(jf, J, sizeof(double) * n3);
        if (p->filter_target == ORC_FILTER_CURRENT && p->filter_passes > 0)
            orc_filter(p, jf, 3, p->filter_passes);
    }
    double *dEp = (double *)malloc(sizeof(double) * n3);
    double *dE = (double *)malloc(sizeof(double) * n3);
    int rc = ORC_OK, total = 0, sw = 0;
    double r = 0.0;
    for (int step = 0; step < nsteps && rc == ORC_OK; ++step) {
        orc_source(p, B, jf, dEp);
        rc = orc_solve(p, dEp, dE, &sw, &r);
        total += sw;
        for (long c = 0; c < n3; ++c) E[c] += dE[c];
        orc_faraday(p, E, B);
        if (p->filter_target == ORC_FILTER_FIELDS && p->filter_passes > 0) {
            orc_filter(p, E, 3, p->filter_passes);
            orc_filter(p, B, 3, p->filter_passes);
        }
    }
    if (st) { st->last_sweeps = sw; st->total_sweeps = total; st->last_resid = r; }
    free(jf); free(dEp); free(dE);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* diagnostics                                                                */
/* ------------------------------------------------------------------------- */

/* out[c] = sum_a D_a B_a at the cell centre (i+1/2, j+1/2, k+1/2) of
 * Eq. gauss_B (forward differences). */
void orc_div_b(const orc_params *p, const double *B, double *out)
{
    shape_t s = shape_of(p);
    const long n = s.ncell;
    double *d = alloc_cells(&s);
    memset(out, 0, sizeof(double) * n);
    for (int a = 0; a < 3; ++a) {
        dbar(&s, B + a * n, d, a, 1);
        axpy(&s, 1.0 / p->d[a], d, out);
    }
    free(d);
}

/* out = D_x(alpha_yz Ex) + D_y(alpha_zx Ey) + D_z(alpha_xy Ez) at the nodes,
 * the left-hand side of Eq. gauss_E (backward differences). */
void orc_gauss_e(const orc_params *p, const double *E, double *out)
{
    shape_t s = shape_of(p);
    double co[ORC_NCOEF];
    orc_coefficients(p, co);
    const long n = s.ncell;
    double *a1 = alloc_cells(&s), *a2 = alloc_cells(&s), *t = alloc_cells(&s);
    memset(out, 0, sizeof(double) * n);
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3, c = (a + 2) % 3;
        alpha(&s, co[ORC_C6], E + a * n, a1, t, b);
        alpha(&s, co[ORC_C6], a1, a2, t, c);
        dbar(&s, a2, a1, a, 0);
        axpy(&s, 1.0 / p->d[a], a1, out);
    }
    free(a1); free(a2); free(t);
}

/* Energy of the converged scheme (derived; the paper does not define a
 * discrete energy): W = sum[E.M E + B^{n-1/2}.S B^{n+1/2}] dV/(8 pi), with
 * M = 1 - A, S = diag(alpha_x, alpha_y, alpha_z) and
 * B^{n-1/2} = B^{n+1/2} + c dt curl E^n.  Also the plain sum
 * (E^2 + B^2) dV/(8 pi). */
void orc_energy(const orc_params *p, const double *E, const double *B, double *w_scheme, double *w_plain)
{
    shape_t s = shape_of(p);
    const long n = s.ncell;
    const long n3 = 3 * n;
    double co[ORC_NCOEF];
    orc_coefficients(p, co);
    double *AE = (double *)malloc(sizeof(double) * n3);
    double *Bm = (double *)malloc(sizeof(double) * n3);
    double *SB = (double *)malloc(sizeof(double) * n3);
    double *t = alloc_cells(&s);
    orc_apply_A(p, E, AE);
    /* B^{n-1/2}: undo one Faraday update with E^n */
    {
        double *negE = (double *)malloc(sizeof(double) * n3);
        for (long c = 0; c < n3; ++c) negE[c] = -E[c];
        memcpy(Bm, B, sizeof(double) * n3);
        orc_faraday(p, negE, Bm);
        free(negE);
    }
    for (int a = 0; a < 3; ++a) alpha(&s, co[ORC_C6], B + a * n, SB + a * n, t, a);
    double dv = 1.0;
    for (int a = 0; a < p->dims; ++a) dv *= p->d[a];
    double ws = 0.0, wp = 0.0;
    for (long c = 0; c < n3; ++c) {
        ws += E[c] * (E[c] - AE[c]) + Bm[c] * SB[c];
        wp += E[c] * E[c] + B[c] * B[c];
    }
    *w_scheme = ws * dv / (8.0 * M_PI);
    *w_plain = wp * dv / (8.0 * M_PI);
    free(AE); free(Bm); free(SB); free(t);
}

/* ------------------------------------------------------------------------- */
/* adjoint of one step (fixed m, current filter or none)                      */
/* ------------------------------------------------------------------------- */

/* The step is linear in (E^n, B^{n+1/2}, j):
 *   dE' = C_b S B - q F j,  dE = P dE',  E1 = E + dE,  B1 = B - C_f E1,
 * with C_f the Faraday curl (forward differences), C_b the source curl
 * (backward differences), S = diag(alpha_x, alpha_y, alpha_z), F the
 * binomial filter and P = sum_{s=0}^{m} A^s (Algorithm 1).  A forward
 * difference transposes to minus the backward one on the periodic lattice,
 * so C_f^T = C_b; A (Eqs. matrixA_*), S and F are symmetric, hence P too.
 * Given Ebar, Bbar = dL/d(E1, B1) this returns, in place, dL/d(E, B) and in
 * jbar the gradient dL/dj:
 *   u = Ebar - C_b Bbar,  Ebar <- u,  w = P u,
 *   Bbar <- Bbar + S C_f w,  jbar = -q F w.
 * Residual mode has no fixed linear map and field filtering is not covered:
 * both return 1. */
int orc_adjoint_step(const orc_params *p, double *Ebar, double *Bbar, double *jbar)
{
    if (p->residual || (p->filter_target == ORC_FILTER_FIELDS && p->filter_passes > 0)) return 1;
    shape_t s = shape_of(p);
    const long n = s.ncell, n3 = 3 * n;
    double co[ORC_NCOEF];
    orc_coefficients(p, co);
    double *u = (double *)malloc(sizeof(double) * n3);
    double *w = (double *)malloc(sizeof(double) * n3);
    double *t = (double *)calloc((size_t)n3, sizeof(double));
    double *tmp = alloc_cells(&s);
    /* u = Ebar - C_b Bbar: the source curl with alpha -> 1 and no current */
    {
        /* C_b Bbar, component by component (the differences of orc_source) */
        const double *Bx = Bbar, *By = Bbar + n, *Bz = Bbar + 2 * n;
        double *d = alloc_cells(&s);
        memset(u, 0, sizeof(double) * n3);
        dbar(&s, Bz, d, 1, 0); axpy(&s, co[ORC_KY], d, u);
        dbar(&s, By, d, 2, 0); axpy(&s, -co[ORC_KZ], d, u);
        dbar(&s, Bx, d, 2, 0); axpy(&s, co[ORC_KZ], d, u + n);
        dbar(&s, Bz, d, 0, 0); axpy(&s, -co[ORC_KX], d, u + n);
        dbar(&s, By, d, 0, 0); axpy(&s, co[ORC_KX], d, u + 2 * n);
        dbar(&s, Bx, d, 1, 0); axpy(&s, -co[ORC_KY], d, u + 2 * n);
        free(d);
        for (long c = 0; c < n3; ++c) u[c] = Ebar[c] - u[c];
    }
    /* w = P u (Algorithm 1 with u as its right-hand side) */
    {
        int sw;
        double r;
        orc_solve(p, u, w, &sw, &r);
    }
    memcpy(Ebar, u, sizeof(double) * n3);
    /* Bbar += S C_f w: orc_faraday subtracts C_f w from a zero field */
    orc_faraday(p, w, t);
    for (int a = 0; a < 3; ++a) {
        double *ta = t + a * n;
        double *sa = (double *)malloc(sizeof(double) * n);
        alpha(&s, co[ORC_C6], ta, sa, tmp, a);
        for (long c = 0; c < n; ++c) Bbar[a * n + c] -= sa[c];
        free(sa);
    }
    /* jbar = -q F w */
    if (jbar) {
        memcpy(jbar, w, sizeof(double) * n3);
        if (p->filter_target == ORC_FILTER_CURRENT && p->filter_passes > 0) orc_filter(p, jbar, 3, p->filter_passes);
        for (long c = 0; c < n3; ++c) jbar[c] *= -co[ORC_Q];
    }
    free(u); free(w); free(t); free(tmp);
    return ORC_OK;
}
