/*
 * fmx_oracle.h -- FP64 CPU oracle for the averaged-Yee Maxwell step
 * (arXiv:1907.13088).  TEST INFRASTRUCTURE ONLY: loaded by tests/, by
 * __graft_entry__.smoke() and by the CPU-baseline leg of bench.py, never by
 * the product path.  Shares no header with the CUDA library.
 */
#ifndef FMX_ORACLE_H
#define FMX_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ENOCONV = 3 };
enum { ORC_FILTER_NONE = 0, ORC_FILTER_CURRENT = 1, ORC_FILTER_FIELDS = 2 };

/* Scalar factors of the step (see orc_coefficients). */
enum {
    ORC_KX = 0, ORC_KY, ORC_KZ, /* c dt / d_i: curl factors */
    ORC_Q,                      /* 4 pi dt: current factor */
    ORC_C6,                     /* 1/6 of alpha = 1 + Dbar^2/6 (0 when lumped) */
    ORC_AX, ORC_AY, ORC_AZ,     /* (sigma_i - 1)/6 */
    ORC_AYZ, ORC_AZX, ORC_AXY,  /* (sigma_i + sigma_j - 1)/36 */
    ORC_BYZ, ORC_BZX, ORC_BXY,  /* -sigma_ij/6 */
    ORC_NCOEF
};

typedef struct {
    int dims;          /* active axes: 1 (x), 2 (x, y) or 3 (x, y, z) */
    long n[3];         /* cells per axis; inactive axes hold 1 */
    double d[3];       /* cell sizes */
    double c;          /* speed of light */
    double dt;         /* time step */
    int m;             /* sweeps of Algorithm 1 in fixed mode */
    int residual;      /* 1: residual-controlled stop */
    double tol;        /* relative residual target */
    int m_max;         /* sweep cap in residual mode */
    int filter_passes; /* binomial passes */
    int filter_target; /* ORC_FILTER_* */
    int lumped;        /* 1: alpha -> 1 (Yee) */
    int coef_f32;      /* 1: round every coefficient to binary32 */
    int cheb;          /* 1: Chebyshev acceleration of the solve (m sweeps, or to tol) */
    double cheb_lo;    /* interval [cheb_lo, cheb_hi] holding the eigenvalues of A */
    double cheb_hi;
} orc_params;

typedef struct {
    int last_sweeps;
    int total_sweeps;
    double last_resid;
} orc_stats;

int orc_threads(int n);
double orc_dt_cfl(const orc_params *p);
void orc_coefficients(const orc_params *p, double co[ORC_NCOEF]);
void orc_filter(const orc_params *p, double *f, int ncomp, int passes);
void orc_source(const orc_params *p, const double *B, const double *J, double *dEp);
void orc_apply_A(const orc_params *p, const double *in, double *out);
int orc_solve(const orc_params *p, const double *dEp, double *dE, int *sweeps, double *resid);
void orc_faraday(const orc_params *p, const double *E, double *B);
int orc_step(const orc_params *p, double *E, double *B, const double *J, int nsteps, orc_stats *st);
void orc_div_b(const orc_params *p, const double *B, double *out);
void orc_gauss_e(const orc_params *p, const double *E, double *out);
void orc_energy(const orc_params *p, const double *E, const double *B, double *w_scheme, double *w_plain);
int orc_adjoint_step(const orc_params *p, double *Ebar, double *Bbar, double *jbar);

#ifdef __cplusplus
}
#endif
#endif
