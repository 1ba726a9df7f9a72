/*
 * fmx.h -- C ABI of the GB300 field advance for the averaged-Yee (unlumped
 * Eastwood finite-element) Maxwell scheme of Lu, Huang, Kilian, Guo, Li and
 * Liang, "An O(N) Maxwell solver with improved numerical dispersion
 * properties" (arXiv:1907.13088).
 *
 * One step advances the state (E^n, B^{n+1/2}) on a periodic staggered Yee
 * grid to (E^{n+1}, B^{n+3/2}):
 *   1. optional binomial low-pass filter of the current (Sec. 4.2, Sec. 5);
 *   2. auxiliary-field source dE' = c dt curl(alpha B) - 4 pi dt j
 *      (Eqs. ampere_aux_x..z);
 *   3. Algorithm 1: dE_(0) = dE', dE_(s+1) = dE' + A dE_(s), with A from
 *      Eqs. matrixA_1st..matrixA_last, either m sweeps or until a relative
 *      residual target (Sec. 2.2.1 weighs both);
 *   4. E^{n+1} = E^n + dE (Sec. 2.2.1);
 *   5. B^{n+3/2} = B^{n+1/2} - c dt curl E^{n+1} (Eqs. faraday_x..z);
 *   6. optional filter of the fields (Sec. 5, "post-process").
 * 2D and 1D grids follow Secs. 2.2.2 and 2.2.3 (D -> 0, alpha -> 1 along the
 * missing axes).  Units are Gaussian (4 pi / c), as in Eqs. ampere_x..z.
 *
 * Storage.  Every field component is its own device array, x fastest:
 * element (i, j, k) at offset (k * n[1] + j) * pitch + i, i < n[0], with
 * pitch >= n[0] and pitch * element size a multiple of 16 bytes, base
 * address 16-byte aligned.  Index (i, j, k) of each component sits at its
 * Yee position (Sec. 2 variable list):
 *   Ex (i+1/2, j, k)   Ey (i, j+1/2, k)   Ez (i, j, k+1/2)
 *   Bx (i, j+1/2, k+1/2)   By (i+1/2, j, k+1/2)   Bz (i+1/2, j+1/2, k)
 * and the current colocated with E.  Boundaries are periodic.
 *
 * Ownership.  The caller allocates every device buffer (fields, their
 * ping-pong partners, current, workspace) and keeps it alive until
 * fmx_destroy; the library borrows them and never allocates or frees device
 * memory.  Host memory passed to a call is only read or written during that
 * call (copies are completed before the call returns when `where` is
 * FMX_HOST).
 *
 * Errors.  Every entry point returns fmx_status (0 = FMX_OK) except
 * fmx_destroy, fmx_strerror, fmx_last_error and the pure queries.  No C++
 * exception crosses the ABI.  A failing call leaves a message in the
 * calling thread's fmx_last_error().  Asynchronous calls (fmx_step,
 * fmx_filter) only enqueue work on the grid's stream; a device-side
 * failure surfaces at the next synchronising call (fmx_get_fields,
 * fmx_diagnostics, fmx_sync).
 */
#ifndef FMX_H
#define FMX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FMX_OK = 0,
    FMX_EINVAL = 1,      /* an argument is out of range or inconsistent      */
    FMX_ECFL = 2,        /* dt above dt_CFL (Eq. dt_cfl_3d and its 2D form)   */
    FMX_ENOCONV = 3,     /* residual mode reached m_max sweeps unconverged    */
    FMX_ECUDA = 4,       /* a CUDA runtime call failed                        */
    FMX_ETIMEOUT = 5,    /* a bounded device-side wait gave up                */
    FMX_ESTATE = 6,      /* call out of order (e.g. stepping before fmx_bind) */
    FMX_EUNSUPPORTED = 7 /* combination the library does not provide         */
} fmx_status;

enum { FMX_F32 = 0, FMX_F64 = 1 };                        /* storage and sweep precision */
/* Solve of (1 - A) dE = dE' (Eq. transform-e-e_aux): Algorithm 1 with m sweeps or
 * to a residual, or Chebyshev semi-iteration (the paper's suggested faster
 * iteration, not its method: the textbook three-term recurrence on an
 * interval holding the eigenvalues of A, see fmx_cheb_interval), m sweeps
 * or to a residual.  Every mode applies A once per sweep; the residual is
 * ||x_(s+1) - x_(s)|| / ||dE'|| in all of them.  The Chebyshev modes run on
 * the staged engine. */
enum { FMX_ITER_FIXED = 0, FMX_ITER_RESIDUAL = 1, FMX_ITER_CHEB_FIXED = 2, FMX_ITER_CHEB_RESIDUAL = 3 };
enum { FMX_FILTER_NONE = 0, FMX_FILTER_CURRENT = 1, FMX_FILTER_FIELDS = 2 };
/* Engines: STAGED, one kernel per stage (every mode and dimension); FUSED, the
 * 2D fixed-m step in one or two kernels per step; RESIDENT, all the steps of
 * an fmx_step call, with Algorithm 1's sweeps (fixed m or to the residual) in
 * one launch of one or more thread-block clusters, for grids of at most
 * 262144 cells (no Chebyshev modes, no field filter); AUTO takes FUSED where
 * it applies, RESIDENT for residual mode on grids of at most 16384 FP64 or
 * 65536 FP32 cells, else STAGED. */
enum { FMX_ENGINE_AUTO = 0, FMX_ENGINE_STAGED = 1, FMX_ENGINE_FUSED = 2, FMX_ENGINE_RESIDENT = 3 };
enum { FMX_HOST = 0, FMX_DEVICE = 1 };                    /* where a copy source/target lives */

/* component bits (index order of the pointer arrays below) */
enum {
    FMX_EX = 1 << 0, FMX_EY = 1 << 1, FMX_EZ = 1 << 2,
    FMX_BX = 1 << 3, FMX_BY = 1 << 4, FMX_BZ = 1 << 5,
    FMX_JX = 1 << 6, FMX_JY = 1 << 7, FMX_JZ = 1 << 8,
    FMX_E = 7, FMX_B = 7 << 3, FMX_J = 7 << 6
};

/* warnings reported by fmx_create */
enum {
    FMX_WARN_ANORM = 1 /* 3D with dt > min(d)/(sqrt(2) c): the App. C bound
                          ||A||_inf < 1 no longer guaranteed (Sec. 2.2.1) */
};

/* Number of coefficients returned by fmx_coefficients. */
#define FMX_NCOEF 14

typedef struct {
    int dims;            /* active axes: 1 (x), 2 (x, y) or 3 (x, y, z)                  */
    int64_t n[3];        /* cells per axis, 1 .. 2^30; inactive axes must be 1; one field
                            array (pitch * n[1] * n[2] elements) at most 2^40 bytes   */
    double d[3];         /* cell sizes (dx, dy, dz) > 0                                 */
    double c;            /* speed of light > 0                                          */
    double dt;           /* time step; if <= 0, dt = courant * dt_CFL                   */
    double courant;      /* fraction of dt_CFL used when dt <= 0, in (0, 1]             */
    int precision;       /* FMX_F32 or FMX_F64                                          */
    int iter_mode;       /* FMX_ITER_*                                                   */
    int m;               /* sweeps in the fixed modes, >= 0                             */
    double tol;          /* residual modes: stop when ||dE_(s+1)-dE_(s)|| <= tol ||dE'|| */
    int m_max;           /* residual modes: sweep cap (FMX_ENOCONV beyond)              */
    int filter_passes;   /* binomial (1/4,1/2,1/4) passes per active axis, >= 0         */
    int filter_target;   /* FMX_FILTER_NONE / _CURRENT (each step, before the source) / _FIELDS (after the update) */
    int lumped;          /* 1: alpha -> 1, A = 0 (the Yee scheme, Sec. 2)               */
    int engine;          /* FMX_ENGINE_*: which kernels run the step                    */
    int64_t pitch;       /* row pitch in elements; 0 = n[0] rounded up to 16 bytes      */
    void *stream;        /* cudaStream_t the grid's work is enqueued on (NULL: legacy)  */
} fmx_params;

/* Device pointers the grid borrows (see Ownership).  E[s][c], B[s][c]:
 * state set s in {0, 1}, component c in {x, y, z}.  Set 0 holds the state
 * after fmx_set_fields; the fused engine alternates between the two sets,
 * the staged engine works in place in the current set.  J[c] may be NULL
 * (vacuum, j = 0).  work: fmx_workspace_bytes() bytes, 256-byte aligned. */
typedef struct {
    void *E[2][3];
    void *B[2][3];
    void *J[3];
    void *work;
    size_t work_bytes;
} fmx_buffers;

/* Diagnostics of the current state, accumulated in FP64 on the device. */
typedef struct {
    double w_scheme;    /* sum[E.(1-A)E + B^{n-1/2}.S B^{n+1/2}] dV/(8 pi): conserved by the converged vacuum step */
    double w_plain;     /* sum[E^2 + B^2] dV/(8 pi)                                       */
    double divb_max;    /* max |D.B| (Eq. gauss_B), cell centres                          */
    double divb_l2;     /* sqrt(sum (D.B)^2)                                              */
    double gauss_max;   /* max |D_x(alpha_yz Ex) + D_y(alpha_zx Ey) + D_z(alpha_xy Ez)| (Eq. gauss_E lhs) */
    double gauss_l2;    /* its L2 norm                                                    */
    double last_resid;  /* residual mode: relative residual of the last solve            */
    int last_sweeps;    /* sweeps of the last solve                                       */
    int64_t total_sweeps; /* sweeps since fmx_bind                                        */
    int64_t steps;      /* steps since fmx_bind                                           */
} fmx_diag;

typedef struct fmx_grid fmx_grid;

/* Validates p and creates a grid handle (host memory only; no device work).
 * Computes dt (from courant when p->dt <= 0) and the coefficients.
 * *warnings receives FMX_WARN_* bits (may be NULL).
 * Errors: FMX_EINVAL (bad sizes, dims, precision, modes, pitch),
 * FMX_ECFL (dt > dt_CFL, Eq. dt_cfl_3d), FMX_EUNSUPPORTED (engine FUSED
 * requested for a case the fused kernel does not cover; a grid that the
 * staged engine would run with n[1] > 524280 or n[2] > 65535, the launch
 * limits of its one-thread-per-cell kernels, which fmx_filter,
 * fmx_diagnostics and fmx_adjoint_step share: those calls return
 * FMX_EUNSUPPORTED for such a grid whatever its engine). */
fmx_status fmx_create(const fmx_params *p, fmx_grid **out, int *warnings);

/* Bytes of one field-component array: pitch * n[1] * n[2] * element size.
 * Returns 0 if p is invalid. */
size_t fmx_field_bytes(const fmx_params *p);

/* Bytes of workspace fmx_bind needs (intermediates of the staged engine,
 * FP64 reduction partials, the device status block).  0 if p is invalid. */
size_t fmx_workspace_bytes(const fmx_params *p);

/* Lends the grid its device buffers (see fmx_buffers).  Checks alignment
 * (16 bytes for fields, 256 for work) and work_bytes.  Resets the step and
 * sweep counters and selects state set 0.  Errors: FMX_EINVAL. */
fmx_status fmx_bind(fmx_grid *g, const fmx_buffers *b);

/* Copies the components in `mask` (FMX_E/FMX_B bits) from src[c] (c = 0..5:
 * Ex, Ey, Ez, Bx, By, Bz; entries outside mask ignored) into the current
 * state set.  Sources are dense (pitch = n[0]) arrays of the grid's
 * precision; `where` (FMX_HOST or FMX_DEVICE; any other value is
 * FMX_EINVAL) says whether they are host or device memory.  E is
 * read as E^n and B as B^{n+1/2}.  Host copies complete before return;
 * device copies are enqueued on the stream.  Errors: FMX_EINVAL,
 * FMX_ESTATE (not bound), FMX_ECUDA. */
fmx_status fmx_set_fields(fmx_grid *g, unsigned mask, const void *const *src, int where);

/* Copies the current j^{n+1/2} (three dense arrays, x, y, z) into the
 * bound J buffers, which are then used unchanged by every following step
 * until the next call.  Errors as fmx_set_fields; FMX_ESTATE if J buffers
 * were bound as NULL. */
fmx_status fmx_set_current(fmx_grid *g, const void *const *src, int where);

/* Time profile of the current, the callback-free form of a current with a
 * fixed spatial shape and a prescribed time dependence (the current enters
 * the step at t = (n + 1/2) dt, Sec. 2): for the next len steps that fmx_step
 * advances, step k of them (k = 0 .. len-1) uses j^{n+1/2} = table[k] * J,
 * J the bound current; after the table runs out, J as it is.  The factor
 * scales the current's coefficient 4 pi dt of that step (computed in FP64,
 * then rounded to the storage precision).  The table (host memory, len
 * doubles) is copied; len = 0 clears it.  It applies to the forward step
 * (also inside fmx_gauss_run), not to fmx_adjoint_step or the batch.
 * Errors: FMX_EINVAL (len < 0, table NULL with len > 0, a non-finite
 * entry), FMX_ESTATE (not bound, or J buffers bound as NULL). */
fmx_status fmx_set_current_profile(fmx_grid *g, const double *table, int len);

/* Enqueues nsteps full steps (1..6 above) on the stream.  Fixed mode never
 * synchronises.  Residual mode reads the device residual back once per chunk
 * of sweeps (synchronising; the first chunk of a step is as long as the
 * previous step's solve, sweeps past the stop do nothing) and returns
 * FMX_ENOCONV if a solve reaches m_max.  On an error the steps enqueued
 * before it stand and are counted (fmx_diagnostics' steps); the state is
 * that after the last of them, except after FMX_ENOCONV, where the failing
 * step's E update and Faraday update have been applied with the unconverged
 * solve.  Errors: FMX_ESTATE, FMX_EINVAL (nsteps < 0), FMX_ECUDA,
 * FMX_ENOCONV. */
fmx_status fmx_step(fmx_grid *g, int nsteps);

/* Applies `passes` binomial passes along every active axis to the
 * components in mask (FMX_E, FMX_B, FMX_J bits), in place on the current
 * state -- the "post-process the fields and currents" option of Sec. 5.
 * Enqueued on the stream.  Errors: FMX_ESTATE, FMX_EINVAL. */
fmx_status fmx_filter(fmx_grid *g, unsigned mask, int passes);

/* Copies the components in mask (FMX_E/FMX_B/FMX_J bits; dst indexed
 * 0..8 as Ex..Bz, Jx, Jy, Jz) out of the current state into dense arrays at
 * dst[c], host or device memory as `where` says (FMX_HOST or FMX_DEVICE).
 * Synchronises the stream.  Errors: FMX_EINVAL, FMX_ESTATE,
 * FMX_ECUDA, FMX_ETIMEOUT (a latched device status). */
fmx_status fmx_get_fields(fmx_grid *g, unsigned mask, void *const *dst, int where);

/* Computes the FP64 diagnostics of the current state.  Synchronises.
 * Errors: FMX_EINVAL (NULL), FMX_ESTATE, FMX_ECUDA. */
fmx_status fmx_diagnostics(fmx_grid *g, fmx_diag *out);

/* Waits for the grid's stream and returns any latched device status.
 * Errors: FMX_EINVAL (NULL), FMX_ECUDA (a failed or pending CUDA call), or
 * the status a kernel latched in the grid's status word. */
fmx_status fmx_sync(fmx_grid *g);

/* The FMX_NCOEF scalar factors the kernels multiply by, after rounding to
 * the grid's precision, as doubles, in this order: c dt/dx, c dt/dy,
 * c dt/dz, 4 pi dt, 1/6 (alpha = 1 + Dbar^2/6), (sigma_x - 1)/6,
 * (sigma_y - 1)/6, (sigma_z - 1)/6, (sigma_y + sigma_z - 1)/36,
 * (sigma_z + sigma_x - 1)/36, (sigma_x + sigma_y - 1)/36, -sigma_yz/6,
 * -sigma_zx/6, -sigma_xy/6; sigma_i = (c dt/d_i)^2, sigma_ij = (c dt/d_i)
 * (c dt/d_j), each evaluated in binary64 in the order written, then
 * rounded once (Eqs. matrixA_1st..matrixA_last).  Lumped grids report 0
 * for entries 4..13.  Host-only; returns FMX_EINVAL if n < FMX_NCOEF. */
fmx_status fmx_coefficients(const fmx_grid *g, double *out, int n);

/* dt in use (after courant * dt_CFL); 0 for a NULL handle. */
double fmx_time_step(const fmx_grid *g);

/* Chebyshev modes: the interval [lo, hi] taken to hold the eigenvalues of A --
 * the extreme eigenvalues of the real symmetric 3x3 symbol of A (Eqs.
 * matrixA_1st..last with Dbar_a -> 2 i s_a, s_a = sin(k_a d_a / 2)) over
 * s_a^2 = j/32, j = 0..32, on every active axis, widened by 0.01 (1 - hi) at
 * both ends.  Errors: FMX_EINVAL (NULL), FMX_ESTATE (not a Chebyshev mode). */
fmx_status fmx_cheb_interval(const fmx_grid *g, double *lo, double *hi);

/* Device pointer of component c (0..5: Ex..Bz of the current state set,
 * 6..8: Jx..Jz), or NULL. */
void *fmx_field_ptr(const fmx_grid *g, int c);

/* Number of device kernels this grid has launched since fmx_bind. */
int64_t fmx_launch_count(const fmx_grid *g);

/* ---- Adjoint (reverse-mode derivative) of the step ----
 * The step is linear in (E^n, B^{n+1/2}, j).  fmx_adjoint_step maps
 * dL/d(E^{n+1}, B^{n+3/2}) (Ebar, Bbar: device arrays in the grid's layout,
 * updated in place) to dL/d(E^n, B^{n+1/2}) and writes dL/dj^{n+1/2} to
 * jbar (may be NULL): u = Ebar - C_b Bbar, Ebar <- u, w = sum_{s<=m} A^s u,
 * Bbar <- Bbar + S C_f w, jbar = -4 pi dt F w, where C_f / C_b are the
 * Faraday / source curls (Eqs. faraday_x..z, ampere_aux_x..z), S the alpha
 * averages, F the current filter; it uses C_f^T = C_b and the symmetry of A
 * (Eqs. matrixA_*), S and F.  Fixed m only; no field filtering.  The work
 * array (fmx_adjoint_workspace_bytes, 256-byte aligned) is caller-owned.
 * Errors: FMX_EINVAL, FMX_ESTATE, FMX_EUNSUPPORTED, FMX_ECUDA. */
size_t fmx_adjoint_workspace_bytes(const fmx_params *p);
fmx_status fmx_adjoint_step(fmx_grid *g, void *const *Ebar, void *const *Bbar, void *const *jbar, void *work,
                            size_t work_bytes);

/* Gaussian-envelope current on a 2D grid (a prescribed source, not part of
 * the paper's scheme): writes j_z(i, j) = sum_p amp[p] exp(-|r_ij - c_p|^2 /
 * (2 width^2)) (periodic distances, r_ij the node (i, j)) and j_x = j_y = 0
 * into the bound current.  cxy: host array (x_p, y_p) pairs, amp: host array;
 * np <= 128.  fmx_gauss_project computes out[p] = sum_ij f(i, j) G_p(i, j)
 * for a device component array f in the grid's layout (FP64 sums; out is a
 * host array; synchronises) -- the projection a source-amplitude gradient
 * needs.  fmx_gauss_accumulate adds weights[p] * sum_ij f G_p to a device
 * accumulator (reset != 0 zeroes it first; asynchronous) and
 * fmx_gauss_accumulated copies the accumulator to out (synchronises).  The
 * host arrays are read before the call returns.  Errors: FMX_EINVAL,
 * FMX_ESTATE, FMX_EUNSUPPORTED (not 2D). */
fmx_status fmx_gauss_source(fmx_grid *g, int np, const double *cxy, const double *amp, double width);
fmx_status fmx_gauss_project(fmx_grid *g, int np, const double *cxy, double width, const void *f, double *out);
fmx_status fmx_gauss_accumulate(fmx_grid *g, int np, const double *cxy, double width, const void *f,
                                const double *weights, int reset);
fmx_status fmx_gauss_accumulated(fmx_grid *g, int np, double *out);

/* Gaussian-source run: the differentiable workload's forward and reverse
 * loops, enqueued on the grid's stream without host synchronisation.
 * fmx_gauss_setup stores np <= 128 sources: centres cxy ((x_p, y_p) pairs),
 * amplitudes theta, phases phi (host arrays, copied before the call returns),
 * the envelope width and the angular frequency omega0.
 * fmx_gauss_run enqueues, for n = n0 .. n0 + nsteps - 1, the current
 *   j_z = sum_p theta_p sin(omega0 (n + 1/2) dt + phi_p) G_p,  j_x = j_y = 0,
 * (G_p as for fmx_gauss_source) followed by one fmx_step.
 * fmx_gauss_adjoint_run enqueues, for n = n0 + nsteps - 1 down to n0, one
 * fmx_adjoint_step (Ebar, Bbar updated in place; jbar[2]: device array in the
 * grid's layout that receives dL/dj_z, jbar[0], jbar[1] untouched) followed by
 *   acc_p += sin(omega0 (n + 1/2) dt + phi_p) sum_ij jbar_z(i, j) G_p(i, j);
 * reset != 0 zeroes acc first.  With Ebar, Bbar starting as dL/d(E^N,
 * B^{N+1/2}) and n0 = 0, nsteps = N, fmx_gauss_accumulated then returns
 * dL/dtheta.  work: as for fmx_adjoint_step.  Errors: FMX_EINVAL, FMX_ESTATE
 * (not bound, no current buffers, no set-up), FMX_EUNSUPPORTED (not 2D; the
 * adjoint's own restrictions), FMX_ECUDA. */
fmx_status fmx_gauss_setup(fmx_grid *g, int np, const double *cxy, const double *theta, const double *phi,
                           double width, double omega0);
fmx_status fmx_gauss_run(fmx_grid *g, int64_t n0, int nsteps);
fmx_status fmx_gauss_adjoint_run(fmx_grid *g, int64_t n0, int nsteps, void *const *Ebar, void *const *Bbar,
                                 void *const *jbar, void *work, size_t work_bytes, int reset);

/* ---- Batched step (many independent 2D grids, one launch per step) ----
 * The grids of a batch are advanced together: every step is one persistent
 * kernel launch whose CTAs loop over (grid, strip, row-segment) tiles of all
 * grids, longest tiles first; the launches of fmx_batch_step are replayed
 * from CUDA graphs (two steps per graph) captured on first use.  Each grid
 * has its own sizes, cell sizes, dt / Courant number and buffers; all share
 * the precision (FP32), m, the current-filter passes, and the stream, which
 * must not be the legacy default stream (graph capture needs a stream of its
 * own).  Grids of the unlumped scheme use the polarisation-split column-pair
 * tiles of the 2D engine, one CTA per TE or TM half of a tile; lumped grids
 * use its single-column tile, in a second launch of the same step when the
 * batch has both kinds.  The same equations as fmx_step (Secs. 2.2.1-2.2.2). */
typedef struct fmx_batch fmx_batch;

/* Validates each of the n parameter sets (2D, FP32, fixed m, equal m,
 * filter passes and target across the batch, stream not NULL) and creates
 * the batch handle (host memory only).  Errors: FMX_EINVAL, FMX_ECFL,
 * FMX_EUNSUPPORTED (an (m, passes) pair without a batched kernel). */
fmx_status fmx_batch_create(const fmx_params *ps, int n, fmx_batch **out);

/* Device bytes the batch needs for its tile descriptors and work list (0
 * for a NULL handle). */
size_t fmx_batch_workspace_bytes(const fmx_batch *b);

/* Lends the batch the buffers of its n grids (bufs[i] as in fmx_bind, set 0
 * and set 1 required, J all NULL or all set in every grid) and a
 * 256-byte-aligned workspace; builds the work list with the automatic tile
 * rows.  The batch counts as bound only once the work list is on the device.
 * Errors: FMX_EINVAL, FMX_ECUDA. */
fmx_status fmx_batch_bind(fmx_batch *b, const fmx_buffers *bufs, void *work, size_t work_bytes);

/* Copy grid i's components in or out of its current state set (as
 * fmx_set_fields / fmx_get_fields; get synchronises).  mask: FMX_E and FMX_B
 * bits only; every component the mask names needs a pointer.  Errors:
 * FMX_EINVAL (bad index, mask, `where` or NULL pointer), FMX_ESTATE (not bound),
 * FMX_ECUDA. */
fmx_status fmx_batch_set_fields(fmx_batch *b, int i, unsigned mask, const void *const *src, int where);
fmx_status fmx_batch_get_fields(fmx_batch *b, int i, unsigned mask, void *const *dst, int where);

/* Rows per tile segment: rows > 0 caps every grid's segment at that many
 * rows; 0 selects the automatic choice.  Rebuilds the work list and drops
 * the captured graphs.  The tile's row extent changes only which rows are
 * recomputed as warm-up, never a result.  A failed rebuild (FMX_EINVAL when
 * the work list outgrows the workspace, FMX_ECUDA) unbinds the batch. */
fmx_status fmx_batch_set_rows(fmx_batch *b, int rows);

/* Tile widths of the column-pair kernels: a CTA of 128 threads runs either
 * one wide tile (256 columns) or two narrow tiles of 128 columns side by
 * side (half the CTA each), all in the same persistent launch.  Rule 0: wide
 * tiles only; 1 (default): narrow tiles for the grids where they compute
 * fewer columns than wide ones (grids narrower than about 114 columns, and
 * widths that leave a wide strip mostly empty); 2: narrow tiles for every
 * grid.  Rebuilds the work list like fmx_batch_set_rows (same errors); no
 * result depends on it. */
fmx_status fmx_batch_set_tiles(fmx_batch *b, int narrow_rule);

/* The current work list: wide and narrow tiles of the column-pair kernels,
 * tiles of the single-column kernel (lumped grids), the rows rule
 * (fmx_batch_set_rows) and the tile rule (fmx_batch_set_tiles); any pointer
 * may be NULL.  Errors: FMX_EINVAL (NULL batch), FMX_ESTATE (not bound). */
fmx_status fmx_batch_tiles(const fmx_batch *b, int *wide, int *narrow, int *single, int *rows, int *narrow_rule);

/* Columns one tile of grid i writes in the current work list (wide or
 * narrow column-pair tile, or the single-column tile), or -1 (NULL batch,
 * not bound, i out of range). */
int fmx_batch_grid_width(const fmx_batch *b, int i);

/* Autotuner: times every pair of tile rule (2, 1, then 0) and row extent
 * (automatic, 1024, 512, 384, 256, 192, 128, 96, 64, 32) over `trial_steps`
 * graph-replayed steps with CUDA events, keeps the fastest pair and returns its row extent
 * in *chosen (0 = automatic; chosen may be NULL; fmx_batch_tiles reports
 * both).  The choice is cached in the process by the batch's signature (m,
 * filter passes, current, every grid's size): a later batch of the same grids
 * takes it without trial steps.  The trial steps advance the grids' state:
 * set the fields afterwards.  Errors: FMX_EINVAL (trial_steps < 2),
 * FMX_ESTATE (not bound), FMX_ECUDA, and those of fmx_batch_set_rows. */
fmx_status fmx_batch_tune(fmx_batch *b, int trial_steps, int *chosen);

/* Enqueues nsteps steps of every grid (graph replays plus at most one
 * plain launch).  Asynchronous.  Errors: FMX_ESTATE, FMX_EINVAL, FMX_ECUDA. */
fmx_status fmx_batch_step(fmx_batch *b, int nsteps);

/* Work items (tiles; a column-pair tile counts once for its TE and TM halves)
 * of the current work list, and kernels launched. */
int fmx_batch_items(const fmx_batch *b);
int64_t fmx_batch_launch_count(const fmx_batch *b);

/* Releases the batch handle and its captured graphs (the borrowed buffers are
 * untouched). */
void fmx_batch_destroy(fmx_batch *b);

/* Per-kernel timing of the fused engine: while enabled, every kernel of
 * fmx_step is bracketed by CUDA events recorded on the grid's stream.
 * fmx_profile_read synchronises, returns one record per kernel kind (the
 * launches, their summed event time, and the algorithmic HBM bytes one
 * launch must move: 4 or 8 bytes per value read or written once) and clears
 * the records.  Not part of the paper; used to measure each kernel against
 * the HBM roofline.  Errors: FMX_ESTATE (not bound), FMX_ECUDA. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    double bytes_per_launch;
} fmx_kernel_stat;
fmx_status fmx_profile_enable(fmx_grid *g, int enable);
fmx_status fmx_profile_read(fmx_grid *g, fmx_kernel_stat *out, int max, int *n);

/* Measured fused multiply-add rate of the current device in the given
 * precision (FMX_F32 or FMX_F64), in flops per second (2 per FMA): a launch
 * of independent FMA chains over every SM, timed with CUDA events on
 * `stream` (cudaStream_t; NULL: legacy stream), best of three after a
 * warm-up; synchronising, nothing allocated.  The arithmetic-roofline
 * denominator reported beside the HBM one (the FP64 step on this class of
 * part is bound by FP64 arithmetic, not by HBM).  Not part of the paper.
 * Errors: FMX_EINVAL (bad precision, NULL output), FMX_ECUDA. */
fmx_status fmx_fma_peak(int precision, void *stream, double *flops_per_s);

/* ---------------------------------------------------------------------
 * NCI closed-form tools (Sec. 3, App. E).  For a cold beam drifting along x
 * at v -> c on a 2D grid (dx, dy) with dt = courant * dt_CFL,
 * dt_CFL = 1 / (c sqrt(1/dx^2 + 1/dy^2)) (2D form of Eq. dt_cfl_3d):
 *   - the resonance curves of Eqs. reson1 and reson2: for every alias
 *     nu = -nu_max..nu_max (Eq. aliasing_x) and every sample k_x, the k_y >= 0
 *     where the beam line omega = c (k_x + 2 pi nu / dx) meets the EM mode
 *     (the mirror -k_y is implied; the trivial meeting at omega = k = 0 is
 *     not a crossing).  The beam is taken without time aliasing
 *     and only where |omega dt| <= pi, the zone of the EM branch: the reading
 *     under which the curves show what Sec. 4.2 states (nu = 0 only for
 *     dt > dt_CFL / sqrt 2, no |nu| >= 2, |k_x| > 2.06 / dx);
 *   - the asymptotic growth rate Gamma of Eq. NCI-growth-rate at each crossing,
 *     with the momentum-conserving interpolation factors of Sec. 3 for a
 *     B-spline particle shape of order shape_order;
 *   - the fastest-growing mode over all crossings.
 * Computed in FP64 on the device. */
#define FMX_NCI_MAX_SHAPE_ORDER 16
#define FMX_NCI_MAX_ALIAS 64
#define FMX_NCI_MAX_KX (1 << 26)

typedef struct {
    double dx, dy;     /* cell sizes (> 0)                                       */
    double c;          /* light speed (> 0)                                      */
    double courant;    /* dt / dt_CFL, in (0, 1]                                 */
    double omega_p;    /* relativistic plasma frequency of the beam (>= 0)       */
    int shape_order;   /* B-spline order l of the particle shape, 0..16          */
    int nu_max;        /* aliases nu = -nu_max..nu_max, 0..64                    */
    int nkx;           /* k_x samples, 1..2^26                                   */
} fmx_nci_params;

/* fmx_nci_resonance -- the k_x samples are the cell centres of the first
 * zone, k_x,i = (2 i + 1 - nkx) pi / (nkx dx), i = 0..nkx-1.
 *   kx    : device double[nkx] receiving those samples, or NULL;
 *   ky    : device double[(2 nu_max + 1) * nkx], row r = nu + nu_max: the
 *           crossing k_y in [0, pi/dy], NaN where the curve of that nu does
 *           not cross that k_x;
 *   gamma : same layout, Gamma at the crossing, 0 where there is none;
 *   best  : device double[4] receiving (Gamma_max, k_x, k_y, nu) of the
 *           fastest-growing crossing (the lowest flat index among equal
 *           maxima), or (0, NaN, NaN, NaN) when nothing crosses; NULL skips
 *           the search.  Its first two words are also the search's working
 *           storage while the call's work runs.
 *   stream: cudaStream_t the work is enqueued on (NULL: legacy stream);
 *           asynchronous, nothing is allocated.
 * Caller-owned buffers, 8-byte aligned.  Errors: FMX_EINVAL (a parameter out
 * of range, ky or gamma NULL), FMX_ECUDA (a launch failed). */
fmx_status fmx_nci_resonance(const fmx_nci_params *p, double *kx, double *ky, double *gamma, double *best,
                             void *stream);

/* Size of the device scratch array behind fmx_step_static (4 MiB). */
#define FMX_STATIC_SCRATCH_BYTES (4u << 20)

/* fmx_step_static -- the paper has no counterpart to this call; it exists for
 * callers that cannot allocate device memory: a host program whose device
 * memory is owned by its own pool or a fixed budget set up front, where an
 * extra cudaMalloc (or a PyTorch allocation) for a workspace is not allowed
 * once the run has started.  It advances nsteps steps exactly like fmx_step
 * with the staged engine (any dims, precision, iteration mode and filter of
 * p; p->engine is ignored), in place on the caller's E[3] and B[3] (device
 * arrays in the layout above with p's pitch), reading J[3] (or J == NULL for
 * vacuum), and allocates nothing: its intermediates live in one file-scope
 * device array of FMX_STATIC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.
 *   Limit: exactly the grids for which fmx_workspace_bytes(p) with
 *   p->engine = FMX_ENGINE_STAGED is at most FMX_STATIC_SCRATCH_BYTES (13
 *   field arrays padded to the pitch and to 256 bytes, plus the reduction
 *   partials and status words: a little under 40 000 cells in FP64 or 80 000
 *   in FP32); larger grids return FMX_EINVAL with a message naming both sizes.
 *   The array lives on the current device, so the fields (and p->stream) must
 *   be on it too: E[0] on another device returns FMX_EINVAL.
 *   The first call on a device resolves the array's device address (with
 *   that device current); make that first call before any stream capture.
 *   Every call on a device shares the same array and it keeps the last call's
 *   contents; each call clears the part that must start at zero (the solver
 *   status) itself.  Calls whose work overlaps on the GPU (other streams,
 *   other host threads) race on the array: serialise them.
 *   Errors as fmx_step (FMX_EINVAL, FMX_ECFL, FMX_ENOCONV, FMX_ECUDA). */
fmx_status fmx_step_static(const fmx_params *p, void *const *E, void *const *B, const void *const *J, int nsteps);

/* Per-grid options of the kernels (not part of the paper):
 *   FMX_OPT_SWEEPS_PER_PASS: sweeps of Algorithm 1 per z-march pass of the
 *     3D FP32 kernels, 1 (one pass per sweep) or 2 (temporal blocking: pairs
 *     of sweeps in one pass, the intermediate sweep kept on chip on a tile
 *     grown by one cell; an odd last sweep takes a pass of its own).  Same
 *     results to FP32 rounding.  Default 1.
 *   FMX_OPT_WAIT_LIMIT_US: how long (microseconds of SM clock at the
 *     device's rated clock) a resident launch over several clusters waits at
 *     its grid barrier before it gives up: the launch then stops between two
 *     phases, the call returns FMX_ETIMEOUT and the fields hold a partly
 *     advanced state.  Default 1000000 (1 s).
 *   FMX_OPT_SELFTEST_LOST_ARRIVAL: 1 makes the resident launch's grid barrier
 *     expect one arrival more than ever comes, so that its first wait runs out
 *     (a test of the time-out path that faults nothing); 0 (default) is the
 *     normal barrier.
 *   FMX_OPT_RESIDENT_CLUSTERS (read only): clusters of the last resident
 *     launch (0 before the first).
 *   FMX_OPT_SEGMENT_ROWS: rows of the row segments that the CTAs of the FP32
 *     2D fused engine (the TE and TM kernels of the step and of the adjoint
 *     step) each march over, a grid of at most that many rows taking one
 *     segment; every segment recomputes a few warm-up rows of the row
 *     pipeline.  0 (default): as many segments as fill one wave of CTAs at
 *     the kernels' occupancy, but none shorter than 3m + 2p + 8 rows (p: the
 *     current's filter passes, 0 without a current).  Same results to the
 *     bit.
 * fmx_set_option returns FMX_EINVAL for an unknown or read-only option or a
 * bad value; fmx_get_option returns the value, or -1 (unknown option or NULL
 * grid). */
enum {
    FMX_OPT_SWEEPS_PER_PASS = 1,
    FMX_OPT_WAIT_LIMIT_US = 2,
    FMX_OPT_SELFTEST_LOST_ARRIVAL = 3,
    FMX_OPT_RESIDENT_CLUSTERS = 4,
    FMX_OPT_SEGMENT_ROWS = 5
};
fmx_status fmx_set_option(fmx_grid *g, int option, int value);
int fmx_get_option(const fmx_grid *g, int option);

/* Streams steps from and to host memory: for each record, the state
 * (E, B) and optionally the current are replaced by host arrays, the grid
 * advances one step, and E, B are copied back out -- the loop a caller runs
 * when every step's inputs come from the host and its result goes back
 * there (not part of the paper).
 *   in[0..5]: E x, y, z and B x, y, z of the step (host or device arrays of
 *             n_x * n_y * n_z values, x fastest, no padding); in[6..8]: J, or
 *             all three NULL to keep the bound current;
 *   out[0..5]: where E, B after the step go (NULL: not read back).
 * Page-locked host memory lets the copies run asynchronously.  On the fused
 * engine the upload of step i+1 and the read-back of step i run concurrently
 * on two copy streams of the grid (created on first use), each step reading
 * state set 0 and writing set 1; the other engines copy and step in order on
 * the grid's stream.  Synchronising: every output is in place on return.
 * Errors: FMX_EINVAL (NULL or partial arrays), FMX_ESTATE (not bound, or a
 * current given with no J bound), the errors of fmx_step, FMX_ECUDA. */
typedef struct {
    const void *in[9];
    void *out[6];
} fmx_host_step;
fmx_status fmx_step_host(fmx_grid *g, const fmx_host_step *io, int count);

/* Releases the handle (host memory only; borrowed buffers are untouched). */
void fmx_destroy(fmx_grid *g);

/* Static description of a status code. */
const char *fmx_strerror(fmx_status s);

/* Message of the last failing call on this thread ("" if none). */
const char *fmx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FMX_H */
