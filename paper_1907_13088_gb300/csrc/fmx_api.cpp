// Host side of the C ABI declared in include/fmx.h: parameter validation,
// the scheme's coefficients, buffer binding, copies, and the dispatch of a
// step to the staged or fused kernels.  No device memory is allocated here:
// every device buffer is borrowed from the caller.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fmx.h"
#include "fmx_internal.h"
#include "fused2d.h"

namespace {

thread_local char g_last_error[512] = "";

fmx_status fail(fmx_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return s;
}

fmx_status cuda_fail(cudaError_t e, const char *what) {
    return fail(FMX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t kAlign = 256;
constexpr size_t kSmallDoubles = 2048;  // workspace room for small per-call parameter arrays
// small-region layout (doubles): Gaussian-source centres, amplitudes or
// weights, projection output of single calls; centres, theta, phi of the
// run set up by fmx_gauss_setup; the gradient accumulator
constexpr size_t kGaussMax = 128;
constexpr size_t kSmCxy = 0, kSmAmp = 256, kSmOut = 384, kSmRunCxy = 512, kSmTheta = 768, kSmPhi = 896,
                 kSmAcc = 1024;
inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

double dt_cfl(const fmx_params *p) {
    double s = 0.0;
    for (int a = 0; a < p->dims; ++a) s += 1.0 / (p->d[a] * p->d[a]);
    return 1.0 / (p->c * sqrt(s));
}

size_t elem_size(int precision) { return precision == FMX_F64 ? 8 : 4; }

int64_t pitch_of(const fmx_params *p) {
    if (p->pitch > 0) return p->pitch;
    const int64_t q = (int64_t)(16 / elem_size(p->precision));
    return (p->n[0] + q - 1) / q * q;
}

// Cells per grid of the resident engine (one cluster of 8-16 SMs runs the
// whole step, so the grid must be small), and the sizes up to which the
// automatic choice prefers it for residual-controlled solves (beyond them
// the staged kernels on every SM win: FP64 arithmetic runs at 1/64 of the
// FP32 rate on this part, so the FP64 limit is lower).
constexpr int64_t kResidentMaxCells = (int64_t)1 << 18;
constexpr int64_t kResidentAutoCells64 = (int64_t)1 << 14;
constexpr int64_t kResidentAutoCells32 = (int64_t)1 << 16;

bool resident_supported(const fmx_params *p) {
    const int64_t cells = p->n[0] * p->n[1] * p->n[2];
    if (cells > kResidentMaxCells) return false;
    if (p->iter_mode != FMX_ITER_FIXED && p->iter_mode != FMX_ITER_RESIDUAL) return false;
    if (p->filter_target == FMX_FILTER_FIELDS && p->filter_passes > 0) return false;
    return true;
}

// The one-thread-per-cell kernels (staged engine, filter, diagnostics, staged
// adjoint) launch (32, 8) blocks on a (n_x/32, n_y/8, n_z) grid, whose y and
// z extents the hardware caps at 65535.
bool cellwise_launch_ok(const fmx_params *p) { return (p->n[1] + 7) / 8 <= 65535 && p->n[2] <= 65535; }
fmx_status cellwise_limit_fail(const char *what) {
    return fail(FMX_EUNSUPPORTED, "%s: one-thread-per-cell kernels need n[1] <= 524280 and n[2] <= 65535", what);
}

// Which engine runs a step of this problem.
int resolve_engine(const fmx_params *p) {
    const bool fusable = fmx::fused2d_supported(p);
    if (p->engine == FMX_ENGINE_FUSED) return fusable ? FMX_ENGINE_FUSED : -1;
    if (p->engine == FMX_ENGINE_STAGED) return FMX_ENGINE_STAGED;
    const bool resident = resident_supported(p);
    if (p->engine == FMX_ENGINE_RESIDENT) return resident ? FMX_ENGINE_RESIDENT : -1;
    if (fusable) return FMX_ENGINE_FUSED;
    const int64_t cells = p->n[0] * p->n[1] * p->n[2];
    const int64_t lim = p->precision == FMX_F64 ? kResidentAutoCells64 : kResidentAutoCells32;
    if (resident && p->iter_mode == FMX_ITER_RESIDUAL && cells <= lim) return FMX_ENGINE_RESIDENT;
    return FMX_ENGINE_STAGED;
}

// Eigenvalues of a real symmetric 3x3 matrix by cyclic Jacobi rotations:
// each rotation in the (p, q) plane by the angle phi with tan(2 phi) =
// 2 a_pq / (a_qq - a_pp) zeroes a_pq; the diagonal converges to the eigenvalues.
void eig_sym3(double a[3][3], double w[3]) {
    for (int sweep = 0; sweep < 64; ++sweep) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        const double dia = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off <= 1e-17 * dia || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double th = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                // a <- G^T a G, G the rotation (cs, sn) in the (p, q) plane
                double b[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) b[i][j] = a[i][j];
                for (int k = 0; k < 3; ++k) {
                    b[k][p] = cs * a[k][p] - sn * a[k][q];
                    b[k][q] = sn * a[k][p] + cs * a[k][q];
                }
                for (int k = 0; k < 3; ++k) {
                    a[p][k] = cs * b[p][k] - sn * b[q][k];
                    a[q][k] = sn * b[p][k] + cs * b[q][k];
                    if (k != p && k != q) a[k][p] = a[p][k], a[k][q] = a[q][k];
                }
                a[p][p] = cs * b[p][p] - sn * b[q][p];
                a[q][q] = sn * b[p][q] + cs * b[q][q];
                a[p][q] = a[q][p] = 0.0;
            }
    }
    for (int i = 0; i < 3; ++i) w[i] = a[i][i];
}

// The Chebyshev interval of fmx_cheb_interval from the step's coefficients
// (co: FMX_NCOEF values in the fmx_coefficients order).
void cheb_interval(int dims, const double *co, double *lo_out, double *hi_out) {
    const double ad[3] = {co[5], co[6], co[7]};
    const double apair[3] = {co[8], co[9], co[10]};  // coefficient of Dbar_bb Dbar_cc in A_aa
    const double bcross[3] = {co[11], co[12], co[13]};  // A_ab by the third axis
    const double c6 = co[4];
    double lo = 1e300, hi = -1e300;
    const int ns = 33;
    const int n1 = dims > 1 ? ns : 1, n2 = dims > 2 ? ns : 1;
    for (int i0 = 0; i0 < ns; ++i0)
        for (int i1 = 0; i1 < n1; ++i1)
            for (int i2 = 0; i2 < n2; ++i2) {
                const double s2[3] = {i0 / 32.0, dims > 1 ? i1 / 32.0 : 0.0, dims > 2 ? i2 / 32.0 : 0.0};
                double sv[3], dd[3];
                for (int a = 0; a < 3; ++a) {
                    sv[a] = sqrt(s2[a]);
                    dd[a] = -4.0 * s2[a];  // Dbar_aa -> -4 s_a^2
                }
                double A[3][3];
                for (int a = 0; a < 3; ++a) {
                    const int b = (a + 1) % 3, c = (a + 2) % 3;
                    A[a][a] = ad[b] * dd[b] + ad[c] * dd[c] + apair[a] * dd[b] * dd[c];
                    // A_ab = b_ab Dbar_a Dbar_b (1 + Dbar_cc / 6) -> -4 b_ab s_a s_b (1 + c6 dd_c)
                    A[a][b] = A[b][a] = -4.0 * bcross[c] * sv[a] * sv[b] * (1.0 + c6 * dd[c]);
                }
                double w[3];
                eig_sym3(A, w);
                for (int k = 0; k < 3; ++k) {
                    lo = w[k] < lo ? w[k] : lo;
                    hi = w[k] > hi ? w[k] : hi;
                }
            }
    *lo_out = lo - 0.01 * (1.0 - hi);
    *hi_out = hi + 0.01 * (1.0 - hi);
}

fmx_status validate(const fmx_params *p, double *dt_out, int *warn) {
    if (!p) return fail(FMX_EINVAL, "params is NULL");
    if (p->dims < 1 || p->dims > 3) return fail(FMX_EINVAL, "dims must be 1, 2 or 3 (got %d)", p->dims);
    for (int a = 0; a < 3; ++a) {
        if (p->n[a] < 1 || p->n[a] > (int64_t)1 << 30) return fail(FMX_EINVAL, "n[%d] out of range", a);
        if (a >= p->dims && p->n[a] != 1) return fail(FMX_EINVAL, "inactive axis %d must have n = 1", a);
        if (a < p->dims && !(p->d[a] > 0.0)) return fail(FMX_EINVAL, "d[%d] must be > 0", a);
    }
    if (!(p->c > 0.0)) return fail(FMX_EINVAL, "c must be > 0");
    if (p->precision != FMX_F32 && p->precision != FMX_F64) return fail(FMX_EINVAL, "bad precision");
    if (p->iter_mode < FMX_ITER_FIXED || p->iter_mode > FMX_ITER_CHEB_RESIDUAL) return fail(FMX_EINVAL, "bad iter_mode");
    const bool fixed = p->iter_mode == FMX_ITER_FIXED || p->iter_mode == FMX_ITER_CHEB_FIXED;
    if (fixed && (p->m < 0 || p->m > 1 << 20)) return fail(FMX_EINVAL, "m out of range");
    if (!fixed && (!(p->tol > 0.0) || p->m_max < 1))
        return fail(FMX_EINVAL, "residual mode needs tol > 0 and m_max >= 1");
    if (p->filter_passes < 0 || p->filter_passes > 1024) return fail(FMX_EINVAL, "filter_passes out of range");
    if (p->filter_target < FMX_FILTER_NONE || p->filter_target > FMX_FILTER_FIELDS)
        return fail(FMX_EINVAL, "bad filter_target");
    if (p->engine < FMX_ENGINE_AUTO || p->engine > FMX_ENGINE_RESIDENT) return fail(FMX_EINVAL, "bad engine");
    const int64_t q = (int64_t)(16 / elem_size(p->precision));
    if (p->pitch != 0 && (p->pitch < p->n[0] || p->pitch % q != 0))
        return fail(FMX_EINVAL, "pitch must be >= n[0] and a multiple of 16 bytes");
    // every size below (cells, bytes per array, workspaces) is a product of
    // the extents; bounding one array at 2^40 bytes keeps them all far from
    // int64 overflow (the extents alone allow 2^90 cells)
    const double array_bytes = (double)pitch_of(p) * (double)p->n[1] * (double)p->n[2] * (double)elem_size(p->precision);
    if (array_bytes > 1099511627776.0)
        return fail(FMX_EINVAL, "one field array would take %.3g bytes (limit 2^40)", array_bytes);
    const double cfl = dt_cfl(p);
    double dt = p->dt;
    if (!(dt > 0.0)) {
        if (!(p->courant > 0.0)) return fail(FMX_EINVAL, "need dt > 0 or courant > 0");
        dt = p->courant * cfl;
    }
    // Eq. dt_cfl_3d: real omega needs c dt <= (sum 1/d_i^2)^(-1/2)
    if (dt > cfl * (1.0 + 1e-12)) return fail(FMX_ECFL, "dt %.17g above dt_CFL %.17g", dt, cfl);
    int w = 0;
    if (p->dims == 3 && !p->lumped) {
        double dmin = p->d[0];
        for (int a = 1; a < 3; ++a) dmin = p->d[a] < dmin ? p->d[a] : dmin;
        if (p->c * dt > dmin / sqrt(2.0)) w |= FMX_WARN_ANORM;  // App. C bound, 3D
    }
    if (resolve_engine(p) < 0)
        return fail(FMX_EUNSUPPORTED, "the %s engine does not cover this problem",
                    p->engine == FMX_ENGINE_FUSED ? "fused" : "resident");
    if (resolve_engine(p) == FMX_ENGINE_STAGED && !cellwise_launch_ok(p)) return cellwise_limit_fail("staged engine");
    *dt_out = dt;
    if (warn) *warn = w;
    return FMX_OK;
}

// The scalar factors of the step, in the order and with the expressions
// documented at fmx_coefficients, evaluated in binary64 (this file is built
// without floating-point contraction) and rounded once to the precision.
void coefficients(const fmx_params *p, double dt, double co[FMX_NCOEF]) {
    const double cdt = p->c * dt;
    double k[3], s[3];
    for (int a = 0; a < 3; ++a) {
        k[a] = cdt / p->d[a];
        s[a] = k[a] * k[a];
    }
    co[0] = k[0];
    co[1] = k[1];
    co[2] = k[2];
    co[3] = (4.0 * M_PI) * dt;
    if (p->lumped) {
        for (int c = 4; c < FMX_NCOEF; ++c) co[c] = 0.0;
    } else {
        co[4] = 1.0 / 6.0;
        co[5] = (s[0] - 1.0) / 6.0;
        co[6] = (s[1] - 1.0) / 6.0;
        co[7] = (s[2] - 1.0) / 6.0;
        co[8] = (s[1] + s[2] - 1.0) / 36.0;
        co[9] = (s[2] + s[0] - 1.0) / 36.0;
        co[10] = (s[0] + s[1] - 1.0) / 36.0;
        co[11] = -(k[1] * k[2]) / 6.0;
        co[12] = -(k[2] * k[0]) / 6.0;
        co[13] = -(k[0] * k[1]) / 6.0;
    }
    if (p->precision == FMX_F32)
        for (int c = 0; c < FMX_NCOEF; ++c) co[c] = (double)(float)co[c];
}

template <typename T>
fmx::Coef<T> make_coef(const double co[FMX_NCOEF]) {
    fmx::Coef<T> c;
    c.kx = (T)co[0];
    c.ky = (T)co[1];
    c.kz = (T)co[2];
    c.q = (T)co[3];
    c.c6 = (T)co[4];
    c.ax = (T)co[5];
    c.ay = (T)co[6];
    c.az = (T)co[7];
    c.ayz = (T)co[8];
    c.azx = (T)co[9];
    c.axy = (T)co[10];
    c.byz = (T)co[11];
    c.bzx = (T)co[12];
    c.bxy = (T)co[13];
    return c;
}

}  // namespace

struct fmx_grid {
    fmx_params p;
    double dt = 0.0;
    double co[FMX_NCOEF];
    std::vector<double> jprof;  // time profile of the current (fmx_set_current_profile)
    size_t jprof_pos = 0;
    int engine = FMX_ENGINE_STAGED;
    fmx::Geo geo;
    size_t elem = 4;
    size_t field_bytes = 0;
    bool bound = false;
    fmx_buffers buf;
    int cur = 0;
    cudaStream_t stream = nullptr;
    // workspace carve
    void *jf[3] = {nullptr, nullptr, nullptr};
    void *tmp = nullptr;
    void *dEp[3] = {nullptr, nullptr, nullptr};
    void *dEa[3] = {nullptr, nullptr, nullptr};
    void *dEb[3] = {nullptr, nullptr, nullptr};
    double *partials = nullptr;
    int64_t nparts = 0;
    double *diag_out = nullptr;
    fmx::DevStatus *st = nullptr;
    double *small = nullptr;  // kSmallDoubles doubles of workspace
    // second stream for the TM chain of the fused 2D engine, with its fork
    // and join events (created on first use)
    cudaStream_t s_tm = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // fmx_step_host: copy-in and copy-out streams and their events (created on
    // first use)
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_in = nullptr, ev_comp = nullptr, ev_out = nullptr;
    // sweeps of Algorithm 1 per z-march pass of the 3D kernels (fmx_set_option)
    int sweeps_per_pass = 1;
    // rows per segment of the FP32 TE/TM kernels, forward and adjoint (0: automatic)
    int seg_rows = 0;
    // resident engine: limit of a wait at its grid barrier, the self-test of
    // that wait, and the clusters of the last launch
    long long wait_limit_us = 1000000;
    int lost_arrival = 0;
    int last_clusters = 0;
    // Chebyshev modes: the interval holding the eigenvalues of A, and the
    // recurrence's constants
    double cheb_lo = 0.0, cheb_hi = 0.0;
    fmx::ChebParams cheb{1.0, 1.0, 1.0};
    // Gaussian-source run (fmx_gauss_setup)
    int gauss_np = 0;
    double gauss_width = 0.0, gauss_omega0 = 0.0;
    // per-kernel timing (fmx_profile_enable): events of each profiled step
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;  // reused across reads
    size_t ev_used = 0;
    int prof_kinds = 0;                // events per step - 1
    // counters
    int64_t steps = 0, total_sweeps = 0, launches = 0;
    int last_sweeps = 0;
    double last_resid = 0.0;
};

namespace {

int staged_arrays(int engine) { return engine == FMX_ENGINE_FUSED ? 1 : 13; }

fmx::Geo geo_of(const fmx_params *p) {
    fmx::Geo g;
    g.nx = (int)p->n[0];
    g.ny = (int)p->n[1];
    g.nz = (int)p->n[2];
    g.pitch = pitch_of(p);
    g.plane = g.pitch * p->n[1];
    return g;
}

size_t workspace_of(const fmx_params *p, int engine) {
    const fmx::Geo g = geo_of(p);
    const size_t fb = align_up((size_t)g.plane * (size_t)g.nz * elem_size(p->precision), kAlign);
    const int64_t slots = fmx::staged_partial_slots(g);
    size_t w = (size_t)staged_arrays(engine) * fb;
    w += align_up((size_t)slots * 8 * sizeof(double), kAlign);
    w += align_up(8 * sizeof(double), kAlign);
    w += align_up(sizeof(fmx::DevStatus), kAlign);
    w += align_up(kSmallDoubles * sizeof(double), kAlign);
    return w;
}

fmx_status check_launch(fmx_grid *g, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what);
    (void)g;
    return FMX_OK;
}

template <typename T>
fmx::StagedPtrs<T> staged_ptrs(fmx_grid *g) {
    fmx::StagedPtrs<T> P;
    for (int c = 0; c < 3; ++c) {
        P.E[c] = (T *)g->buf.E[g->cur][c];
        P.B[c] = (T *)g->buf.B[g->cur][c];
        P.J[c] = (const T *)g->buf.J[c];
        P.jf[c] = (T *)g->jf[c];
        P.dEp[c] = (T *)g->dEp[c];
        P.dEa[c] = (T *)g->dEa[c];
        P.dEb[c] = (T *)g->dEb[c];
    }
    P.tmp = (T *)g->tmp;
    P.partials = g->partials;
    P.st = g->st;
    return P;
}

// `passes` binomial passes along every active axis of one component, in
// place on f, ping-ponging with the tmp scratch array.
template <typename T>
fmx_status filter_in_place(fmx_grid *g, T *f, int passes) {
    const int n = passes * g->p.dims;
    if (n == 0) return FMX_OK;
    T *tmp = (T *)g->tmp;
    const T *src = f;
    for (int q = 0; q < n; ++q) {
        T *dst = (q % 2 == 0) ? tmp : f;
        g->launches += fmx::launch_filter_pass<T>(g->geo, g->p.dims, src, dst, q % g->p.dims, g->stream);
        src = dst;
    }
    if (src != f) {
        cudaError_t e = cudaMemcpyAsync(f, src, g->field_bytes, cudaMemcpyDeviceToDevice, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (filter)");
    }
    return check_launch(g, "filter kernel launch");
}

// Filters the current into the jf workspace (out of place; J is unchanged)
// and returns in jsrc the arrays the source stage should read.
template <typename T>
fmx_status filtered_current(fmx_grid *g, const T *jsrc[3]) {
    const bool have_j = g->buf.J[0] != nullptr;
    for (int c = 0; c < 3; ++c) jsrc[c] = have_j ? (const T *)g->buf.J[c] : nullptr;
    if (!have_j || g->p.filter_target != FMX_FILTER_CURRENT || g->p.filter_passes == 0) return FMX_OK;
    const int n = g->p.filter_passes * g->p.dims;
    for (int c = 0; c < 3; ++c) {
        const T *src = (const T *)g->buf.J[c];
        T *jf = (T *)g->jf[c];
        T *tmp = (T *)g->tmp;
        for (int q = 0; q < n; ++q) {
            // choose the first target so that the last pass lands in jf
            T *dst = ((n - 1 - q) % 2 == 0) ? jf : tmp;
            g->launches += fmx::launch_filter_pass<T>(g->geo, g->p.dims, src, dst, q % g->p.dims, g->stream);
            src = dst;
        }
        jsrc[c] = jf;
    }
    return check_launch(g, "current filter launch");
}

// coefficients of the next step: the current's 4 pi dt times the next entry of
// the time profile while one is left (consumed here)
template <typename T>
fmx::Coef<T> step_coef(fmx_grid *g) {
    fmx::Coef<T> c = make_coef<T>(g->co);
    if (g->jprof_pos < g->jprof.size()) c.q = (T)(g->co[3] * g->jprof[g->jprof_pos++]);
    return c;
}

template <typename T>
fmx_status staged_step(fmx_grid *g) {
    const fmx::Coef<T> c = step_coef<T>(g);
    fmx::StagedPtrs<T> P = staged_ptrs<T>(g);
    const int mode = g->p.iter_mode;
    const bool cheb = mode == FMX_ITER_CHEB_FIXED || mode == FMX_ITER_CHEB_RESIDUAL;
    const bool resid = mode == FMX_ITER_RESIDUAL || mode == FMX_ITER_CHEB_RESIDUAL;
    const bool have_j = g->buf.J[0] != nullptr;
    const int jpasses = (have_j && g->p.filter_target == FMX_FILTER_CURRENT) ? g->p.filter_passes : 0;
    // 3D, Algorithm 1 with fixed m, at most one filter pass on the current: the
    // z-marching kernels (source with the filter fused, sweeps from a plane ring)
    // (their offsets within a plane are 32-bit: larger planes take the staged kernels)
    const bool march = mode == FMX_ITER_FIXED && fmx::march3d_supported(g->p.dims, jpasses) &&
                       (int64_t)g->geo.ny * g->geo.pitch < ((int64_t)1 << 31);
    const T *jsrc[3];
    fmx_status s = FMX_OK;
    if (march) {
        const T *jraw[3] = {have_j ? P.J[0] : nullptr, have_j ? P.J[1] : nullptr, have_j ? P.J[2] : nullptr};
        const T *b[3] = {P.B[0], P.B[1], P.B[2]};
        g->launches += fmx::launch_march3d_source<T>(g->geo, c, b, jraw, jpasses, P.dEp, g->stream);
    } else {
        s = filtered_current<T>(g, jsrc);
        if (s != FMX_OK) return s;
        // the solve's device-side status starts from ||dE'|| (residual and Chebyshev modes)
        g->launches += fmx::launch_staged_source<T>(g->geo, g->p.dims, c, P, jsrc, g->stream, resid || cheb);
    }
    if (mode == FMX_ITER_FIXED) {
        const T *in[3] = {P.dEp[0], P.dEp[1], P.dEp[2]};
        const T *dp[3] = {P.dEp[0], P.dEp[1], P.dEp[2]};
        bool updated = false;
        for (int it = 0; it < g->p.m; ++it) {
            // two sweeps per z-march pass (temporal blocking) where the grid asks
            // for it; the pass that ends the solve also applies the update
            if (march && g->sweeps_per_pass == 2 && it + 2 <= g->p.m) {
                const bool last = it + 2 == g->p.m;
                T *out[3];
                for (int q = 0; q < 3; ++q) out[q] = last ? P.E[q] : (in[0] == P.dEa[0] ? P.dEb[q] : P.dEa[q]);
                const int n = fmx::launch_march3d_sweeps2<T>(g->geo, c, dp, in, out, g->stream, last);
                if (n) {
                    g->launches += n;
                    ++it;  // two sweeps done
                    if (last) {
                        updated = true;
                        break;
                    }
                    for (int q = 0; q < 3; ++q) in[q] = out[q];
                    continue;
                }
            }
            // the z-marching FP32 sweep can apply E^{n+1} = E^n + dE in its last pass
            if (march && it == g->p.m - 1) {
                const int n = fmx::launch_march3d_sweep<T>(g->geo, c, dp, in, P.E, g->stream, true);
                g->launches += n;
                if (n) {
                    updated = true;
                    break;
                }
            }
            T *out[3];
            for (int q = 0; q < 3; ++q) out[q] = in[0] == P.dEa[0] ? P.dEb[q] : P.dEa[q];
            g->launches += march ? fmx::launch_march3d_sweep<T>(g->geo, c, dp, in, out, g->stream)
                                 : fmx::launch_staged_sweep<T>(g->geo, g->p.dims, c, P, in, out, false, g->stream);
            for (int q = 0; q < 3; ++q) in[q] = out[q];
        }
        if (!updated) g->launches += fmx::launch_update_e<T>(g->geo, P.E, in, g->stream);
        g->last_sweeps = g->p.m;
        g->total_sweeps += g->p.m;
    } else {
        // sweeps counted on the device (DevStatus): Algorithm 1 to a residual, or
        // Chebyshev acceleration for m sweeps or to a residual
        g->launches += fmx::launch_resid_init(g->partials, g->nparts, g->st, g->stream);
        fmx::DevStatus hs;
        const double tol2 = g->p.tol * g->p.tol;
        auto sweep = [&]() {
            if (cheb) {
                g->launches += fmx::launch_cheb_sweep<T>(g->geo, g->p.dims, c, P, g->cheb, g->stream);
                g->launches += fmx::launch_cheb_update(g->partials, g->nparts, g->st, g->cheb, resid, tol2,
                                                       g->p.m_max, g->stream);
            } else {
                g->launches += fmx::launch_resid_sweep<T>(g->geo, g->p.dims, c, P, g->stream);
                g->launches += fmx::launch_resid_update(g->partials, g->nparts, g->st, tol2, g->p.m_max, g->stream);
            }
        };
        if (!resid) {  // Chebyshev, fixed m
            for (int it = 0; it < g->p.m; ++it) sweep();
        }
        // residual mode: the first chunk as long as the previous step's solve (the
        // next one usually needs about as many sweeps), then chunks of 8; sweeps
        // past the stop are no-ops on the device
        int chunk = g->last_sweeps > 8 ? g->last_sweeps : 8;
        for (;;) {
            if (resid) {
                for (int q = 0; q < chunk; ++q) sweep();
                chunk = 8;
            }
            s = check_launch(g, "residual sweep launch");
            if (s != FMX_OK) return s;
            cudaError_t e = cudaMemcpyAsync(&hs, g->st, sizeof(hs), cudaMemcpyDeviceToHost, g->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
            if (e != cudaSuccess) return cuda_fail(e, "residual status read-back");
            if (hs.done || !resid) break;
        }
        g->launches += fmx::launch_update_e_resid<T>(g->geo, P, g->stream);
        g->last_sweeps = hs.count;
        g->total_sweeps += hs.count;
        g->last_resid = hs.nrm2 > 0.0 ? sqrt(hs.r2 / hs.nrm2) : 0.0;
        if (hs.noconv) {
            g->launches += fmx::launch_faraday<T>(g->geo, g->p.dims, c, P.E, P.B, g->stream);
            return fail(FMX_ENOCONV, "residual %.3g above tol after %d sweeps", g->last_resid, hs.count);
        }
    }
    {
        const T *e[3] = {P.E[0], P.E[1], P.E[2]};
        const int n = march ? fmx::launch_march3d_faraday<T>(g->geo, c, e, P.B, g->stream) : 0;
        g->launches += n ? n : fmx::launch_faraday<T>(g->geo, g->p.dims, c, P.E, P.B, g->stream);
    }
    s = check_launch(g, "staged step launch");
    if (s != FMX_OK) return s;
    if (g->p.filter_target == FMX_FILTER_FIELDS && g->p.filter_passes > 0) {
        for (int q = 0; q < 3; ++q) {
            if ((s = filter_in_place<T>(g, P.E[q], g->p.filter_passes)) != FMX_OK) return s;
            if ((s = filter_in_place<T>(g, P.B[q], g->p.filter_passes)) != FMX_OK) return s;
        }
    }
    return FMX_OK;
}

// Resident engine: nsteps steps in one launch (one cluster, or several in a
// cooperative launch).  The status word is cleared first (arrival count,
// generation, latched error).  Residual mode, and any launch over several
// clusters, reads the status back once (synchronising: it reports FMX_ENOCONV,
// FMX_ETIMEOUT and the sweep counts); fixed m on one cluster stays
// asynchronous.
template <typename T>
fmx_status resident_steps(fmx_grid *g, int nsteps) {
    if (nsteps == 0) return FMX_OK;
    const fmx::Coef<T> c = make_coef<T>(g->co);
    const fmx::StagedPtrs<T> P = staged_ptrs<T>(g);
    const bool resid = g->p.iter_mode == FMX_ITER_RESIDUAL;
    const bool have_j = g->buf.J[0] != nullptr;
    const int jpasses = (have_j && g->p.filter_target == FMX_FILTER_CURRENT) ? g->p.filter_passes : 0;
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) khz = 2000000;
    fmx::ResidentWait wait;
    wait.limit_cycles = (long long)g->wait_limit_us * (long long)khz / 1000;
    wait.lost_arrival = g->lost_arrival;
    cudaError_t e = cudaMemsetAsync(g->st, 0, sizeof(fmx::DevStatus), g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (status)");
    const int ncl = fmx::launch_resident<T>(g->geo, g->p.dims, c, P, nsteps, resid, g->p.m, g->p.tol * g->p.tol,
                                            g->p.m_max, jpasses, wait, g->stream);
    if (ncl < 0) return cuda_fail(cudaGetLastError(), "resident launch");
    g->launches += 1;
    fmx_status s = check_launch(g, "resident launch");
    if (s != FMX_OK) return s;
    g->last_clusters = ncl;
    if (!resid && ncl == 1 && !wait.lost_arrival) {
        g->last_sweeps = g->p.m;
        g->total_sweeps += (int64_t)g->p.m * nsteps;
        g->steps += nsteps;
        return FMX_OK;
    }
    fmx::DevStatus hs;
    e = cudaMemcpyAsync(&hs, g->st, sizeof(hs), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "resident status read-back");
    if (hs.err) {
        // a grid-barrier wait ran out: the launch stopped between two phases and
        // the fields hold a partly advanced state
        const fmx_status err = (fmx_status)hs.err;
        cudaMemsetAsync(&g->st->err, 0, sizeof(int), g->stream);
        return fail(err, "resident launch over %d cluster(s): a wait at the grid barrier ran out after %lld us", ncl,
                    g->wait_limit_us);
    }
    if (!resid) {
        g->last_sweeps = g->p.m;
        g->total_sweeps += (int64_t)g->p.m * nsteps;
        g->steps += nsteps;
        return FMX_OK;
    }
    g->last_sweeps = hs.count;
    g->total_sweeps += hs.sweeps_total;
    g->last_resid = hs.nrm2 > 0.0 ? sqrt(hs.r2 / hs.nrm2) : 0.0;
    if (hs.noconv) {
        // as the staged engine: the failing step is applied but not counted
        g->steps += hs.steps - 1;
        return fail(FMX_ENOCONV, "residual %.3g above tol after %d sweeps", g->last_resid, hs.count);
    }
    g->steps += nsteps;
    return FMX_OK;
}

// Next n events of the profiling pool (created on first use, then reused).
cudaEvent_t *profile_events(fmx_grid *g, size_t n) {
    while (g->ev_pool.size() < g->ev_used + n) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g->ev_pool.push_back(e);
    }
    cudaEvent_t *p = g->ev_pool.data() + g->ev_used;
    g->ev_used += n;
    return p;
}

// pre (optional): work that step k needs first, enqueued on the stream the
// TM set runs on (step 0: the grid's stream, before the fork, so both sets see it)
typedef fmx_status (*StepPre)(fmx_grid *g, int k, cudaStream_t s);

template <typename T>
fmx_status fused_step(fmx_grid *g, int nsteps, StepPre pre = nullptr) {
    const fmx::Coef<T> c0 = make_coef<T>(g->co);
    // TE/TM kernels: the TE and TM chains touch disjoint components, so the TM
    // launches go to a second stream, forked from and joined back into the
    // grid's stream (not when profiling: the events time one stream)
    bool two = false;
    if constexpr (sizeof(T) == 4)
        two = nsteps > 0 && !g->prof && fmx::fused2d_pol_supported(g->geo) && c0.c6 == 1.f / 6.f;
    if (pre && nsteps > 0) {
        fmx_status s = pre(g, 0, g->stream);
        if (s != FMX_OK) return s;
    }
    if (two) {
        cudaError_t e = cudaSuccess;
        if (!g->s_tm) e = cudaStreamCreateWithFlags(&g->s_tm, cudaStreamNonBlocking);
        if (e == cudaSuccess && !g->ev_fork) e = cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess && !g->ev_join) e = cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(g->ev_fork, g->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->s_tm, g->ev_fork, 0);
        if (e != cudaSuccess) return cuda_fail(e, "TM stream fork");
    }
    // after the fork every exit goes through the join below, so that work
    // enqueued later on the grid's stream waits for the TM launches already made
    fmx_status st = FMX_OK;
    for (int n = 0; n < nsteps; ++n) {
        if (pre && n > 0) {
            st = pre(g, n, two ? g->s_tm : g->stream);
            if (st != FMX_OK) break;
        }
        const fmx::Coef<T> c = step_coef<T>(g);
        const int nxt = 1 - g->cur;
        fmx::Fused2dArgs<T> a{};
        for (int q = 0; q < 3; ++q) {
            a.E[q] = (const T *)g->buf.E[g->cur][q];
            a.B[q] = (const T *)g->buf.B[g->cur][q];
            a.J[q] = (const T *)g->buf.J[q];
            a.Eo[q] = (T *)g->buf.E[nxt][q];
            a.Bo[q] = (T *)g->buf.B[nxt][q];
        }
        a.m = g->p.m;
        a.passes = (g->p.filter_target == FMX_FILTER_CURRENT && g->buf.J[0]) ? g->p.filter_passes : 0;
        cudaEvent_t *ev = g->prof ? profile_events(g, 3) : nullptr;
        int nl;
        if constexpr (sizeof(T) == 4) {
            // the TE/TM kernels take alpha's 1/6 as a compile-time constant (lumped mode zeroes it)
            if (fmx::fused2d_pol_supported(g->geo) && c.c6 == 1.f / 6.f) {
                nl = fmx::launch_fused2d_pol(g->geo, c, a, g->stream, ev, two ? g->s_tm : nullptr, g->seg_rows);
                g->prof_kinds = 2;
            } else {
                if (ev) cudaEventRecord(ev[0], g->stream);
                nl = fmx::launch_fused2d<T>(g->geo, c, a, g->stream);
                if (ev) cudaEventRecord(ev[1], g->stream), cudaEventRecord(ev[2], g->stream);
                g->prof_kinds = 1;
            }
        } else {
            if (ev) cudaEventRecord(ev[0], g->stream);
            nl = fmx::launch_fused2d<T>(g->geo, c, a, g->stream);
            if (ev) cudaEventRecord(ev[1], g->stream), cudaEventRecord(ev[2], g->stream);
            g->prof_kinds = 1;
        }
        if (nl < 0) {
            st = fail(FMX_EUNSUPPORTED, "fused 2D kernel: configuration not instantiated");
            break;
        }
        g->launches += nl;
        g->cur = nxt;
        g->steps += 1;
        g->last_sweeps = g->p.m;
        g->total_sweeps += g->p.m;
    }
    if (two) {
        cudaError_t e = cudaEventRecord(g->ev_join, g->s_tm);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->ev_join, 0);
        if (e != cudaSuccess && st == FMX_OK) st = cuda_fail(e, "TM stream join");
    }
    if (st != FMX_OK) return st;
    return check_launch(g, "fused step launch");
}

// One component between a dense host or device array (rows of n_x values)
// and the grid's pitched array: one 1D copy when the rows are contiguous on
// both sides, else a 2D copy; on `stream` (the grid's stream by default).
fmx_status copy_rows(fmx_grid *g, void *dst, size_t dpitch, const void *src, size_t spitch, bool sync,
                     cudaStream_t stream = nullptr) {
    const cudaStream_t st = stream ? stream : g->stream;
    const size_t width = (size_t)g->geo.nx * g->elem;
    const size_t rows = (size_t)g->geo.ny * (size_t)g->geo.nz;
    cudaError_t e;
    if (dpitch == width && spitch == width)
        e = cudaMemcpyAsync(dst, src, width * rows, cudaMemcpyDefault, st);
    else
        e = cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy of a component");
    if (sync) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return FMX_OK;
}

// Whether the fused FP32 2D adjoint kernels cover the grid (grids stepped by
// the fused engine; the staged engine's grids keep the staged adjoint), and
// the filter passes they apply to jbar.
bool adjoint_fused_ok(const fmx_grid *g, int *passes) {
    *passes = g->p.filter_target == FMX_FILTER_CURRENT ? g->p.filter_passes : 0;
    return g->p.precision == FMX_F32 && g->p.dims == 2 && g->engine == FMX_ENGINE_FUSED &&
           g->p.iter_mode == FMX_ITER_FIXED && !(g->p.filter_target == FMX_FILTER_FIELDS && g->p.filter_passes > 0) &&
           (float)g->co[4] == 1.f / 6.f && fmx::adjoint2d_supported(g->geo, g->p.m, *passes);
}

// One fused adjoint step from (Eb, Bb) into (Ebo, Bbo) (out of place), jbar
// components whose pointer is set.
fmx_status adjoint_fused(fmx_grid *g, float *const Eb[3], float *const Bb[3], float *const Ebo[3],
                         float *const Bbo[3], float *const jb[3], int passes) {
    fmx::Adj2dArgs<float> a{};
    for (int q = 0; q < 3; ++q) {
        a.Eb[q] = Eb[q];
        a.Bb[q] = Bb[q];
        a.Ebo[q] = Ebo[q];
        a.Bbo[q] = Bbo[q];
        a.Jbo[q] = jb[q];
    }
    a.m = g->p.m;
    a.passes = passes;
    const int n = fmx::launch_adjoint2d(g->geo, make_coef<float>(g->co), a, g->stream, g->seg_rows);
    if (n < 0) return fail(FMX_EUNSUPPORTED, "fused 2D adjoint: configuration not instantiated");
    g->launches += n;
    return check_launch(g, "fused adjoint launch");
}

// the workspace arrays the fused adjoint writes into (the staged layout's
// dEa and dEb: jf[3], tmp, dEp[3], dEa[3], dEb[3])
void adjoint_scratch(const fmx_grid *g, void *work, float *Ebo[3], float *Bbo[3]) {
    char *w = (char *)work;
    const size_t fb = align_up(g->field_bytes, kAlign);
    for (int c = 0; c < 3; ++c) {
        Ebo[c] = (float *)(w + (7 + c) * fb);
        Bbo[c] = (float *)(w + (10 + c) * fb);
    }
}

fmx_status copy_back(fmx_grid *g, float *const dst[6], float *const src[6]) {
    for (int q = 0; q < 6; ++q) {
        cudaError_t e = cudaMemcpyAsync(dst[q], src[q], g->field_bytes, cudaMemcpyDeviceToDevice, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (adjoint)");
    }
    return FMX_OK;
}

// jmask: components of jbar to write (bit c = component c)
template <typename T>
fmx_status adjoint_impl(fmx_grid *g, void *const *Eb_, void *const *Bb_, void *const *jb_, void *work,
                        size_t work_bytes, unsigned jmask = 7u) {
    if (g->p.iter_mode != FMX_ITER_FIXED) return fail(FMX_EUNSUPPORTED, "the adjoint covers fixed m only");
    if (!cellwise_launch_ok(&g->p)) return cellwise_limit_fail("adjoint step");
    if (g->p.filter_target == FMX_FILTER_FIELDS && g->p.filter_passes > 0)
        return fail(FMX_EUNSUPPORTED, "the adjoint does not cover field filtering");
    const size_t need = workspace_of(&g->p, FMX_ENGINE_STAGED);
    if (!work || work_bytes < need) return fail(FMX_EINVAL, "adjoint workspace of %zu bytes needed", need);
    if ((uintptr_t)work % kAlign) return fail(FMX_EINVAL, "adjoint workspace must be 256-byte aligned");
    T *Eb[3], *Bb[3], *jb[3];
    for (int c = 0; c < 3; ++c) {
        if (!Eb_[c] || !Bb_[c]) return fail(FMX_EINVAL, "NULL adjoint field");
        Eb[c] = (T *)Eb_[c];
        Bb[c] = (T *)Bb_[c];
        jb[c] = (jb_ && (jmask >> c & 1u)) ? (T *)jb_[c] : nullptr;
    }
    if constexpr (sizeof(T) == 4) {
        int passes;
        if (adjoint_fused_ok(g, &passes)) {
            float *Eo[3], *Bo[3];
            adjoint_scratch(g, work, Eo, Bo);
            fmx_status s = adjoint_fused(g, Eb, Bb, Eo, Bo, jb, passes);
            if (s != FMX_OK) return s;
            float *dst[6] = {Eb[0], Eb[1], Eb[2], Bb[0], Bb[1], Bb[2]};
            float *src[6] = {Eo[0], Eo[1], Eo[2], Bo[0], Bo[1], Bo[2]};
            return copy_back(g, dst, src);
        }
    }
    // staged layout: jf[3], tmp, dEp[3], dEa[3], dEb[3]
    char *w = (char *)work;
    const size_t fb = align_up(g->field_bytes, kAlign);
    w += 4 * fb;
    fmx::StagedPtrs<T> P;
    for (int c = 0; c < 3; ++c) {
        P.E[c] = nullptr;
        P.B[c] = nullptr;
        P.J[c] = nullptr;
        P.jf[c] = nullptr;
        P.dEp[c] = (T *)(w + c * fb);
        P.dEa[c] = (T *)(w + (3 + c) * fb);
        P.dEb[c] = (T *)(w + (6 + c) * fb);
    }
    P.tmp = nullptr;
    P.partials = nullptr;
    P.st = nullptr;
    const fmx::Coef<T> c = make_coef<T>(g->co);
    g->launches += fmx::launch_adj_source<T>(g->geo, g->p.dims, c, Eb, Bb, P.dEp, g->stream);
    const T *in[3] = {P.dEp[0], P.dEp[1], P.dEp[2]};
    for (int it = 0; it < g->p.m; ++it) {
        T *out[3];
        for (int q = 0; q < 3; ++q) out[q] = (it % 2 == 0) ? P.dEa[q] : P.dEb[q];
        g->launches += fmx::launch_staged_sweep<T>(g->geo, g->p.dims, c, P, in, out, false, g->stream);
        for (int q = 0; q < 3; ++q) in[q] = out[q];
    }
    T *wv[3] = {const_cast<T *>(in[0]), const_cast<T *>(in[1]), const_cast<T *>(in[2])};
    for (int q = 0; q < 3; ++q) {
        cudaError_t e = cudaMemcpyAsync(Eb[q], P.dEp[q], g->field_bytes, cudaMemcpyDeviceToDevice, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (adjoint)");
    }
    g->launches += fmx::launch_adj_faraday<T>(g->geo, g->p.dims, c, wv, Bb, g->stream);
    if (jb[0] || jb[1] || jb[2]) {
        g->launches += fmx::launch_scale_copy<T>(g->geo, -c.q, wv, jb, g->stream);
        if (g->p.filter_target == FMX_FILTER_CURRENT && g->p.filter_passes > 0)
            for (int q = 0; q < 3; ++q) {
                if (!jb[q]) continue;
                fmx_status s = filter_in_place<T>(g, jb[q], g->p.filter_passes);
                if (s != FMX_OK) return s;
            }
    }
    return check_launch(g, "adjoint launch");
}

// Chebyshev modes: the interval of A's eigenvalues and the recurrence's
// constants, from the coefficients already in g->co (the other modes leave
// them unused).
void set_cheb_constants(fmx_grid *g) {
    if (g->p.iter_mode != FMX_ITER_CHEB_FIXED && g->p.iter_mode != FMX_ITER_CHEB_RESIDUAL) return;
    cheb_interval(g->p.dims, g->co, &g->cheb_lo, &g->cheb_hi);
    const double al = 1.0 - g->cheb_hi, be = 1.0 - g->cheb_lo;
    g->cheb.theta = 0.5 * (be + al);
    g->cheb.delta = 0.5 * (be - al);
    g->cheb.sig = g->cheb.theta / g->cheb.delta;
}

}  // namespace

extern "C" {

fmx_status fmx_create(const fmx_params *p, fmx_grid **out, int *warnings) {
    if (!out) return fail(FMX_EINVAL, "out is NULL");
    *out = nullptr;
    double dt = 0.0;
    fmx_status s = validate(p, &dt, warnings);
    if (s != FMX_OK) return s;
    fmx_grid *g = new (std::nothrow) fmx_grid;
    if (!g) return fail(FMX_EINVAL, "out of host memory");
    g->p = *p;
    g->dt = dt;
    coefficients(p, dt, g->co);
    set_cheb_constants(g);
    g->engine = resolve_engine(p);
    g->geo = geo_of(p);
    g->elem = elem_size(p->precision);
    g->field_bytes = (size_t)g->geo.plane * (size_t)g->geo.nz * g->elem;
    g->stream = (cudaStream_t)p->stream;
    memset(&g->buf, 0, sizeof(g->buf));
    *out = g;
    return FMX_OK;
}

size_t fmx_field_bytes(const fmx_params *p) {
    double dt;
    if (validate(p, &dt, nullptr) != FMX_OK) return 0;
    const fmx::Geo g = geo_of(p);
    return (size_t)g.plane * (size_t)g.nz * elem_size(p->precision);
}

size_t fmx_workspace_bytes(const fmx_params *p) {
    double dt;
    if (validate(p, &dt, nullptr) != FMX_OK) return 0;
    return workspace_of(p, resolve_engine(p));
}

fmx_status fmx_bind(fmx_grid *g, const fmx_buffers *b) {
    if (!g || !b) return fail(FMX_EINVAL, "NULL argument");
    for (int s = 0; s < 2; ++s)
        for (int c = 0; c < 3; ++c) {
            const void *e = b->E[s][c], *bb = b->B[s][c];
            const bool need = s == 0 || g->engine == FMX_ENGINE_FUSED;
            if (need && (!e || !bb)) return fail(FMX_EINVAL, "state set %d component %d is NULL", s, c);
            if (((uintptr_t)e | (uintptr_t)bb) % 16) return fail(FMX_EINVAL, "field buffers must be 16-byte aligned");
        }
    const bool any_j = b->J[0] || b->J[1] || b->J[2];
    if (any_j && !(b->J[0] && b->J[1] && b->J[2])) return fail(FMX_EINVAL, "bind all three J buffers or none");
    for (int c = 0; c < 3; ++c)
        if ((uintptr_t)b->J[c] % 16) return fail(FMX_EINVAL, "J buffers must be 16-byte aligned");
    const size_t need = workspace_of(&g->p, g->engine);
    if (!b->work || b->work_bytes < need)
        return fail(FMX_EINVAL, "workspace of %zu bytes needed (got %zu)", need, b->work_bytes);
    if ((uintptr_t)b->work % kAlign) return fail(FMX_EINVAL, "workspace must be 256-byte aligned");
    g->buf = *b;
    char *w = (char *)b->work;
    const size_t fb = align_up(g->field_bytes, kAlign);
    if (g->engine != FMX_ENGINE_FUSED) {
        for (int c = 0; c < 3; ++c) { g->jf[c] = w; w += fb; }
        g->tmp = w; w += fb;
        for (int c = 0; c < 3; ++c) { g->dEp[c] = w; w += fb; }
        for (int c = 0; c < 3; ++c) { g->dEa[c] = w; w += fb; }
        for (int c = 0; c < 3; ++c) { g->dEb[c] = w; w += fb; }
    } else {
        g->tmp = w; w += fb;
    }
    const int64_t slots = fmx::staged_partial_slots(g->geo);
    g->partials = (double *)w;
    g->nparts = slots * 8;
    w += align_up((size_t)slots * 8 * sizeof(double), kAlign);
    g->diag_out = (double *)w;
    w += align_up(8 * sizeof(double), kAlign);
    g->st = (fmx::DevStatus *)w;
    w += align_up(sizeof(fmx::DevStatus), kAlign);
    g->small = (double *)w;
    // status partials count for the residual reductions is one per block
    g->nparts = slots;
    cudaError_t e = cudaMemsetAsync(g->st, 0, sizeof(fmx::DevStatus), g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync (status)");
    g->cur = 0;
    g->steps = g->total_sweeps = g->launches = 0;
    g->last_sweeps = 0;
    g->last_resid = 0.0;
    g->bound = true;
    return FMX_OK;
}

fmx_status fmx_set_fields(fmx_grid *g, unsigned mask, const void *const *src, int where) {
    if (!g || !src) return fail(FMX_EINVAL, "NULL argument");
    if (where != FMX_HOST && where != FMX_DEVICE) return fail(FMX_EINVAL, "where must be FMX_HOST or FMX_DEVICE");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (mask & ~(unsigned)(FMX_E | FMX_B)) return fail(FMX_EINVAL, "mask holds bits other than E and B");
    const size_t sp = (size_t)g->geo.nx * g->elem, dp = (size_t)g->geo.pitch * g->elem;
    for (int c = 0; c < 6; ++c) {
        if (!(mask & (1u << c))) continue;
        if (!src[c]) return fail(FMX_EINVAL, "src[%d] is NULL", c);
        void *dst = c < 3 ? g->buf.E[g->cur][c] : g->buf.B[g->cur][c - 3];
        fmx_status s = copy_rows(g, dst, dp, src[c], sp, false);
        if (s != FMX_OK) return s;
    }
    if (where == FMX_HOST) {
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return FMX_OK;
}

fmx_status fmx_set_current_profile(fmx_grid *g, const double *table, int len) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (!g->buf.J[0]) return fail(FMX_ESTATE, "no J buffers bound");
    if (len < 0 || (len > 0 && !table)) return fail(FMX_EINVAL, "bad table");
    for (int k = 0; k < len; ++k)
        if (!std::isfinite(table[k])) return fail(FMX_EINVAL, "table[%d] is not finite", k);
    g->jprof.assign(table, table + len);
    g->jprof_pos = 0;
    return FMX_OK;
}

fmx_status fmx_set_current(fmx_grid *g, const void *const *src, int where) {
    if (!g || !src) return fail(FMX_EINVAL, "NULL argument");
    if (where != FMX_HOST && where != FMX_DEVICE) return fail(FMX_EINVAL, "where must be FMX_HOST or FMX_DEVICE");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (!g->buf.J[0]) return fail(FMX_ESTATE, "no J buffers bound");
    const size_t sp = (size_t)g->geo.nx * g->elem, dp = (size_t)g->geo.pitch * g->elem;
    for (int c = 0; c < 3; ++c) {
        if (!src[c]) return fail(FMX_EINVAL, "src[%d] is NULL", c);
        fmx_status s = copy_rows(g, g->buf.J[c], dp, src[c], sp, false);
        if (s != FMX_OK) return s;
    }
    if (where == FMX_HOST) {
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return FMX_OK;
}

fmx_status fmx_step(fmx_grid *g, int nsteps) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (nsteps < 0) return fail(FMX_EINVAL, "nsteps < 0");
    if (g->engine == FMX_ENGINE_FUSED) {
        return g->p.precision == FMX_F64 ? fused_step<double>(g, nsteps) : fused_step<float>(g, nsteps);
    }
    // the resident launch applies one current factor to all its steps: a time
    // profile still being consumed takes the staged kernels
    if (g->engine == FMX_ENGINE_RESIDENT && g->jprof_pos >= g->jprof.size()) {
        return g->p.precision == FMX_F64 ? resident_steps<double>(g, nsteps) : resident_steps<float>(g, nsteps);
    }
    for (int n = 0; n < nsteps; ++n) {
        fmx_status s = g->p.precision == FMX_F64 ? staged_step<double>(g) : staged_step<float>(g);
        if (s != FMX_OK) return s;
        g->steps += 1;
    }
    return FMX_OK;
}

fmx_status fmx_filter(fmx_grid *g, unsigned mask, int passes) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (passes < 0) return fail(FMX_EINVAL, "passes < 0");
    if (mask & ~(unsigned)(FMX_E | FMX_B | FMX_J)) return fail(FMX_EINVAL, "bad mask");
    if ((mask & FMX_J) && !g->buf.J[0]) return fail(FMX_ESTATE, "no J buffers bound");
    if (mask && passes > 0 && !cellwise_launch_ok(&g->p)) return cellwise_limit_fail("fmx_filter");
    for (int c = 0; c < 9; ++c) {
        if (!(mask & (1u << c))) continue;
        void *f = c < 3 ? g->buf.E[g->cur][c] : (c < 6 ? g->buf.B[g->cur][c - 3] : g->buf.J[c - 6]);
        fmx_status s = g->p.precision == FMX_F64 ? filter_in_place<double>(g, (double *)f, passes)
                                                 : filter_in_place<float>(g, (float *)f, passes);
        if (s != FMX_OK) return s;
    }
    return FMX_OK;
}

fmx_status fmx_get_fields(fmx_grid *g, unsigned mask, void *const *dst, int where) {
    if (!g || !dst) return fail(FMX_EINVAL, "NULL argument");
    if (where != FMX_HOST && where != FMX_DEVICE) return fail(FMX_EINVAL, "where must be FMX_HOST or FMX_DEVICE");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (mask & ~(unsigned)(FMX_E | FMX_B | FMX_J)) return fail(FMX_EINVAL, "bad mask");
    if ((mask & FMX_J) && !g->buf.J[0]) return fail(FMX_ESTATE, "no J buffers bound");
    const size_t dp = (size_t)g->geo.nx * g->elem, sp = (size_t)g->geo.pitch * g->elem;
    for (int c = 0; c < 9; ++c) {
        if (!(mask & (1u << c))) continue;
        if (!dst[c]) return fail(FMX_EINVAL, "dst[%d] is NULL", c);
        const void *f = c < 3 ? g->buf.E[g->cur][c] : (c < 6 ? g->buf.B[g->cur][c - 3] : g->buf.J[c - 6]);
        fmx_status s = copy_rows(g, dst[c], dp, f, sp, false);
        if (s != FMX_OK) return s;
    }
    return fmx_sync(g);
}

fmx_status fmx_diagnostics(fmx_grid *g, fmx_diag *out) {
    if (!g || !out) return fail(FMX_EINVAL, "NULL argument");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (!cellwise_launch_ok(&g->p)) return cellwise_limit_fail("fmx_diagnostics");
    double co[FMX_NCOEF];
    memcpy(co, g->co, sizeof(co));
    const fmx::Coef<double> c = make_coef<double>(co);
    int nl;
    if (g->p.precision == FMX_F64) {
        double *E[3], *B[3];
        for (int q = 0; q < 3; ++q) { E[q] = (double *)g->buf.E[g->cur][q]; B[q] = (double *)g->buf.B[g->cur][q]; }
        nl = fmx::launch_diagnostics<double>(g->geo, g->p.dims, c, g->p.d, E, B, g->partials,
                                             fmx::staged_partial_slots(g->geo) * 8, g->diag_out, g->stream);
    } else {
        float *E[3], *B[3];
        for (int q = 0; q < 3; ++q) { E[q] = (float *)g->buf.E[g->cur][q]; B[q] = (float *)g->buf.B[g->cur][q]; }
        nl = fmx::launch_diagnostics<float>(g->geo, g->p.dims, c, g->p.d, E, B, g->partials,
                                            fmx::staged_partial_slots(g->geo) * 8, g->diag_out, g->stream);
    }
    if (nl < 0) return fail(FMX_EINVAL, "diagnostics partial buffer too small");
    g->launches += nl;
    fmx_status s = check_launch(g, "diagnostics launch");
    if (s != FMX_OK) return s;
    double h[6];
    cudaError_t e = cudaMemcpyAsync(h, g->diag_out, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics read-back");
    double dv = 1.0;
    for (int a = 0; a < g->p.dims; ++a) dv *= g->p.d[a];
    out->w_scheme = h[0] * dv / (8.0 * M_PI);
    out->w_plain = h[1] * dv / (8.0 * M_PI);
    out->divb_max = h[2];
    out->divb_l2 = sqrt(h[3]);
    out->gauss_max = h[4];
    out->gauss_l2 = sqrt(h[5]);
    out->last_resid = g->last_resid;
    out->last_sweeps = g->last_sweeps;
    out->total_sweeps = g->total_sweeps;
    out->steps = g->steps;
    return FMX_OK;
}

fmx_status fmx_sync(fmx_grid *g) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pending CUDA error");
    if (g->bound && g->st) {
        // on the grid's own stream: the legacy default stream may hold other work
        fmx::DevStatus hs;
        e = cudaMemcpyAsync(&hs, g->st, sizeof(hs), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "status read-back");
        if (hs.err) return fail((fmx_status)hs.err, "device reported status %d", hs.err);
    }
    return FMX_OK;
}

size_t fmx_adjoint_workspace_bytes(const fmx_params *p) {
    double dt;
    if (validate(p, &dt, nullptr) != FMX_OK) return 0;
    return workspace_of(p, FMX_ENGINE_STAGED);
}

fmx_status fmx_adjoint_step(fmx_grid *g, void *const *Ebar, void *const *Bbar, void *const *jbar, void *work,
                            size_t work_bytes) {
    if (!g || !Ebar || !Bbar) return fail(FMX_EINVAL, "NULL argument");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    return g->p.precision == FMX_F64 ? adjoint_impl<double>(g, Ebar, Bbar, jbar, work, work_bytes)
                                     : adjoint_impl<float>(g, Ebar, Bbar, jbar, work, work_bytes);
}

fmx_status fmx_gauss_source(fmx_grid *g, int np, const double *cxy, const double *amp, double width) {
    if (!g || !cxy || !amp || np < 1 || !(width > 0.0)) return fail(FMX_EINVAL, "bad arguments");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (!g->buf.J[0]) return fail(FMX_ESTATE, "no J buffers bound");
    if (g->p.dims != 2) return fail(FMX_EUNSUPPORTED, "the Gaussian source is 2D");
    if ((size_t)np > kGaussMax) return fail(FMX_EINVAL, "at most %zu sources", kGaussMax);
    cudaError_t e = cudaMemcpyAsync(g->small + kSmCxy, cxy, sizeof(double) * 2 * np, cudaMemcpyHostToDevice,
                                    g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->small + kSmAmp, amp, sizeof(double) * np, cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "source parameter upload");
    const fmx::GaussSrc gs{np, g->small + kSmCxy, g->small + kSmAmp, nullptr, nullptr, 0.0, 0.0, width};
    if (g->p.precision == FMX_F64) {
        double *J[3] = {(double *)g->buf.J[0], (double *)g->buf.J[1], (double *)g->buf.J[2]};
        g->launches += fmx::launch_gauss_source<double>(g->geo, gs, J, true, g->stream);
    } else {
        float *J[3] = {(float *)g->buf.J[0], (float *)g->buf.J[1], (float *)g->buf.J[2]};
        g->launches += fmx::launch_gauss_source<float>(g->geo, gs, J, true, g->stream);
    }
    return check_launch(g, "Gaussian source launch");
}

// Projection of a device array f on the envelopes: into `out` (device) or,
// with weights (device) or phases (device, weights sin(omega0 t + phi)), added
// to the accumulator.
static fmx_status gauss_project_dev(fmx_grid *g, const fmx::GaussSrc &gs, const void *f, const double *weights,
                                    double *out) {
    const int64_t cap = fmx::staged_partial_slots(g->geo) * 8;
    const int n = g->p.precision == FMX_F64
                      ? fmx::launch_gauss_project<double>(g->geo, gs, (const double *)f, g->partials, cap, weights,
                                                          out, g->stream)
                      : fmx::launch_gauss_project<float>(g->geo, gs, (const float *)f, g->partials, cap, weights, out,
                                                         g->stream);
    if (n < 0) return fail(FMX_EINVAL, "workspace too small for %d projections", gs.np);
    g->launches += n;
    return check_launch(g, "Gaussian projection launch");
}

static fmx_status gauss_project_impl(fmx_grid *g, int np, const double *cxy, double width, const void *f,
                                     const double *weights, double *out_host) {
    if (!g || !cxy || !f || np < 1 || !(width > 0.0)) return fail(FMX_EINVAL, "bad arguments");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (g->p.dims != 2) return fail(FMX_EUNSUPPORTED, "the Gaussian source is 2D");
    if ((size_t)np > kGaussMax) return fail(FMX_EINVAL, "at most %zu sources", kGaussMax);
    cudaError_t e = cudaMemcpyAsync(g->small + kSmCxy, cxy, sizeof(double) * 2 * np, cudaMemcpyHostToDevice,
                                    g->stream);
    if (e == cudaSuccess && weights)
        e = cudaMemcpyAsync(g->small + kSmAmp, weights, sizeof(double) * np, cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "projection parameter upload");
    const fmx::GaussSrc gs{np, g->small + kSmCxy, nullptr, nullptr, nullptr, 0.0, 0.0, width};
    double *dout = weights ? g->small + kSmAcc : g->small + kSmOut;
    fmx_status s = gauss_project_dev(g, gs, f, weights ? g->small + kSmAmp : nullptr, dout);
    if (s != FMX_OK || !out_host) return s;
    e = cudaMemcpyAsync(out_host, dout, sizeof(double) * np, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "projection read-back");
    return FMX_OK;
}

fmx_status fmx_gauss_project(fmx_grid *g, int np, const double *cxy, double width, const void *f, double *out) {
    if (!out) return fail(FMX_EINVAL, "NULL output");
    return gauss_project_impl(g, np, cxy, width, f, nullptr, out);
}

static fmx_status gauss_reset_acc(fmx_grid *g, int np) {
    cudaError_t e = cudaMemsetAsync(g->small + kSmAcc, 0, sizeof(double) * np, g->stream);
    return e == cudaSuccess ? FMX_OK : cuda_fail(e, "cudaMemsetAsync");
}

fmx_status fmx_gauss_accumulate(fmx_grid *g, int np, const double *cxy, double width, const void *f,
                                const double *weights, int reset) {
    if (!g || !weights) return fail(FMX_EINVAL, "NULL argument");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (np < 1 || (size_t)np > kGaussMax) return fail(FMX_EINVAL, "1 to %zu sources", kGaussMax);
    if (reset) {
        fmx_status s = gauss_reset_acc(g, np);
        if (s != FMX_OK) return s;
    }
    return gauss_project_impl(g, np, cxy, width, f, weights, nullptr);
}

fmx_status fmx_gauss_accumulated(fmx_grid *g, int np, double *out) {
    if (!g || !out || np < 1 || (size_t)np > kGaussMax) return fail(FMX_EINVAL, "bad arguments");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    cudaError_t e = cudaMemcpyAsync(out, g->small + kSmAcc, sizeof(double) * np, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "accumulator read-back");
    return FMX_OK;
}

fmx_status fmx_gauss_setup(fmx_grid *g, int np, const double *cxy, const double *theta, const double *phi,
                           double width, double omega0) {
    if (!g || !cxy || !theta || !phi || !(width > 0.0) || !isfinite(omega0)) return fail(FMX_EINVAL, "bad arguments");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (g->p.dims != 2) return fail(FMX_EUNSUPPORTED, "the Gaussian source is 2D");
    if (np < 1 || (size_t)np > kGaussMax) return fail(FMX_EINVAL, "1 to %zu sources", kGaussMax);
    cudaError_t e = cudaMemcpyAsync(g->small + kSmRunCxy, cxy, sizeof(double) * 2 * np, cudaMemcpyHostToDevice,
                                    g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->small + kSmTheta, theta, sizeof(double) * np, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->small + kSmPhi, phi, sizeof(double) * np, cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);  // host arrays are read before return
    if (e != cudaSuccess) return cuda_fail(e, "source set-up upload");
    g->gauss_np = np;
    g->gauss_width = width;
    g->gauss_omega0 = omega0;
    return FMX_OK;
}

static fmx::GaussSrc gauss_run_src(const fmx_grid *g, int64_t n) {
    return fmx::GaussSrc{g->gauss_np, g->small + kSmRunCxy, nullptr, g->small + kSmTheta, g->small + kSmPhi,
                         g->gauss_omega0, ((double)n + 0.5) * g->dt, g->gauss_width};
}

// the synthesis of step k of the running fmx_gauss_run (it writes j_z, read
// by the TM set only, so it runs on the TM stream; step 0 also zeroes j_x, j_y)
static thread_local int64_t t_gauss_n0 = 0;
static fmx_status gauss_pre(fmx_grid *g, int k, cudaStream_t s) {
    float *J[3] = {(float *)g->buf.J[0], (float *)g->buf.J[1], (float *)g->buf.J[2]};
    g->launches += fmx::launch_gauss_source<float>(g->geo, gauss_run_src(g, t_gauss_n0 + k), J, k == 0, s);
    return check_launch(g, "Gaussian source launch");
}

fmx_status fmx_gauss_run(fmx_grid *g, int64_t n0, int nsteps) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (!g->buf.J[0]) return fail(FMX_ESTATE, "no J buffers bound");
    if (g->gauss_np < 1) return fail(FMX_ESTATE, "fmx_gauss_setup not called");
    if (nsteps < 0) return fail(FMX_EINVAL, "nsteps < 0");
    if (g->engine == FMX_ENGINE_FUSED && g->p.precision == FMX_F32) {
        // one fused run: the TE chain and the synthesis + TM chain overlap across steps
        t_gauss_n0 = n0;
        return fused_step<float>(g, nsteps, gauss_pre);
    }
    for (int k = 0; k < nsteps; ++k) {
        const fmx::GaussSrc gs = gauss_run_src(g, n0 + k);
        if (g->p.precision == FMX_F64) {
            double *J[3] = {(double *)g->buf.J[0], (double *)g->buf.J[1], (double *)g->buf.J[2]};
            g->launches += fmx::launch_gauss_source<double>(g->geo, gs, J, k == 0, g->stream);
        } else {
            float *J[3] = {(float *)g->buf.J[0], (float *)g->buf.J[1], (float *)g->buf.J[2]};
            g->launches += fmx::launch_gauss_source<float>(g->geo, gs, J, k == 0, g->stream);
        }
        fmx_status s = check_launch(g, "Gaussian source launch");
        if (s == FMX_OK) s = fmx_step(g, 1);
        if (s != FMX_OK) return s;
    }
    return FMX_OK;
}

fmx_status fmx_gauss_adjoint_run(fmx_grid *g, int64_t n0, int nsteps, void *const *Ebar, void *const *Bbar,
                                 void *const *jbar, void *work, size_t work_bytes, int reset) {
    if (!g || !Ebar || !Bbar || !jbar || !jbar[2]) return fail(FMX_EINVAL, "NULL argument");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (g->gauss_np < 1) return fail(FMX_ESTATE, "fmx_gauss_setup not called");
    if (nsteps < 0) return fail(FMX_EINVAL, "nsteps < 0");
    if (reset) {
        fmx_status s = gauss_reset_acc(g, g->gauss_np);
        if (s != FMX_OK) return s;
    }
    int passes;
    if (adjoint_fused_ok(g, &passes)) {
        // fused adjoint, ping-pong between the caller's arrays and the
        // workspace; one copy back at the end when the result sits in the latter
        const size_t need = workspace_of(&g->p, FMX_ENGINE_STAGED);
        if (!work || work_bytes < need) return fail(FMX_EINVAL, "adjoint workspace of %zu bytes needed", need);
        if ((uintptr_t)work % kAlign) return fail(FMX_EINVAL, "adjoint workspace must be 256-byte aligned");
        float *set[2][6];
        for (int q = 0; q < 3; ++q) {
            if (!Ebar[q] || !Bbar[q]) return fail(FMX_EINVAL, "NULL adjoint field");
            set[0][q] = (float *)Ebar[q];
            set[0][3 + q] = (float *)Bbar[q];
        }
        adjoint_scratch(g, work, set[1], set[1] + 3);
        float *jz[3] = {nullptr, nullptr, (float *)jbar[2]};  // only dL/dj_z enters the source gradient
        int cur = 0;
        for (int k = nsteps - 1; k >= 0; --k) {
            fmx_status s = adjoint_fused(g, set[cur], set[cur] + 3, set[1 - cur], set[1 - cur] + 3, jz, passes);
            if (s == FMX_OK) s = gauss_project_dev(g, gauss_run_src(g, n0 + k), jbar[2], nullptr, g->small + kSmAcc);
            if (s != FMX_OK) return s;
            cur = 1 - cur;
        }
        return cur == 0 ? FMX_OK : copy_back(g, set[0], set[1]);
    }
    for (int k = nsteps - 1; k >= 0; --k) {
        // only dL/dj_z enters the source gradient
        fmx_status s = g->p.precision == FMX_F64 ? adjoint_impl<double>(g, Ebar, Bbar, jbar, work, work_bytes, 4u)
                                                 : adjoint_impl<float>(g, Ebar, Bbar, jbar, work, work_bytes, 4u);
        if (s == FMX_OK) s = gauss_project_dev(g, gauss_run_src(g, n0 + k), jbar[2], nullptr, g->small + kSmAcc);
        if (s != FMX_OK) return s;
    }
    return FMX_OK;
}

fmx_status fmx_coefficients(const fmx_grid *g, double *out, int n) {
    if (!g || !out) return fail(FMX_EINVAL, "NULL argument");
    if (n < FMX_NCOEF) return fail(FMX_EINVAL, "need room for %d coefficients", FMX_NCOEF);
    memcpy(out, g->co, sizeof(g->co));
    return FMX_OK;
}

double fmx_time_step(const fmx_grid *g) { return g ? g->dt : 0.0; }

fmx_status fmx_cheb_interval(const fmx_grid *g, double *lo, double *hi) {
    if (!g || !lo || !hi) return fail(FMX_EINVAL, "NULL argument");
    if (g->p.iter_mode != FMX_ITER_CHEB_FIXED && g->p.iter_mode != FMX_ITER_CHEB_RESIDUAL)
        return fail(FMX_ESTATE, "not a Chebyshev mode");
    *lo = g->cheb_lo;
    *hi = g->cheb_hi;
    return FMX_OK;
}

void *fmx_field_ptr(const fmx_grid *g, int c) {
    if (!g || !g->bound || c < 0 || c > 8) return nullptr;
    if (c < 3) return g->buf.E[g->cur][c];
    if (c < 6) return g->buf.B[g->cur][c - 3];
    return g->buf.J[c - 6];
}

int64_t fmx_launch_count(const fmx_grid *g) { return g ? g->launches : 0; }

fmx_status fmx_profile_enable(fmx_grid *g, int enable) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (g->engine != FMX_ENGINE_FUSED) return fail(FMX_EUNSUPPORTED, "per-kernel timing covers the fused engine");
    g->prof = enable != 0;
    return FMX_OK;
}

fmx_status fmx_profile_read(fmx_grid *g, fmx_kernel_stat *out, int max, int *n) {
    if (!g || !out || !n) return fail(FMX_EINVAL, "NULL argument");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    *n = 0;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const int kinds = g->prof_kinds;
    if (kinds == 0 || g->ev_used == 0) {
        g->ev_used = 0;
        return FMX_OK;
    }
    const double cells = (double)g->geo.nx * g->geo.ny * g->geo.nz;
    const bool hj = g->buf.J[0] != nullptr;
    const double esz = (double)g->elem;
    const char *names[2];
    double bytes[2];
    if (kinds == 2) {
        names[0] = "k_pol2d TE (Ex, Ey, Bz)";
        names[1] = "k_pol2d TM (Ez, Bx, By)";
        bytes[0] = cells * esz * ((hj ? 5 : 3) + 3);
        bytes[1] = cells * esz * ((hj ? 4 : 3) + 3);
    } else {
        names[0] = "k_fused2d";
        bytes[0] = cells * esz * ((hj ? 9 : 6) + 6);
    }
    double tot[2] = {0.0, 0.0};
    const size_t steps = g->ev_used / 3;
    for (size_t k = 0; k < steps; ++k) {
        cudaEvent_t *ev = g->ev_pool.data() + 3 * k;
        for (int q = 0; q < kinds; ++q) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[q], ev[q + 1]);
            if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
            tot[q] += ms;
        }
    }
    for (int q = 0; q < kinds && q < max; ++q) {
        memset(&out[q], 0, sizeof(out[q]));
        snprintf(out[q].name, sizeof(out[q].name), "%s", names[q]);
        out[q].launches = (int64_t)steps;
        out[q].total_ms = tot[q];
        out[q].bytes_per_launch = bytes[q];
        ++*n;
    }
    g->ev_used = 0;
    return FMX_OK;
}

fmx_status fmx_set_option(fmx_grid *g, int option, int value) {
    if (!g) return fail(FMX_EINVAL, "NULL grid");
    switch (option) {
        case FMX_OPT_SWEEPS_PER_PASS:
            if (value != 1 && value != 2) return fail(FMX_EINVAL, "sweeps per pass must be 1 or 2 (got %d)", value);
            g->sweeps_per_pass = value;
            return FMX_OK;
        case FMX_OPT_WAIT_LIMIT_US:
            if (value < 1) return fail(FMX_EINVAL, "wait limit must be >= 1 us (got %d)", value);
            g->wait_limit_us = value;
            return FMX_OK;
        case FMX_OPT_SELFTEST_LOST_ARRIVAL:
            if (value != 0 && value != 1) return fail(FMX_EINVAL, "lost-arrival self-test is 0 or 1 (got %d)", value);
            g->lost_arrival = value;
            return FMX_OK;
        case FMX_OPT_SEGMENT_ROWS:
            if (value < 0) return fail(FMX_EINVAL, "segment rows must be >= 0 (got %d)", value);
            g->seg_rows = value;
            return FMX_OK;
    }
    return fail(FMX_EINVAL, "unknown option %d", option);
}

int fmx_get_option(const fmx_grid *g, int option) {
    if (!g) return -1;
    switch (option) {
        case FMX_OPT_SWEEPS_PER_PASS: return g->sweeps_per_pass;
        case FMX_OPT_WAIT_LIMIT_US: return (int)g->wait_limit_us;
        case FMX_OPT_SELFTEST_LOST_ARRIVAL: return g->lost_arrival;
        case FMX_OPT_RESIDENT_CLUSTERS: return g->last_clusters;
        case FMX_OPT_SEGMENT_ROWS: return g->seg_rows;
    }
    return -1;
}

fmx_status fmx_step_host(fmx_grid *g, const fmx_host_step *io, int count) {
    if (!g || (!io && count > 0)) return fail(FMX_EINVAL, "NULL argument");
    if (!g->bound) return fail(FMX_ESTATE, "grid not bound");
    if (count < 0) return fail(FMX_EINVAL, "count < 0");
    for (int i = 0; i < count; ++i) {
        for (int c = 0; c < 6; ++c)
            if (!io[i].in[c]) return fail(FMX_EINVAL, "step %d: in[%d] is NULL", i, c);
        const bool any_j = io[i].in[6] || io[i].in[7] || io[i].in[8];
        if (any_j && !(io[i].in[6] && io[i].in[7] && io[i].in[8]))
            return fail(FMX_EINVAL, "step %d: give all three current components or none", i);
        if (any_j && !g->buf.J[0]) return fail(FMX_ESTATE, "step %d: a current is given but no J buffers are bound", i);
    }
    const size_t sp = (size_t)g->geo.nx * g->elem, dp = (size_t)g->geo.pitch * g->elem;
    auto dst_in = [&](int set, int c) -> void * {
        return c < 3 ? g->buf.E[set][c] : (c < 6 ? g->buf.B[set][c - 3] : g->buf.J[c - 6]);
    };
    auto step1 = [&]() {
        return g->p.precision == FMX_F64 ? (g->engine == FMX_ENGINE_FUSED ? fused_step<double>(g, 1)
                                                                          : fmx_step(g, 1))
                                         : (g->engine == FMX_ENGINE_FUSED ? fused_step<float>(g, 1) : fmx_step(g, 1));
    };
    if (g->engine != FMX_ENGINE_FUSED) {
        // in-place engines: upload, step and read back in order on the grid's stream
        for (int i = 0; i < count; ++i) {
            fmx_status s = FMX_OK;
            for (int c = 0; c < 9 && s == FMX_OK; ++c)
                if (io[i].in[c]) s = copy_rows(g, dst_in(g->cur, c), dp, io[i].in[c], sp, false);
            if (s == FMX_OK) s = step1();
            for (int c = 0; c < 6 && s == FMX_OK; ++c)
                if (io[i].out[c]) s = copy_rows(g, io[i].out[c], sp, dst_in(g->cur, c), dp, false);
            if (s != FMX_OK) return s;
        }
        cudaError_t e = cudaStreamSynchronize(g->stream);
        return e == cudaSuccess ? FMX_OK : cuda_fail(e, "cudaStreamSynchronize");
    }
    // fused engine: every step reads state set 0 and writes set 1, so the
    // upload of step i+1 (into set 0, on the copy-in stream, after step i has
    // read it) overlaps the read-back of step i (from set 1, on the copy-out
    // stream); step i+1 waits for both
    cudaError_t e = cudaSuccess;
    if (!g->s_in) e = cudaStreamCreateWithFlags(&g->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !g->s_out) e = cudaStreamCreateWithFlags(&g->s_out, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&g->ev_in, &g->ev_comp, &g->ev_out})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    // the copies start after whatever the grid's stream already holds
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_comp, g->stream);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_out, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "host-streaming set-up");
    for (int i = 0; i < count; ++i) {
        e = cudaStreamWaitEvent(g->s_in, g->ev_comp, 0);  // step i-1 has read set 0 and J
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        for (int c = 0; c < 9; ++c) {
            if (!io[i].in[c]) continue;
            fmx_status s = copy_rows(g, dst_in(0, c), dp, io[i].in[c], sp, false, g->s_in);
            if (s != FMX_OK) return s;
        }
        e = cudaEventRecord(g->ev_in, g->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->ev_in, 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->stream, g->ev_out, 0);  // step i-1's read-back of set 1
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        g->cur = 0;
        fmx_status s = step1();
        if (s != FMX_OK) return s;
        e = cudaEventRecord(g->ev_comp, g->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(g->s_out, g->ev_comp, 0);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
        for (int c = 0; c < 6; ++c) {
            if (!io[i].out[c]) continue;
            s = copy_rows(g, io[i].out[c], sp, dst_in(1, c), dp, false, g->s_out);
            if (s != FMX_OK) return s;
        }
        e = cudaEventRecord(g->ev_out, g->s_out);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    }
    // later work on the grid's stream follows the last read-back
    e = cudaStreamWaitEvent(g->stream, g->ev_out, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->s_out);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    return e == cudaSuccess ? FMX_OK : cuda_fail(e, "host-streaming synchronise");
}

void fmx_destroy(fmx_grid *g) {
    if (!g) return;
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : {g->ev_fork, g->ev_join, g->ev_in, g->ev_comp, g->ev_out})
        if (e) cudaEventDestroy(e);
    // their work was joined into the grid's stream or synchronised
    for (cudaStream_t s : {g->s_tm, g->s_in, g->s_out})
        if (s) cudaStreamDestroy(s);
    delete g;
}

const char *fmx_strerror(fmx_status s) {
    switch (s) {
        case FMX_OK: return "ok";
        case FMX_EINVAL: return "invalid argument";
        case FMX_ECFL: return "time step above the CFL limit";
        case FMX_ENOCONV: return "iteration did not converge within m_max sweeps";
        case FMX_ECUDA: return "CUDA runtime error";
        case FMX_ETIMEOUT: return "bounded device wait expired";
        case FMX_ESTATE: return "call out of order";
        case FMX_EUNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

const char *fmx_last_error(void) { return g_last_error; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Helpers for entry points that supply their own workspace (static_scratch.cu).
// ---------------------------------------------------------------------------
namespace fmx {

void set_last_error(const char *msg) { fail(FMX_EINVAL, "%s", msg); }

size_t staged_workspace_bytes(const fmx_params *p) {
    if (!p) return 0;
    fmx_params q = *p;
    q.engine = FMX_ENGINE_STAGED;
    double dt;
    if (validate(&q, &dt, nullptr) != FMX_OK) return 0;
    return workspace_of(&q, FMX_ENGINE_STAGED);
}

fmx_status staged_steps_on(const fmx_params *p, void *const E[3], void *const B[3], const void *const J[3],
                           void *work, size_t work_bytes, int nsteps) {
    if (!p || !E || !B) return fail(FMX_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(FMX_EINVAL, "nsteps < 0");
    fmx_params q = *p;
    q.engine = FMX_ENGINE_STAGED;
    double dt = 0.0;
    fmx_status s = validate(&q, &dt, nullptr);
    if (s != FMX_OK) return s;
    fmx_grid g;  // on the stack: this path performs no allocation of any kind
    g.p = q;
    g.dt = dt;
    coefficients(&q, dt, g.co);
    set_cheb_constants(&g);
    g.engine = FMX_ENGINE_STAGED;
    g.geo = geo_of(&q);
    g.elem = elem_size(q.precision);
    g.field_bytes = (size_t)g.geo.plane * (size_t)g.geo.nz * g.elem;
    g.stream = (cudaStream_t)q.stream;
    fmx_buffers b;
    memset(&b, 0, sizeof(b));
    for (int c = 0; c < 3; ++c) {
        b.E[0][c] = E[c];
        b.B[0][c] = B[c];
        b.J[c] = J ? const_cast<void *>(J[c]) : nullptr;
    }
    b.work = work;
    b.work_bytes = work_bytes;
    s = fmx_bind(&g, &b);
    if (s != FMX_OK) return s;
    for (int n = 0; n < nsteps; ++n) {
        s = q.precision == FMX_F64 ? staged_step<double>(&g) : staged_step<float>(&g);
        if (s != FMX_OK) return s;
    }
    return FMX_OK;
}

}  // namespace fmx

// ---------------------------------------------------------------------------
// Batched step
// ---------------------------------------------------------------------------

struct fmx_batch {
    int n = 0;
    std::vector<fmx_params> p;
    std::vector<fmx::BatchGrid> grids;  // host copy of the descriptors
    int m = 0, passes = 0;
    bool hj = false;
    cudaStream_t stream = nullptr;
    int threads = 0, halo = 0, width = 0, bps = 1, sms = 1;
    size_t smem = 0;
    // polarisation-split column-pair tiles (unlumped grids), when instantiated
    bool pol_ok = false;
    int pwidth = 0, pbps = 1;
    size_t psmem = 0;
    // narrow tiles (half a CTA each, two per CTA) and the rule that picks them
    int pwidth_n = 0;
    size_t pnbytes = 0;
    int narrow_policy = 1;
    int nwide = 0, nnarrow = 0;
    bool bound = false;
    fmx::BatchGrid *d_grids = nullptr;
    fmx::BatchItem *d_items = nullptr;  // pol items, then single-column items
    size_t max_items = 0;
    int nitems = 0, npol = 0;
    int rows_policy = 0;
    int parity = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int64_t launches = 0, steps = 0;
};

namespace {

void batch_drop_graphs(fmx_batch *b) {
    for (int q = 0; q < 2; ++q)
        if (b->graph[q]) {
            cudaGraphExecDestroy(b->graph[q]);
            b->graph[q] = nullptr;
        }
}

// Rows per segment of grid i under the current policy.  The automatic choice
// aims at about four tiles per resident CTA slot over the whole batch.
int batch_rows(const fmx_batch *b, int i) {
    const int ny = (int)b->p[i].n[1];
    if (b->rows_policy > 0) return b->rows_policy < ny ? b->rows_policy : ny;
    double work = 0.0;  // total (strips x rows) of the batch
    for (int k = 0; k < b->n; ++k) {
        const int ns = ((int)b->p[k].n[0] + b->width - 1) / b->width;
        work += (double)ns * b->p[k].n[1];
    }
    const double target = 4.0 * b->bps * b->sms;
    int L = (int)(work / target) + 1;
    if (L < 32) L = 32;
    return L < ny ? L : ny;
}

// grid i runs on the polarisation-split kernels: the unlumped scheme (the
// kernels take 1/6 as a compile-time constant), 32-bit offsets
bool batch_pol_grid(const fmx_batch *b, int i) {
    const fmx::BatchGrid &G = b->grids[i];
    return b->pol_ok && G.c.c6 == 1.f / 6.f && (int64_t)G.g.ny * G.g.pitch < ((int64_t)1 << 31);
}

// Whether a grid of the polarisation kernels takes narrow tiles: never
// (policy 0), where they compute fewer columns than wide ones (policy 1), or
// always (policy 2).
bool batch_narrow(const fmx_batch *b, int i) {
    if (b->narrow_policy == 0 || b->pwidth_n <= 0) return false;
    if (b->narrow_policy == 2) return true;
    const int nx = (int)b->p[i].n[0];
    const int64_t wide = (int64_t)((nx + b->pwidth - 1) / b->pwidth) * 2 * b->threads;
    const int64_t narrow = (int64_t)((nx + b->pwidth_n - 1) / b->pwidth_n) * b->threads;
    return narrow < wide;
}

fmx_status batch_build(fmx_batch *b) {
    std::vector<fmx::BatchItem> items[3];  // [0] wide pol, [1] narrow pol, [2] single column
    std::vector<double> cost[3];
    const int warm = 3 * b->m + 2 * b->passes + 8;
    for (int i = 0; i < b->n; ++i) {
        fmx::BatchGrid &G = b->grids[i];
        const int kind = batch_pol_grid(b, i) ? (batch_narrow(b, i) ? 1 : 0) : 2;
        G.L = batch_rows(b, i);
        G.W = kind == 0 ? b->pwidth : (kind == 1 ? b->pwidth_n : b->width);
        G.nstrip = (G.g.nx + G.W - 1) / G.W;
        const int nseg = (G.g.ny + G.L - 1) / G.L;
        for (int st = 0; st < G.nstrip; ++st)
            for (int sg = 0; sg < nseg; ++sg) {
                items[kind].push_back({i, st, sg});
                const int rows = (sg + 1) * G.L <= G.g.ny ? G.L : G.g.ny - sg * G.L;
                cost[kind].push_back((double)rows + warm);
            }
    }
    if (items[0].size() + items[1].size() + items[2].size() > b->max_items)
        return fail(FMX_EINVAL, "batch work list larger than its workspace");
    // each list longest tiles first (narrow tiles pair up with their neighbours
    // in this order, so the two halves of a CTA get similar row counts)
    std::vector<fmx::BatchItem> sorted;
    for (int kind = 0; kind < 3; ++kind) {
        std::vector<size_t> order(items[kind].size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = k;
        std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[kind][x] > cost[kind][y]; });
        for (size_t k = 0; k < order.size(); ++k) sorted.push_back(items[kind][order[k]]);
    }
    b->nwide = (int)items[0].size();
    b->nnarrow = (int)items[1].size();
    b->npol = b->nwide + b->nnarrow;
    b->nitems = (int)sorted.size();
    cudaError_t e = cudaMemcpyAsync(b->d_grids, b->grids.data(), sizeof(fmx::BatchGrid) * b->n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_items, sorted.data(), sizeof(fmx::BatchItem) * sorted.size(), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
    batch_drop_graphs(b);
    return FMX_OK;
}

// one launch per kind of tile present: the polarisation kernels (each item a
// TE and a TM half) and the single-column kernel
fmx_status batch_launch(fmx_batch *b, int parity) {
    const int nscal = b->nitems - b->npol;
    if (b->npol > 0) {
        const int slots = b->pbps * b->sms, want = 2 * (b->nwide + (b->nnarrow + 1) / 2);
        const int nl = fmx::launch_fused2d_pol_batch(b->m, b->passes, b->hj, b->d_grids, b->d_items, b->nwide,
                                                     b->nnarrow, parity, want < slots ? want : slots, b->psmem,
                                                     b->pnbytes, b->stream);
        if (nl < 0) return fail(FMX_EUNSUPPORTED, "batched kernel not instantiated");
        b->launches += nl;
    }
    if (nscal > 0) {
        const int slots = b->bps * b->sms;
        const int nl = fmx::launch_fused2d_batch(b->m, b->passes, b->hj, b->d_grids, b->d_items + b->npol, nscal,
                                                 parity, nscal < slots ? nscal : slots, b->smem, b->stream);
        if (nl < 0) return fail(FMX_EUNSUPPORTED, "batched kernel not instantiated");
        b->launches += nl;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batched kernel launch");
    return FMX_OK;
}

// graph of two steps starting from `parity` (captured once per parity)
fmx_status batch_graph(fmx_batch *b, int parity, cudaGraphExec_t *out) {
    if (b->graph[parity]) {
        *out = b->graph[parity];
        return FMX_OK;
    }
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    const int64_t l0 = b->launches;
    fmx_status s1 = batch_launch(b, parity);
    fmx_status s2 = s1 == FMX_OK ? batch_launch(b, 1 - parity) : s1;
    b->launches = l0;  // captured, not run
    e = cudaStreamEndCapture(b->stream, &gr);
    if (s2 != FMX_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s2;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph[parity], gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    *out = b->graph[parity];
    return FMX_OK;
}

}  // namespace

extern "C" {

fmx_status fmx_batch_create(const fmx_params *ps, int n, fmx_batch **out) {
    if (!ps || !out || n < 1) return fail(FMX_EINVAL, "bad arguments");
    *out = nullptr;
    for (int i = 0; i < n; ++i) {
        const fmx_params &q = ps[i];
        if (q.dims != 2 || q.precision != FMX_F32 || q.iter_mode != FMX_ITER_FIXED)
            return fail(FMX_EINVAL, "grid %d: the batch takes 2D FP32 grids with fixed m", i);
        if (q.filter_target == FMX_FILTER_FIELDS && q.filter_passes > 0)
            return fail(FMX_EINVAL, "grid %d: field filtering is not part of the batched step", i);
        if (q.m != ps[0].m || q.filter_passes != ps[0].filter_passes || q.filter_target != ps[0].filter_target ||
            q.stream != ps[0].stream)
            return fail(FMX_EINVAL, "grid %d: m, filter and stream must match across the batch", i);
    }
    if (!ps[0].stream) return fail(FMX_EINVAL, "the batch needs a stream other than the legacy default stream");
    fmx_batch *b = new (std::nothrow) fmx_batch;
    if (!b) return fail(FMX_EINVAL, "out of host memory");
    b->n = n;
    b->p.assign(ps, ps + n);
    b->grids.resize(n);
    b->m = ps[0].m;
    b->passes = ps[0].filter_target == FMX_FILTER_CURRENT ? ps[0].filter_passes : 0;
    b->stream = (cudaStream_t)ps[0].stream;
    for (int i = 0; i < n; ++i) {
        fmx_params q = ps[i];
        q.engine = FMX_ENGINE_STAGED;
        double dt = 0.0;
        fmx_status s = validate(&q, &dt, nullptr);
        if (s != FMX_OK) {
            delete b;
            return s;
        }
        double co[FMX_NCOEF];
        coefficients(&q, dt, co);
        memset(&b->grids[i], 0, sizeof(fmx::BatchGrid));
        b->grids[i].g = geo_of(&q);
        b->grids[i].c = make_coef<float>(co);
    }
    // geometry with and without a current (bind decides)
    if (fmx::fused2d_batch_geometry(b->m, 0, false, &b->threads, &b->halo, &b->width, &b->smem, &b->bps) != 0) {
        delete b;
        return fail(FMX_EUNSUPPORTED, "no batched kernel for m = %d", ps[0].m);
    }
    int pt = 0, ph = 0;
    b->pol_ok = fmx::fused2d_pol_batch_geometry(b->m, 0, false, &pt, &ph, &b->pwidth, &b->psmem, &b->pbps,
                                                &b->pwidth_n, &b->pnbytes) == 0;
    *out = b;
    return FMX_OK;
}

size_t fmx_batch_workspace_bytes(const fmx_batch *b) {
    if (!b) return 0;
    // work list bound: the smallest row extent the tuner tries (32 rows)
    size_t items = 0;
    int width = b->width > 0 ? b->width : 1;
    if (b->pol_ok && b->pwidth > 0 && b->pwidth < width) width = b->pwidth;
    if (b->pol_ok && b->pwidth_n > 0 && b->pwidth_n < width) width = b->pwidth_n;
    for (int i = 0; i < b->n; ++i) {
        const size_t ns = ((size_t)b->p[i].n[0] + width - 1) / width;
        items += ns * (((size_t)b->p[i].n[1] + 31) / 32 + 1);
    }
    return align_up(sizeof(fmx::BatchGrid) * b->n, kAlign) + align_up(sizeof(fmx::BatchItem) * items, kAlign);
}

fmx_status fmx_batch_bind(fmx_batch *b, const fmx_buffers *bufs, void *work, size_t work_bytes) {
    if (!b || !bufs || !work) return fail(FMX_EINVAL, "NULL argument");
    if ((uintptr_t)work % kAlign) return fail(FMX_EINVAL, "workspace must be 256-byte aligned");
    const size_t need = fmx_batch_workspace_bytes(b);
    if (work_bytes < need) return fail(FMX_EINVAL, "batch workspace of %zu bytes needed", need);
    const bool hj = bufs[0].J[0] != nullptr;
    for (int i = 0; i < b->n; ++i) {
        fmx::BatchGrid &G = b->grids[i];
        for (int s = 0; s < 2; ++s)
            for (int c = 0; c < 3; ++c) {
                if (!bufs[i].E[s][c] || !bufs[i].B[s][c]) return fail(FMX_EINVAL, "grid %d: NULL field buffer", i);
                if (((uintptr_t)bufs[i].E[s][c] | (uintptr_t)bufs[i].B[s][c]) % 16)
                    return fail(FMX_EINVAL, "grid %d: field buffers must be 16-byte aligned", i);
                G.E[s][c] = (const float *)bufs[i].E[s][c];
                G.B[s][c] = (const float *)bufs[i].B[s][c];
            }
        for (int c = 0; c < 3; ++c) {
            if ((bufs[i].J[c] != nullptr) != hj) return fail(FMX_EINVAL, "grid %d: J buffers all set or all NULL", i);
            G.J[c] = (const float *)bufs[i].J[c];
        }
    }
    b->hj = hj;
    if (fmx::fused2d_batch_geometry(b->m, b->hj ? b->passes : 0, b->hj, &b->threads, &b->halo, &b->width, &b->smem,
                                    &b->bps) != 0)
        return fail(FMX_EUNSUPPORTED, "no batched kernel for m = %d, passes = %d", b->m, b->passes);
    {
        int pt = 0, ph = 0;
        b->pol_ok = fmx::fused2d_pol_batch_geometry(b->m, b->hj ? b->passes : 0, b->hj, &pt, &ph, &b->pwidth,
                                                    &b->psmem, &b->pbps, &b->pwidth_n, &b->pnbytes) == 0;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b->sms = 1;
    char *w = (char *)work;
    b->d_grids = (fmx::BatchGrid *)w;
    w += align_up(sizeof(fmx::BatchGrid) * b->n, kAlign);
    b->d_items = (fmx::BatchItem *)w;
    b->max_items = (work_bytes - align_up(sizeof(fmx::BatchGrid) * b->n, kAlign)) / sizeof(fmx::BatchItem);
    b->parity = 0;
    b->launches = b->steps = 0;
    // bound only once the work list is on the device
    const fmx_status s = batch_build(b);
    b->bound = s == FMX_OK;
    return s;
}

fmx_status fmx_batch_set_fields(fmx_batch *b, int i, unsigned mask, const void *const *src, int where) {
    if (!b || !src || i < 0 || i >= b->n) return fail(FMX_EINVAL, "bad arguments");
    if (where != FMX_HOST && where != FMX_DEVICE) return fail(FMX_EINVAL, "where must be FMX_HOST or FMX_DEVICE");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    if (mask & ~(unsigned)(FMX_E | FMX_B)) return fail(FMX_EINVAL, "mask holds bits other than E and B");
    const fmx::BatchGrid &G = b->grids[i];
    const size_t sp = (size_t)G.g.nx * 4, dp = (size_t)G.g.pitch * 4;
    for (int c = 0; c < 6; ++c) {
        if (!(mask & (1u << c))) continue;
        if (!src[c]) return fail(FMX_EINVAL, "src[%d] is NULL", c);
        void *dst = (void *)(c < 3 ? G.E[b->parity][c] : G.B[b->parity][c - 3]);
        cudaError_t e = cudaMemcpy2DAsync(dst, dp, src[c], sp, sp, (size_t)G.g.ny, cudaMemcpyDefault, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
    }
    if (where == FMX_HOST) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return FMX_OK;
}

fmx_status fmx_batch_get_fields(fmx_batch *b, int i, unsigned mask, void *const *dst, int where) {
    if (!b || !dst || i < 0 || i >= b->n) return fail(FMX_EINVAL, "bad arguments");
    if (where != FMX_HOST && where != FMX_DEVICE) return fail(FMX_EINVAL, "where must be FMX_HOST or FMX_DEVICE");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    if (mask & ~(unsigned)(FMX_E | FMX_B)) return fail(FMX_EINVAL, "mask holds bits other than E and B");
    const fmx::BatchGrid &G = b->grids[i];
    const size_t dpch = (size_t)G.g.nx * 4, sp = (size_t)G.g.pitch * 4;
    for (int c = 0; c < 6; ++c) {
        if (!(mask & (1u << c))) continue;
        if (!dst[c]) return fail(FMX_EINVAL, "dst[%d] is NULL", c);
        const void *src = c < 3 ? G.E[b->parity][c] : G.B[b->parity][c - 3];
        cudaError_t e = cudaMemcpy2DAsync(dst[c], dpch, src, sp, dpch, (size_t)G.g.ny, cudaMemcpyDefault, b->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy2DAsync");
    }
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return FMX_OK;
}

fmx_status fmx_batch_set_rows(fmx_batch *b, int rows) {
    if (!b || rows < 0) return fail(FMX_EINVAL, "bad arguments");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    b->rows_policy = rows;
    // a failed rebuild leaves descriptors and work list out of step: unbind
    const fmx_status s = batch_build(b);
    if (s != FMX_OK) b->bound = false;
    return s;
}

fmx_status fmx_batch_set_tiles(fmx_batch *b, int narrow_policy) {
    if (!b || narrow_policy < 0 || narrow_policy > 2) return fail(FMX_EINVAL, "bad arguments");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    b->narrow_policy = narrow_policy;
    const fmx_status s = batch_build(b);
    if (s != FMX_OK) b->bound = false;
    return s;
}

fmx_status fmx_batch_tiles(const fmx_batch *b, int *wide, int *narrow, int *single, int *rows, int *narrow_policy) {
    if (!b) return fail(FMX_EINVAL, "NULL batch");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    if (wide) *wide = b->nwide;
    if (narrow) *narrow = b->nnarrow;
    if (single) *single = b->nitems - b->npol;
    if (rows) *rows = b->rows_policy;
    if (narrow_policy) *narrow_policy = b->narrow_policy;
    return FMX_OK;
}

int fmx_batch_grid_width(const fmx_batch *b, int i) {
    if (!b || !b->bound || i < 0 || i >= b->n) return -1;
    return b->grids[i].W;
}

fmx_status fmx_batch_step(fmx_batch *b, int nsteps) {
    if (!b) return fail(FMX_EINVAL, "NULL batch");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    if (nsteps < 0) return fail(FMX_EINVAL, "nsteps < 0");
    int left = nsteps;
    if (left % 2) {
        fmx_status s = batch_launch(b, b->parity);
        if (s != FMX_OK) return s;
        b->parity = 1 - b->parity;
        --left;
    }
    if (left > 0) {
        cudaGraphExec_t ge = nullptr;
        fmx_status s = batch_graph(b, b->parity, &ge);
        if (s != FMX_OK) return s;
        for (int k = 0; k < left / 2; ++k) {
            cudaError_t e = cudaGraphLaunch(ge, b->stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        }
        // kernels per step: one per kind of tile present
        b->launches += (int64_t)left * ((b->npol > 0) + (b->nitems > b->npol));
    }
    b->steps += nsteps;
    return FMX_OK;
}

}  // extern "C"

namespace {
// tuner choices by batch signature (m, passes, current, every grid's size):
// a later batch of the same grids reuses them without trial steps
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;

std::string batch_signature(const fmx_batch *b) {
    std::string k = std::to_string(b->m) + "/" + std::to_string(b->passes) + "/" + std::to_string((int)b->hj);
    for (int i = 0; i < b->n; ++i) k += ":" + std::to_string(b->p[i].n[0]) + "x" + std::to_string(b->p[i].n[1]);
    return k;
}
}  // namespace

extern "C" {

fmx_status fmx_batch_tune(fmx_batch *b, int trial_steps, int *chosen) {
    if (!b || trial_steps < 2) return fail(FMX_EINVAL, "bad arguments");
    if (!b->bound) return fail(FMX_ESTATE, "batch not bound");
    const std::string key = batch_signature(b);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->narrow_policy = it->second.second;
            if (chosen) *chosen = it->second.first;
            return fmx_batch_set_rows(b, it->second.first);
        }
    }
    // tile rule (narrow tiles everywhere, where they compute fewer columns,
    // or wide tiles only) x rows per segment (automatic, then fixed heights)
    const int rule[] = {2, 1, 0};
    const int cand[] = {0, 1024, 512, 384, 256, 192, 128, 96, 64, 32};
    float best = 1e30f;
    int best_rows = 0, best_rule = 2;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(FMX_ECUDA, "cudaEventCreate");
    fmx_status s = FMX_OK;
    for (int nr : rule) {
        b->narrow_policy = nr;
        for (int rows : cand) {
            if ((s = fmx_batch_set_rows(b, rows)) != FMX_OK) break;
            if ((s = fmx_batch_step(b, 2)) != FMX_OK) break;  // capture + warm
            cudaEventRecord(e0, b->stream);
            if ((s = fmx_batch_step(b, trial_steps / 2 * 2)) != FMX_OK) break;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_rows = rows;
                best_rule = nr;
            }
        }
        if (s != FMX_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != FMX_OK) return s;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = {best_rows, best_rule};
    }
    if (chosen) *chosen = best_rows;
    b->narrow_policy = best_rule;
    return fmx_batch_set_rows(b, best_rows);
}

int fmx_batch_items(const fmx_batch *b) { return b ? b->nitems : 0; }

int64_t fmx_batch_launch_count(const fmx_batch *b) { return b ? b->launches : 0; }

void fmx_batch_destroy(fmx_batch *b) {
    if (!b) return;
    batch_drop_graphs(b);
    delete b;
}

}  // extern "C"
