// Staged engine: one kernel per stage of the step, every intermediate in
// global memory.  General path: 1D/2D/3D, FP32/FP64, fixed or
// residual-controlled iteration, current or field filtering.  Each kernel
// is a plain one-thread-per-cell periodic stencil; the fused 2D engine
// (fused2d.cu) is the throughput path.
//
// Stencils (paper arXiv:1907.13088):
//   Dbar_a f: forward f[+1] - f[0] when f sits on an integer position along
//     a, backward f[0] - f[-1] when it sits half a cell off (Sec. 2);
//   alpha_a f = f + (1/6) Dbar_aa f (the (1/6, 2/3, 1/6) stencil);
//   source: Eqs. ampere_aux_x..z; A: Eqs. matrixA_1st..matrixA_last;
//   Faraday: Eqs. faraday_x..z.  Inactive axes (2D, 1D) drop every term
//   that differentiates along them and alpha becomes 1 (Secs. 2.2.2-2.2.3).
#include <cuda_runtime.h>

#include "fmx_internal.h"
#include "stencil.cuh"

namespace fmx {
namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ bool cell(const Geo &g, Pos &p, int64_t &idx) {
    p.i = blockIdx.x * BX + threadIdx.x;
    p.j = blockIdx.y * BY + threadIdx.y;
    p.k = blockIdx.z;
    idx = (int64_t)p.k * g.plane + (int64_t)p.j * g.pitch + p.i;
    return p.i < g.nx && p.j < g.ny;
}

__device__ __forceinline__ int64_t block_slot() {
    return (int64_t)blockIdx.x + (int64_t)gridDim.x * ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
}

// FP64 block sum of v (all threads call), thread 0 writes out[block_slot()]
__device__ __forceinline__ void block_sum_to(double v, double *out) {
    __shared__ double red[BX * BY / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int t = threadIdx.y * BX + threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < BX * BY / 32; ++w) s += red[w];
        out[block_slot()] = s;
    }
}

template <typename T>
__global__ void k_filter_pass(Geo g, const T *__restrict__ in, T *__restrict__ out, int axis) {
    Pos p;
    int64_t idx;
    if (!cell(g, p, idx)) return;
    Field<T, T> f{in, g};
    int dx, dy, dz;
    unit(axis, 1, dx, dy, dz);
    out[idx] = T(0.25) * f(p, -dx, -dy, -dz) + T(0.5) * f(p, 0, 0, 0) + T(0.25) * f(p, dx, dy, dz);
}

template <typename T, int DIM>
__global__ void k_source(Geo g, Coef<T> c, StagedPtrs<T> P, const T *jx, const T *jy, const T *jz, int norm) {
    Pos p;
    int64_t idx;
    bool in = cell(g, p, idx);
    double s = 0.0;
    if (in) {
        Field<T, T> b[3] = {{P.B[0], g}, {P.B[1], g}, {P.B[2], g}};
        T ex = curl_alpha_b<T, DIM, 0>(b, p, c);
        T ey = curl_alpha_b<T, DIM, 1>(b, p, c);
        T ez = curl_alpha_b<T, DIM, 2>(b, p, c);
        if (jx) ex -= c.q * jx[idx];
        if (jy) ey -= c.q * jy[idx];
        if (jz) ez -= c.q * jz[idx];
        P.dEp[0][idx] = ex;
        P.dEp[1][idx] = ey;
        P.dEp[2][idx] = ez;
        s = (double)ex * ex + (double)ey * ey + (double)ez * ez;
    }
    if (norm) block_sum_to(s, P.partials);
}

template <typename T, int DIM>
__device__ __forceinline__ double sweep_cell(const Geo &g, const Coef<T> &c, const T *const dEp[3],
                                             const T *const in[3], T *const out[3], Pos p, int64_t idx) {
    Field<T, T> f[3] = {{in[0], g}, {in[1], g}, {in[2], g}};
    T nx_ = dEp[0][idx] + apply_a<T, DIM, 0>(f, p, c);
    T ny_ = dEp[1][idx] + apply_a<T, DIM, 1>(f, p, c);
    T nz_ = dEp[2][idx] + apply_a<T, DIM, 2>(f, p, c);
    T ox = in[0][idx], oy = in[1][idx], oz = in[2][idx];
    out[0][idx] = nx_;
    out[1][idx] = ny_;
    out[2][idx] = nz_;
    T dx = nx_ - ox, dy = ny_ - oy, dz = nz_ - oz;
    return (double)dx * dx + (double)dy * dy + (double)dz * dz;
}

template <typename T, int DIM>
__global__ void k_sweep(Geo g, Coef<T> c, const T *p0, const T *p1, const T *p2, const T *i0, const T *i1,
                        const T *i2, T *o0, T *o1, T *o2, double *partials) {
    Pos p;
    int64_t idx;
    bool inb = cell(g, p, idx);
    double s = 0.0;
    const T *dEp[3] = {p0, p1, p2};
    const T *in[3] = {i0, i1, i2};
    T *out[3] = {o0, o1, o2};
    if (inb) s = sweep_cell<T, DIM>(g, c, dEp, in, out, p, idx);
    if (partials) block_sum_to(s, partials);
}

// Residual mode: the sweep index lives on the device (DevStatus.count);
// a stopped solve turns the remaining launches of a chunk into no-ops.
template <typename T, int DIM>
__global__ void k_resid_sweep(Geo g, Coef<T> c, StagedPtrs<T> P) {
    if (P.st->done) return;
    const int s = P.st->count;
    Pos p;
    int64_t idx;
    bool inb = cell(g, p, idx);
    const T *in[3];
    T *out[3];
    for (int q = 0; q < 3; ++q) {
        in[q] = s == 0 ? P.dEp[q] : ((s & 1) ? P.dEa[q] : P.dEb[q]);
        out[q] = ((s + 1) & 1) ? P.dEa[q] : P.dEb[q];
    }
    const T *dEp[3] = {P.dEp[0], P.dEp[1], P.dEp[2]};
    double v = 0.0;
    if (inb) v = sweep_cell<T, DIM>(g, c, dEp, in, out, p, idx);
    block_sum_to(v, P.partials);
}

// Chebyshev semi-iteration (textbook three-term recurrence) for
// (1 - A) x = dE', x_0 = dE': sweep s computes r = dE' - x_s + A x_s,
// d = c1 d + c2 r, x_{s+1} = x_s + d, with c1 = 0, c2 = 1/theta for s = 0 and
// rho_s = 1 / (2 sig - rho_{s-1}), c1 = rho_s rho_{s-1}, c2 = 2 rho_s / delta
// after (rho_0 = 1 / sig, kept in DevStatus.cheb_rho by the update kernel).
template <typename T, int DIM>
__global__ void k_cheb_sweep(Geo g, Coef<T> c, StagedPtrs<T> P, ChebParams cp) {
    if (P.st->done) return;
    const int s = P.st->count;
    double c1 = 0.0, c2 = 1.0 / cp.theta;
    if (s > 0) {
        const double rp = P.st->cheb_rho, rn = 1.0 / (2.0 * cp.sig - rp);
        c1 = rn * rp;
        c2 = 2.0 * rn / cp.delta;
    }
    Pos p;
    int64_t idx;
    bool inb = cell(g, p, idx);
    double v = 0.0;
    if (inb) {
        const T *in[3];
        T *out[3];
        for (int q = 0; q < 3; ++q) {
            in[q] = s == 0 ? P.dEp[q] : ((s & 1) ? P.dEa[q] : P.dEb[q]);
            out[q] = ((s + 1) & 1) ? P.dEa[q] : P.dEb[q];
        }
        Field<T, T> f[3] = {{in[0], g}, {in[1], g}, {in[2], g}};
        const T ax[3] = {apply_a<T, DIM, 0>(f, p, c), apply_a<T, DIM, 1>(f, p, c), apply_a<T, DIM, 2>(f, p, c)};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const T x = in[q][idx];
            const T r = P.dEp[q][idx] - x + ax[q];
            const T d = (s == 0 ? T(0) : T(c1) * P.jf[q][idx]) + T(c2) * r;
            P.jf[q][idx] = d;
            out[q][idx] = x + d;
            v += (double)d * (double)d;
        }
    }
    block_sum_to(v, P.partials);
}

__device__ __forceinline__ double reduce_partials(const double *partials, int64_t n) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x) s += partials[q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

__global__ void k_resid_init(const double *partials, int64_t n, DevStatus *st) {
    double t = reduce_partials(partials, n);
    if (threadIdx.x == 0) {
        st->nrm2 = t;
        st->r2 = 0.0;
        st->count = 0;
        st->done = t == 0.0 ? 1 : 0;
        st->noconv = 0;
    }
}

__global__ void k_resid_update(const double *partials, int64_t n, DevStatus *st, double tol2, int m_max) {
    if (st->done) return;
    double t = reduce_partials(partials, n);
    if (threadIdx.x == 0) {
        st->r2 = t;
        st->count += 1;
        if (t <= tol2 * st->nrm2) {
            st->done = 1;
        } else if (st->count >= m_max) {
            st->done = 1;
            st->noconv = 1;
        }
    }
}

__global__ void k_cheb_update(const double *partials, int64_t n, DevStatus *st, ChebParams cp, int resid, double tol2,
                              int m_max) {
    if (st->done) return;
    double t = reduce_partials(partials, n);
    if (threadIdx.x == 0) {
        const int s = st->count;
        st->cheb_rho = s == 0 ? 1.0 / cp.sig : 1.0 / (2.0 * cp.sig - st->cheb_rho);
        st->r2 = t;
        st->count = s + 1;
        if (resid) {
            if (t <= tol2 * st->nrm2) {
                st->done = 1;
            } else if (st->count >= m_max) {
                st->done = 1;
                st->noconv = 1;
            }
        }
    }
}

template <typename T>
__global__ void k_update_e(Geo g, T *e0, T *e1, T *e2, const T *d0, const T *d1, const T *d2_) {
    Pos p;
    int64_t idx;
    if (!cell(g, p, idx)) return;
    e0[idx] += d0[idx];
    e1[idx] += d1[idx];
    e2[idx] += d2_[idx];
}

template <typename T>
__global__ void k_update_e_resid(Geo g, StagedPtrs<T> P) {
    Pos p;
    int64_t idx;
    if (!cell(g, p, idx)) return;
    const int s = P.st->count;
    for (int q = 0; q < 3; ++q) {
        const T *d = s == 0 ? P.dEp[q] : ((s & 1) ? P.dEa[q] : P.dEb[q]);
        P.E[q][idx] += d[idx];
    }
}

template <typename T, int DIM>
__global__ void k_faraday(Geo g, Coef<T> c, const T *e0, const T *e1, const T *e2, T *b0, T *b1, T *b2) {
    Pos p;
    int64_t idx;
    if (!cell(g, p, idx)) return;
    Field<T, T> e[3] = {{e0, g}, {e1, g}, {e2, g}};
    b0[idx] -= curl_e<T, DIM, 0>(e, p, c);
    b1[idx] -= curl_e<T, DIM, 1>(e, p, c);
    b2[idx] -= curl_e<T, DIM, 2>(e, p, c);
}

inline dim3 grid_of(const Geo &g) { return dim3((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz); }

}  // namespace

int64_t staged_partial_slots(const Geo &g) {
    dim3 gr = grid_of(g);
    return (int64_t)gr.x * gr.y * gr.z;
}

template <typename T>
int launch_filter_pass(const Geo &g, int dims, const T *in, T *out, int axis, cudaStream_t s) {
    (void)dims;
    k_filter_pass<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, in, out, axis);
    return 1;
}

template <typename T>
int launch_staged_source(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p,
                         const T *const jsrc[3], cudaStream_t s, bool norm) {
    const T *jx = jsrc ? jsrc[0] : nullptr, *jy = jsrc ? jsrc[1] : nullptr, *jz = jsrc ? jsrc[2] : nullptr;
    if (dims == 3)
        k_source<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p, jx, jy, jz, norm);
    else if (dims == 2)
        k_source<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p, jx, jy, jz, norm);
    else
        k_source<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p, jx, jy, jz, norm);
    return 1;
}

template <typename T>
int launch_staged_sweep(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p, const T *const in[3],
                        T *const out[3], bool resid, cudaStream_t s) {
    double *part = resid ? p.partials : nullptr;
    if (dims == 3)
        k_sweep<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p.dEp[0], p.dEp[1], p.dEp[2], in[0], in[1], in[2],
                                                          out[0], out[1], out[2], part);
    else if (dims == 2)
        k_sweep<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p.dEp[0], p.dEp[1], p.dEp[2], in[0], in[1], in[2],
                                                          out[0], out[1], out[2], part);
    else
        k_sweep<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p.dEp[0], p.dEp[1], p.dEp[2], in[0], in[1], in[2],
                                                          out[0], out[1], out[2], part);
    return 1;
}

template <typename T>
int launch_resid_sweep(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p, cudaStream_t s) {
    if (dims == 3)
        k_resid_sweep<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p);
    else if (dims == 2)
        k_resid_sweep<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p);
    else
        k_resid_sweep<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p);
    return 1;
}

int launch_resid_init(double *partials, int64_t nparts, DevStatus *st, cudaStream_t s) {
    k_resid_init<<<1, 1024, 0, s>>>(partials, nparts, st);
    return 1;
}

template <typename T>
int launch_cheb_sweep(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p, const ChebParams &cp,
                      cudaStream_t s) {
    if (dims == 3)
        k_cheb_sweep<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p, cp);
    else if (dims == 2)
        k_cheb_sweep<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p, cp);
    else
        k_cheb_sweep<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, p, cp);
    return 1;
}

int launch_cheb_update(double *partials, int64_t nparts, DevStatus *st, const ChebParams &cp, bool resid,
                       double tol2, int m_max, cudaStream_t s) {
    k_cheb_update<<<1, 1024, 0, s>>>(partials, nparts, st, cp, resid ? 1 : 0, tol2, m_max);
    return 1;
}

int launch_resid_update(double *partials, int64_t nparts, DevStatus *st, double tol2, int m_max, cudaStream_t s) {
    k_resid_update<<<1, 1024, 0, s>>>(partials, nparts, st, tol2, m_max);
    return 1;
}

template <typename T>
int launch_update_e(const Geo &g, T *const E[3], const T *const dE[3], cudaStream_t s) {
    k_update_e<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, E[0], E[1], E[2], dE[0], dE[1], dE[2]);
    return 1;
}

template <typename T>
int launch_update_e_resid(const Geo &g, const StagedPtrs<T> &p, cudaStream_t s) {
    k_update_e_resid<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, p);
    return 1;
}

template <typename T>
int launch_faraday(const Geo &g, int dims, const Coef<T> &c, T *const E[3], T *const B[3], cudaStream_t s) {
    if (dims == 3)
        k_faraday<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, E[0], E[1], E[2], B[0], B[1], B[2]);
    else if (dims == 2)
        k_faraday<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, E[0], E[1], E[2], B[0], B[1], B[2]);
    else
        k_faraday<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, E[0], E[1], E[2], B[0], B[1], B[2]);
    return 1;
}

#define FMX_INST(T)                                                                                           \
    template int launch_filter_pass<T>(const Geo &, int, const T *, T *, int, cudaStream_t);                  \
    template int launch_staged_source<T>(const Geo &, int, const Coef<T> &, const StagedPtrs<T> &,            \
                                         const T *const[3], cudaStream_t, bool);                              \
    template int launch_staged_sweep<T>(const Geo &, int, const Coef<T> &, const StagedPtrs<T> &,             \
                                        const T *const[3], T *const[3], bool, cudaStream_t);                  \
    template int launch_resid_sweep<T>(const Geo &, int, const Coef<T> &, const StagedPtrs<T> &, cudaStream_t); \
    template int launch_cheb_sweep<T>(const Geo &, int, const Coef<T> &, const StagedPtrs<T> &, const ChebParams &, \
                                      cudaStream_t);                                                         \
    template int launch_update_e<T>(const Geo &, T *const[3], const T *const[3], cudaStream_t);               \
    template int launch_update_e_resid<T>(const Geo &, const StagedPtrs<T> &, cudaStream_t);                  \
    template int launch_faraday<T>(const Geo &, int, const Coef<T> &, T *const[3], T *const[3], cudaStream_t);
FMX_INST(float)
FMX_INST(double)
#undef FMX_INST

}  // namespace fmx
