// Adjoint of one field step and the Gaussian-envelope current source.
//
// The step is linear in (E^n, B^{n+1/2}, j):  dE' = C_b S B - q F j,
// dE = P dE' (P = sum_{s<=m} A^s, Algorithm 1), E1 = E + dE, B1 = B - C_f E1,
// with C_f the Faraday curl (forward differences, Eqs. faraday_x..z) and C_b
// the source curl (backward differences, Eqs. ampere_aux_x..z).  On the
// periodic lattice C_f^T = C_b, and A (Eqs. matrixA_*), S = diag(alpha) and
// the binomial filter F are symmetric, so the adjoint of the step maps
// (Ebar, Bbar) = dL/d(E1, B1) to
//   u = Ebar - C_b Bbar,  Ebar <- u,  w = P u,  Bbar <- Bbar + S C_f w,
//   jbar = -q F w,
// i.e. the same curls, the same m sweeps and the same filter as the forward
// step, applied in reverse order.
#include <cuda_runtime.h>

#include "fmx_internal.h"
#include "stencil.cuh"

namespace fmx {
namespace {

constexpr int BX = 32, BY = 8;

__device__ __forceinline__ bool cell_of(const Geo &g, Pos &p, int64_t &idx) {
    p.i = blockIdx.x * BX + threadIdx.x;
    p.j = blockIdx.y * BY + threadIdx.y;
    p.k = blockIdx.z;
    idx = (int64_t)p.k * g.plane + (int64_t)p.j * g.pitch + p.i;
    return p.i < g.nx && p.j < g.ny;
}

inline dim3 grid_of(const Geo &g) { return dim3((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz); }

// u = Ebar - C_b Bbar  (c.c6 must be 0: no averaging in the transposed Faraday curl)
template <typename T, int DIM>
__global__ void k_adj_source(Geo g, Coef<T> c, const T *e0, const T *e1, const T *e2, const T *b0, const T *b1,
                             const T *b2, T *u0, T *u1, T *u2) {
    Pos p;
    int64_t idx;
    if (!cell_of(g, p, idx)) return;
    Field<T, T> b[3] = {{b0, g}, {b1, g}, {b2, g}};
    u0[idx] = e0[idx] - curl_alpha_b<T, DIM, 0>(b, p, c);
    u1[idx] = e1[idx] - curl_alpha_b<T, DIM, 1>(b, p, c);
    u2[idx] = e2[idx] - curl_alpha_b<T, DIM, 2>(b, p, c);
}

// Bbar_a += alpha_a (C_f w)_a, alpha along the component's own axis
template <typename T, int DIM, int A>
__device__ __forceinline__ T alpha_curl(const Field<T, T> w[3], const Geo &g, Pos p, const Coef<T> &c) {
    T t0 = curl_e<T, DIM, A>(w, p, c);
    if (A < DIM) {
        Pos pp = p, pm = p;
        if (A == 0) { pp.i = wrapc(p.i + 1, g.nx); pm.i = wrapc(p.i - 1, g.nx); }
        if (A == 1) { pp.j = wrapc(p.j + 1, g.ny); pm.j = wrapc(p.j - 1, g.ny); }
        if (A == 2) { pp.k = wrapc(p.k + 1, g.nz); pm.k = wrapc(p.k - 1, g.nz); }
        const T tp = curl_e<T, DIM, A>(w, pp, c), tm = curl_e<T, DIM, A>(w, pm, c);
        t0 += c.c6 * (tp - T(2) * t0 + tm);
    }
    return t0;
}

template <typename T, int DIM>
__global__ void k_adj_faraday(Geo g, Coef<T> c, const T *w0, const T *w1, const T *w2, T *b0, T *b1, T *b2) {
    Pos p;
    int64_t idx;
    if (!cell_of(g, p, idx)) return;
    Field<T, T> w[3] = {{w0, g}, {w1, g}, {w2, g}};
    b0[idx] += alpha_curl<T, DIM, 0>(w, g, p, c);
    b1[idx] += alpha_curl<T, DIM, 1>(w, g, p, c);
    b2[idx] += alpha_curl<T, DIM, 2>(w, g, p, c);
}

template <typename T>
__global__ void k_scale_copy(Geo g, T s, const T *i0, const T *i1, const T *i2, T *o0, T *o1, T *o2) {
    Pos p;
    int64_t idx;
    if (!cell_of(g, p, idx)) return;
    o0[idx] = s * i0[idx];
    o1[idx] = s * i1[idx];
    o2[idx] = s * i2[idx];
}

// Gaussian-envelope current: j_z(i, j) = sum_p amp_p exp(-|r_ij - c_p|^2 / (2 w^2)),
// distances taken periodically; 2D, j_z sits on the node (i, j).  The
// arithmetic is in the storage precision T.
template <typename T>
__device__ __forceinline__ T pdist(T d, T n) {
    return d - n * floor(d / n + T(0.5));
}

template <typename T>
__device__ __forceinline__ T gexp(T e) {
    if constexpr (sizeof(T) == 4) return __expf(e);
    else return exp(e);
}

template <typename T>
__global__ void k_gauss_source(Geo g, int np, const double *cxy, const double *amp, double inv2w2, T *jx, T *jy,
                               T *jz) {
    Pos p;
    int64_t idx;
    if (!cell_of(g, p, idx)) return;
    const T nx = (T)g.nx, ny = (T)g.ny, k = (T)inv2w2;
    T acc = T(0);
    for (int q = 0; q < np; ++q) {
        const T dx = pdist<T>((T)p.i - (T)cxy[2 * q], nx);
        const T dy = pdist<T>((T)p.j - (T)cxy[2 * q + 1], ny);
        acc += (T)amp[q] * gexp<T>(-(dx * dx + dy * dy) * k);
    }
    jx[idx] = T(0);
    jy[idx] = T(0);
    jz[idx] = acc;
}

// partials[q * nblk + b] = sum over the cells of block b of f * G_q (G in the
// storage precision, sums in FP64)
template <typename T>
__global__ void k_gauss_project(Geo g, int np, const double *cxy, double inv2w2, const T *f, double *partials,
                                int nblk) {
    const int q = blockIdx.y;
    const int64_t ncell = (int64_t)g.nx * g.ny;
    const T nx = (T)g.nx, ny = (T)g.ny, k = (T)inv2w2, cx = (T)cxy[2 * q], cy = (T)cxy[2 * q + 1];
    double acc = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)nblk * blockDim.x) {
        const int i = (int)(c % g.nx), j = (int)(c / g.nx);
        const T dx = pdist<T>((T)i - cx, nx), dy = pdist<T>((T)j - cy, ny);
        acc += (double)(f[(int64_t)j * g.pitch + i] * gexp<T>(-(dx * dx + dy * dy) * k));
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        partials[(int64_t)q * nblk + blockIdx.x] = s;
    }
}

// out[q] = sum_b partials (weights == nullptr), or acc[q] += weights[q] * sum_b partials
__global__ void k_gauss_project_final(const double *partials, int nblk, int np, const double *weights, double *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partials[(int64_t)q * nblk + b];
    if (weights) out[q] += weights[q] * s;
    else out[q] = s;
}

}  // namespace

template <typename T>
int launch_adj_source(const Geo &g, int dims, const Coef<T> &c, T *const Eb[3], T *const Bb[3], T *const u[3],
                      cudaStream_t s) {
    Coef<T> c0 = c;
    c0.c6 = T(0);
    if (dims == 3)
        k_adj_source<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c0, Eb[0], Eb[1], Eb[2], Bb[0], Bb[1], Bb[2], u[0], u[1], u[2]);
    else if (dims == 2)
        k_adj_source<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c0, Eb[0], Eb[1], Eb[2], Bb[0], Bb[1], Bb[2], u[0], u[1], u[2]);
    else
        k_adj_source<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c0, Eb[0], Eb[1], Eb[2], Bb[0], Bb[1], Bb[2], u[0], u[1], u[2]);
    return 1;
}

template <typename T>
int launch_adj_faraday(const Geo &g, int dims, const Coef<T> &c, T *const w[3], T *const Bb[3], cudaStream_t s) {
    if (dims == 3)
        k_adj_faraday<T, 3><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, w[0], w[1], w[2], Bb[0], Bb[1], Bb[2]);
    else if (dims == 2)
        k_adj_faraday<T, 2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, w[0], w[1], w[2], Bb[0], Bb[1], Bb[2]);
    else
        k_adj_faraday<T, 1><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, c, w[0], w[1], w[2], Bb[0], Bb[1], Bb[2]);
    return 1;
}

template <typename T>
int launch_scale_copy(const Geo &g, T sc, T *const in[3], T *const out[3], cudaStream_t s) {
    k_scale_copy<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, sc, in[0], in[1], in[2], out[0], out[1], out[2]);
    return 1;
}

template <typename T>
int launch_gauss_source(const Geo &g, int np, const double *cxy, const double *amp, double width, T *const J[3],
                        cudaStream_t s) {
    k_gauss_source<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, np, cxy, amp, 1.0 / (2.0 * width * width), J[0], J[1],
                                                          J[2]);
    return 1;
}

template <typename T>
int launch_gauss_project(const Geo &g, int np, const double *cxy, double width, const T *f, double *partials,
                         int nblk, const double *weights, double *out, cudaStream_t s) {
    k_gauss_project<T><<<dim3(nblk, np), 256, 0, s>>>(g, np, cxy, 1.0 / (2.0 * width * width), f, partials, nblk);
    k_gauss_project_final<<<(np + 127) / 128, 128, 0, s>>>(partials, nblk, np, weights, out);
    return 2;
}

#define FMX_ADJ_INST(T)                                                                                         \
    template int launch_adj_source<T>(const Geo &, int, const Coef<T> &, T *const[3], T *const[3], T *const[3], \
                                      cudaStream_t);                                                           \
    template int launch_adj_faraday<T>(const Geo &, int, const Coef<T> &, T *const[3], T *const[3], cudaStream_t); \
    template int launch_scale_copy<T>(const Geo &, T, T *const[3], T *const[3], cudaStream_t);                  \
    template int launch_gauss_source<T>(const Geo &, int, const double *, const double *, double, T *const[3],  \
                                        cudaStream_t);                                                         \
    template int launch_gauss_project<T>(const Geo &, int, const double *, double, const T *, double *, int,    \
                                         const double *, double *, cudaStream_t);
FMX_ADJ_INST(float)
FMX_ADJ_INST(double)
#undef FMX_ADJ_INST

}  // namespace fmx
