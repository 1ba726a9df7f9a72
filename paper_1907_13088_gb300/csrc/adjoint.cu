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
    // a null output component is skipped (callers may want only some)
    if (o0) o0[idx] = s * i0[idx];
    if (o1) o1[idx] = s * i1[idx];
    if (o2) o2[idx] = s * i2[idx];
}

// Gaussian-envelope current: j_z(i, j) = sum_p a_p G_p(i, j) with
// G_p = exp(-|r_ij - c_p|^2 / (2 w^2)), distances taken periodically per axis;
// 2D, j_z sits on the node (i, j).  The envelope factorises per axis,
// G_p(i, j) = gx_p(i) gy_p(j), so a tile of GTX columns x GTY rows needs
// np (GTX + GTY) exponentials instead of np GTX GTY: the tile's 1D profiles
// go to shared memory and every cell is a sum of np products.  Amplitudes
// are given (amp) or formed in the kernel as a_p = theta_p sin(omega0 t +
// phi_p) (FP64).  The arithmetic is otherwise in the storage precision T.
constexpr int GTX = 32, GTY = 64, GRY = 8;  // tile; rows per thread (256 threads)

template <typename T>
__device__ __forceinline__ T pdist(T d, T n) {
    return d - n * floor(d / n + T(0.5));
}

template <typename T>
__device__ __forceinline__ T gexp(T e) {
    if constexpr (sizeof(T) == 4) return __expf(e);
    else return exp(e);
}

struct GaussArgs {
    const double *cxy;    // (x_p, y_p)
    const double *amp;    // a_p, or nullptr: theta, phi, omega0, t below
    const double *theta;
    const double *phi;
    double omega0, t;
    double inv2w2;        // 1 / (2 w^2)
    int np;
};

// shared layout: par[3][np] (source centre x, y and, in the synthesis, the
// amplitude, in T), gx[np][GTX], gy[np][GTY] (gy pre-scaled by a_p in the
// source).  The per-source values are converted from FP64 once per block
// (FP64 work is slow on this part: doing it per profile element cost more
// than the rest of the kernel).
template <typename T>
__device__ __forceinline__ void gauss_params(const GaussArgs &a, bool scale, T *par) {
    for (int p = threadIdx.x; p < a.np; p += blockDim.x) {
        par[p] = (T)a.cxy[2 * p];
        par[a.np + p] = (T)a.cxy[2 * p + 1];
        if (scale) par[2 * a.np + p] = (T)(a.amp ? a.amp[p] : a.theta[p] * sin(a.omega0 * a.t + a.phi[p]));
    }
}

// the tile's 1D profiles from par (gauss_params, synchronised before)
template <typename T>
__device__ __forceinline__ void gauss_profiles(const Geo &g, const GaussArgs &a, int x0, int y0, bool scale, T *gx,
                                               T *gy, const T *par) {
    const T nx = (T)g.nx, ny = (T)g.ny, k = (T)a.inv2w2;
    for (int q = threadIdx.x; q < a.np * GTX; q += blockDim.x) {
        const int p = q / GTX, i = x0 + q % GTX;
        const T dx = pdist<T>((T)i - par[p], nx);
        gx[q] = gexp<T>(-dx * dx * k);
    }
    for (int q = threadIdx.x; q < a.np * GTY; q += blockDim.x) {
        const int p = q / GTY, j = y0 + q % GTY;
        const T dy = pdist<T>((T)j - par[a.np + p], ny);
        T v = gexp<T>(-dy * dy * k);
        if (scale) v *= par[2 * a.np + p];
        gy[q] = v;
    }
}

// bytes of the par block, padded to 16
template <typename T>
__host__ __device__ constexpr int gauss_par_bytes(int np) {
    return (int)((3 * np * sizeof(T) + 15) / 16 * 16);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gauss_source(Geo g, GaussArgs a, T *jx, T *jy, T *jz, int zero_xy) {
    extern __shared__ __align__(16) unsigned char gsm[];
    T *par = reinterpret_cast<T *>(gsm);  // [3][np]
    T *gx = reinterpret_cast<T *>(gsm + gauss_par_bytes<T>(a.np));
    T *gy = gx + a.np * GTX;
    const int x0 = blockIdx.x * GTX, y0 = blockIdx.y * GTY;
    gauss_params<T>(a, true, par);
    __syncthreads();
    gauss_profiles<T>(g, a, x0, y0, true, gx, gy, par);
    __syncthreads();
    const int tx = threadIdx.x % GTX, ty = threadIdx.x / GTX;
    T acc[GRY];
#pragma unroll
    for (int r = 0; r < GRY; ++r) acc[r] = T(0);
    // several sources in flight: the row profile of a source is one broadcast
    // 16-byte load per four rows (FP32)
#pragma unroll 4
    for (int p = 0; p < a.np; ++p) {
        const T xv = gx[p * GTX + tx];
        const T *yr = gy + p * GTY + ty * GRY;
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int h = 0; h < GRY; h += 4) {
                const float4 y4 = *reinterpret_cast<const float4 *>(yr + h);
                acc[h + 0] += y4.x * xv;
                acc[h + 1] += y4.y * xv;
                acc[h + 2] += y4.z * xv;
                acc[h + 3] += y4.w * xv;
            }
        } else {
#pragma unroll
            for (int r = 0; r < GRY; ++r) acc[r] += yr[r] * xv;
        }
    }
    const int i = x0 + tx;
    if (i >= g.nx) return;
#pragma unroll
    for (int r = 0; r < GRY; ++r) {
        const int j = y0 + ty * GRY + r;
        if (j >= g.ny) break;
        const int64_t idx = (int64_t)j * g.pitch + i;
        jz[idx] = acc[r];
        if (zero_xy) {
            jx[idx] = T(0);
            jy[idx] = T(0);
        }
    }
}

// partials[q * nblk + b] = sum over the tiles of block b of f * G_q: products
// and the sum over one warp's 256 cells in T, everything above in FP64
template <typename T>
__global__ void __launch_bounds__(256) k_gauss_project(Geo g, GaussArgs a, const T *f, double *partials, int nblk) {
    extern __shared__ __align__(16) unsigned char gsm[];
    double *wsum = reinterpret_cast<double *>(gsm);  // [8 warps][np]
    T *par = reinterpret_cast<T *>(wsum + 8 * a.np);  // [3][np]
    T *gx = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(par) + gauss_par_bytes<T>(a.np));
    T *gy = gx + a.np * GTX;
    const int tilesx = (g.nx + GTX - 1) / GTX, ntiles = tilesx * ((g.ny + GTY - 1) / GTY);
    const int tx = threadIdx.x % GTX, ty = threadIdx.x / GTX, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < 8 * a.np; q += blockDim.x) wsum[q] = 0.0;
    gauss_params<T>(a, false, par);  // synchronised by the first tile's barrier
    for (int tile = blockIdx.x; tile < ntiles; tile += nblk) {
        const int x0 = (tile % tilesx) * GTX, y0 = (tile / tilesx) * GTY;
        __syncthreads();  // previous tile's profiles are consumed
        gauss_profiles<T>(g, a, x0, y0, false, gx, gy, par);
        __syncthreads();
        const int i = x0 + tx;
        T fv[GRY];
#pragma unroll
        for (int r = 0; r < GRY; ++r) {
            const int j = y0 + ty * GRY + r;
            fv[r] = (i < g.nx && j < g.ny) ? f[(int64_t)j * g.pitch + i] : T(0);
        }
        // the sources in chunks of 32: each lane forms its products for all 32
        // (zero past np), then a reduce-scatter over the warp (halving
        // exchanges, 31 shuffles) leaves lane l with the warp's sum for source
        // p0 + l, which it adds to the warp's FP64 slot
        for (int p0 = 0; p0 < a.np; p0 += 32) {
            T v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int p = p0 + i;
                T s = T(0);
                if (p < a.np) {
                    const T *yr = gy + p * GTY + ty * GRY;
                    if constexpr (sizeof(T) == 4) {
#pragma unroll
                        for (int h = 0; h < GRY; h += 4) {
                            const float4 y4 = *reinterpret_cast<const float4 *>(yr + h);
                            s += y4.x * fv[h + 0];
                            s += y4.y * fv[h + 1];
                            s += y4.z * fv[h + 2];
                            s += y4.w * fv[h + 3];
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < GRY; ++r) s += yr[r] * fv[r];
                    }
                    s *= gx[p * GTX + tx];
                }
                v[i] = s;
            }
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                const int o = 16 >> r;  // the half kept: upper when this lane's bit o is set
                const bool up = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < o; ++i) {
                    const T send = up ? v[i] : v[i + o];
                    const T keep = up ? v[i + o] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            if (p0 + lane < a.np) wsum[warp * a.np + p0 + lane] += (double)v[0];
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < a.np; p += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += wsum[w * a.np + p];
        partials[(int64_t)p * nblk + blockIdx.x] = s;
    }
}

// out[q] = sum_b partials (no weights), or acc[q] += w_q * sum_b partials with
// w_q = weights[q] or, when weights is nullptr and phi is given,
// w_q = sin(omega0 t + phi_q).  One block per q; fixed summation order.
constexpr int GFT = 128;
__global__ void __launch_bounds__(GFT) k_gauss_project_final(const double *partials, int nblk, int np,
                                                             const double *weights, const double *phi, double omega0,
                                                             double t, double *out) {
    const int q = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += GFT) s += partials[(int64_t)q * nblk + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[GFT / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    s = 0.0;
    for (int w = 0; w < GFT / 32; ++w) s += red[w];
    if (weights) out[q] += weights[q] * s;
    else if (phi) out[q] += sin(omega0 * t + phi[q]) * s;
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

// the source adds np doubles for the amplitudes, the projection 8 np for the
// per-warp sums (both in front of the profiles, so these stay 8-byte aligned)
template <typename T>
size_t gauss_smem(int np, bool project) {
    // [wsum: 8 np doubles, projection only][par, padded to 16 bytes][gx][gy]:
    // the profiles start 16-byte aligned for 16-byte loads
    return (size_t)np * (GTX + GTY) * sizeof(T) + (project ? (size_t)8 * np * sizeof(double) : 0) +
           (size_t)gauss_par_bytes<T>(np);
}

template <typename T>
int launch_gauss_source(const Geo &g, const GaussSrc &gs, T *const J[3], bool zero_xy, cudaStream_t s) {
    GaussArgs a{gs.cxy, gs.amp, gs.theta, gs.phi, gs.omega0, gs.t, 1.0 / (2.0 * gs.width * gs.width), gs.np};
    const size_t sm = gauss_smem<T>(gs.np, false);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gauss_source<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gauss_smem<T>(128, true));
        attr = true;
    }
    const dim3 grid((g.nx + GTX - 1) / GTX, (g.ny + GTY - 1) / GTY);
    k_gauss_source<T><<<grid, 256, sm, s>>>(g, a, J[0], J[1], J[2], zero_xy ? 1 : 0);
    return 1;
}

template <typename T>
int launch_gauss_project(const Geo &g, const GaussSrc &gs, const T *f, double *partials, int64_t cap,
                         const double *weights, double *out, cudaStream_t s) {
    GaussArgs a{gs.cxy, nullptr, nullptr, nullptr, 0.0, 0.0, 1.0 / (2.0 * gs.width * gs.width), gs.np};
    const int ntiles = ((g.nx + GTX - 1) / GTX) * ((g.ny + GTY - 1) / GTY);
    int64_t nblk = cap / gs.np;
    if (nblk > ntiles) nblk = ntiles;
    if (nblk > 1024) nblk = 1024;
    if (nblk < 1) return -1;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gauss_project<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gauss_smem<T>(128, true));
        attr = true;
    }
    k_gauss_project<T><<<(int)nblk, 256, gauss_smem<T>(gs.np, true), s>>>(g, a, f, partials, (int)nblk);
    k_gauss_project_final<<<gs.np, GFT, 0, s>>>(partials, (int)nblk, gs.np, weights, gs.phi, gs.omega0, gs.t, out);
    return 2;
}

#define FMX_ADJ_INST(T)                                                                                         \
    template int launch_adj_source<T>(const Geo &, int, const Coef<T> &, T *const[3], T *const[3], T *const[3], \
                                      cudaStream_t);                                                           \
    template int launch_adj_faraday<T>(const Geo &, int, const Coef<T> &, T *const[3], T *const[3], cudaStream_t); \
    template int launch_scale_copy<T>(const Geo &, T, T *const[3], T *const[3], cudaStream_t);                  \
    template int launch_gauss_source<T>(const Geo &, const GaussSrc &, T *const[3], bool, cudaStream_t);        \
    template int launch_gauss_project<T>(const Geo &, const GaussSrc &, const T *, double *, int64_t,          \
                                         const double *, double *, cudaStream_t);
FMX_ADJ_INST(float)
FMX_ADJ_INST(double)
#undef FMX_ADJ_INST

}  // namespace fmx
