// FP64 diagnostics of a state (E^n, B^{n+1/2}):
//   energy of the converged scheme  sum[E.(1-A)E + B^{n-1/2}.S B^{n+1/2}]
//     with B^{n-1/2} = B^{n+1/2} + c dt curl E^n and S = diag(alpha_x,
//     alpha_y, alpha_z) (derived from the symmetry of A and S; the paper
//     does not define a discrete energy);
//   plain sum (E^2 + B^2);
//   D.B at cell centres (Eq. gauss_B);
//   D_x(alpha_yz Ex) + D_y(alpha_zx Ey) + D_z(alpha_xy Ez) at nodes
//     (left-hand side of Eq. gauss_E).
// Every cell's terms are evaluated in FP64 from the stored precision; block
// partials are combined by a single-block kernel in a fixed order.
#include <cuda_runtime.h>

#include "fmx_internal.h"
#include "stencil.cuh"

namespace fmx {
namespace {

constexpr int BX = 32, BY = 8, NT = BX * BY, NQ = 6;

template <typename T, int DIM>
__global__ void k_diag(Geo g, Coef<double> c, double idx_, double idy_, double idz_, const T *e0, const T *e1,
                       const T *e2, const T *b0, const T *b1, const T *b2, double *partials) {
    Pos p;
    p.i = blockIdx.x * BX + threadIdx.x;
    p.j = blockIdx.y * BY + threadIdx.y;
    p.k = blockIdx.z;
    const bool in = p.i < g.nx && p.j < g.ny;
    double v[NQ] = {0, 0, 0, 0, 0, 0};
    if (in) {
        Field<T, double> E[3] = {{e0, g}, {e1, g}, {e2, g}};
        Field<T, double> B[3] = {{b0, g}, {b1, g}, {b2, g}};
        const double inv_d[3] = {idx_, idy_, idz_};
        const int o0[3] = {0, 0, 0};
        double ae[3] = {apply_a<double, DIM, 0>(E, p, c), apply_a<double, DIM, 1>(E, p, c),
                        apply_a<double, DIM, 2>(E, p, c)};
        double ce[3] = {curl_e<double, DIM, 0>(E, p, c), curl_e<double, DIM, 1>(E, p, c),
                        curl_e<double, DIM, 2>(E, p, c)};
        double ws = 0.0, wp = 0.0, div = 0.0, gs = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double ea = E[a](p, 0, 0, 0), ba = B[a](p, 0, 0, 0);
            double sb = ba;
            if (a < DIM) sb += c.c6 * d2<double>(B[a], p, o0, a);
            ws += ea * (ea - ae[a]) + (ba + ce[a]) * sb;
            wp += ea * ea + ba * ba;
            if (a < DIM) div += (at_sh(B[a], p, o0, a, 1) - ba) * inv_d[a];
        }
        // node divergence of alpha_bc E_a, backward along a
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int b = (a + 1) % 3, cc = (a + 2) % 3;
            double val[2];
            for (int s = 0; s < 2; ++s) {
                int o[3] = {0, 0, 0};
                o[a] = -s;
                // alpha_c (alpha_b E_a) at o
                double w[3];
                for (int t = -1; t <= 1; ++t) {
                    int q[3] = {o[0], o[1], o[2]};
                    if (cc < DIM) q[cc] += t;
                    else if (t != 0) { w[t + 1] = 0.0; continue; }
                    double u = E[a](p, q[0], q[1], q[2]);
                    if (b < DIM) u += c.c6 * d2<double>(E[a], p, q, b);
                    w[t + 1] = u;
                }
                val[s] = cc < DIM ? w[1] + c.c6 * (w[2] - 2.0 * w[1] + w[0]) : w[1];
            }
            gs += (val[0] - val[1]) * inv_d[a];
        }
        v[0] = ws;
        v[1] = wp;
        v[2] = fabs(div);
        v[3] = div * div;
        v[4] = fabs(gs);
        v[5] = gs * gs;
    }
    __shared__ double red[NQ][NT / 32];
    const int t = threadIdx.y * BX + threadIdx.x;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        double x = v[q];
        const bool mx = q == 2 || q == 4;
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            x = mx ? fmax(x, y) : x + y;
        }
        if ((t & 31) == 0) red[q][t >> 5] = x;
    }
    __syncthreads();
    if (t < NQ) {
        const bool mx = t == 2 || t == 4;
        double x = 0.0;
        for (int w = 0; w < NT / 32; ++w) x = mx ? fmax(x, red[t][w]) : x + red[t][w];
        const int64_t slot =
            (int64_t)blockIdx.x + (int64_t)gridDim.x * ((int64_t)blockIdx.y + (int64_t)gridDim.y * blockIdx.z);
        partials[slot * NQ + t] = x;
    }
}

__global__ void k_diag_final(const double *partials, int64_t nslots, double *out) {
    __shared__ double red[NQ][32];
    double v[NQ] = {0, 0, 0, 0, 0, 0};
    for (int64_t s = threadIdx.x; s < nslots; s += blockDim.x)
        for (int q = 0; q < NQ; ++q) {
            double x = partials[s * NQ + q];
            v[q] = (q == 2 || q == 4) ? fmax(v[q], x) : v[q] + x;
        }
    for (int q = 0; q < NQ; ++q) {
        double x = v[q];
        const bool mx = q == 2 || q == 4;
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_down_sync(0xffffffffu, x, o);
            x = mx ? fmax(x, y) : x + y;
        }
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        const int q = threadIdx.x;
        const bool mx = q == 2 || q == 4;
        double x = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = mx ? fmax(x, red[q][w]) : x + red[q][w];
        out[q] = x;
    }
}

}  // namespace

template <typename T>
int launch_diagnostics(const Geo &g, int dims, const Coef<double> &c, const double d[3], T *const E[3],
                       T *const B[3], double *partials, int64_t nparts, double *out_dev, cudaStream_t s) {
    dim3 grid((g.nx + BX - 1) / BX, (g.ny + BY - 1) / BY, g.nz);
    const int64_t nslots = (int64_t)grid.x * grid.y * grid.z;
    if (nslots * NQ > nparts) return -1;
    const double ix = 1.0 / d[0], iy = 1.0 / d[1], iz = 1.0 / d[2];
    if (dims == 3)
        k_diag<T, 3><<<grid, dim3(BX, BY), 0, s>>>(g, c, ix, iy, iz, E[0], E[1], E[2], B[0], B[1], B[2], partials);
    else if (dims == 2)
        k_diag<T, 2><<<grid, dim3(BX, BY), 0, s>>>(g, c, ix, iy, iz, E[0], E[1], E[2], B[0], B[1], B[2], partials);
    else
        k_diag<T, 1><<<grid, dim3(BX, BY), 0, s>>>(g, c, ix, iy, iz, E[0], E[1], E[2], B[0], B[1], B[2], partials);
    k_diag_final<<<1, 1024, 0, s>>>(partials, nslots, out_dev);
    return 2;
}

template int launch_diagnostics<float>(const Geo &, int, const Coef<double> &, const double[3], float *const[3],
                                       float *const[3], double *, int64_t, double *, cudaStream_t);
template int launch_diagnostics<double>(const Geo &, int, const Coef<double> &, const double[3], double *const[3],
                                        double *const[3], double *, int64_t, double *, cudaStream_t);

}  // namespace fmx
