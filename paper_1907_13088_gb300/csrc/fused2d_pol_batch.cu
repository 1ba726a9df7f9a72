// Launches of the polarisation tiles (pol_tile.cuh) beyond the single-grid
// kernels of even n_x: grids with odd n_x, where the strips that cross the
// periodic seam load single columns (SEAM tile) and the others column pairs,
// and the batched step over many independent grids.
#include <cuda_runtime.h>

#include "fused2d.h"
#include "pol_tile.cuh"

namespace fmx {
namespace {

using namespace pair2;
using pol2d::coef2_of;
using pol2d::PolGeom;
using pol2d::pol_tile;

// odd n_x: the strips that cross the periodic seam take the SEAM tile, the
// others the pair tile
template <int POL, int M, int P, bool HJ, int NT>
__global__ void __launch_bounds__(NT, 3)
    k_pol2d_odd(Fused2dArgs<float> a, Geo g, Coef2 c, int W, int L, int nstrip) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *sm = reinterpret_cast<float *>(smraw);
    const int strip = blockIdx.x % nstrip, seg = blockIdx.x / nstrip;
    const int xs = strip * W - PolGeom<M, P, HJ>::HC;
    if (xs >= 0 && xs + 2 * NT <= g.nx) pol_tile<POL, M, P, HJ, NT, false>(a, g, c, W, L, strip, seg, sm);
    else pol_tile<POL, M, P, HJ, NT, true>(a, g, c, W, L, strip, seg, sm);
}

// Batched step on the polarisation kernels: a persistent loop over tasks.
// Task v < nwide is the TE half of the wide tile items[v] (the whole CTA, NT
// column pairs) and task nwide + v its TM half; the tasks after them take the
// narrow tiles (NT/2 column pairs) two at a time, one per half of the CTA,
// both in the same polarisation, again all TE pairs before all TM pairs (an
// SM then mostly runs one tile body at a time).  One launch per step covers
// both halves of every tile.
template <int M, int P, bool HJ, int NT>
__global__ void __launch_bounds__(NT, 3)
    k_pol2d_batch(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items, int nwide, int nnarrow,
                  int parity, int narrow_floats) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *sm = reinterpret_cast<float *>(smraw);
    constexpr int NH = NT / 2;
    const int npair = (nnarrow + 1) / 2;
    for (int v = blockIdx.x; v < 2 * (nwide + npair); v += gridDim.x) {
        __syncthreads();  // both halves are done with the previous task's shared memory
        const bool narrow = v >= 2 * nwide;
        const int half = narrow ? (int)threadIdx.x / NH : 0;
        // the TE halves of a kind of tile before its TM halves
        const int vk = narrow ? v - 2 * nwide : v, nk = narrow ? npair : nwide;
        const int tm = vk >= nk, k = vk - tm * nk;
        const int it = narrow ? nwide + 2 * k + half : k;
        if (narrow && it >= nwide + nnarrow) continue;  // the odd last narrow tile has one half idle
        const BatchItem w = items[it];
        const BatchGrid &G = grids[w.grid];
        Fused2dArgs<float> a{};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            a.E[q] = G.E[parity][q];
            a.B[q] = G.B[parity][q];
            a.J[q] = HJ ? G.J[q] : nullptr;
            a.Eo[q] = const_cast<float *>(G.E[1 - parity][q]);
            a.Bo[q] = const_cast<float *>(G.B[1 - parity][q]);
        }
        a.m = M;
        a.passes = P;
        const Geo g = G.g;
        const Coef2 c = coef2_of(G.c, P);
        if (!narrow) {
            const int xs = w.strip * G.W - PolGeom<M, P, HJ>::HC;
            const bool seam = (g.nx & 1) && !(xs >= 0 && xs + 2 * NT <= g.nx);
            if (!seam) {
                if (tm) pol_tile<TM, M, P, HJ, NT>(a, g, c, G.W, G.L, w.strip, w.seg, sm);
                else pol_tile<TE, M, P, HJ, NT>(a, g, c, G.W, G.L, w.strip, w.seg, sm);
            } else {
                if (tm) pol_tile<TM, M, P, HJ, NT, true>(a, g, c, G.W, G.L, w.strip, w.seg, sm);
                else pol_tile<TE, M, P, HJ, NT, true>(a, g, c, G.W, G.L, w.strip, w.seg, sm);
            }
        } else {
            float *smh = sm + half * narrow_floats;
            const int xs = w.strip * G.W - PolGeom<M, P, HJ>::HC;
            const bool seam = (g.nx & 1) && !(xs >= 0 && xs + 2 * NH <= g.nx);
            if (!seam) {
                if (tm) pol_tile<TM, M, P, HJ, NH, false, true>(a, g, c, G.W, G.L, w.strip, w.seg, smh, half);
                else pol_tile<TE, M, P, HJ, NH, false, true>(a, g, c, G.W, G.L, w.strip, w.seg, smh, half);
            } else {
                if (tm) pol_tile<TM, M, P, HJ, NH, true, true>(a, g, c, G.W, G.L, w.strip, w.seg, smh, half);
                else pol_tile<TE, M, P, HJ, NH, true, true>(a, g, c, G.W, G.L, w.strip, w.seg, smh, half);
            }
        }
    }
}

}  // namespace

namespace pol2d {

template <int POL, int M, int P, bool HJ>
void launch_odd(const Geo &g, const Coef2 &c, const Fused2dArgs<float> &a, int W, int L, int nstrip, int nblocks,
                cudaStream_t s) {
    constexpr int NT = 128;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_pol2d_odd<POL, M, P, HJ, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes<POL, M, P, HJ>());
        attr = true;
    }
    k_pol2d_odd<POL, M, P, HJ, NT><<<nblocks, NT, smem_bytes<POL, M, P, HJ>(), s>>>(a, g, c, W, L, nstrip);
}

#define FMX_POL_ODD_MP(M, P, HJ)                                                                                \
    template void launch_odd<TE, M, P, HJ>(const Geo &, const Coef2 &, const Fused2dArgs<float> &, int, int, int, \
                                           int, cudaStream_t);                                                    \
    template void launch_odd<TM, M, P, HJ>(const Geo &, const Coef2 &, const Fused2dArgs<float> &, int, int, int, \
                                           int, cudaStream_t);
#define FMX_POL_ODD_M(M)                                                                             \
    FMX_POL_ODD_MP(M, 0, false) FMX_POL_ODD_MP(M, 0, true) FMX_POL_ODD_MP(M, 1, true) FMX_POL_ODD_MP(M, 2, true) \
    FMX_POL_ODD_MP(M, 3, true)
FMX_POL_ODD_M(0)
FMX_POL_ODD_M(1)
FMX_POL_ODD_M(2)
FMX_POL_ODD_M(3)
FMX_POL_ODD_M(4)
#undef FMX_POL_ODD_M
#undef FMX_POL_ODD_MP

}  // namespace pol2d

int fused2d_pol_batch_geometry(int m, int passes, bool hj, int *threads, int *halo, int *width, size_t *smem,
                               int *blocks_per_sm, int *width_narrow, size_t *narrow_bytes) {
    int rc = -1;
#define FMX_PBG(MM, PP, HH)                                                                                    \
    if (m == MM && passes == PP && hj == HH) {                                                               \
        using Gm = PolGeom<MM, PP, HH>;                                                                     \
        constexpr int NT = 128;                                                                             \
        const size_t te = pol2d::smem_bytes<TE, MM, PP, HH>(), tm = pol2d::smem_bytes<TM, MM, PP, HH>(); \
        const size_t te2 = pol2d::smem_bytes<TE, MM, PP, HH, NT / 2>(),                                  \
                     tm2 = pol2d::smem_bytes<TM, MM, PP, HH, NT / 2>();                                  \
        const size_t nb2 = ((te2 > tm2 ? te2 : tm2) + 15) / 16 * 16;                                        \
        *threads = NT;                                                                                      \
        *halo = Gm::HC;                                                                                     \
        *width = 2 * NT - 2 * Gm::HC - 2;                                                                   \
        *width_narrow = NT - 2 * Gm::HC - 2;                                                                \
        *narrow_bytes = nb2;                                                                                \
        *smem = te > tm ? te : tm;                                                                          \
        if (2 * nb2 > *smem) *smem = 2 * nb2;                                                              \
        auto k = k_pol2d_batch<MM, PP, HH, NT>;                                                             \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);                   \
        int nb = 0;                                                                                         \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, *smem) != cudaSuccess || nb < 1) nb = 1; \
        *blocks_per_sm = nb;                                                                                \
        rc = 0;                                                                                             \
    }
    FMX_PBG(4, 0, false) FMX_PBG(4, 3, true) FMX_PBG(2, 0, false) FMX_PBG(1, 0, false) FMX_PBG(0, 0, false)
#undef FMX_PBG
    return rc;
}

int launch_fused2d_pol_batch(int m, int passes, bool hj, const BatchGrid *grids, const BatchItem *items, int nwide,
                             int nnarrow, int parity, int nblocks, size_t smem, size_t narrow_bytes, cudaStream_t s) {
    const int nf = (int)(narrow_bytes / sizeof(float));
#define FMX_PBL(MM, PP, HH)                                                                                    \
    if (m == MM && passes == PP && hj == HH) {                                                               \
        k_pol2d_batch<MM, PP, HH, 128><<<nblocks, 128, smem, s>>>(grids, items, nwide, nnarrow, parity, nf); \
        return 1;                                                                                            \
    }
    FMX_PBL(4, 0, false) FMX_PBL(4, 3, true) FMX_PBL(2, 0, false) FMX_PBL(1, 0, false) FMX_PBL(0, 0, false)
#undef FMX_PBL
    return -1;
}

}  // namespace fmx
