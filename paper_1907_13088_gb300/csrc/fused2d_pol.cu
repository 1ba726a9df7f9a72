// FP32 fused 2D step split by polarisation (Sec. 2.2.2: the TE set Ex, Ey,
// Bz; jx, jy and the TM set Ez, Bx, By; jz decouple exactly), two columns per
// thread: the single-grid kernels.  One step is one TE launch and one TM
// launch over (strip, row-segment) tiles; the tile, its row pipeline and its
// shared-memory layout are in pol_tile.cuh.  Grids with odd n_x launch the
// kernels of fused2d_pol_batch.cu, which also holds the batched step; they
// are kept apart because instantiating the tile's SEAM variant in this
// translation unit was measured to slow the even-n_x TE kernel by 11%.
#include <cuda_runtime.h>
#include <math.h>

#include "fused2d.h"
#include "pol_tile.cuh"

namespace fmx {
namespace {

using namespace pair2;
using pol2d::PolGeom;
using pol2d::pol_tile;

// rows per segment asked for by the caller of the current launch (0:
// automatic, see PolLauncher::shape), and whether its tiles prefetch their
// input rows into L1 (fused2d_l1_prefetch)
thread_local int t_rows = 0;
thread_local bool t_l1pf = false;

template <int POL, int M, int P, bool HJ, int NT, bool L1PF>
__global__ void __launch_bounds__(NT, 3)
    k_pol2d(Fused2dArgs<float> a, Geo g, Coef2 c, int W, int L, int nstrip) {
    extern __shared__ __align__(16) unsigned char smraw[];
    pol_tile<POL, M, P, HJ, NT, false, false, L1PF>(a, g, c, W, L, blockIdx.x % nstrip, blockIdx.x / nstrip,
                                                    reinterpret_cast<float *>(smraw));
}

template <int POL, int M, int P, bool HJ>
struct PolLauncher {
    static constexpr int NT = 128;
    static size_t smem_bytes() { return pol2d::smem_bytes<POL, M, P, HJ>(); }
    static int blocks_per_sm() {
        static int b = -1;
        if (b < 0) {
            auto k = k_pol2d<POL, M, P, HJ, NT, false>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
            cudaFuncSetAttribute(k_pol2d<POL, M, P, HJ, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes());
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, smem_bytes()) != cudaSuccess || n < 1) n = 1;
            b = n;
        }
        return b;
    }
    static Fused2dShape shape(const Geo &g) {
        using Gm = PolGeom<M, P, HJ>;
        Fused2dShape sh;
        sh.threads = NT;
        sh.halo = Gm::HC;
        sh.width = 2 * NT - 2 * Gm::HC - 2;
        sh.strips = (g.nx + sh.width - 1) / sh.width;
        static int sms = -1;
        if (sms < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        }
        // automatic: one wave of CTAs at the measured occupancy, but no
        // segment shorter than the rows its pipeline recomputes to warm up
        // (3m + 2p + 8): on small grids fewer, longer segments are faster
        // (1024^2, m = 4, p = 3: 12-row segments 38.6 us per step, 24-row 30.7)
        const int target = blocks_per_sm() * sms;
        int nseg = target / sh.strips;
        if (nseg < 1) nseg = 1;
        if (nseg > g.ny) nseg = g.ny;
        int rows = (g.ny + nseg - 1) / nseg;
        const int warm = 3 * M + 2 * (HJ ? P : 0) + 8;
        if (rows < warm) rows = warm;
        if (t_rows > 0) rows = t_rows;
        sh.rows = rows < g.ny ? rows : g.ny;
        sh.segments = (g.ny + sh.rows - 1) / sh.rows;
        return sh;
    }
    static void run(const Geo &g, const Coef2 &c, const Fused2dArgs<float> &a, cudaStream_t s) {
        const Fused2dShape sh = shape(g);
        if (g.nx % 2 == 0 && t_l1pf)
            k_pol2d<POL, M, P, HJ, NT, true><<<sh.strips * sh.segments, NT, smem_bytes(), s>>>(a, g, c, sh.width, sh.rows,
                                                                                              sh.strips);
        else if (g.nx % 2 == 0)
            k_pol2d<POL, M, P, HJ, NT, false><<<sh.strips * sh.segments, NT, smem_bytes(), s>>>(a, g, c, sh.width,
                                                                                               sh.rows, sh.strips);
        else
            pol2d::launch_odd<POL, M, P, HJ>(g, c, a, sh.width, sh.rows, sh.strips, sh.strips * sh.segments, s);
    }
};

// events (optional): ev[0] before the TE launch, ev[1] between, ev[2] after TM;
// the TM launch goes to t_tm when set
thread_local cudaEvent_t *t_ev = nullptr;
thread_local cudaStream_t t_tm = nullptr;

template <int M, int P, bool HJ>
int run_both(const Geo &g, const Coef2 &c, const Fused2dArgs<float> &a, cudaStream_t s, Fused2dShape *sh) {
    if (sh) {
        *sh = PolLauncher<TE, M, P, HJ>::shape(g);
        return 0;
    }
    if (t_ev) cudaEventRecord(t_ev[0], s);
    PolLauncher<TE, M, P, HJ>::run(g, c, a, s);
    if (t_ev) cudaEventRecord(t_ev[1], s);
    PolLauncher<TM, M, P, HJ>::run(g, c, a, t_tm ? t_tm : s);
    if (t_ev) cudaEventRecord(t_ev[2], s);
    return 2;
}

template <int M>
int pol_p(const Geo &g, const Coef2 &c, const Fused2dArgs<float> &a, cudaStream_t s, bool hj, int p,
          Fused2dShape *sh) {
    if (!hj) return run_both<M, 0, false>(g, c, a, s, sh);
    switch (p) {
        case 0: return run_both<M, 0, true>(g, c, a, s, sh);
        case 1: return run_both<M, 1, true>(g, c, a, s, sh);
        case 2: return run_both<M, 2, true>(g, c, a, s, sh);
        case 3: return run_both<M, 3, true>(g, c, a, s, sh);
    }
    return -1;
}

int pol_dispatch(const Geo &g, const Coef2 &c, const Fused2dArgs<float> &a, cudaStream_t s, int m, bool hj, int p,
                 Fused2dShape *sh) {
    switch (m) {
        case 0: return pol_p<0>(g, c, a, s, hj, p, sh);
        case 1: return pol_p<1>(g, c, a, s, hj, p, sh);
        case 2: return pol_p<2>(g, c, a, s, hj, p, sh);
        case 3: return pol_p<3>(g, c, a, s, hj, p, sh);
        case 4: return pol_p<4>(g, c, a, s, hj, p, sh);
    }
    return -1;
}

Coef2 make_coef2(const Coef<float> &c, int passes) { return pol2d::coef2_of(c, passes); }

}  // namespace

// 32-bit element offsets within one component (any n_x: strips of an odd-n_x
// grid that cross the periodic seam load their column pairs one column at a
// time)
bool fused2d_pol_supported(const Geo &g) { return (int64_t)g.ny * g.pitch < ((int64_t)1 << 31); }

bool fused2d_l1_prefetch(const Geo &g) {
    static long long l2 = -1;
    if (l2 < 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        l2 = cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) == cudaSuccess && v > 0 ? v : (1LL << 27);
    }
    return 60.0 * (double)g.nx * (double)g.ny > 1.5 * (double)l2;
}

int launch_fused2d_pol(const Geo &g, const Coef<float> &c, const Fused2dArgs<float> &a, cudaStream_t s,
                       cudaEvent_t *ev, cudaStream_t s_tm, int seg_rows) {
    const bool hj = a.J[0] != nullptr;
    const int p = hj ? a.passes : 0;
    if (c.c6 != 1.f / 6.f) return -1;  // the kernels use 1/6 as a compile-time constant
    t_ev = ev;
    t_tm = s_tm;
    t_rows = seg_rows;
    t_l1pf = fused2d_l1_prefetch(g);
    const int n = pol_dispatch(g, make_coef2(c, p), a, s, a.m, hj, p, nullptr);
    t_ev = nullptr;
    t_tm = nullptr;
    t_rows = 0;
    t_l1pf = false;
    return n;
}

Fused2dShape fused2d_pol_shape(const Geo &g, int m, int passes, int seg_rows) {
    Fused2dShape sh{0, 0, 0, 0, 0, 0};
    Fused2dArgs<float> a{};
    Coef<float> c{};
    t_rows = seg_rows;
    pol_dispatch(g, make_coef2(c, passes >= 0 ? passes : 0), a, nullptr, m, passes >= 0, passes >= 0 ? passes : 0,
                 &sh);
    t_rows = 0;
    return sh;
}

}  // namespace fmx
