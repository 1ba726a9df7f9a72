// Resident engine: every step of an fmx_step call -- current filter, source,
// the whole solve of Algorithm 1 (fixed m or to the residual stop), E update
// and Faraday -- in ONE launch, for grids small enough to live in L2 (the
// latency-bound case: a 64 x 64 FP64 grid has 4096 cells, far too few to fill
// the GPU, and one host read-back per step cost more than the step).
//
// The launch is one thread-block cluster (16 CTAs where the device schedules
// clusters of 16, else 8, one CTA per SM) or, where the arithmetic needs more
// SMs (FP64 runs at 1/64 of the FP32 rate on this class of part: grids above
// ~4096 FP64 cells), up to 8 clusters in one cooperative launch (every CTA
// co-resident).  Each CTA owns a contiguous
// range of cells (linear index, x fastest).  Phases are separated by
//   - one cluster: the cluster's hardware barrier (barrier.cluster
//     arrive.release / wait.acquire);
//   - several clusters: a cluster barrier, then the cluster's leader thread
//     arrives at a grid barrier in global memory (an atomic arrival count and
//     a generation the last arrival advances with release semantics) and
//     waits for the generation to move with a bounded spin (a limit in SM
//     clock cycles, FMX_ETIMEOUT latched in the status word when it runs out,
//     a wait that gives up as soon as another cluster has), then a second
//     cluster barrier releases the cluster with the leader's verdict.
// Field data other CTAs wrote is read through L2 (ld.global.cg).  The
// residual of a sweep is reduced in FP64: warp shuffles, then the warps of a
// CTA in a fixed order, then every CTA writes its partial into each CTA of
// its cluster (distributed shared memory) and sums the cluster's partials in
// rank order; with several clusters each leader publishes its cluster's sum
// and every thread adds the clusters' sums in cluster order after the grid
// barrier.  All threads therefore hold bit-identical norms and take the same
// stop decision: control flow stays uniform and every barrier is reached by
// every thread (or every wait gives up within its limit).
//
// Arithmetic per cell is the staged engine's (stencil.cuh): source Eqs.
// ampere_aux_x..z, A of Eqs. matrixA_1st..matrixA_last, Algorithm 1, Eqs.
// faraday_x..z; residual ||dE_(s+1) - dE_(s)||_2 <= tol ||dE'||_2 with at
// least one sweep, none when dE' = 0, FMX_ENOCONV past m_max.
//
// Phase order of one step n (the E update of step n-1 is folded into step
// n's source phase: the source reads only B):
//   S  : E += dE_(n-1) (own cells; n > 0), dE' = c dt curl(alpha B) - q j_f,
//        ||dE'||^2                                                    | barrier
//   W_s: dE_(s+1) = dE' + A dE_(s), ||dE_(s+1) - dE_(s)||^2          | barrier
//   F  : B -= c dt curl(E + dE) (E^{n+1} formed on the fly)          | barrier
// and after the last step one more E += dE.  The current is filtered once per
// launch into the jf workspace (it is constant over the launch).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "fmx_internal.h"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace fmx {
namespace {

constexpr int kNT = 256;         // threads per CTA
constexpr int kMaxCluster = 16;  // CTAs per cluster
constexpr int kMaxClusters = 8;  // clusters per launch (DevStatus::xpart)

// value at a periodic shift, read through L2
template <typename T>
struct FieldL2 {
    const T *__restrict__ p;
    Geo g;
    __device__ __forceinline__ T operator()(Pos b, int dx, int dy, int dz) const {
        int x = wrapc(b.i + dx, g.nx), y = wrapc(b.j + dy, g.ny), z = wrapc(b.k + dz, g.nz);
        return __ldcg(p + (int64_t)z * g.plane + (int64_t)y * g.pitch + x);
    }
};

// E^{n+1} = E^n + dE at a periodic shift, rounded to T as the staged update stores it
template <typename T>
struct SumL2 {
    const T *__restrict__ e;
    const T *__restrict__ d;
    Geo g;
    __device__ __forceinline__ T operator()(Pos b, int dx, int dy, int dz) const {
        int x = wrapc(b.i + dx, g.nx), y = wrapc(b.j + dy, g.ny), z = wrapc(b.k + dz, g.nz);
        const int64_t o = (int64_t)z * g.plane + (int64_t)y * g.pitch + x;
        return __ldcg(e + o) + __ldcg(d + o);
    }
};

struct Cells {
    int lo, hi;  // linear cell range of this CTA
    Geo g;
    __device__ __forceinline__ void at(int q, Pos &p, int64_t &idx) const {
        p.i = q % g.nx;
        const int r = q / g.nx;
        p.j = r % g.ny;
        p.k = r / g.ny;
        idx = (int64_t)p.k * g.plane + (int64_t)p.j * g.pitch + p.i;
    }
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The phase barrier of a launch (see the file comment).  Every thread calls
// barrier(); it returns false once the launch has given up (a grid wait ran
// out), after which every thread leaves its loops.
struct Sync {
    cg::cluster_group cl;
    DevStatus *st;
    int ncl, cid, crank;
    long long limit;  // SM clock cycles a leader waits at the grid barrier
    int lost;         // self-test: the grid barrier expects one arrival more than come
    int *abort_s;     // this CTA's copy of the leader's verdict (shared memory)

    __device__ bool grid() const { return ncl > 1 || lost; }

    // the leader's arrival and bounded wait at the grid barrier: 1 when every
    // cluster arrived, 0 when the wait ran out or another cluster gave up
    __device__ int grid_wait() const {
        const unsigned target = (unsigned)(ncl + lost);
        const unsigned g0 = ld_acquire_gpu(&st->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&st->bar_count, 1u) + 1u;
        if (arrived == target) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            st_release_gpu(&st->bar_gen, g0 + 1u);
            return 1;
        }
        const long long t0 = clock64();
        while (ld_acquire_gpu(&st->bar_gen) == g0) {
            if (ld_relaxed_gpu(&st->err) != 0) return 0;
            if (clock64() - t0 > limit) {
                atomicCAS(&st->err, 0, (int)FMX_ETIMEOUT);
                return 0;
            }
            __nanosleep(64);
        }
        return 1;
    }

    __device__ bool barrier() const {
        if (!grid()) {
            cl.sync();
            return true;
        }
        __threadfence();
        cl.sync();  // the cluster's phase is done
        if (crank == 0 && threadIdx.x == 0) {
            const int verdict = grid_wait() ? 0 : 1;
            for (int r = 0; r < (int)cl.num_blocks(); ++r) *cl.map_shared_rank(abort_s, r) = verdict;
        }
        cl.sync();  // every cluster's phase is done (or the launch gave up)
        return *abort_s == 0;
    }
};

// Launch-wide FP64 sum of v (every thread calls it and gets the same value,
// or ok = false when the launch gave up).  xs: this CTA's [2][kMaxCluster]
// partial slots, alternated by `par` so that the next reduction never
// overwrites slots (or DevStatus::xpart entries) a slower CTA still reads.
__device__ __forceinline__ double launch_sum(const Sync &S, double v, double *red, double *xs, int par, bool &ok) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int t = threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    const int C = (int)S.cl.num_blocks();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kNT / 32; ++w) s += red[w];
        for (int r = 0; r < C; ++r) S.cl.map_shared_rank(xs + par * kMaxCluster, r)[S.crank] = s;
    }
    S.cl.sync();
    double tot = 0.0;
    for (int r = 0; r < C; ++r) tot += xs[par * kMaxCluster + r];
    if (!S.grid()) {
        ok = true;
        return tot;
    }
    if (S.crank == 0 && t == 0) __stcg(&S.st->xpart[par][S.cid], tot);
    ok = S.barrier();
    if (!ok) return 0.0;
    double all = 0.0;
    for (int k = 0; k < S.ncl; ++k) all += __ldcg(&S.st->xpart[par][k]);
    return all;
}

template <typename T>
struct ResidentArgs {
    StagedPtrs<T> P;   // E, B in place; J raw; jf, tmp, dEp, dEa, dEb workspace
    Coef<T> c;
    int nsteps;
    int resid;         // 1: Algorithm 1 to the residual stop; 0: m sweeps
    int m, m_max;
    double tol2;
    int jpasses;       // current filter passes per active axis (0: j used as is)
    int have_j;
    long long limit;   // grid-barrier wait limit, SM clock cycles
    int lost;          // self-test of the wait's time-out
};

template <typename T, int DIM>
__global__ void __launch_bounds__(kNT) k_resident(ResidentArgs<T> a, Geo g) {
    __shared__ double red[kNT / 32];
    __shared__ double xs[2 * kMaxCluster];
    __shared__ int abort_s;
    Sync S{cg::this_cluster(), a.P.st, 0, 0, 0, a.limit, a.lost, &abort_s};
    const int C = (int)S.cl.num_blocks();
    S.crank = (int)S.cl.block_rank();
    S.ncl = (int)(gridDim.x / C);
    S.cid = (int)(blockIdx.x / C);  // the clusters tile the 1D grid in order
    const int b = S.cid * C + S.crank, NB = S.ncl * C;
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    Cells cells{(int)(N * b / NB), (int)(N * (b + 1) / NB), g};
    const int t = threadIdx.x;
    StagedPtrs<T> &P = a.P;
    const Coef<T> &c = a.c;
    int par = 0;
    bool ok = true;

    // the current: p binomial passes per active axis (axis order x, y, z, x, ...
    // as the staged filter), ping-ponging between tmp and jf so the last pass
    // lands in jf
    const T *jsrc[3] = {a.have_j ? P.J[0] : nullptr, a.have_j ? P.J[1] : nullptr, a.have_j ? P.J[2] : nullptr};
    if (a.have_j && a.jpasses > 0) {
        const int n = a.jpasses * DIM;
        for (int comp = 0; comp < 3 && ok; ++comp) {
            const T *src = P.J[comp];
            for (int q = 0; q < n && ok; ++q) {
                T *dst = ((n - 1 - q) % 2 == 0) ? P.jf[comp] : P.tmp;
                const int axis = q % DIM;
                FieldL2<T> f{src, g};
                int dx, dy, dz;
                unit(axis, 1, dx, dy, dz);
                for (int qq = cells.lo + t; qq < cells.hi; qq += kNT) {
                    Pos p;
                    int64_t idx;
                    cells.at(qq, p, idx);
                    dst[idx] = T(0.25) * f(p, -dx, -dy, -dz) + T(0.5) * f(p, 0, 0, 0) + T(0.25) * f(p, dx, dy, dz);
                }
                ok = S.barrier();
                src = dst;
            }
            jsrc[comp] = P.jf[comp];
        }
    }

    const T *dfin[3] = {nullptr, nullptr, nullptr};  // dE of the previous step (E update pending)
    int last = 0, steps_done = 0, noconv = 0;
    long long total = 0;
    double n2 = 0.0, r2 = 0.0;
    FieldL2<T> bf[3] = {{P.B[0], g}, {P.B[1], g}, {P.B[2], g}};
    for (int n = 0; n < a.nsteps && ok; ++n) {
        // ---- S: pending E update, source, ||dE'||^2
        double v = 0.0;
        for (int q = cells.lo + t; q < cells.hi; q += kNT) {
            Pos p;
            int64_t idx;
            cells.at(q, p, idx);
            if (dfin[0]) {
#pragma unroll
                for (int k = 0; k < 3; ++k) P.E[k][idx] = __ldcg(P.E[k] + idx) + __ldcg(dfin[k] + idx);
            }
            T ex = curl_alpha_b<T, DIM, 0>(bf, p, c);
            T ey = curl_alpha_b<T, DIM, 1>(bf, p, c);
            T ez = curl_alpha_b<T, DIM, 2>(bf, p, c);
            if (jsrc[0]) ex -= c.q * __ldcg(jsrc[0] + idx);
            if (jsrc[1]) ey -= c.q * __ldcg(jsrc[1] + idx);
            if (jsrc[2]) ez -= c.q * __ldcg(jsrc[2] + idx);
            P.dEp[0][idx] = ex;
            P.dEp[1][idx] = ey;
            P.dEp[2][idx] = ez;
            v += (double)ex * ex + (double)ey * ey + (double)ez * ez;
        }
        if (a.resid) {
            n2 = launch_sum(S, v, red, xs, par, ok);
            par ^= 1;
        } else {
            ok = S.barrier();
        }
        if (!ok) break;
        // ---- W_s: sweeps of Algorithm 1
        int s = 0;
        bool stop = a.resid ? n2 == 0.0 : a.m == 0;
        while (!stop) {
            const T *in[3];
            T *out[3];
            for (int k = 0; k < 3; ++k) {
                in[k] = s == 0 ? P.dEp[k] : ((s & 1) ? P.dEa[k] : P.dEb[k]);
                out[k] = ((s + 1) & 1) ? P.dEa[k] : P.dEb[k];
            }
            FieldL2<T> f[3] = {{in[0], g}, {in[1], g}, {in[2], g}};
            double w = 0.0;
            for (int q = cells.lo + t; q < cells.hi; q += kNT) {
                Pos p;
                int64_t idx;
                cells.at(q, p, idx);
                const T nx_ = __ldcg(P.dEp[0] + idx) + apply_a<T, DIM, 0>(f, p, c);
                const T ny_ = __ldcg(P.dEp[1] + idx) + apply_a<T, DIM, 1>(f, p, c);
                const T nz_ = __ldcg(P.dEp[2] + idx) + apply_a<T, DIM, 2>(f, p, c);
                const T dx = nx_ - __ldcg(in[0] + idx), dy = ny_ - __ldcg(in[1] + idx),
                        dz = nz_ - __ldcg(in[2] + idx);
                out[0][idx] = nx_;
                out[1][idx] = ny_;
                out[2][idx] = nz_;
                w += (double)dx * dx + (double)dy * dy + (double)dz * dz;
            }
            ++s;
            if (a.resid) {
                r2 = launch_sum(S, w, red, xs, par, ok);
                par ^= 1;
                if (!ok) break;
                if (r2 <= a.tol2 * n2) {
                    stop = true;
                } else if (s >= a.m_max) {
                    stop = true;
                    noconv = 1;
                }
            } else {
                ok = S.barrier();
                if (!ok) break;
                stop = s >= a.m;
            }
        }
        if (!ok) break;
        for (int k = 0; k < 3; ++k) dfin[k] = s == 0 ? P.dEp[k] : ((s & 1) ? P.dEa[k] : P.dEb[k]);
        last = s;
        total += s;
        // ---- F: Faraday with E^{n+1} = E^n + dE formed on the fly
        {
            SumL2<T> e[3] = {{P.E[0], dfin[0], g}, {P.E[1], dfin[1], g}, {P.E[2], dfin[2], g}};
            for (int q = cells.lo + t; q < cells.hi; q += kNT) {
                Pos p;
                int64_t idx;
                cells.at(q, p, idx);
                const T c0 = curl_e<T, DIM, 0>(e, p, c), c1 = curl_e<T, DIM, 1>(e, p, c),
                        c2 = curl_e<T, DIM, 2>(e, p, c);
                P.B[0][idx] = __ldcg(P.B[0] + idx) - c0;
                P.B[1][idx] = __ldcg(P.B[1] + idx) - c1;
                P.B[2][idx] = __ldcg(P.B[2] + idx) - c2;
            }
            ok = S.barrier();
        }
        if (!ok) break;
        ++steps_done;
        if (noconv) break;
    }
    if (!ok) return;  // a grid wait ran out: FMX_ETIMEOUT is latched in the status word
    // the last step's E update (everyone has passed the Faraday barrier)
    if (dfin[0]) {
        for (int q = cells.lo + t; q < cells.hi; q += kNT) {
            Pos p;
            int64_t idx;
            cells.at(q, p, idx);
#pragma unroll
            for (int k = 0; k < 3; ++k) P.E[k][idx] = __ldcg(P.E[k] + idx) + __ldcg(dfin[k] + idx);
        }
    }
    if (b == 0 && t == 0) {
        DevStatus *st = P.st;
        st->nrm2 = n2;
        st->r2 = r2;
        st->count = last;
        st->done = 1;
        st->noconv = noconv;
        st->steps = steps_done;
        st->sweeps_total = total;
    }
}

template <typename T, int DIM>
struct ResidentLauncher {
    // dynamic shared memory (unused) of more than half an SM's: one CTA per SM,
    // so that a cluster's CTAs spread over as many SMs (and FP64 pipes) as it has
    static size_t spread_bytes() {
        static size_t b = (size_t)-1;
        if (b == (size_t)-1) {
            int dev = 0, per_sm = 0, per_block = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&per_block, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
            size_t want = (size_t)per_sm / 2 + 1024;
            if (want > (size_t)per_block) want = 0;
            if (want > 0 &&
                cudaFuncSetAttribute(k_resident<T, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want) !=
                    cudaSuccess)
                want = 0;
            cudaGetLastError();
            b = want;
        }
        return b;
    }
    static cudaLaunchAttribute cluster_attr(int cs) {
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeClusterDimension;
        at.val.clusterDim.x = cs;
        at.val.clusterDim.y = 1;
        at.val.clusterDim.z = 1;
        return at;
    }
    // cluster size: 16 CTAs where the device runs clusters of 16, else 8
    static int cluster() {
        static int cs = -1;
        if (cs < 0) {
            auto k = k_resident<T, DIM>;
            cs = 8;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute at[1] = {cluster_attr(16)};
                cfg.gridDim = dim3(16);
                cfg.blockDim = dim3(kNT);
                cfg.dynamicSmemBytes = spread_bytes();
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) cs = 16;
            }
            cudaGetLastError();
        }
        return cs;
    }
    // clusters the device can hold at once (cooperative launches need them all
    // resident), capped by the status word's partial slots
    static int max_clusters() {
        static int mc = -1;
        if (mc < 0) {
            const int cs = cluster();
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1] = {cluster_attr(cs)};
            cfg.gridDim = dim3(cs);
            cfg.blockDim = dim3(kNT);
            cfg.dynamicSmemBytes = spread_bytes();
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, k_resident<T, DIM>, &cfg) != cudaSuccess || n < 1) n = 1;
            cudaGetLastError();
            mc = n < kMaxClusters ? n : kMaxClusters;
        }
        return mc;
    }
    // set once a cooperative launch over clusters has been refused
    static bool &coop_refused() {
        static bool r = false;
        return r;
    }
    // A grid barrier costs ~3 us per phase (an L2 atomic round trip and a
    // poll); another cluster pays when it takes more FP64 work off the
    // cluster's SMs than that.  Measured (FP64, Algorithm 1 to 1e-13): 64^2,
    // one cluster 0.090 ms per step, four 0.133; 128^2, one 0.161, two 0.126,
    // four 0.097, seven 0.108.  So about 256 cells per CTA in FP64; FP32
    // arithmetic is 64x cheaper.
    static int clusters_for(int64_t cells, bool lost) {
        if (coop_refused()) return 1;
        const int64_t per_cta = sizeof(T) == 8 ? 256 : 4096;
        const int64_t want = (cells + per_cta * cluster() - 1) / (per_cta * cluster());
        int n = (int)(want < 1 ? 1 : want);
        const int mc = max_clusters();
        if (n > mc) n = mc;
        (void)lost;
        return n;
    }
    static cudaError_t run(const Geo &g, const ResidentArgs<T> &a, int &ncl, cudaStream_t s) {
        const int cs = cluster();
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2] = {cluster_attr(cs), {}};
        at[1].id = cudaLaunchAttributeCooperative;
        at[1].val.cooperative = 1;
        cfg.gridDim = dim3(cs * ncl);
        cfg.blockDim = dim3(kNT);
        cfg.dynamicSmemBytes = spread_bytes();
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = ncl > 1 ? 2 : 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_resident<T, DIM>, a, g);
        if (e != cudaSuccess && ncl > 1) {
            // this device or driver does not co-schedule clusters cooperatively:
            // one cluster from now on
            cudaGetLastError();
            coop_refused() = true;
            ncl = 1;
            cfg.gridDim = dim3(cs);
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, k_resident<T, DIM>, a, g);
        }
        return e;
    }
};

}  // namespace

template <typename T>
int resident_cluster_size(int dims) {
    return dims == 3 ? ResidentLauncher<T, 3>::cluster()
                     : (dims == 2 ? ResidentLauncher<T, 2>::cluster() : ResidentLauncher<T, 1>::cluster());
}

template <typename T>
int resident_clusters(int dims, int64_t cells, bool lost_arrival) {
    return dims == 3 ? ResidentLauncher<T, 3>::clusters_for(cells, lost_arrival)
                     : (dims == 2 ? ResidentLauncher<T, 2>::clusters_for(cells, lost_arrival)
                                  : ResidentLauncher<T, 1>::clusters_for(cells, lost_arrival));
}

template <typename T>
int launch_resident(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &P, int nsteps, bool resid, int m,
                    double tol2, int m_max, int jpasses, const ResidentWait &wait, cudaStream_t s) {
    ResidentArgs<T> a;
    a.P = P;
    a.c = c;
    a.nsteps = nsteps;
    a.resid = resid ? 1 : 0;
    a.m = m;
    a.m_max = m_max;
    a.tol2 = tol2;
    a.jpasses = jpasses;
    a.have_j = P.J[0] != nullptr;
    a.limit = wait.limit_cycles;
    a.lost = wait.lost_arrival ? 1 : 0;
    const int64_t cells = (int64_t)g.nx * g.ny * g.nz;
    int ncl = resident_clusters<T>(dims, cells, a.lost != 0);
    cudaError_t e = dims == 3 ? ResidentLauncher<T, 3>::run(g, a, ncl, s)
                              : (dims == 2 ? ResidentLauncher<T, 2>::run(g, a, ncl, s)
                                           : ResidentLauncher<T, 1>::run(g, a, ncl, s));
    return e == cudaSuccess ? ncl : -1;
}

template int resident_cluster_size<float>(int);
template int resident_cluster_size<double>(int);
template int resident_clusters<float>(int, int64_t, bool);
template int resident_clusters<double>(int, int64_t, bool);
template int launch_resident<float>(const Geo &, int, const Coef<float> &, const StagedPtrs<float> &, int, bool, int,
                                    double, int, int, const ResidentWait &, cudaStream_t);
template int launch_resident<double>(const Geo &, int, const Coef<double> &, const StagedPtrs<double> &, int, bool,
                                     int, double, int, int, const ResidentWait &, cudaStream_t);

}  // namespace fmx
