// Resident engine: every step of an fmx_step call -- current filter, source,
// the whole solve of Algorithm 1 (fixed m or to the residual stop), E update
// and Faraday -- in ONE launch of one thread-block cluster, for grids small
// enough to live in L2 (the latency-bound case: a 64 x 64 FP64 grid has 4096
// cells, far too few to fill the GPU, and one host read-back per step cost
// more than the step).
//
// Each CTA of the cluster owns a contiguous range of cells (linear index,
// x fastest).  Phases are separated by the cluster's hardware barrier
// (barrier.cluster arrive.release / wait.acquire); field data other CTAs
// wrote is read through L2 (ld.global.cg), never from a stale L1 line.  The
// residual of a sweep is reduced in FP64: warp shuffles, then the warps of a
// CTA in a fixed order, then every CTA writes its partial into each CTA's
// shared memory (distributed shared memory) before the barrier, and every
// thread sums the cluster's partials in rank order.  All threads therefore
// hold bit-identical norms and take the same stop decision, so the control
// flow stays uniform across the cluster and every barrier is reached by all
// threads.  Nothing spins in software: the only waits are the hardware
// cluster barriers.
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

constexpr int kNT = 256;       // threads per CTA
constexpr int kMaxCluster = 16;

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

// Cluster-wide FP64 sum of v (every thread of every CTA calls it; every
// thread gets the same value).  xs: this CTA's [2][kMaxCluster] partial
// slots, alternated by `par` so that the next reduction never overwrites
// slots a slower CTA is still reading.
__device__ __forceinline__ double cluster_sum(cg::cluster_group &cl, double v, double *red, double *xs, int par) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int t = threadIdx.x;
    if ((t & 31) == 0) red[t >> 5] = v;
    __syncthreads();
    const int C = (int)cl.num_blocks();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < kNT / 32; ++w) s += red[w];
        const int me = (int)cl.block_rank();
        for (int r = 0; r < C; ++r) {
            double *dst = cl.map_shared_rank(xs + par * kMaxCluster, r);
            dst[me] = s;
        }
    }
    __threadfence();
    cl.sync();
    double tot = 0.0;
    for (int r = 0; r < C; ++r) tot += xs[par * kMaxCluster + r];
    return tot;
}

__device__ __forceinline__ void cluster_barrier(cg::cluster_group &cl) {
    __threadfence();
    cl.sync();
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
};

template <typename T, int DIM>
__global__ void __launch_bounds__(kNT) k_resident(ResidentArgs<T> a, Geo g) {
    cg::cluster_group cl = cg::this_cluster();
    __shared__ double red[kNT / 32];
    __shared__ double xs[2 * kMaxCluster];
    const int C = (int)cl.num_blocks(), b = (int)cl.block_rank();
    const int64_t N = (int64_t)g.nx * g.ny * g.nz;
    Cells cells{(int)(N * b / C), (int)(N * (b + 1) / C), g};
    const int t = threadIdx.x;
    StagedPtrs<T> &P = a.P;
    const Coef<T> &c = a.c;
    int par = 0;

    // the current: p binomial passes per active axis (axis order x, y, z, x, ...
    // as the staged filter), ping-ponging between tmp and jf so the last pass
    // lands in jf
    const T *jsrc[3] = {a.have_j ? P.J[0] : nullptr, a.have_j ? P.J[1] : nullptr, a.have_j ? P.J[2] : nullptr};
    if (a.have_j && a.jpasses > 0) {
        const int n = a.jpasses * DIM;
        for (int comp = 0; comp < 3; ++comp) {
            const T *src = P.J[comp];
            for (int q = 0; q < n; ++q) {
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
                cluster_barrier(cl);
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
    for (int n = 0; n < a.nsteps; ++n) {
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
            n2 = cluster_sum(cl, v, red, xs, par);
            par ^= 1;
        } else {
            cluster_barrier(cl);
        }
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
                r2 = cluster_sum(cl, w, red, xs, par);
                par ^= 1;
                if (r2 <= a.tol2 * n2) {
                    stop = true;
                } else if (s >= a.m_max) {
                    stop = true;
                    noconv = 1;
                }
            } else {
                cluster_barrier(cl);
                stop = s >= a.m;
            }
        }
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
            cluster_barrier(cl);
        }
        ++steps_done;
        if (noconv) break;
    }
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
    // cluster size: 16 CTAs where the device runs clusters of 16, else 8
    static int cluster() {
        static int cs = -1;
        if (cs < 0) {
            auto k = k_resident<T, DIM>;
            cs = 8;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeClusterDimension;
                at[0].val.clusterDim.x = 16;
                at[0].val.clusterDim.y = 1;
                at[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3(16);
                cfg.blockDim = dim3(kNT);
                cfg.attrs = at;
                cfg.numAttrs = 1;
                int n = 0;
                if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) cs = 16;
            }
            cudaGetLastError();
        }
        return cs;
    }
    static cudaError_t run(const Geo &g, const ResidentArgs<T> &a, cudaStream_t s) {
        const int cs = cluster();
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kNT);
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_resident<T, DIM>, a, g);
    }
};

}  // namespace

template <typename T>
int resident_cluster_size(int dims) {
    return dims == 3 ? ResidentLauncher<T, 3>::cluster()
                     : (dims == 2 ? ResidentLauncher<T, 2>::cluster() : ResidentLauncher<T, 1>::cluster());
}

template <typename T>
int launch_resident(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &P, int nsteps, bool resid, int m,
                    double tol2, int m_max, int jpasses, cudaStream_t s) {
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
    cudaError_t e = dims == 3 ? ResidentLauncher<T, 3>::run(g, a, s)
                              : (dims == 2 ? ResidentLauncher<T, 2>::run(g, a, s) : ResidentLauncher<T, 1>::run(g, a, s));
    return e == cudaSuccess ? 1 : -1;
}

template int resident_cluster_size<float>(int);
template int resident_cluster_size<double>(int);
template int launch_resident<float>(const Geo &, int, const Coef<float> &, const StagedPtrs<float> &, int, bool, int,
                                    double, int, int, cudaStream_t);
template int launch_resident<double>(const Geo &, int, const Coef<double> &, const StagedPtrs<double> &, int, bool,
                                     int, double, int, int, cudaStream_t);

}  // namespace fmx
