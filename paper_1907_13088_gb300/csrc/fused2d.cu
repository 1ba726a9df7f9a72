// Fused 2D step of the averaged-Yee scheme (arXiv:1907.13088, Sec. 2.2.2).
//
// One launch advances the whole grid by one step.  A CTA owns a strip of NT
// consecutive columns (one column per thread, periodic in x) and marches up
// a segment of rows.  Every stage of the step is a row pipeline stage:
//
//   J   : raw current row r+1+P -> y-binomial (2P+1 taps, registers) -> jy
//   Bp  : B row r+2 -> alpha_y B_y (registers) ; Bx, Bz, alpha_y B_y -> smem
//   S0  : source row r: x-binomial of jy, dE' (Eqs. ampere_aux_x..z, 2D)
//   S_s : sweep s = 1..M of Algorithm 1 on row r - 2s (A of Eqs.
//         matrixA_1st_2d..matrixA_last_2d)
//   E   : E^{n+1} = E^n + dE_(M) on row r - 2M
//   F   : Faraday update (Eqs. faraday_x..z, 2D) on row r - 2M - 1
//
// Stage s reads the outputs of stage s-1 from the three previous iterations
// only, so one __syncthreads per row is enough.  A thread's own column of
// each stage's recent outputs is kept in registers (the y-neighbours); the
// x-neighbours go through shared-memory row rings.  Only E, B and j are
// read from HBM and only E^{n+1}, B^{n+3/2} written: 60 bytes per cell and
// step in FP32 with a current (48 without).  The columns of the x-halo and
// the warm-up rows of a segment are recomputed, never exchanged.
#include <cuda_runtime.h>

#include "fused2d.h"

namespace fmx {
namespace {

// binomial weight C(2P, k) / 4^P of the P-pass (1/4, 1/2, 1/4) filter
__host__ __device__ constexpr double binom_w(int P, int k) {
    double c = 1.0;
    for (int i = 0; i < k; ++i) c = c * (2 * P - i) / (i + 1);
    double d = 1.0;
    for (int i = 0; i < P; ++i) d *= 4.0;
    return c / d;
}

template <typename T>
struct Cfg {
    static constexpr int NT = sizeof(T) == 4 ? 256 : 128;
};

template <int M, int P, bool HJ>
struct Geom {
    static constexpr int PX = (HJ && P > 1) ? P : 1;  // smem row padding
    static constexpr int H = PX + M;                  // left halo of the strip
    static constexpr int D0 = (2 * M + 1) > 4 ? (2 * M + 1) : 4;  // dE' ring depth
    static constexpr int NS = M > 1 ? M - 1 : 0;      // rings of sweeps 1..M-1
    static constexpr int TJ = HJ ? 2 * P + 1 : 1;     // y-filter taps
    static constexpr int WU = TJ > 3 ? TJ : 3;        // warm-up of the current/B chain
};

template <typename T, int M, int P, bool HJ, int NT>
__host__ __device__ constexpr size_t smem_elems() {
    using G = Geom<M, P, HJ>;
    constexpr size_t RW = NT + 2 * G::PX;
    return RW * ((HJ ? 2 * 3 : 0) + 4 + 4 + 2 + G::D0 * 3 + G::NS * 4 * 3 + 2 * 2);
}

__device__ __forceinline__ int wrap_row(int r, int n) {
    int y = r % n;
    return y < 0 ? y + n : y;
}

template <int D>
__device__ __forceinline__ int ring(int r) {
    int q = r % D;
    return q < 0 ? q + D : q;
}

// One tile: columns [strip W, strip W + W) and rows [seg L, seg L + L) of the
// output, with the x-halo and warm-up rows recomputed.  Ends after a barrier,
// so a persistent caller may start another tile right away.
template <typename T, int M, int P, bool HJ, int NT>
__device__ __forceinline__ void fused2d_tile(const Fused2dArgs<T> &a, const Geo &g, const Coef<T> &c, int W, int L,
                                             int strip, int seg) {
    using G = Geom<M, P, HJ>;
    constexpr int PX = G::PX, H = G::H, D0 = G::D0, NS = G::NS, TJ = G::TJ;
    constexpr int RW = NT + 2 * PX;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);
    T *s_jy = sm;                                  // [2][3][RW]
    T *s_bx = s_jy + (HJ ? 2 * 3 * RW : 0);        // [4][RW]
    T *s_bz = s_bx + 4 * RW;                       // [4][RW]
    T *s_ay = s_bz + 4 * RW;                       // [2][RW]   alpha_y B_y
    T *s_dp = s_ay + 2 * RW;                       // [D0][3][RW] dE'
    T *s_sw = s_dp + D0 * 3 * RW;                  // [NS][4][3][RW]
    T *s_e = s_sw + NS * 4 * 3 * RW;               // [2][2][RW]  Ey, Ez of E^{n+1}
    constexpr int total = (int)smem_elems<T, M, P, HJ, NT>();

    const int tid = threadIdx.x;
    for (int q = tid; q < total; q += NT) sm[q] = T(0);

    const int x0 = strip * W;
    const int y0 = seg * L;
    const int y1 = min(y0 + L, g.ny);
    const int xg = x0 - H + tid;
    int xc = xg % g.nx;
    if (xc < 0) xc += g.nx;
    const bool xout = tid >= H && tid < H + W && xg < g.nx;
    const int col = tid + PX;

    const T *__restrict__ Ex = a.E[0];
    const T *__restrict__ Ey = a.E[1];
    const T *__restrict__ Ez = a.E[2];
    const T *__restrict__ Bx = a.B[0];
    const T *__restrict__ By = a.B[1];
    const T *__restrict__ Bz = a.B[2];
    const T *__restrict__ Jx = a.J[0];
    const T *__restrict__ Jy = a.J[1];
    const T *__restrict__ Jz = a.J[2];

    const int r0 = y0 - M - G::WU - 1;
    const int r1 = y1 + 2 * M + 1;

    // register state
    T jw[3][TJ];        // raw current, own column, rows r+1+P (0) .. r+1-P
    T byw[3];           // By rows r+2, r+1, r
    T bz_prev = T(0), axbx_prev = T(0);
    T win[M > 0 ? M : 1][3][3];  // stage s input: outputs of s-1 at t-1, t-2, t-3
    T dxx[M > 0 ? M : 1][3];     // Dbar_xx dEz of stage s-1 at rows rho+1, rho, rho-1
    T hh[M > 0 ? M : 1][2];      // Dbar_x dEx (backward) at rows rho+1, rho
    T en[3], enp[3];             // E^{n+1} own column, current and previous row
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int k = 0; k < TJ; ++k) jw[q][k] = T(0);
        byw[q] = T(0);
        en[q] = enp[q] = T(0);
    }
#pragma unroll
    for (int s = 0; s < (M > 0 ? M : 1); ++s) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
#pragma unroll
            for (int k = 0; k < 3; ++k) win[s][q][k] = T(0);
            dxx[s][q] = T(0);
        }
        hh[s][0] = hh[s][1] = T(0);
    }

    // prefetched own-column loads for the current iteration
    T pj[3] = {T(0), T(0), T(0)}, pb[3], pe[3], pf[3];
    auto load_row = [&](int r, T out_j[3], T out_b[3], T out_e[3], T out_f[3]) {
        const int64_t oj = (int64_t)wrap_row(r + 1 + P, g.ny) * g.pitch + xc;
        const int64_t ob = (int64_t)wrap_row(r + 2, g.ny) * g.pitch + xc;
        const int64_t oe = (int64_t)wrap_row(r - 2 * M, g.ny) * g.pitch + xc;
        const int64_t of = (int64_t)wrap_row(r - 2 * M - 1, g.ny) * g.pitch + xc;
        if (HJ) {
            out_j[0] = __ldg(Jx + oj);
            out_j[1] = __ldg(Jy + oj);
            out_j[2] = __ldg(Jz + oj);
        }
        out_b[0] = __ldg(Bx + ob);
        out_b[1] = __ldg(By + ob);
        out_b[2] = __ldg(Bz + ob);
        out_e[0] = __ldg(Ex + oe);
        out_e[1] = __ldg(Ey + oe);
        out_e[2] = __ldg(Ez + oe);
        out_f[0] = __ldg(Bx + of);
        out_f[1] = __ldg(By + of);
        out_f[2] = __ldg(Bz + of);
    };
    load_row(r0, pj, pb, pe, pf);
    __syncthreads();

    for (int r = r0; r < r1; ++r) {
        // current iteration's inputs; issue next iteration's loads
        T cj[3], cb[3], ce[3], cf[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            cj[q] = pj[q];
            cb[q] = pb[q];
            ce[q] = pe[q];
            cf[q] = pf[q];
        }
        if (r + 1 < r1) load_row(r + 1, pj, pb, pe, pf);

        const int rhoM = r - 2 * M;  // row of the last sweep and of the E update
        const int rhoF = rhoM - 1;   // row of the Faraday update
        T oM[3];                     // output of stage M on row rhoM

        // ---------------- sweeps M..1 (decreasing, so windows still hold t-1) --------
#pragma unroll
        for (int s = M; s >= 1; --s) {
            const int rho = r - 2 * s;
            // ring of stage s-1 (dE' for s = 1)
            const T *rx_p1, *ry_0, *ry_m1, *rz_p1;  // rows rho+1 (Ex, Ez), rho, rho-1 (Ey)
            if (s == 1) {
                rx_p1 = s_dp + (ring<D0>(rho + 1) * 3 + 0) * RW;
                ry_0 = s_dp + (ring<D0>(rho) * 3 + 1) * RW;
                ry_m1 = s_dp + (ring<D0>(rho - 1) * 3 + 1) * RW;
                rz_p1 = s_dp + (ring<D0>(rho + 1) * 3 + 2) * RW;
            } else {
                const T *base = s_sw + (s - 2) * 4 * 3 * RW;
                rx_p1 = base + (((rho + 1) & 3) * 3 + 0) * RW;
                ry_0 = base + ((rho & 3) * 3 + 1) * RW;
                ry_m1 = base + (((rho - 1) & 3) * 3 + 1) * RW;
                rz_p1 = base + (((rho + 1) & 3) * 3 + 2) * RW;
            }
            T(&X)[3] = win[s - 1][0];
            T(&Y)[3] = win[s - 1][1];
            T(&Z)[3] = win[s - 1][2];
            const T eym = ry_0[col - 1], eyp = ry_0[col + 1], eyp_m1 = ry_m1[col + 1];
            const T exm = rx_p1[col - 1];
            const T ezm = rz_p1[col - 1], ezp = rz_p1[col + 1];
            // windows of derived differences: new row rho+1
            dxx[s - 1][2] = dxx[s - 1][1];
            dxx[s - 1][1] = dxx[s - 1][0];
            dxx[s - 1][0] = ezp - T(2) * Z[0] + ezm;
            hh[s - 1][1] = hh[s - 1][0];
            hh[s - 1][0] = X[0] - exm;
            const T *dp = s_dp + ring<D0>(rho) * 3 * RW;
            const T px = dp[col], py = dp[RW + col], pz = dp[2 * RW + col];
            const T g_own = Y[1] - Y[2];
            const T g_nb = eyp - eyp_m1;
            const T *D = dxx[s - 1];
            T nx_ = px + c.ay * (X[0] - T(2) * X[1] + X[2]) + c.bxy * (g_nb - g_own);
            T ny_ = py + c.ax * (eyp - T(2) * Y[1] + eym) + c.bxy * (hh[s - 1][0] - hh[s - 1][1]);
            T nz_ = pz + c.ax * D[1] + c.ay * (Z[0] - T(2) * Z[1] + Z[2]) + c.axy * (D[0] - T(2) * D[1] + D[2]);
            if (s == M) {
                oM[0] = nx_;
                oM[1] = ny_;
                oM[2] = nz_;
            } else {
                T *o = s_sw + (s - 1) * 4 * 3 * RW + (rho & 3) * 3 * RW;
                o[col] = nx_;
                o[RW + col] = ny_;
                o[2 * RW + col] = nz_;
                // push into the window of stage s+1
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    win[s][q][2] = win[s][q][1];
                    win[s][q][1] = win[s][q][0];
                }
                win[s][0][0] = nx_;
                win[s][1][0] = ny_;
                win[s][2][0] = nz_;
            }
            if (s == M) {
                // ---------------- E update and Faraday ----------------
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    enp[q] = en[q];
                    en[q] = ce[q] + oM[q];
                }
                const bool yE = rhoM >= y0 && rhoM < y1;
                if (yE && xout) {
                    const int64_t o = (int64_t)rhoM * g.pitch + xc;
                    a.Eo[0][o] = en[0];
                    a.Eo[1][o] = en[1];
                    a.Eo[2][o] = en[2];
                }
                T *se = s_e + (rhoM & 1) * 2 * RW;
                se[col] = en[1];
                se[RW + col] = en[2];
                const T *sf = s_e + (rhoF & 1) * 2 * RW;
                const T ey_p = sf[col + 1], ez_p = sf[RW + col + 1];
                T bx_ = cf[0] - c.ky * (en[2] - enp[2]);
                T by_ = cf[1] + c.kx * (ez_p - enp[2]);
                T bz_ = cf[2] - c.kx * (ey_p - enp[1]) + c.ky * (en[0] - enp[0]);
                const bool yF = rhoF >= y0 && rhoF < y1;
                if (yF && xout) {
                    const int64_t o = (int64_t)rhoF * g.pitch + xc;
                    a.Bo[0][o] = bx_;
                    a.Bo[1][o] = by_;
                    a.Bo[2][o] = bz_;
                }
            }
        }

        // ---------------- source, row r ----------------
        {
            T jf[3] = {T(0), T(0), T(0)};
            if (HJ) {
                const T *jr = s_jy + (r & 1) * 3 * RW;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    T acc = T(0);
#pragma unroll
                    for (int k = 0; k < 2 * P + 1; ++k) acc += T(binom_w(P, k)) * jr[q * RW + col + k - P];
                    jf[q] = acc;
                }
            }
            const T *sbx = s_bx + (r & 3) * RW;
            const T *sbz = s_bz + (r & 3) * RW;
            const T *say = s_ay + (r & 1) * RW;
            const T bx0 = sbx[col];
            const T axbx = bx0 + c.c6 * (sbx[col + 1] - T(2) * bx0 + sbx[col - 1]);
            const T bz0 = sbz[col], bzm = sbz[col - 1];
            const T ay0 = say[col], aym = say[col - 1];
            T ex_ = c.ky * (bz0 - bz_prev);
            T ey_ = -(c.kx * (bz0 - bzm));
            T ez_ = c.kx * (ay0 - aym) - c.ky * (axbx - axbx_prev);
            if (HJ) {
                ex_ -= c.q * jf[0];
                ey_ -= c.q * jf[1];
                ez_ -= c.q * jf[2];
            }
            bz_prev = bz0;
            axbx_prev = axbx;
            T *dp = s_dp + ring<D0>(r) * 3 * RW;
            dp[col] = ex_;
            dp[RW + col] = ey_;
            dp[2 * RW + col] = ez_;
            if (M > 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    win[0][q][2] = win[0][q][1];
                    win[0][q][1] = win[0][q][0];
                }
                win[0][0][0] = ex_;
                win[0][1][0] = ey_;
                win[0][2][0] = ez_;
            } else {
                // no sweeps: dE = dE' feeds the E update directly
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    enp[q] = en[q];
                }
                en[0] = ce[0] + ex_;
                en[1] = ce[1] + ey_;
                en[2] = ce[2] + ez_;
                const bool yE = rhoM >= y0 && rhoM < y1;
                if (yE && xout) {
                    const int64_t o = (int64_t)rhoM * g.pitch + xc;
                    a.Eo[0][o] = en[0];
                    a.Eo[1][o] = en[1];
                    a.Eo[2][o] = en[2];
                }
                T *se = s_e + (rhoM & 1) * 2 * RW;
                se[col] = en[1];
                se[RW + col] = en[2];
                const T *sf = s_e + (rhoF & 1) * 2 * RW;
                const T ey_p = sf[col + 1], ez_p = sf[RW + col + 1];
                T bx_ = cf[0] - c.ky * (en[2] - enp[2]);
                T by_ = cf[1] + c.kx * (ez_p - enp[2]);
                T bz_ = cf[2] - c.kx * (ey_p - enp[1]) + c.ky * (en[0] - enp[0]);
                const bool yF = rhoF >= y0 && rhoF < y1;
                if (yF && xout) {
                    const int64_t o = (int64_t)rhoF * g.pitch + xc;
                    a.Bo[0][o] = bx_;
                    a.Bo[1][o] = by_;
                    a.Bo[2][o] = bz_;
                }
            }
        }

        // ---------------- current: y-binomial of row r+1 ----------------
        if (HJ) {
            T *jo = s_jy + ((r + 1) & 1) * 3 * RW;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
#pragma unroll
                for (int k = TJ - 1; k > 0; --k) jw[q][k] = jw[q][k - 1];
                jw[q][0] = cj[q];
                T acc = T(0);
#pragma unroll
                for (int k = 0; k < TJ; ++k) acc += T(binom_w(P, k)) * jw[q][k];
                jo[q * RW + col] = acc;
            }
        }

        // ---------------- B prep: row r+2 ----------------
        {
            byw[2] = byw[1];
            byw[1] = byw[0];
            byw[0] = cb[1];
            s_bx[((r + 2) & 3) * RW + col] = cb[0];
            s_bz[((r + 2) & 3) * RW + col] = cb[2];
            s_ay[((r + 1) & 1) * RW + col] = byw[1] + c.c6 * (byw[0] - T(2) * byw[1] + byw[2]);
        }
        __syncthreads();
    }
}

template <typename T, int M, int P, bool HJ, int NT>
__global__ void __launch_bounds__(NT, 2)
    k_fused2d(Fused2dArgs<T> a, Geo g, Coef<T> c, int W, int L, int nstrip) {
    fused2d_tile<T, M, P, HJ, NT>(a, g, c, W, L, blockIdx.x % nstrip, blockIdx.x / nstrip);
}

// Batched step: a persistent grid-stride loop over (grid, strip, segment)
// tiles of many independent grids (longest tiles first), one launch per step;
// the batch runs its lumped grids here (the unlumped ones on the column-pair
// tiles of fused2d_pol_batch.cu).
template <int M, int P, bool HJ, int NT>
__global__ void __launch_bounds__(NT, 2)
    k_fused2d_batch(const BatchGrid *__restrict__ grids, const BatchItem *__restrict__ items, int nitems, int parity) {
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const BatchItem w = items[it];
        const BatchGrid &G = grids[w.grid];
        Fused2dArgs<float> a{};
        for (int q = 0; q < 3; ++q) {
            a.E[q] = G.E[parity][q];
            a.B[q] = G.B[parity][q];
            a.J[q] = HJ ? G.J[q] : nullptr;
            a.Eo[q] = const_cast<float *>(G.E[1 - parity][q]);
            a.Bo[q] = const_cast<float *>(G.B[1 - parity][q]);
        }
        a.m = M;
        a.passes = P;
        fused2d_tile<float, M, P, HJ, NT>(a, G.g, G.c, G.W, G.L, w.strip, w.seg);
    }
}

template <typename T, int M, int P, bool HJ>
struct Launcher {
    static constexpr int NT = Cfg<T>::NT;
    static size_t smem_bytes() { return smem_elems<T, M, P, HJ, NT>() * sizeof(T); }
    static int blocks_per_sm() {
        static int b = -1;
        if (b < 0) {
            auto k = k_fused2d<T, M, P, HJ, NT>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, smem_bytes()) != cudaSuccess || n < 1) n = 1;
            b = n;
        }
        return b;
    }
    static Fused2dShape shape(const Geo &g) {
        using Gm = Geom<M, P, HJ>;
        Fused2dShape sh;
        sh.threads = NT;
        sh.halo = Gm::H;
        sh.width = NT - 2 * Gm::H - 1;
        sh.strips = (g.nx + sh.width - 1) / sh.width;
        static int sms = -1;
        if (sms < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        }
        const int target = blocks_per_sm() * sms;
        int nseg = target / sh.strips;
        if (nseg < 1) nseg = 1;
        if (nseg > g.ny) nseg = g.ny;
        sh.rows = (g.ny + nseg - 1) / nseg;
        sh.segments = (g.ny + sh.rows - 1) / sh.rows;
        return sh;
    }
    static int run(const Geo &g, const Coef<T> &c, const Fused2dArgs<T> &a, cudaStream_t s) {
        const Fused2dShape sh = shape(g);
        k_fused2d<T, M, P, HJ, NT><<<sh.strips * sh.segments, NT, smem_bytes(), s>>>(a, g, c, sh.width, sh.rows,
                                                                                     sh.strips);
        return 1;
    }
};

constexpr int kMaxM = 4, kMaxP = 3;

template <typename T, int M>
int dispatch_p(const Geo &g, const Coef<T> &c, const Fused2dArgs<T> &a, cudaStream_t s, bool hj, int p,
               Fused2dShape *sh) {
    if (!hj) {
        if (sh) { *sh = Launcher<T, M, 0, false>::shape(g); return 0; }
        return Launcher<T, M, 0, false>::run(g, c, a, s);
    }
    switch (p) {
        case 0: if (sh) { *sh = Launcher<T, M, 0, true>::shape(g); return 0; } return Launcher<T, M, 0, true>::run(g, c, a, s);
        case 1: if (sh) { *sh = Launcher<T, M, 1, true>::shape(g); return 0; } return Launcher<T, M, 1, true>::run(g, c, a, s);
        case 2: if (sh) { *sh = Launcher<T, M, 2, true>::shape(g); return 0; } return Launcher<T, M, 2, true>::run(g, c, a, s);
        case 3: if (sh) { *sh = Launcher<T, M, 3, true>::shape(g); return 0; } return Launcher<T, M, 3, true>::run(g, c, a, s);
    }
    return -1;
}

template <typename T>
int dispatch(const Geo &g, const Coef<T> &c, const Fused2dArgs<T> &a, cudaStream_t s, int m, bool hj, int p,
             Fused2dShape *sh) {
    switch (m) {
        case 0: return dispatch_p<T, 0>(g, c, a, s, hj, p, sh);
        case 1: return dispatch_p<T, 1>(g, c, a, s, hj, p, sh);
        case 2: return dispatch_p<T, 2>(g, c, a, s, hj, p, sh);
        case 3: return dispatch_p<T, 3>(g, c, a, s, hj, p, sh);
        case 4: return dispatch_p<T, 4>(g, c, a, s, hj, p, sh);
    }
    return -1;
}

}  // namespace

bool fused2d_supported(const fmx_params *p) {
    if (p->dims != 2 || p->iter_mode != FMX_ITER_FIXED) return false;
    if (p->filter_target == FMX_FILTER_FIELDS && p->filter_passes > 0) return false;
    if (p->m < 0 || p->m > kMaxM) return false;
    if (p->filter_target == FMX_FILTER_CURRENT && p->filter_passes > kMaxP) return false;
    return p->n[0] <= (1 << 24) && p->n[1] <= (1 << 24);
}

template <typename T>
int launch_fused2d(const Geo &g, const Coef<T> &c, const Fused2dArgs<T> &a, cudaStream_t s) {
    const bool hj = a.J[0] != nullptr;
    return dispatch<T>(g, c, a, s, a.m, hj, hj ? a.passes : 0, nullptr);
}

template <typename T>
Fused2dShape fused2d_shape(const Geo &g, int m, int passes) {
    Fused2dShape sh{0, 0, 0, 0, 0, 0};
    Fused2dArgs<T> a{};
    Coef<T> c{};
    dispatch<T>(g, c, a, nullptr, m, passes >= 0, passes >= 0 ? passes : 0, &sh);
    return sh;
}

int fused2d_batch_geometry(int m, int passes, bool hj, int *threads, int *halo, int *width, size_t *smem,
                           int *blocks_per_sm) {
    int rc = -1;
#define FMX_BG(MM, PP, HH)                                                                                   \
    if (m == MM && passes == PP && hj == HH) {                                                              \
        using Gm = Geom<MM, PP, HH>;                                                                       \
        constexpr int NT = Cfg<float>::NT;                                                                 \
        *threads = NT;                                                                                     \
        *halo = Gm::H;                                                                                     \
        *width = NT - 2 * Gm::H - 1;                                                                       \
        *smem = smem_elems<float, MM, PP, HH, NT>() * sizeof(float);                                       \
        auto k = k_fused2d_batch<MM, PP, HH, NT>;                                                          \
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);                  \
        int nb = 0;                                                                                        \
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, NT, *smem) != cudaSuccess || nb < 1) nb = 1; \
        *blocks_per_sm = nb;                                                                               \
        rc = 0;                                                                                            \
    }
    FMX_BG(4, 0, false) FMX_BG(4, 3, true) FMX_BG(2, 0, false) FMX_BG(1, 0, false) FMX_BG(0, 0, false)
#undef FMX_BG
    return rc;
}

int launch_fused2d_batch(int m, int passes, bool hj, const BatchGrid *grids, const BatchItem *items, int nitems,
                         int parity, int nblocks, size_t smem, cudaStream_t s) {
#define FMX_BL(MM, PP, HH)                                                                       \
    if (m == MM && passes == PP && hj == HH) {                                                  \
        k_fused2d_batch<MM, PP, HH, Cfg<float>::NT><<<nblocks, Cfg<float>::NT, smem, s>>>(grids, items, nitems, parity); \
        return 1;                                                                              \
    }
    FMX_BL(4, 0, false) FMX_BL(4, 3, true) FMX_BL(2, 0, false) FMX_BL(1, 0, false) FMX_BL(0, 0, false)
#undef FMX_BL
    return -1;
}

template int launch_fused2d<float>(const Geo &, const Coef<float> &, const Fused2dArgs<float> &, cudaStream_t);
template int launch_fused2d<double>(const Geo &, const Coef<double> &, const Fused2dArgs<double> &, cudaStream_t);
template Fused2dShape fused2d_shape<float>(const Geo &, int, int);
template Fused2dShape fused2d_shape<double>(const Geo &, int, int);

}  // namespace fmx
