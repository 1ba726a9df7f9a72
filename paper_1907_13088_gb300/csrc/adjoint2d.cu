// Fused 2D adjoint of one FP32 step, split by polarisation like the forward
// kernels (fused2d_pol.cu): one TE launch (Ex, Ey, Bz) and one TM launch
// (Ez, Bx, By) per step.
//
// The forward step is linear, dE' = C_b S B - q F j, w = P dE' with
// P = sum_{s<=m} A^s (Algorithm 1), E1 = E + w, B1 = B - C_f E1.  On the
// periodic lattice C_f^T = C_b (Eqs. faraday_x..z, ampere_aux_x..z), and A
// (Eqs. matrixA_*), S = diag(alpha) and the binomial filter F are symmetric,
// so given (Ebar, Bbar) = dL/d(E1, B1):
//   u = Ebar - C_b Bbar          (row r; no alpha: C_f^T carries none)
//   Ebar' = u
//   w = P u                      (the forward sweeps, u in place of dE')
//   Bbar' = Bbar + S C_f w       (TE: Bz, no alpha in 2D; TM: Bx averaged
//                                 along x, By along y, one row later)
//   jbar = -q F w                (y binomial over a register window of w,
//                                 then x from shared memory)
// Row pipeline, shared-memory split rows and packed FP32x2 arithmetic as in
// the forward kernels; each stage two rows behind its producer, one
// __syncthreads per row.  HBM traffic per cell: TE reads 3 and writes 3 (+2
// with jbar) values, TM reads 3 and writes 3 (+1).
#include <cuda_runtime.h>
#include <math.h>

#include "fused2d.h"
#include "pair2.cuh"

namespace fmx {
namespace {

using namespace pair2;

template <int POL, int M, int P, bool HJB>
struct AdjGeom {
    // extra rows the first stage must lead by: the jbar window (P) and the TM
    // averaging of the Faraday curl along y (1)
    static constexpr int EJ = (HJB && P > (POL == TM ? 1 : 0)) ? P : (POL == TM ? 1 : 0);
    // lag of the last stage behind row r: Faraday (TE 2M+1, TM 2M+2), jbar (2M+P+1)
    static constexpr int LAST = 2 * M + ((HJB && P + 1 > (POL == TM ? 2 : 1)) ? P + 1 : (POL == TM ? 2 : 1));
    // left halo: source curl 1 + M sweeps + (TM x-average 1 | jbar x-filter P), even
    static constexpr int REACH = 1 + M + ((HJB && P > 1) ? P : 1);
    static constexpr int HC = (REACH + 1) / 2 * 2;
    static constexpr int PADP = (HJB && P > 1) ? (P + 1) / 2 : 1;  // smem pad, in pairs
    static constexpr int NS = M > 1 ? M - 1 : 0;
    static constexpr int TJ = HJB ? 2 * P + 1 : 1;
    static constexpr int D0 = 12;  // dE' (here u) ring depth: >= 2M+1, a multiple of 4
};

// Shared-memory map (floats); RP = floats per half row.
template <int POL, int M, int P, bool HJB, int RP>
struct AdjSmem {
    using G = AdjGeom<POL, M, P, HJB>;
    static constexpr int NC = POL == TE ? 2 : 1;
    static constexpr int B = 0;                               // TE: Bbar_z, TM: Bbar_y rows [4] full
    static constexpr int DP = B + 8 * RP;                     // u: [D0][NC] full
    static constexpr int SW = DP + G::D0 * NC * 2 * RP;       // sweeps 1..M-1: [NS][4]
    static constexpr int SWS = POL == TE ? 3 * RP : 2 * RP;   //   TE: Ex odd half + Ey full; TM: Ez full
    static constexpr int EN = SW + G::NS * 4 * SWS;           // w (TE: w_y, TM: w_z) [2] even half
    static constexpr int CX = EN + 2 * RP;                    // TM: ky D_y w [2] full
    static constexpr int JB = CX + (POL == TM ? 4 * RP : 0);  // y-filtered w: [2][NC] full
    static constexpr int TOTAL = JB + (HJB ? 2 * NC * 2 * RP : 0);
};

// rows ahead of the register prefetch per stream: Ebar, Bbar, Bbar again for
// the Faraday stage (an L2 hit)
template <int POL>
struct AdjPrefetch {
    static constexpr int PE = POL == TM ? 4 : 2, PB = POL == TM ? 4 : 2, PF = POL == TM ? 4 : 2;
    static constexpr int L1 = 2;  // rows beyond those whose Ebar, Bbar lines go to L1 (Adj2dArgs::l1pf)
};

template <int POL, int M, int P, bool HJB, int NT>
__global__ void __launch_bounds__(NT, 3)
    k_adj2d(Adj2dArgs<float> a, Geo g, Coef2 c, int W, int L, int nstrip) {
    using G = AdjGeom<POL, M, P, HJB>;
    constexpr int HC = G::HC, PADP = G::PADP, TJ = G::TJ, D0 = G::D0;
    constexpr int RP = NT + 2 * PADP;
    using S = AdjSmem<POL, M, P, HJB, RP>;
    constexpr int NC = S::NC;
    extern __shared__ __align__(16) unsigned char smraw[];
    float *sm = reinterpret_cast<float *>(smraw);
    float *s_b = sm + S::B;
    float *s_dp = sm + S::DP;
    float *s_sw = sm + S::SW;
    float *s_e = sm + S::EN;
    float *s_cx = sm + S::CX;
    float *s_jb = sm + S::JB;

    const int tid = threadIdx.x;
    for (int q = tid; q < S::TOTAL; q += NT) sm[q] = 0.f;

    const int strip = blockIdx.x % nstrip, seg = blockIdx.x / nstrip;
    const int x0 = strip * W;
    const int y0 = seg * L;
    const int y1 = min(y0 + L, g.ny);
    const int cg = x0 - HC + 2 * tid;  // first column of the pair
    int xc = cg % g.nx;
    if (xc < 0) xc += g.nx;
    const bool xout = 2 * tid >= HC && 2 * tid < HC + W && cg < g.nx;
    const int pc = tid + PADP;
    auto lft = [&](const float *row) { return row[RP + pc - 1]; };
    auto rgt = [&](const float *row) { return row[pc + 1]; };
    auto own = [&](const float *row) { return mk(row[pc], row[RP + pc]); };
    auto put = [&](float *row, f2 v) {
        row[pc] = v.x;
        row[RP + pc] = v.y;
    };

    // streams of the set: TE Ebar_x, Ebar_y, Bbar_z; TM Ebar_z, Bbar_x, Bbar_y
    const float *__restrict__ inE0 = POL == TE ? a.Eb[0] : a.Eb[2];
    const float *__restrict__ inE1 = a.Eb[1];
    const float *__restrict__ inB0 = POL == TE ? a.Bb[2] : a.Bb[0];
    const float *__restrict__ inB1 = a.Bb[1];
    float *__restrict__ oE0 = POL == TE ? a.Ebo[0] : a.Ebo[2];
    float *__restrict__ oE1 = a.Ebo[1];
    float *__restrict__ oB0 = POL == TE ? a.Bbo[2] : a.Bbo[0];
    float *__restrict__ oB1 = a.Bbo[1];
    float *__restrict__ oJ0 = POL == TE ? a.Jbo[0] : a.Jbo[2];
    float *__restrict__ oJ1 = a.Jbo[1];

    // first row: the first stage's earliest needed row y0 - M - EJ, less 3:
    // Bbar rows reach shared memory (and TM's Bbar_x delay line) two
    // iterations after their load, and the previous row's Bbar one more
    int r0 = y0 - M - G::EJ - 3;
    r0 -= ((r0 % 4) + 4) % 4;
    int r1 = y1 + G::LAST;
    r1 += (4 - ((r1 - r0) % 4)) % 4;

    // Faraday stage row behind r: TE rhoF = r - 2M - 1; TM rhoB = r - 2M - 2
    constexpr int FL = POL == TE ? 2 * M + 1 : 2 * M + 2;
    const int pitch = (int)g.pitch, plane = g.ny * pitch;
    auto row_off = [&](int r) {
        int y = r % g.ny;
        if (y < 0) y += g.ny;
        return y * pitch + xc;
    };
    int oe = row_off(r0), ob = row_off(r0 + 2), of = row_off(r0 - FL);
    auto adv = [&](int &o) {
        o += pitch;
        if (o >= plane) o -= plane;
    };
    // L1 prefetch of the rows AdjPrefetch::L1 beyond the register loads
    int le = row_off(r0 + AdjPrefetch<POL>::PE + AdjPrefetch<POL>::L1),
        lb = row_off(r0 + 2 + AdjPrefetch<POL>::PB + AdjPrefetch<POL>::L1);

    const f2 z2 = mk(0.f, 0.f);
    f2 win[M > 0 ? M : 1][NC][3];
    f2 aux[M > 0 ? M : 1][3];
    float eyrp[M > 0 ? M : 1];
    f2 en[NC], enp[NC];
    f2 bprev = z2;            // TE: Bbar_z row r-1; TM: Bbar_x row r-1
    f2 bxd[2] = {z2, z2};     // TM: Bbar_x of rows r, r+1 (own pair), slot = row parity
    f2 cyw[3] = {z2, z2, z2}; // TM: -kx D_x w of rows rhoF, rhoF-1, rhoF-2
    f2 cxp = z2;              // TM: ky D_y w of row rhoF-1 (own pair)
    f2 jw[NC][TJ];            // w rows rhoM .. rhoM-2P (own pair)
    f2 jdj[NC];               // y-filtered w of the previous row (own pair)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        en[q] = enp[q] = jdj[q] = z2;
#pragma unroll
        for (int k = 0; k < TJ; ++k) jw[q][k] = z2;
    }
#pragma unroll
    for (int s = 0; s < (M > 0 ? M : 1); ++s) {
#pragma unroll
        for (int q = 0; q < NC; ++q) win[s][q][0] = win[s][q][1] = win[s][q][2] = z2;
        aux[s][0] = aux[s][1] = aux[s][2] = z2;
        eyrp[s] = 0.f;
    }

    auto ld2 = [&](const float *p, int o) { return __ldg(reinterpret_cast<const float2 *>(p + o)); };
    using PF_ = AdjPrefetch<POL>;
    constexpr int PE = PF_::PE, PB = PF_::PB, PFD = PF_::PF;
    f2 pe0[PE], pe1[PE], pb0[PB], pb1[PB], pf0[PFD], pf1[PFD];
    auto ldE = [&](int k) {
        pe0[k] = ld2(inE0, oe);
        pe1[k] = POL == TE ? ld2(inE1, oe) : z2;
        adv(oe);
    };
    auto ldB = [&](int k) {
        pb0[k] = ld2(inB0, ob);
        pb1[k] = POL == TM ? ld2(inB1, ob) : z2;
        adv(ob);
    };
    auto ldF = [&](int k) {
        pf0[k] = ld2(inB0, of);
        pf1[k] = POL == TM ? ld2(inB1, of) : z2;
        adv(of);
    };
#pragma unroll
    for (int k = 0; k < PE; ++k) ldE(k);
#pragma unroll
    for (int k = 0; k < PB; ++k) ldB(k);
#pragma unroll
    for (int k = 0; k < PFD; ++k) ldF(k);
    int b0 = ((r0 % D0) + D0) % D0;  // u ring slot of row r0 (a multiple of 4)
    __syncthreads();

    for (int rb = r0; rb < r1; rb += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = rb + u;
            // this row's inputs, then the loads `depth` rows ahead (past the
            // segment: valid wrapped rows, unused)
            const f2 ce0 = pe0[u % PE], ce1 = pe1[u % PE], cb0 = pb0[u % PB], cb1 = pb1[u % PB],
                     cf0 = pf0[u % PFD], cf1 = pf1[u % PFD];
            ldE(u % PE);
            ldB(u % PB);
            ldF(u % PFD);
            if (a.l1pf) {
                prefetch_l1(inE0 + le);
                if (POL == TE) prefetch_l1(inE1 + le);
                prefetch_l1(inB0 + lb);
                if (POL == TM) prefetch_l1(inB1 + lb);
                adv(le);
                adv(lb);
            }
            const int rhoM = r - 2 * M, rhoF = rhoM - 1;
            // u ring row of row r - k (u, k compile-time; b0 in {0, 4, 8})
            auto dprow = [&](int k) {
                int sl = b0 + u - k;
                return s_dp + (sl < 0 ? sl + D0 : sl) * NC * 2 * RP;
            };
            // w = dE_(M) of row rhoM: Faraday transpose and jbar
            auto finish = [&](f2 o0, f2 o1) {
                enp[0] = en[0];
                en[0] = o0;
                if (POL == TE) {
                    enp[1] = en[1];
                    en[1] = o1;
                }
                // neighbours read column 2t+2 (even) of TE: w_y, TM: w_z
                s_e[(u & 1) * RP + pc] = POL == TE ? en[1].x : en[0].x;
                const float er = s_e[((u + 1) & 1) * RP + pc + 1];  // row rhoF
                if constexpr (POL == TE) {
                    // Bbar_z += kx (w_y[i+1] - w_y[i]) - ky (w_x[j+1] - w_x[j]), row rhoF
                    const f2 dxwy = fma(enp[1], m1(), mk(enp[1].y, er));
                    const f2 dywx = fma(enp[0], m1(), en[0]);
                    const f2 bo0 = fma(c.kx, dxwy, fma(mul(c.ky, dywx), m1(), cf0));
                    if (rhoF >= y0 && rhoF < y1 && xout) *reinterpret_cast<float2 *>(oB0 + rhoF * pitch + xc) = bo0;
                } else {
                    // row rhoF: cx = ky (w[j+1] - w[j]), cy = -kx (w[i+1] - w[i])
                    const f2 cx = mul(c.ky, fma(enp[0], m1(), en[0]));
                    const f2 cy = mul(c.kx, fma(mk(enp[0].y, er), m1(), enp[0]));
                    // row rhoB = rhoF - 1: Bbar_x += alpha_x cx, Bbar_y += alpha_y cy
                    const float *sx = s_cx + ((u + 1) & 1) * 2 * RP;
                    const f2 bxo = fma(c6(), fma(cxp, m2(), add(mk(lft(sx), cxp.x), mk(cxp.y, rgt(sx)))), add(cf0, cxp));
                    cyw[2] = cyw[1];
                    cyw[1] = cyw[0];
                    cyw[0] = cy;
                    const f2 byo = fma(c6(), fma(cyw[1], m2(), add(cyw[0], cyw[2])), add(cf1, cyw[1]));
                    put(s_cx + (u & 1) * 2 * RP, cx);
                    cxp = cx;
                    const int rhoB = rhoF - 1;
                    if (rhoB >= y0 && rhoB < y1 && xout) {
                        const int o = rhoB * pitch + xc;
                        *reinterpret_cast<float2 *>(oB0 + o) = bxo;
                        *reinterpret_cast<float2 *>(oB1 + o) = byo;
                    }
                }
                if constexpr (HJB) {
                    // x binomial of the y-filtered row rhoM-P-1 (previous slot), then
                    // the y binomial of row rhoM-P into this slot
                    const int rhoJ = rhoM - P - 1;
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        const float *row = s_jb + (((u + 1) & 1) * NC + q) * 2 * RP;
                        float col[2 * P + 2];
#pragma unroll
                        for (int i = 0; i < 2 * P + 2; ++i) {
                            const int off = i - P;
                            col[i] = off == 0        ? jdj[q].x
                                     : off == 1      ? jdj[q].y
                                     : (off & 1) == 0 ? row[pc + off / 2]
                                                      : row[RP + pc + (off - 1) / 2];
                        }
                        f2 taps[2 * P + 1];
#pragma unroll
                        for (int k = 0; k < 2 * P + 1; ++k) taps[k] = mk(col[k], col[k + 1]);
                        const f2 jb = mul(c.qf, fma(binom_taps<P>(taps), m1(), z2));  // -q F w
                        float *oj = q == 0 ? oJ0 : oJ1;
                        if (oj && rhoJ >= y0 && rhoJ < y1 && xout)
                            *reinterpret_cast<float2 *>(oj + rhoJ * pitch + xc) = jb;
#pragma unroll
                        for (int k = TJ - 1; k > 0; --k) jw[q][k] = jw[q][k - 1];
                        jw[q][0] = q == 0 ? en[0] : en[1];
                        const f2 acc = binom_taps<P>(jw[q]);
                        put(s_jb + ((u & 1) * NC + q) * 2 * RP, acc);
                        jdj[q] = acc;
                    }
                }
            };

            // ---------------- sweeps M..1 ----------------
#pragma unroll
            for (int s = M; s >= 1; --s) {
                // input rows of sweep s (outputs of stage s-1): rho+1 and rho.
                // TE: xo = odd half of Ex, ey = full Ey; TM: ez = full Ez.
                const float *xo_p1, *ey_0, *ez_p1;
                if (s == 1) {
                    const float *rp1 = dprow(2 * s - 1), *r0w = dprow(2 * s);
                    xo_p1 = rp1 + RP;
                    ey_0 = r0w + 2 * RP;
                    ez_p1 = rp1;
                } else {
                    const float *base = s_sw + (s - 2) * 4 * S::SWS;
                    const float *rp1 = base + ((u - 2 * s + 1 + 16) & 3) * S::SWS;
                    const float *r0w = base + ((u - 2 * s + 16) & 3) * S::SWS;
                    xo_p1 = rp1;
                    ey_0 = r0w + RP;
                    ez_p1 = rp1;
                }
                // dE' of row rho (own pair): sweep 1 holds it in its window
                f2 dp0, dp1 = z2;
                if (s == 1) {
                    dp0 = win[0][0][1];
                    if (POL == TE) dp1 = win[0][1][1];
                } else {
                    const float *dr = dprow(2 * s);
                    dp0 = own(dr);
                    if (POL == TE) dp1 = own(dr + 2 * RP);
                }
                f2 o0, o1 = z2;
                if constexpr (POL == TE) {
                    const f2 *X = win[s - 1][0];
                    const f2 *Y = win[s - 1][1];
                    // h = Dbar_x(bwd) Ex at row rho+1: X0 - (Ex[2t-1], X0.x)
                    const float exl = xo_p1[pc - 1];
                    aux[s - 1][1] = aux[s - 1][0];
                    aux[s - 1][0] = fma(mk(exl, X[0].x), m1(), X[0]);
                    const float eyl = lft(ey_0), eyr = rgt(ey_0), eyr_m = eyrp[s - 1];
                    eyrp[s - 1] = eyr;
                    const f2 g_own = fma(Y[2], m1(), Y[1]);
                    const f2 g_nb = mk(g_own.y, eyr - eyr_m);
                    const f2 dyyx = fma(X[1], m2(), add(X[0], X[2]));
                    const f2 dxxy = fma(Y[1], m2(), add(mk(eyl, Y[1].x), mk(Y[1].y, eyr)));
                    o0 = fma(c.ay, dyyx, dp0);
                    o0 = fma(c.bxy, fma(g_own, m1(), g_nb), o0);
                    o1 = fma(c.ax, dxxy, dp1);
                    o1 = fma(c.bxy, fma(aux[s - 1][1], m1(), aux[s - 1][0]), o1);
                } else {
                    const f2 *Z = win[s - 1][0];
                    const float ezl = lft(ez_p1), ezr = rgt(ez_p1);
                    aux[s - 1][2] = aux[s - 1][1];
                    aux[s - 1][1] = aux[s - 1][0];
                    aux[s - 1][0] = fma(Z[0], m2(), add(mk(ezl, Z[0].x), mk(Z[0].y, ezr)));
                    const f2 *D = aux[s - 1];
                    const f2 dyy = fma(Z[1], m2(), add(Z[0], Z[2]));
                    const f2 dxxyy = fma(D[1], m2(), add(D[0], D[2]));
                    o0 = fma(c.ax, D[1], dp0);
                    o0 = fma(c.ay, dyy, o0);
                    o0 = fma(c.axy, dxxyy, o0);
                }
                if (s < M) {
                    float *o = s_sw + (s - 1) * 4 * S::SWS + ((u - 2 * s + 16) & 3) * S::SWS;
                    if (POL == TE) {
                        o[pc] = o0.y;     // Ex: neighbours read the odd column only
                        put(o + RP, o1);  // Ey: both
                    } else {
                        put(o, o0);
                    }
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        win[s][q][2] = win[s][q][1];
                        win[s][q][1] = win[s][q][0];
                    }
                    win[s][0][0] = o0;
                    if (POL == TE) win[s][1][0] = o1;
                } else {
                    finish(o0, o1);
                }
            }


            // ---------------- u = Ebar - C_b Bbar, row r ----------------
            {
                const float *sb = s_b + (u & 3) * 2 * RP;
                f2 d0, d1 = z2;
                if constexpr (POL == TE) {
                    // u_x = Ebar_x - ky (Bbar_z[j] - Bbar_z[j-1]);  u_y = Ebar_y + kx (Bbar_z[i] - Bbar_z[i-1])
                    const f2 bz0 = own(sb);
                    d0 = fma(c.ky, fma(bz0, m1(), bprev), ce0);
                    d1 = fma(c.kx, fma(mk(lft(sb), bz0.x), m1(), bz0), ce1);
                    bprev = bz0;
                } else {
                    // u_z = Ebar_z - kx (Bbar_y[i] - Bbar_y[i-1]) + ky (Bbar_x[j] - Bbar_x[j-1])
                    const f2 by0 = own(sb);
                    const f2 bx0 = bxd[u & 1];
                    const f2 dxby = fma(mk(lft(sb), by0.x), m1(), by0);
                    d0 = fma(mul(c.kx, dxby), m1(), fma(c.ky, fma(bprev, m1(), bx0), ce0));
                    bprev = bx0;
                }
                if (r >= y0 && r < y1 && xout) {
                    const int o = r * pitch + xc;
                    *reinterpret_cast<float2 *>(oE0 + o) = d0;
                    if (POL == TE) *reinterpret_cast<float2 *>(oE1 + o) = d1;
                }
                if (M > 0) {
                    float *dr = dprow(0);
                    put(dr, d0);
                    if (POL == TE) put(dr + 2 * RP, d1);
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        win[0][q][2] = win[0][q][1];
                        win[0][q][1] = win[0][q][0];
                    }
                    win[0][0][0] = d0;
                    if (POL == TE) win[0][1][0] = d1;
                } else {
                    finish(d0, d1);  // no sweeps: w = u
                }
            }

            // ---------------- Bbar prep, row r+2 ----------------
            put(s_b + ((u + 2) & 3) * 2 * RP, POL == TE ? cb0 : cb1);  // TE: Bbar_z, TM: Bbar_y
            if (POL == TM) bxd[u & 1] = cb0;                          // TM: Bbar_x
            __syncthreads();
        }
        b0 += 4;
        if (b0 >= D0) b0 -= D0;
    }
}

// rows per segment asked for by the caller of the current launch (0:
// automatic, see AdjLauncher::run)
thread_local int t_adj_rows = 0;

template <int POL, int M, int P, bool HJB>
struct AdjLauncher {
    static constexpr int NT = 128;
    using Gm = AdjGeom<POL, M, P, HJB>;
    static size_t smem_bytes() { return (size_t)AdjSmem<POL, M, P, HJB, NT + 2 * Gm::PADP>::TOTAL * sizeof(float); }
    static int blocks_per_sm() {
        static int b = -1;
        if (b < 0) {
            auto k = k_adj2d<POL, M, P, HJB, NT>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, smem_bytes()) != cudaSuccess || n < 1) n = 1;
            b = n;
        }
        return b;
    }
    static void run(const Geo &g, const Coef2 &c, const Adj2dArgs<float> &a, cudaStream_t s) {
        const int width = 2 * NT - 2 * Gm::HC - 2;
        const int strips = (g.nx + width - 1) / width;
        static int sms = -1;
        if (sms < 0) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
        }
        // automatic: one wave of CTAs at the measured occupancy, but no
        // segment shorter than its warm-up rows (3m + 2p + 8), as the forward
        int nseg = blocks_per_sm() * sms / strips;
        if (nseg < 1) nseg = 1;
        if (nseg > g.ny) nseg = g.ny;
        int rows = (g.ny + nseg - 1) / nseg;
        if (rows < 3 * M + 2 * P + 8) rows = 3 * M + 2 * P + 8;
        if (t_adj_rows > 0) rows = t_adj_rows;
        if (rows > g.ny) rows = g.ny;
        const int segs = (g.ny + rows - 1) / rows;
        k_adj2d<POL, M, P, HJB, NT><<<strips * segs, NT, smem_bytes(), s>>>(a, g, c, width, rows, strips);
    }
};

// TE writes jbar_x, jbar_y when either is asked for; TM writes jbar_z when asked
template <int M, int P>
int adj_pair(const Geo &g, const Coef2 &c, const Adj2dArgs<float> &a, cudaStream_t s) {
    if (a.Jbo[0] || a.Jbo[1]) AdjLauncher<TE, M, P, true>::run(g, c, a, s);
    else AdjLauncher<TE, M, P, false>::run(g, c, a, s);
    if (a.Jbo[2]) AdjLauncher<TM, M, P, true>::run(g, c, a, s);
    else AdjLauncher<TM, M, P, false>::run(g, c, a, s);
    return 2;
}

template <int M>
int adj_p(const Geo &g, const Coef2 &c, const Adj2dArgs<float> &a, cudaStream_t s, int p) {
    switch (p) {
        case 0: return adj_pair<M, 0>(g, c, a, s);
        case 1: return adj_pair<M, 1>(g, c, a, s);
        case 2: return adj_pair<M, 2>(g, c, a, s);
        case 3: return adj_pair<M, 3>(g, c, a, s);
    }
    return -1;
}

}  // namespace

bool adjoint2d_supported(const Geo &g, int m, int passes) {
    return g.nz == 1 && g.nx % 2 == 0 && (int64_t)g.ny * g.pitch < ((int64_t)1 << 31) && m >= 0 && m <= 4 &&
           passes >= 0 && passes <= 3;
}

int launch_adjoint2d(const Geo &g, const Coef<float> &c, const Adj2dArgs<float> &a, cudaStream_t s, int seg_rows) {
    if (!adjoint2d_supported(g, a.m, a.passes) || c.c6 != 1.f / 6.f) return -1;
    struct RowsScope {  // the segment rows of this call's launches
        explicit RowsScope(int r) { t_adj_rows = r; }
        ~RowsScope() { t_adj_rows = 0; }
    } rows_scope(seg_rows);
    Coef2 k;
    auto b = [](float v) { return make_float2(v, v); };
    k.kx = b(c.kx);
    k.ky = b(c.ky);
    k.qf = b(ldexpf(c.q, -4 * a.passes));  // q / 4^(2p), exact
    k.ax = b(c.ax);
    k.ay = b(c.ay);
    k.axy = b(c.axy);
    k.bxy = b(c.bxy);
    Adj2dArgs<float> a2 = a;
    a2.l1pf = fused2d_l1_prefetch(g) ? 1 : 0;
    switch (a.m) {
        case 0: return adj_p<0>(g, k, a2, s, a.passes);
        case 1: return adj_p<1>(g, k, a2, s, a.passes);
        case 2: return adj_p<2>(g, k, a2, s, a.passes);
        case 3: return adj_p<3>(g, k, a2, s, a.passes);
        case 4: return adj_p<4>(g, k, a2, s, a.passes);
    }
    return -1;
}

}  // namespace fmx
