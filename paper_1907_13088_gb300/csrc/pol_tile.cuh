// Tile of the FP32 fused 2D step split by polarisation (TE or TM), two
// columns per thread: the shared device code of the single-grid kernels
// (fused2d_pol.cu) and of the odd-n_x and batched launches
// (fused2d_pol_batch.cu).  Internal.
//
// In 2D the scheme decouples exactly into the TE set (Ex, Ey, Bz; jx, jy)
// and the TM set (Ez, Bx, By; jz) (Sec. 2.2.2: E_z is solved independently
// of E_x and E_y, and Eqs. faraday_x_2d..ampere_aux_z_2d couple nothing
// across the two sets).  Each set gets its own kernel; one step is one TE
// launch and one TM launch.  Each kernel keeps the row pipeline of
// fused2d.cu (J -> B prep -> source -> M sweeps -> E update -> Faraday, each
// stage two rows behind its producer, one __syncthreads per row) but a
// thread owns two adjacent columns and does the arithmetic on column pairs
// with packed FP32x2 instructions.  Ring slots are compile-time constants: the
// row loop runs in blocks of four rows from a row index that is a multiple of
// four.  HBM traffic per cell and step: TE reads 5 and writes 3 FP32 values,
// TM reads 4 and writes 3 (60 bytes together).  Global loads and stores move
// column pairs (8 bytes); with odd n_x, strips that cross the periodic seam
// load single columns and the last column is stored alone.
//
// Shared memory only carries what a thread's neighbours read.  A row is
// stored split: the even columns (pair.x) in one array of RP floats and the
// odd columns (pair.y) in the next, so the neighbour values a thread needs
// (column 2t-1 = pair t-1 odd, column 2t+2 = pair t+1 even) are unit-stride
// 4-byte loads, one wavefront per warp and free of bank conflicts.  Where
// neighbours read only one parity, only that half is stored.  Where registers
// allow (TE: the filtered current, sweep inputs; TM: sweep inputs), a thread's
// own values of a row come from registers instead of back from shared memory.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "fused2d.h"
#include "pair2.cuh"

namespace fmx {
namespace pol2d {

using namespace pair2;

// Input prefetch into registers, rows ahead per input stream (each divides
// 4): the current, B, E, and B again for the Faraday update (that re-read of
// rows the CTA loaded 2m+3 rows earlier hits L2).  The depths fit the 168
// registers of 3 blocks/SM.
template <int POL>
struct PolPrefetch {
    static constexpr int PJ = POL == TM ? 4 : 2, PB = POL == TM ? 4 : 2, PE = POL == TM ? 4 : 2,
                         PF = POL == TM ? 4 : 2;
    // rows beyond those register loads whose j, B and E lines are prefetched
    // into L1 by the L1PF tiles (no register holds them).  4096^2, m = 4, p = 3: 65.3 Gcell/s without, 72.1 with 2
    // rows (1 to 4 rows, for TE and TM apart, all within 71.6-72.1; 8 rows 71.0)
    static constexpr int L1 = 2;
};

template <int M, int P, bool HJ>
struct PolGeom {
    static constexpr int PX = (HJ && P > 1) ? P : 1;            // columns of x-reach of the source
    static constexpr int HC = ((PX + M) + 1) / 2 * 2;           // left halo, even
    static constexpr int PADP = (HJ && P > 1) ? (P + 1) / 2 : 1; // smem pad, in pairs
    static constexpr int NS = M > 1 ? M - 1 : 0;
    static constexpr int TJ = HJ ? 2 * P + 1 : 1;
    static constexpr int WU = TJ > 3 ? TJ : 3;
};

// Shared-memory map of one polarisation kernel, in floats.  RP = floats per
// half row (pairs of the strip plus pads).  "full" = both halves (2 RP),
// "half" = one parity (RP).
template <int POL, int M, int P, bool HJ, int RP>
struct PolSmem {
    using G = PolGeom<M, P, HJ>;
    static constexpr int NC = POL == TE ? 2 : 1;                     // E components of the set
    // dE' ring depth: >= 2M+1 rows, a multiple of 4 (16, with a mask for the
    // slot wrap, measured slower in both kernels: more shared memory, less L1)
    static constexpr int D0 = 12;
    static_assert(2 * M + 1 <= D0 && D0 % 4 == 0, "dE' ring too shallow");
    static constexpr int J = 0;                                      // y-filtered j: [2][NC] full
    static constexpr int B = J + (HJ ? 2 * NC * 2 * RP : 0);         // TE: Bz, TM: Bx [4] full
    static constexpr int AY = B + 8 * RP;                            // TM: alpha_y By [2] full
    static constexpr int DP = AY + (POL == TM ? 4 * RP : 0);         // dE': [D0][NC] full
    static constexpr int SW = DP + D0 * NC * 2 * RP;              // sweeps 1..M-1: [NS][4] slots
    static constexpr int SWS = POL == TE ? 3 * RP : 2 * RP;          //   TE: Ex odd half + Ey full; TM: Ez full
    static constexpr int EN = SW + G::NS * 4 * SWS;                  // E^{n+1} (TE: Ey, TM: Ez): [2] even half
    static constexpr int TOTAL = EN + 2 * RP;
};

// One tile: strip `strip` (W columns written) and segment `seg` (L rows) of a
// grid, in the shared memory `sm` (PolSmem layout).  HALF: the tile is run by
// one half of the CTA (threads half * NT .. half * NT + NT - 1), which
// synchronises on its own named barrier 1 + half, so that a CTA can carry
// two independent narrow tiles; otherwise the whole CTA runs it.  L1PF: the
// input rows are also prefetched into L1 PolPrefetch::L1 rows beyond the
// register loads (for grids whose rows come from HBM).
template <int POL, int M, int P, bool HJ, int NT, bool SEAM = false, bool HALF = false, bool L1PF = false>
__device__ __forceinline__ void pol_tile(const Fused2dArgs<float> &a, const Geo &g, const Coef2 &c, int W, int L,
                                         int strip, int seg, float *sm, int half = 0) {
    using G = PolGeom<M, P, HJ>;
    constexpr int HC = G::HC, PADP = G::PADP, TJ = G::TJ;
    constexpr int RP = NT + 2 * PADP;  // pairs (floats of a half row) per smem row
    using S = PolSmem<POL, M, P, HJ, RP>;
    constexpr int D0 = S::D0;
    constexpr int NC = S::NC;
    // own values from registers (TE) or read back from smem (TM: 4 blocks/SM leave no room)
    constexpr bool RJ = POL == TE;
    float *s_j = sm + S::J;
    float *s_b = sm + S::B;
    float *s_ay = sm + S::AY;
    float *s_dp = sm + S::DP;
    float *s_sw = sm + S::SW;
    float *s_e = sm + S::EN;

    const int tid = HALF ? (int)threadIdx.x - half * NT : (int)threadIdx.x;
    auto row_barrier = [&]() {
        if constexpr (HALF) asm volatile("bar.sync %0, %1;" ::"r"(1 + half), "n"(NT) : "memory");
        else __syncthreads();
    };
    for (int q = tid; q < S::TOTAL; q += NT) sm[q] = 0.f;

    const int x0 = strip * W;
    const int y0 = seg * L;
    const int y1 = min(y0 + L, g.ny);
    const int cg = x0 - HC + 2 * tid;  // first column of the pair
    int xc = cg % g.nx;
    if (xc < 0) xc += g.nx;
    // SEAM (odd n_x, a strip whose columns cross the periodic seam): a pair
    // may straddle the seam or start at an odd column, so its two columns are
    // loaded one at a time, and the grid's last column is stored alone
    const bool xout = 2 * tid >= HC && 2 * tid < HC + W && cg < g.nx;
    [[maybe_unused]] int dxc = 1;         // SEAM: 1, or 1 - n_x across the seam
    [[maybe_unused]] bool xlast = false;  // SEAM: the pair's second column lies past the grid
    if constexpr (SEAM) {
        int xc1 = (cg + 1) % g.nx;
        if (xc1 < 0) xc1 += g.nx;
        dxc = xc1 - xc;
        xlast = cg + 1 >= g.nx;
    }
    const int pc = tid + PADP;  // pair index in an smem row
    // full row: column 2t-1 (left), 2t+2 (right), own pair, store
    auto lft = [&](const float *row) { return row[RP + pc - 1]; };
    auto rgt = [&](const float *row) { return row[pc + 1]; };
    auto own = [&](const float *row) { return mk(row[pc], row[RP + pc]); };
    auto put = [&](float *row, f2 v) {
        row[pc] = v.x;
        row[RP + pc] = v.y;
    };

    // inputs of the set
    const float *__restrict__ inJ0 = POL == TE ? a.J[0] : a.J[2];
    const float *__restrict__ inJ1 = a.J[1];
    const float *__restrict__ inB0 = POL == TE ? a.B[2] : a.B[0];  // TE: Bz   TM: Bx
    const float *__restrict__ inB1 = a.B[1];                        // TM: By
    const float *__restrict__ inE0 = POL == TE ? a.E[0] : a.E[2];  // TE: Ex   TM: Ez
    const float *__restrict__ inE1 = a.E[1];                        // TE: Ey
    float *__restrict__ oE0 = POL == TE ? a.Eo[0] : a.Eo[2];
    float *__restrict__ oE1 = a.Eo[1];
    float *__restrict__ oB0 = POL == TE ? a.Bo[2] : a.Bo[0];
    float *__restrict__ oB1 = a.Bo[1];

    // first row, aligned down to a multiple of 4 (extra warm-up rows are harmless)
    int r0 = y0 - M - G::WU - 1;
    r0 -= ((r0 % 4) + 4) % 4;
    int r1 = y1 + 2 * M + 1;
    r1 += (4 - ((r1 - r0) % 4)) % 4;

    // running row offsets (element index of (row, xc)) of the four input rows;
    // 32-bit: the launcher requires ny * pitch < 2^31
    const int pitch = (int)g.pitch, plane = g.ny * pitch;
    auto row_off = [&](int r) {
        int y = r % g.ny;
        if (y < 0) y += g.ny;
        return y * pitch + xc;
    };
    int oj = row_off(r0 + 1 + P), ob = row_off(r0 + 2), oe = row_off(r0 - 2 * M), of = row_off(r0 - 2 * M - 1);
    auto adv = [&](int &o) {
        o += pitch;
        if (o >= plane) o -= plane;
    };
    // L1 prefetch: the rows PolPrefetch::L1 beyond the register loads
    constexpr int L1D = PolPrefetch<POL>::L1;
    int lj = 0, lb = 0, le = 0;
    if constexpr (L1PF) {
        lj = row_off(r0 + 1 + P + PolPrefetch<POL>::PJ + L1D);
        lb = row_off(r0 + 2 + PolPrefetch<POL>::PB + L1D);
        le = row_off(r0 - 2 * M + PolPrefetch<POL>::PE + L1D);
    }

    // register state (pairs)
    f2 jw[NC][TJ];
    f2 jd[NC];           // TE: y-filtered j of row r (own pair; TM reads it back from smem)
    f2 byw[3];           // TM: By rows r+2, r+1, r
    f2 bprev;            // TE: Bz row r-1   TM: alpha_x Bx row r-1
    f2 win[M > 0 ? M : 1][NC][3];
    f2 aux[M > 0 ? M : 1][3];  // TE: h = Dbar_x Ex (rows rho+1, rho)   TM: Dbar_xx Ez (rho+1, rho, rho-1)
    float eyrp[M > 0 ? M : 1];  // TE: Ey at column 2t+2, row rho-1 of each sweep's input
    f2 en[NC], enp[NC];
    const f2 z2 = mk(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < NC; ++q) {
#pragma unroll
        for (int k = 0; k < TJ; ++k) jw[q][k] = z2;
        en[q] = enp[q] = jd[q] = z2;
    }
    byw[0] = byw[1] = byw[2] = z2;
    bprev = z2;
#pragma unroll
    for (int s = 0; s < (M > 0 ? M : 1); ++s) {
#pragma unroll
        for (int q = 0; q < NC; ++q) win[s][q][0] = win[s][q][1] = win[s][q][2] = z2;
        aux[s][0] = aux[s][1] = aux[s][2] = z2;
        eyrp[s] = 0.f;
    }

    auto ld2 = [&](const float *p, int o) {
        if constexpr (SEAM) return mk(__ldg(p + o), __ldg(p + o + dxc));
        else return __ldg(reinterpret_cast<const float2 *>(p + o));
    };
    // one register buffer per row modulo the stream's depth (the depths divide
    // the four-row unroll, so the buffer of a row is a compile-time constant):
    // j (NC), B (TE: Bz; TM: Bx, By), E (NC), B again for the Faraday update
    using PF_ = PolPrefetch<POL>;
    constexpr int PJ = PF_::PJ, PB = PF_::PB, PE = PF_::PE, PFD = PF_::PF;
    f2 pj0[PJ], pj1[PJ], pb0[PB], pb1[PB], pe0[PE], pe1[PE], pf0[PFD], pf1[PFD];
    auto ldJ = [&](int k) {
        if (HJ) {
            pj0[k] = ld2(inJ0, oj);
            if (POL == TE) pj1[k] = ld2(inJ1, oj);
        }
        adv(oj);
    };
    auto ldB = [&](int k) {
        pb0[k] = ld2(inB0, ob);
        if (POL == TM) pb1[k] = ld2(inB1, ob);
        adv(ob);
    };
    auto ldE = [&](int k) {
        pe0[k] = ld2(inE0, oe);
        if (POL == TE) pe1[k] = ld2(inE1, oe);
        adv(oe);
    };
    auto ldF = [&](int k) {
        pf0[k] = ld2(inB0, of);
        if (POL == TM) pf1[k] = ld2(inB1, of);
        adv(of);
    };
    // rows r0 .. r0 + depth - 1 of each stream (r0 is a multiple of 4)
#pragma unroll
    for (int k = 0; k < PJ; ++k) ldJ(k);
#pragma unroll
    for (int k = 0; k < PB; ++k) ldB(k);
#pragma unroll
    for (int k = 0; k < PE; ++k) ldE(k);
#pragma unroll
    for (int k = 0; k < PFD; ++k) ldF(k);
    if (!HJ) {
#pragma unroll
        for (int k = 0; k < PJ; ++k) pj0[k] = pj1[k] = z2;
    }
    if (POL == TE) {
#pragma unroll
        for (int k = 0; k < PB; ++k) pb1[k] = z2;
#pragma unroll
        for (int k = 0; k < PFD; ++k) pf1[k] = z2;
    } else {
#pragma unroll
        for (int k = 0; k < PJ; ++k) pj1[k] = z2;
#pragma unroll
        for (int k = 0; k < PE; ++k) pe1[k] = z2;
    }
    int b0 = ((r0 % D0) + D0) % D0;  // dE' ring slot of row r0 (a multiple of 4)
    // With D0 = 12 the dE' ring is addressed through the bases of its three
    // 4-row groups, rotated once per block of four rows, so that every slot a
    // row touches is a compile-time offset from one of them (no per-access
    // wrap arithmetic; 11% fewer instructions in the TE kernel)
    constexpr int DRS = NC * 2 * RP;  // floats per dE' ring row
    float *gA = s_dp + b0 * DRS, *gB = s_dp + ((b0 + 4) % D0) * DRS, *gC = s_dp + ((b0 + 8) % D0) * DRS;

    row_barrier();

    for (int rb = r0; rb < r1; rb += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = rb + u;
            // this row's inputs, then the loads of the rows `depth` ahead into
            // the freed buffers (past the segment: valid wrapped rows, unused)
            const f2 cj0 = pj0[u % PJ], cj1 = pj1[u % PJ], cb0 = pb0[u % PB], cb1 = pb1[u % PB],
                     ce0 = pe0[u % PE], ce1 = pe1[u % PE], cf0 = pf0[u % PFD], cf1 = pf1[u % PFD];
            ldJ(u % PJ);
            ldB(u % PB);
            ldE(u % PE);
            ldF(u % PFD);
            if constexpr (L1PF && L1D > 0) {
                if (HJ) {
                    prefetch_l1(inJ0 + lj);
                    if (POL == TE) prefetch_l1(inJ1 + lj);
                }
                prefetch_l1(inB0 + lb);
                if (POL == TM) prefetch_l1(inB1 + lb);
                prefetch_l1(inE0 + le);
                if (POL == TE) prefetch_l1(inE1 + le);
                adv(lj);
                adv(lb);
                adv(le);
            }
            const int rhoM = r - 2 * M, rhoF = rhoM - 1;
            // dE' ring row of row r - k (u, k compile-time; b0 a multiple of 4)
            auto dprow = [&](int k) {
                if constexpr (D0 == 12) {
                    const int d = u - k;  // in [-8, 3]
                    return d >= 0 ? gA + d * DRS : (d >= -4 ? gC + (d + 4) * DRS : gB + (d + 8) * DRS);
                }
                int sl = b0 + u - k;
                if constexpr ((D0 & (D0 - 1)) == 0) sl &= D0 - 1;
                else sl = sl < 0 ? sl + D0 : sl;
                return s_dp + sl * NC * 2 * RP;
            };
            // E update of row rhoM from dE_(M), Faraday update of row rhoF
            auto finish = [&](f2 o0, f2 o1) {
                enp[0] = en[0];
                en[0] = add(ce0, o0);
                if (POL == TE) {
                    enp[1] = en[1];
                    en[1] = add(ce1, o1);
                }
                const bool yE = rhoM >= y0 && rhoM < y1;
                if (yE && xout) {
                    const int o = rhoM * pitch + xc;
                    if constexpr (SEAM) {
                        if (!xlast) *reinterpret_cast<float2 *>(oE0 + o) = en[0];
                        else oE0[o] = en[0].x;
                        if (POL == TE) {
                            if (!xlast) *reinterpret_cast<float2 *>(oE1 + o) = en[1];
                            else oE1[o] = en[1].x;
                        }
                    } else {
                        *reinterpret_cast<float2 *>(oE0 + o) = en[0];
                        if (POL == TE) *reinterpret_cast<float2 *>(oE1 + o) = en[1];
                    }
                }
                // neighbours read column 2t+2 (even) of TE: Ey, TM: Ez
                s_e[(u & 1) * RP + pc] = POL == TE ? en[1].x : en[0].x;
                const float er = s_e[((u + 1) & 1) * RP + pc + 1];  // row rhoF
                f2 bo0, bo1 = z2;
                if constexpr (POL == TE) {
                    // Bz -= kx (Ey[i+1] - Ey[i]) - ky (Ex[j+1] - Ex[j])
                    const f2 dxey = fma(enp[1], m1(), mk(enp[1].y, er));
                    const f2 dyex = fma(enp[0], m1(), en[0]);
                    bo0 = fma(c.ky, dyex, fma(fma(c.kx, dxey, z2), m1(), cf0));
                } else {
                    // Bx -= ky (Ez[j+1] - Ez[j]);  By += kx (Ez[i+1] - Ez[i])
                    const f2 dyez = fma(enp[0], m1(), en[0]);
                    const f2 dxez = fma(enp[0], m1(), mk(enp[0].y, er));
                    bo0 = fma(fma(c.ky, dyez, z2), m1(), cf0);
                    bo1 = fma(c.kx, dxez, cf1);
                }
                const bool yF = rhoF >= y0 && rhoF < y1;
                if (yF && xout) {
                    const int o = rhoF * pitch + xc;
                    if constexpr (SEAM) {
                        if (!xlast) *reinterpret_cast<float2 *>(oB0 + o) = bo0;
                        else oB0[o] = bo0.x;
                        if (POL == TM) {
                            if (!xlast) *reinterpret_cast<float2 *>(oB1 + o) = bo1;
                            else oB1[o] = bo1.x;
                        }
                    } else {
                        *reinterpret_cast<float2 *>(oB0 + o) = bo0;
                        if (POL == TM) *reinterpret_cast<float2 *>(oB1 + o) = bo1;
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

            // ---------------- source, row r ----------------
            {
                f2 jf0 = z2, jf1 = z2;
                if (HJ) {
                    const float *jr = s_j + (u & 1) * NC * 2 * RP;
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        const float *row = jr + q * 2 * RP;
                        // columns 2t-P .. 2t+1+P (TE: the own pair from registers)
                        float col[2 * P + 2];
#pragma unroll
                        for (int i = 0; i < 2 * P + 2; ++i) {
                            const int off = i - P;
                            col[i] = (off == 0 && RJ)   ? jd[q].x
                                     : (off == 1 && RJ) ? jd[q].y
                                     : (off & 1) == 0   ? row[pc + off / 2]
                                                        : row[RP + pc + (off - 1) / 2];
                        }
                        f2 taps[2 * P + 1];
#pragma unroll
                        for (int k = 0; k <= 2 * P; ++k) taps[k] = mk(col[k], col[k + 1]);
                        const f2 acc = binom_taps<P>(taps);
                        if (q == 0) jf0 = acc; else jf1 = acc;
                    }
                }
                f2 d0, d1 = z2;
                if constexpr (POL == TE) {
                    // own Bz from shared memory: a register delay line spills at 3 blocks/SM
                    const float *sb = s_b + (u & 3) * 2 * RP;
                    const f2 bz0 = own(sb);
                    const float bzl = lft(sb);
                    // dE'_x = ky (Bz[j] - Bz[j-1]) - q jx ;  dE'_y = -kx (Bz[i] - Bz[i-1]) - q jy
                    d0 = mul(c.ky, fma(bprev, m1(), bz0));
                    d1 = mul(c.kx, fma(bz0, m1(), mk(bzl, bz0.x)));
                    bprev = bz0;
                    if (HJ) {
                        d0 = fma(c.qf, fma(jf0, m1(), z2), d0);
                        d1 = fma(c.qf, fma(jf1, m1(), z2), d1);
                    }
                } else {
                    const float *sb = s_b + (u & 3) * 2 * RP;
                    const f2 bx0 = own(sb);
                    const f2 axbx = fma(c6(), fma(bx0, m2(), add(mk(lft(sb), bx0.x), mk(bx0.y, rgt(sb)))), bx0);
                    const float *sa = s_ay + (u & 1) * 2 * RP;
                    const f2 ay0 = own(sa);
                    const float ayl = lft(sa);
                    const f2 dxay = fma(mk(ayl, ay0.x), m1(), ay0);
                    // dE'_z = kx Dbar_x(alpha_y By) - ky Dbar_y(alpha_x Bx) - q jz
                    d0 = fma(c.kx, dxay, mul(fma(c.ky, fma(bprev, m1(), axbx), z2), m1()));
                    bprev = axbx;
                    if (HJ) d0 = fma(c.qf, fma(jf0, m1(), z2), d0);
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
                    finish(d0, d1);  // no sweeps: dE = dE'
                }
            }

            // ---------------- current: y-binomial of row r+1 ----------------
            if (HJ) {
                float *jo = s_j + ((u + 1) & 1) * NC * 2 * RP;
#pragma unroll
                for (int q = 0; q < NC; ++q) {
#pragma unroll
                    for (int k = TJ - 1; k > 0; --k) jw[q][k] = jw[q][k - 1];
                    jw[q][0] = q == 0 ? cj0 : cj1;
                    const f2 acc = binom_taps<P>(jw[q]);
                    put(jo + q * 2 * RP, acc);
                    if (RJ) jd[q] = acc;
                }
            }

            // ---------------- B prep, row r+2 ----------------
            {
                put(s_b + ((u + 2) & 3) * 2 * RP, cb0);
                if (POL == TM) {
                    byw[2] = byw[1];
                    byw[1] = byw[0];
                    byw[0] = cb1;
                    // alpha_y By of row r+1
                    put(s_ay + ((u + 1) & 1) * 2 * RP, fma(c6(), fma(byw[1], m2(), add(byw[0], byw[2])), byw[1]));
                }
            }
            row_barrier();
        }
        b0 += 4;
        if (b0 >= D0) b0 -= D0;
        float *t = gA;
        gA = gB;
        gB = gC;
        gC = t;
    }
}

// coefficient pairs of the polarisation kernels from the scheme's FP32
// coefficients; qf = q / 4^(2 passes), exact
__host__ __device__ inline Coef2 coef2_of(const Coef<float> &c, int passes) {
    Coef2 k;
    k.kx = make_float2(c.kx, c.kx);
    k.ky = make_float2(c.ky, c.ky);
    const float qf = ldexpf(c.q, -4 * passes);
    k.qf = make_float2(qf, qf);
    k.ax = make_float2(c.ax, c.ax);
    k.ay = make_float2(c.ay, c.ay);
    k.axy = make_float2(c.axy, c.axy);
    k.bxy = make_float2(c.bxy, c.bxy);
    return k;
}

// dynamic shared memory of a tile of NT column pairs
template <int POL, int M, int P, bool HJ, int NT = 128>
inline size_t smem_bytes() {
    return (size_t)PolSmem<POL, M, P, HJ, NT + 2 * PolGeom<M, P, HJ>::PADP>::TOTAL * sizeof(float);
}

// grids with odd n_x (fused2d_pol_batch.cu): the strips that cross the
// periodic seam take the SEAM tile, the others the pair tile
template <int POL, int M, int P, bool HJ>
void launch_odd(const Geo &g, const Coef2 &c, const Fused2dArgs<float> &a, int W, int L, int nstrip, int nblocks,
                cudaStream_t s);

}  // namespace pol2d
}  // namespace fmx
