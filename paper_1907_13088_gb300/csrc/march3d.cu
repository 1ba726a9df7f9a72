// 3D z-marching kernels for the source (with the one-pass current filter) and
// the sweeps of Algorithm 1.  A CTA owns a TX x TY column tile and walks a
// segment of z planes; each input plane of the tile, with a one-cell halo in
// x and y, is copied once into a shared-memory ring, so that every stencil of
// the step (the A operator of Eqs. matrixA_1st..matrixA_last, the averaged
// curl of Eqs. ampere_aux_x..z, the 27-point binomial) reads its neighbours
// from shared memory.  The planes travel by cp.async, several planes ahead
// of the one being computed, so no register holds data in flight: planes
// k-1..k+1 are read while planes k+2..k+RS-2 are on their way (RS ring
// slots), and the sweep's dE' of the thread's own cell rides in a second ring
// of the same depth.  One __syncthreads per plane; the slot refilled after it
// was last read in the previous plane's iteration.  The stencil arithmetic of
// these one-column kernels (FP64, odd n_x) is the staged engine's
// (stencil.cuh), read through a ring accessor.  The FP32 column-pair kernels
// further down factor the A operator and the averaged curl into in-plane
// stencils and 3-point combinations along z, so that they read one plane per
// iteration and carry the z-combinations in registers.
#include <cuda_runtime.h>

#include <type_traits>

#include "fmx_internal.h"
#include "pair2.cuh"
#include "stencil.cuh"

namespace fmx {
namespace {

constexpr int TX = 32, TY = 8, NTH = TX * TY;  // tile and threads
constexpr int RW = TX + 2, RH = TY + 2, PL = RW * RH;  // a tile plane with its halo
constexpr int ZSEG = 32;                                // planes per CTA

// ring slots: 8 for FP32 (five planes in flight), 4 for FP64 (one)
template <typename T>
struct RingDepth {
    static constexpr int RS = sizeof(T) == 4 ? 8 : 4;
    static constexpr int LA = RS - 3;  // copy groups in flight ahead of the plane computed
};

// component c of the ring at a shift (dx, dy in [-1, 1], dz in [-1, 1]) of
// the thread's cell in plane k
template <typename T>
struct Ring {
    const T *base;        // this component's slot-0 plane; slots are `stride` floats apart
    int sm1, s0, sp1;     // slot offsets of planes k-1, k, k+1
    int cell;             // (ty + 1) * RW + tx + 1
    __device__ __forceinline__ T operator()(Pos, int dx, int dy, int dz) const {
        const int so = dz < 0 ? sm1 : (dz > 0 ? sp1 : s0);
        return base[so + cell + dy * RW + dx];
    }
};

__device__ __forceinline__ int wrapm(int v, int n) { return ((v % n) + n) % n; }

// one element, global -> shared, asynchronous (cp.async, 4 or 8 bytes)
template <typename T>
__device__ __forceinline__ void cp_async_el(T *dst, const T *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_pair(float *dst, const float *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Copies of the tile's planes with their halo: a thread owns cells q = tid and
// q = tid + NTH (when < PL) of every plane; their in-plane offsets are fixed,
// so they are computed once.  issue(k) starts the copy of plane k (periodic)
// of the N components into ring slot k mod RS.
template <typename T, int N, int RS>
struct AsyncPlanes {
    const T *src[N];
    int off0, off1;  // in-plane offsets of the thread's cells (off1 < 0: none)
    int q0, q1;
    __device__ __forceinline__ void init(const T *const s[N], const Geo &g, int x0, int y0) {
#pragma unroll
        for (int c = 0; c < N; ++c) src[c] = s[c];
        const int tid = threadIdx.y * TX + threadIdx.x;
        q0 = tid;
        q1 = tid + NTH < PL ? tid + NTH : -1;
        auto off = [&](int q) {
            const int x = wrapm(x0 - 1 + q % RW, g.nx), y = wrapm(y0 - 1 + q / RW, g.ny);
            return y * (int)g.pitch + x;
        };
        off0 = off(q0);
        off1 = q1 >= 0 ? off(q1) : -1;
    }
    __device__ __forceinline__ void issue(T *ring, const Geo &g, int k) const {
        const int64_t base = (int64_t)wrapm(k, g.nz) * g.plane;
        const int slot = k & (RS - 1);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            cp_async_el(ring + (slot * N + c) * PL + q0, src[c] + base + off0);
            if (q1 >= 0) cp_async_el(ring + (slot * N + c) * PL + q1, src[c] + base + off1);
        }
    }
};

template <typename T, int N, int RS>
__device__ __forceinline__ void ring_fields(Ring<T> f[N], const T *ring, int k) {
    const int cell = (threadIdx.y + 1) * RW + threadIdx.x + 1;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        f[c].base = ring + c * PL;
        f[c].sm1 = ((k - 1) & (RS - 1)) * N * PL;
        f[c].s0 = (k & (RS - 1)) * N * PL;
        f[c].sp1 = ((k + 1) & (RS - 1)) * N * PL;
        f[c].cell = cell;
    }
}

// out = dEp + A in (one sweep of Algorithm 1), 3D.  (A register window of the
// 3 x 3 x 3 neighbourhood per component, read once per plane, was measured
// slower: 111 registers leave 2 CTAs per SM.)
template <typename T>
__global__ void __launch_bounds__(NTH) k3_sweep(Geo g, Coef<T> c, const T *p0, const T *p1, const T *p2,
                                                const T *i0, const T *i1, const T *i2, T *o0, T *o1, T *o2) {
    constexpr int RS = RingDepth<T>::RS, LA = RingDepth<T>::LA;
    extern __shared__ __align__(16) unsigned char m3raw[];
    T *ring = reinterpret_cast<T *>(m3raw);  // [RS][3][PL] input planes with halo
    T *own = ring + RS * 3 * PL;             // [RS][3][NTH] dE' of each thread's cell
    const T *in[3] = {i0, i1, i2};
    const T *dp[3] = {p0, p1, p2};
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    const int tid = threadIdx.y * TX + threadIdx.x;
    AsyncPlanes<T, 3, RS> ld;
    ld.init(in, g, x0, y0);
    Pos p;
    p.i = x0 + threadIdx.x;
    p.j = y0 + threadIdx.y;
    const bool inside = p.i < g.nx && p.j < g.ny;
    const int64_t cell = (int64_t)p.j * g.pitch + p.i;
    // copy group m: input plane z0+1+m and dE' plane z0+m (group 0 also planes
    // z0-1 and z0); planes past the segment are not copied (empty groups keep
    // the count)
    auto issue = [&](int m) {
        if (m == 0) {
            ld.issue(ring, g, z0 - 1);
            ld.issue(ring, g, z0);
        }
        if (z0 + 1 + m <= z1) ld.issue(ring, g, z0 + 1 + m);
        const int kd = z0 + m;
        if (inside && kd < z1) {
            const int slot = kd & (RS - 1);
#pragma unroll
            for (int q = 0; q < 3; ++q) cp_async_el(own + (slot * 3 + q) * NTH + tid, dp[q] + (int64_t)kd * g.plane + cell);
        }
        cp_async_commit();
    };
#pragma unroll
    for (int m = 0; m < LA; ++m) issue(m);
    for (int k = z0; k < z1; ++k) {
        cp_async_wait<LA - 1>();  // this thread's copies of group k - z0
        __syncthreads();          // everyone's, and every read of the slots refilled next is done
        issue(k - z0 + LA);
        if (inside) {
            p.k = k;
            Ring<T> f[3];
            ring_fields<T, 3, RS>(f, ring, k);
            const T *d = own + (k & (RS - 1)) * 3 * NTH + tid;
            const int64_t idx = (int64_t)k * g.plane + cell;
            o0[idx] = d[0] + apply_a<T, 3, 0>(f, p, c);
            o1[idx] = d[NTH] + apply_a<T, 3, 1>(f, p, c);
            o2[idx] = d[2 * NTH] + apply_a<T, 3, 2>(f, p, c);
        }
    }
    cp_async_wait<0>();
}

// dE' = C_b (alpha B) - q F j, 3D, F = one (1/4, 1/2, 1/4) pass along each
// axis (PASSES = 1) or none (PASSES = 0); HJ: a current is bound
template <typename T, int PASSES, bool HJ>
__global__ void __launch_bounds__(NTH) k3_source(Geo g, Coef<T> c, const T *b0, const T *b1, const T *b2,
                                                 const T *j0, const T *j1, const T *j2, T *o0, T *o1, T *o2) {
    constexpr int N = HJ ? 6 : 3;
    constexpr int RS = RingDepth<T>::RS, LA = RingDepth<T>::LA;
    extern __shared__ __align__(16) unsigned char m3raw[];
    T *ring = reinterpret_cast<T *>(m3raw);  // [RS][N][PL]
    const T *src[6] = {b0, b1, b2, j0, j1, j2};
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    AsyncPlanes<T, N, RS> ld;
    ld.init(src, g, x0, y0);
    // copy group m: plane z0+1+m (group 0 also planes z0-1 and z0)
    auto issue = [&](int m) {
        if (m == 0) {
            ld.issue(ring, g, z0 - 1);
            ld.issue(ring, g, z0);
        }
        if (z0 + 1 + m <= z1) ld.issue(ring, g, z0 + 1 + m);
        cp_async_commit();
    };
#pragma unroll
    for (int m = 0; m < LA; ++m) issue(m);
    Pos p;
    p.i = x0 + threadIdx.x;
    p.j = y0 + threadIdx.y;
    const bool inside = p.i < g.nx && p.j < g.ny;
    for (int k = z0; k < z1; ++k) {
        cp_async_wait<LA - 1>();
        __syncthreads();
        issue(k - z0 + LA);
        if (inside) {
            p.k = k;
            Ring<T> f[N];
            ring_fields<T, N, RS>(f, ring, k);
            T d[3] = {curl_alpha_b<T, 3, 0>(f, p, c), curl_alpha_b<T, 3, 1>(f, p, c), curl_alpha_b<T, 3, 2>(f, p, c)};
            if constexpr (HJ) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    T jf;
                    if constexpr (PASSES == 1) {
                        // separable binomial: weights (1, 2, 1)/4 per axis
                        jf = T(0);
#pragma unroll
                        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
                            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                                for (int dx = -1; dx <= 1; ++dx) {
                                    const T w = T((2 - dx * dx) * (2 - dy * dy) * (2 - dz * dz)) * T(1.0 / 64.0);
                                    jf += w * f[3 + a](p, dx, dy, dz);
                                }
                    } else {
                        jf = f[3 + a](p, 0, 0, 0);
                    }
                    d[a] -= c.q * jf;
                }
            }
            const int64_t idx = (int64_t)k * g.plane + (int64_t)p.j * g.pitch + p.i;
            o0[idx] = d[0];
            o1[idx] = d[1];
            o2[idx] = d[2];
        }
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// FP32 sweep, two adjacent columns per thread (even n_x).  The tile is 64
// columns x 8 rows; a smem row holds column x0 + j at index j + 2 (j = -1..64),
// so a thread's own pair sits at an even index and is one 8-byte load, and its
// x-neighbours (columns 2t-1 and 2t+2) are single loads.  The A operator is
// evaluated on column pairs with packed FP32x2 arithmetic.  The planes arrive
// by cp.async like the scalar kernel's (8-byte copies of column pairs, 4-byte
// copies of the two halo columns); dE' of the thread's own pair is prefetched
// into registers two planes ahead (E^n, when the sweep also applies the update
// E^{n+1} = E^n + dE, one plane ahead).
using pair2::f2;
constexpr int TXP = 32, TX2 = 2 * TXP;              // threads along x, columns of the tile
constexpr int RW2 = TX2 + 4, PL2 = RW2 * RH;         // smem row and plane (one component)
constexpr int NPC = TXP * RH, NCP2 = NPC + 2 * RH;  // pair copies and halo copies per plane
constexpr int SWEEP_RS = 8;  // ring slots of the pair sweep: one plane read, seven in flight

struct Coef3P {
    f2 ax, ay, az, ayz, azx, axy, byz, bzx, bxy, c6, kx, ky, kz, q;
    f2 q64;  // q / 64: the one-pass 3D binomial with integer weights (exact power-of-two scaling)
};
template <int AX>
__device__ __forceinline__ f2 ck(const Coef3P &c) {
    return AX == 0 ? c.kx : (AX == 1 ? c.ky : c.kz);
}

template <int AX>
__device__ __forceinline__ f2 cdiag(const Coef3P &c) {
    return AX == 0 ? c.ax : (AX == 1 ? c.ay : c.az);
}
template <int AX>
__device__ __forceinline__ f2 cpair(const Coef3P &c) {
    return AX == 0 ? c.ayz : (AX == 1 ? c.azx : c.axy);
}
template <int THIRD>
__device__ __forceinline__ f2 ccross(const Coef3P &c) {
    return THIRD == 0 ? c.byz : (THIRD == 1 ? c.bzx : c.bxy);
}

// Dbar_{ax ax} of component q at offset (ox, oy, oz), on pairs
template <int Q, int AX, typename F>
__device__ __forceinline__ f2 d2p(const F &V, int ox, int oy, int oz) {
    constexpr int ex = AX == 0, ey = AX == 1, ez = AX == 2;
    return pair2::fma(V(Q, ox, oy, oz), pair2::m2(), pair2::add(V(Q, ox + ex, oy + ey, oz + ez), V(Q, ox - ex, oy - ey, oz - ez)));
}

// (A dE)_A on a column pair: the operator of apply_a (stencil.cuh) in 3D
template <int A, typename F>
__device__ __forceinline__ f2 apply_a2(const F &V, const Coef3P &c) {
    using namespace pair2;
    constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
    constexpr int bx = B == 0, by = B == 1, bz = B == 2, cx = C == 0, cy = C == 1, cz = C == 2;
    const f2 dB = d2p<A, B>(V, 0, 0, 0);
    f2 r = mul(cdiag<B>(c), dB);
    r = fma(cdiag<C>(c), d2p<A, C>(V, 0, 0, 0), r);
    const f2 dd = fma(dB, m2(), add(d2p<A, B>(V, cx, cy, cz), d2p<A, B>(V, -cx, -cy, -cz)));
    r = fma(cpair<A>(c), dd, r);
    // A_AB E_B with weight (1 + Dbar_CC / 6) at (o_A, o_B) = (1,0), (1,-1), (0,0), (0,-1)
    auto wb = [&](int oa, int ob) {
        const int ox = (A == 0) * oa + bx * ob, oy = (A == 1) * oa + by * ob, oz = (A == 2) * oa + bz * ob;
        return fma(c.c6, d2p<B, C>(V, ox, oy, oz), V(B, ox, oy, oz));
    };
    r = fma(ccross<C>(c), fma(add(wb(1, -1), wb(0, 0)), m1(), add(wb(1, 0), wb(0, -1))), r);
    // A_AC E_C with weight (1 + Dbar_BB / 6) at (o_A, o_C) = (1,0), (1,-1), (0,0), (0,-1)
    auto wc = [&](int oa, int oc) {
        const int ox = (A == 0) * oa + cx * oc, oy = (A == 1) * oa + cy * oc, oz = (A == 2) * oa + cz * oc;
        return fma(c.c6, d2p<C, B>(V, ox, oy, oz), V(C, ox, oy, oz));
    };
    r = fma(ccross<B>(c), fma(add(wc(1, -1), wc(0, 0)), m1(), add(wc(1, 0), wc(0, -1))), r);
    return r;
}

// a thread's (at most two) copy items of a component plane, and the plane the
// z-march copies next: its index unwrapped (which picks the ring slot) and
// the element offset of the plane wrapped periodically, advanced one plane
// per copy so that no plane index is divided by n_z on the way
struct PairCopies {
    int s[2], o[2];  // smem index within a component plane (-1: none), global in-plane offset
    bool w[2];       // column pair (8 bytes) or halo column (4 bytes)
    int ku;          // next plane, unwrapped
    int64_t off;     // element offset of that plane wrapped into [0, n_z)
    __device__ __forceinline__ void init(const Geo &g, int x0, int y0, int k0) {
        const int tid = threadIdx.y * TXP + threadIdx.x;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int q = tid + r * NTH;
            s[r] = -1;
            o[r] = 0;
            w[r] = false;
            if (q < NCP2) {
                int row, j;
                if (q < NPC) {
                    row = q / TXP;
                    j = 2 * (q % TXP);
                    w[r] = true;
                } else {
                    const int h = q - NPC;
                    row = h / 2;
                    j = (h & 1) ? TX2 : -1;
                }
                const int x = wrapm(x0 + j, g.nx), y = wrapm(y0 - 1 + row, g.ny);
                s[r] = row * RW2 + 2 + j;
                o[r] = y * (int)g.pitch + x;
            }
        }
        ku = k0;
        off = (int64_t)wrapm(k0, g.nz) * g.plane;
    }
    // copies plane ku of the N components into ring slot ku mod RS, then
    // moves on to the next plane
    template <int RS, int N = 3>
    __device__ __forceinline__ void issue_next(float *ring, const float *const src[N], const Geo &g) {
        float *slot = ring + (ku & (RS - 1)) * N * PL2;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (s[r] < 0) continue;
            const int64_t go = off + o[r];
#pragma unroll
            for (int c = 0; c < N; ++c) {
                float *dst = slot + c * PL2 + s[r];
                const float *sp = src[c] + go;
                if (w[r]) cp_async_pair(dst, sp);
                else cp_async_el(dst, sp);
            }
        }
        ++ku;
        off += g.plane;
        if (off == (int64_t)g.nz * g.plane) off = 0;
    }
};

// The A operator factored for a z-march.  Operators along different axes
// commute, so every element of A (Eqs. matrixA_1st..matrixA_last, 3D) is an
// in-plane (x, y) stencil of one z-plane followed by a 3-point combination
// along z:
//   (A dE)_x(k) = a_y P_k + a_z Dzz Ex + a_yz Dzz P + b_xy (G_k + c6 Dzz G) + b_zx (N_k - N_(k-1)),
//   (A dE)_y(k) = a_x Q_k + a_z Dzz Ey + a_zx Dzz Q + b_xy (G'_k + c6 Dzz G') + b_yz (N'_k - N'_(k-1)),
//   (A dE)_z(k) = T_k + H_(k+1) - H_k,
// with Dzz f = f_(k+1) - 2 f_k + f_(k-1) and the in-plane fields
//   P = Dbar_yy Ex,  G = Dbar_x(fwd) Dbar_y(bwd) Ey,  N = Dbar_x(fwd) (Ez + c6 Dbar_yy Ez),
//   Q = Dbar_xx Ey,  G' = Dbar_y(fwd) Dbar_x(bwd) Ex,  N' = Dbar_y(fwd) (Ez + c6 Dbar_xx Ez),
//   T = (a_x Dbar_xx + a_y Dbar_yy + a_xy Dbar_xx Dbar_yy) Ez,
//   H = b_zx Dbar_x(bwd) (Ex + c6 Dbar_yy Ex) + b_yz Dbar_y(bwd) (Ey + c6 Dbar_xx Ey).
// Plane j of the sweep's input therefore reaches outputs j-1, j and j+1
// through the combinations below, computed once from plane j alone (21
// shared-memory loads per column pair against 51 for the 27-point form).
struct PlaneTerms {
    f2 x1, x0, xl;  // x: to outputs j-1 and j+1 (x1), to j (x0), to j+1 (xl = x1 - b_zx N)
    f2 y1, y0, yl;  // y: the same with G', N', Q
    f2 zh, zt;      // z: H to output j-1, T - H to output j
};

template <typename F>
__device__ __forceinline__ PlaneTerms plane_terms(const F &V, const Coef3P &c, f2 bxy6) {
    using namespace pair2;
    auto d2 = [](f2 p, f2 o, f2 m) { return fma(o, m2(), add(p, m)); };  // p - 2 o + m
    auto sub = [](f2 a, f2 b) { return fma(b, m1(), a); };
    // Ex at columns x-1, x and rows y-1, y, y+1
    const f2 ex_m = V(0, 0, -1), ex_0 = V(0, 0, 0), ex_p = V(0, 0, 1);
    const f2 exl_m = V(0, -1, -1), exl_0 = V(0, -1, 0), exl_p = V(0, -1, 1);
    // Ey at columns x-1, x, x+1 and rows y-1, y
    const f2 ey_m = V(1, 0, -1), ey_0 = V(1, 0, 0);
    const f2 eyl_m = V(1, -1, -1), eyl_0 = V(1, -1, 0), eyr_m = V(1, 1, -1), eyr_0 = V(1, 1, 0);
    // Ez at columns x-1..x+1 and rows y-1..y+1: ez[dy + 1][dx + 1]
    f2 ez[3][3];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) ez[dy + 1][dx + 1] = V(2, dx, dy);
    const f2 P = d2(ex_p, ex_0, ex_m), Pl = d2(exl_p, exl_0, exl_m);  // Dbar_yy Ex at x, x-1
    const f2 Q = d2(eyr_0, ey_0, eyl_0), Qm = d2(eyr_m, ey_m, eyl_m);  // Dbar_xx Ey at y, y-1
    const f2 G = sub(sub(eyr_0, ey_0), sub(eyr_m, ey_m));
    const f2 Gp = sub(sub(ex_p, exl_p), sub(ex_0, exl_0));
    const f2 dxz_m = d2(ez[0][2], ez[0][1], ez[0][0]), dxz_0 = d2(ez[1][2], ez[1][1], ez[1][0]),
             dxz_p = d2(ez[2][2], ez[2][1], ez[2][0]);  // Dbar_xx Ez at y-1, y, y+1
    const f2 dyz_0 = d2(ez[2][1], ez[1][1], ez[0][1]), dyz_r = d2(ez[2][2], ez[1][2], ez[0][2]);  // Dbar_yy Ez at x, x+1
    const f2 N = sub(fma(c.c6, dyz_r, ez[1][2]), fma(c.c6, dyz_0, ez[1][1]));
    const f2 Np = sub(fma(c.c6, dxz_p, ez[2][1]), fma(c.c6, dxz_0, ez[1][1]));
    const f2 T = fma(c.axy, d2(dxz_p, dxz_0, dxz_m), fma(c.ay, dyz_0, mul(c.ax, dxz_0)));
    const f2 X = sub(fma(c.c6, P, ex_0), fma(c.c6, Pl, exl_0));
    const f2 Y = sub(fma(c.c6, Q, ey_0), fma(c.c6, Qm, ey_m));
    PlaneTerms t;
    t.zh = fma(c.byz, Y, mul(c.bzx, X));
    t.zt = sub(T, t.zh);
    const f2 bN = mul(c.bzx, N), bNp = mul(c.byz, Np);
    t.x1 = fma(bxy6, G, fma(c.ayz, P, mul(c.az, ex_0)));
    t.x0 = fma(t.x1, m2(), add(bN, fma(c.bxy, G, mul(c.ay, P))));
    t.xl = sub(t.x1, bN);
    t.y1 = fma(bxy6, Gp, fma(c.azx, Q, mul(c.az, ey_0)));
    t.y0 = fma(t.y1, m2(), add(bNp, fma(c.bxy, Gp, mul(c.ax, Q))));
    t.yl = sub(t.y1, bNp);
    return t;
}

// out = dEp + A in, or with UPD: E = E + dEp + A in (the last sweep and the
// update of the step in one pass; E in place).  The CTA marches its input
// planes z0-1..z1 once each: iteration i reads plane z0-1+i from the ring
// (nothing else of the plane is read again), adds its terms to the partial
// outputs held in registers, and completes output plane z0+i-2.  One plane
// is read while the next RS-1 are on their way; one barrier per plane.
template <bool UPD>
__global__ void __launch_bounds__(NTH, UPD ? 2 : 3) k3_sweep2(Geo g, Coef3P c, const float *p0, const float *p1,
                                                             const float *p2, const float *i0, const float *i1,
                                                             const float *i2, float *o0, float *o1, float *o2) {
    using namespace pair2;
    constexpr int RS = SWEEP_RS;
    extern __shared__ __align__(16) unsigned char m3raw[];
    float *ring = reinterpret_cast<float *>(m3raw);  // [RS][3][PL2]
    const float *in[3] = {i0, i1, i2};
    const float *dp[3] = {p0, p1, p2};
    float *out[3] = {o0, o1, o2};
    const int x0 = blockIdx.x * TX2, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    const int np = z1 - z0 + 2;  // input planes z0-1 .. z1
    PairCopies cp;
    cp.init(g, x0, y0, z0 - 1);
    const int px = x0 + 2 * threadIdx.x, py = y0 + threadIdx.y;
    const bool inside = px < g.nx && py < g.ny;
    const int c0 = (threadIdx.y + 1) * RW2 + 2 + 2 * threadIdx.x;
    // copy group i: input plane z0-1+i (empty past the last)
    auto issue = [&](int i) {
        if (i < np) cp.issue_next<RS>(ring, in, g);
        cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < RS - 1; ++i) issue(i);
    // own-pair offsets: of the output completed next, and of the one two
    // planes later (the register prefetch); outputs lie in [z0, z1), no wrap
    int64_t ocell = (int64_t)z0 * g.plane + (int64_t)py * g.pitch + px;
    int64_t pcell = ocell;
    // dE' (and E^n) of the own pair of outputs o and o+1: two register buffers
    f2 pd[2][3], pe[2][3];
    auto prefetch = [&](int b, bool ok) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            pd[b][q] = mk(0.f, 0.f);
            pe[b][q] = mk(0.f, 0.f);
            if (ok) {
                pd[b][q] = __ldg(reinterpret_cast<const float2 *>(dp[q] + pcell));
                if (UPD) pe[b][q] = *reinterpret_cast<const float2 *>(out[q] + pcell);
            }
        }
        pcell += g.plane;
    };
    prefetch(0, inside);
    prefetch(1, inside && z0 + 1 < z1);
    const f2 bxy6 = mul(c.bxy, c.c6);
    f2 xa = mk(0.f, 0.f), xb = xa, ya = xa, yb = xa, za = xa;  // partial outputs o, o+1
    auto step = [&](int i, auto bsel) {
        constexpr int b = decltype(bsel)::value;
        cp_async_wait<RS - 2>();
        __syncthreads();
        issue(i + RS - 1);
        if (inside) {
            const float *pl = ring + ((z0 - 1 + i) & (RS - 1)) * 3 * PL2 + c0;  // the copy's slot of plane z0-1+i
            auto V = [&](int q, int dx, int dy) -> f2 {
                const float *row = pl + q * PL2 + dy * RW2;
                const f2 pr = *reinterpret_cast<const float2 *>(row);
                return dx == 0 ? pr : (dx > 0 ? mk(pr.y, row[2]) : mk(row[-1], pr.x));
            };
            const PlaneTerms t = plane_terms(V, c, bxy6);
            if (i >= 2) {
                // output plane z0 + i - 2 is complete
                f2 r[3] = {add(xa, t.x1), add(ya, t.y1), add(za, t.zh)};
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    r[q] = add(pd[b][q], r[q]);
                    if (UPD) r[q] = add(pe[b][q], r[q]);
                    *reinterpret_cast<float2 *>(out[q] + ocell) = r[q];
                }
                ocell += g.plane;
                prefetch(b, z0 + i < z1);  // output z0 + i, two iterations on
            }
            xa = add(xb, t.x0);
            xb = t.xl;
            ya = add(yb, t.y0);
            yb = t.yl;
            za = t.zt;
        }
    };
    for (int i = 0; i < np; i += 2) {
        step(i, std::integral_constant<int, 0>());
        if (i + 1 < np) step(i + 1, std::integral_constant<int, 1>());
    }
    cp_async_wait<0>();
}

// dE' = C_b (alpha B) - q F j on a column pair, 3D (the source of k3_source,
// curl_alpha_b in stencil.cuh); F = one (1/4, 1/2, 1/4) pass along each axis
// (PASSES = 1) or none.  The averaged curl (Eqs. ampere_aux_x..z) factored
// like the sweep's A, the z-differences moved outside:
//   x: k_y (V_k + c6 Dzz V) - k_z (U_k - U_(k-1)),    V = Dbar_y(bwd) Bz,  U = By + c6 Dbar_yy By,
//   y: k_z (W_k - W_(k-1)) - k_x (V'_k + c6 Dzz V'),  V' = Dbar_x(bwd) Bz, W = Bx + c6 Dbar_xx Bx,
//   z: k_x Dbar_x(bwd) U - k_y Dbar_y(bwd) W          (in-plane),
// so plane j of B reaches outputs j-1, j, j+1 through terms of plane j alone.
struct CurlTerms {
    f2 x1, x0, xl;  // x: to outputs j-1 and j+1 (x1), to j (x0), to j+1 (xl = x1 + k_z U)
    f2 y1, y0, yl;  // y: the same with V' and W
    f2 z;           // z: to output j
};

template <typename F>
__device__ __forceinline__ CurlTerms curl_plane_terms(const F &V, const Coef3P &c, f2 nkxc6, f2 kyc6) {
    using namespace pair2;
    auto d2 = [](f2 p, f2 o, f2 m) { return fma(o, m2(), add(p, m)); };  // p - 2 o + m
    auto sub = [](f2 a, f2 b) { return fma(b, m1(), a); };
    // Bx at columns x-1..x+1 and rows y-1, y
    const f2 bx_m = V(0, 0, -1), bx_0 = V(0, 0, 0);
    const f2 bxl_m = V(0, -1, -1), bxl_0 = V(0, -1, 0), bxr_m = V(0, 1, -1), bxr_0 = V(0, 1, 0);
    // By at columns x-1, x and rows y-1..y+1
    const f2 by_m = V(1, 0, -1), by_0 = V(1, 0, 0), by_p = V(1, 0, 1);
    const f2 byl_m = V(1, -1, -1), byl_0 = V(1, -1, 0), byl_p = V(1, -1, 1);
    // Bz at (x, y-1), (x, y), (x-1, y)
    const f2 bz_m = V(2, 0, -1), bz_0 = V(2, 0, 0), bzl_0 = V(2, -1, 0);
    const f2 U = fma(c.c6, d2(by_p, by_0, by_m), by_0), Ul = fma(c.c6, d2(byl_p, byl_0, byl_m), byl_0);
    const f2 W = fma(c.c6, d2(bxr_0, bx_0, bxl_0), bx_0), Wm = fma(c.c6, d2(bxr_m, bx_m, bxl_m), bx_m);
    const f2 Vy = sub(bz_0, bz_m), Vx = sub(bz_0, bzl_0);
    const f2 kzU = mul(c.kz, U), kzW = mul(c.kz, W);
    CurlTerms t;
    t.x1 = mul(kyc6, Vy);
    t.x0 = fma(t.x1, m2(), sub(mul(c.ky, Vy), kzU));
    t.xl = add(t.x1, kzU);
    t.y1 = mul(nkxc6, Vx);
    t.y0 = fma(t.y1, m2(), sub(kzW, mul(c.kx, Vx)));
    t.yl = sub(t.y1, kzW);
    t.z = sub(mul(c.kx, sub(U, Ul)), mul(c.ky, sub(W, Wm)));
    return t;
}

// Ring: B (and j) planes of the 64 x 8 tile, RS slots.  The CTA marches its
// input planes z0-1..z1 once each, like the sweep: iteration i reads plane
// z0-1+i (B for the curl terms, j for its x-y binomial), and completes output
// plane z0+i-2; the z part of the binomial combines the x-y results of the
// last three planes, kept in registers.  One plane is read while the next
// RS-1 are on their way; one barrier per plane.
template <int RS, int PASSES, bool HJ>
__global__ void __launch_bounds__(NTH, 3) k3_source2(Geo g, Coef3P c, const float *b0, const float *b1,
                                                    const float *b2, const float *j0, const float *j1,
                                                    const float *j2, float *o0, float *o1, float *o2) {
    using namespace pair2;
    constexpr int N = HJ ? 6 : 3;
    extern __shared__ __align__(16) unsigned char m3raw[];
    float *ring = reinterpret_cast<float *>(m3raw);  // [RS][N][PL2]
    const float *src[6] = {b0, b1, b2, j0, j1, j2};
    float *out[3] = {o0, o1, o2};
    const int x0 = blockIdx.x * TX2, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    const int np = z1 - z0 + 2;  // input planes z0-1 .. z1
    PairCopies cp;
    cp.init(g, x0, y0, z0 - 1);
    const int px = x0 + 2 * threadIdx.x, py = y0 + threadIdx.y;
    const bool inside = px < g.nx && py < g.ny;
    const int c0 = (threadIdx.y + 1) * RW2 + 2 + 2 * threadIdx.x;
    // copy group i: input plane z0-1+i (empty past the last)
    auto issue = [&](int i) {
        if (i < np) cp.issue_next<RS, N>(ring, src, g);
        cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < RS - 1; ++i) issue(i);
    int64_t ocell = (int64_t)z0 * g.plane + (int64_t)py * g.pitch + px;
    const f2 nkxc6 = mul(mul(c.kx, c.c6), m1()), kyc6 = mul(c.ky, c.c6);
    f2 xa = mk(0.f, 0.f), xb = xa, ya = xa, yb = xa, za = xa;  // partial outputs o, o+1
    // PASSES = 1: x-y binomial of the current of planes j-2, j-1 (own pair);
    // PASSES = 0: the raw current of plane j-1 in jz[a][1]
    f2 jz[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a) jz[a][0] = jz[a][1] = xa;
    for (int i = 0; i < np; ++i) {
        cp_async_wait<RS - 2>();
        __syncthreads();
        issue(i + RS - 1);
        if (inside) {
            const float *pl = ring + ((z0 - 1 + i) & (RS - 1)) * N * PL2 + c0;  // the copy's slot of plane z0-1+i
            auto V = [&](int q, int dx, int dy) -> f2 {
                const float *row = pl + q * PL2 + dy * RW2;
                const f2 pr = *reinterpret_cast<const float2 *>(row);
                return dx == 0 ? pr : (dx > 0 ? mk(pr.y, row[2]) : mk(row[-1], pr.x));
            };
            const CurlTerms t = curl_plane_terms(V, c, nkxc6, kyc6);
            f2 jn[3];
            if constexpr (HJ) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if constexpr (PASSES == 1) {
                        // separable binomial with integer weights (1, 2, 1) per axis,
                        // the 1/64 folded into q: the x-y part here
                        f2 acc = mk(0.f, 0.f);
#pragma unroll
                        for (int dy = -1; dy <= 1; ++dy) {
                            const f2 rowf = fma(V(3 + a, 0, dy), cst(2), add(V(3 + a, -1, dy), V(3 + a, 1, dy)));
                            acc = fma(cst(2 - dy * dy), rowf, acc);
                        }
                        jn[a] = acc;
                    } else {
                        jn[a] = V(3 + a, 0, 0);
                    }
                }
            }
            if (i >= 2) {
                // output plane z0 + i - 2 is complete
                f2 d[3] = {add(xa, t.x1), add(ya, t.y1), za};
                if constexpr (HJ) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        if constexpr (PASSES == 1) {
                            const f2 jsum = fma(jz[a][1], cst(2), add(jz[a][0], jn[a]));
                            d[a] = fma(mul(c.q64, jsum), m1(), d[a]);
                        } else {
                            d[a] = fma(mul(c.q, jz[a][1]), m1(), d[a]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) *reinterpret_cast<float2 *>(out[q] + ocell) = d[q];
                ocell += g.plane;
            }
            xa = add(xb, t.x0);
            xb = t.xl;
            ya = add(yb, t.y0);
            yb = t.yl;
            za = t.z;
            if constexpr (HJ) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    jz[a][0] = jz[a][1];
                    jz[a][1] = jn[a];
                }
            }
        }
    }
    cp_async_wait<0>();
}

// B -= c dt curl E^{n+1} (Eqs. faraday_x..z) on a column pair, 3D: forward
// differences (curl_e in stencil.cuh) of E from the plane ring
template <int A, typename F>
__device__ __forceinline__ f2 curl_e2(const F &V, const Coef3P &c) {
    using namespace pair2;
    constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
    constexpr int bx = B == 0, by = B == 1, bz = B == 2, cx = C == 0, cy = C == 1, cz = C == 2;
    const f2 r = mul(ck<B>(c), fma(V(C, 0, 0, 0), m1(), V(C, bx, by, bz)));
    return fma(mul(ck<C>(c), fma(V(B, 0, 0, 0), m1(), V(B, cx, cy, cz))), m1(), r);
}

__global__ void __launch_bounds__(NTH, 3) k3_faraday2(Geo g, Coef3P c, const float *e0, const float *e1,
                                                     const float *e2, float *b0, float *b1, float *b2) {
    using namespace pair2;
    constexpr int RS = RingDepth<float>::RS, LA = RingDepth<float>::LA;
    extern __shared__ __align__(16) unsigned char m3raw[];
    float *ring = reinterpret_cast<float *>(m3raw);  // [RS][3][PL2] E^{n+1} planes
    const float *in[3] = {e0, e1, e2};
    float *bo[3] = {b0, b1, b2};
    const int x0 = blockIdx.x * TX2, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    PairCopies cp;
    cp.init(g, x0, y0, z0);
    const int px = x0 + 2 * threadIdx.x, py = y0 + threadIdx.y;
    const bool inside = px < g.nx && py < g.ny;
    const int64_t cell = (int64_t)py * g.pitch + px;
    const int c0 = (threadIdx.y + 1) * RW2 + 2 + 2 * threadIdx.x;
    // copy group m: planes z0, z0+1 (m = 0), plane z0+1+m (m >= 1, up to z1)
    auto issue = [&](int m) {
        if (m == 0) cp.issue_next<RS>(ring, in, g);
        if (z0 + 1 + m <= z1) cp.issue_next<RS>(ring, in, g);
        cp_async_commit();
    };
    // B of the own pair, planes k and k+1: two register buffers
    f2 pb[2][3];
    auto ldown = [&](int k, int b) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            pb[b][q] = mk(0.f, 0.f);
            if (inside && k < z1) pb[b][q] = *reinterpret_cast<const float2 *>(bo[q] + (int64_t)k * g.plane + cell);
        }
    };
#pragma unroll
    for (int m = 0; m < LA; ++m) issue(m);
    ldown(z0, 0);
    ldown(z0 + 1, 1);
    auto step = [&](int k, auto bsel) {
        constexpr int b = decltype(bsel)::value;
        cp_async_wait<LA - 1>();
        __syncthreads();
        issue(k - z0 + LA);
        f2 bv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) bv[q] = pb[b][q];
        ldown(k + 2, b);
        if (inside) {
            const int s0 = (k & (RS - 1)) * 3 * PL2, sp1 = ((k + 1) & (RS - 1)) * 3 * PL2;
            auto V = [&](int q, int dx, int dy, int dz) -> f2 {
                const float *row = ring + (dz > 0 ? sp1 : s0) + q * PL2 + c0 + dy * RW2;
                const f2 pr = *reinterpret_cast<const float2 *>(row);
                return dx == 0 ? pr : (dx > 0 ? mk(pr.y, row[2]) : mk(row[-1], pr.x));
            };
            const f2 r[3] = {curl_e2<0>(V, c), curl_e2<1>(V, c), curl_e2<2>(V, c)};
            const int64_t idx = (int64_t)k * g.plane + cell;
#pragma unroll
            for (int q = 0; q < 3; ++q) *reinterpret_cast<float2 *>(bo[q] + idx) = fma(r[q], m1(), bv[q]);
        }
    };
    for (int k = z0; k < z1; k += 2) {
        step(k, std::integral_constant<int, 0>());
        if (k + 1 < z1) step(k + 1, std::integral_constant<int, 1>());
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Two sweeps of Algorithm 1 in one z-march (temporal blocking, FP32 column
// pairs, even n_x): dE_(s+2) = dE' + A (dE' + A dE_(s)), both sweeps in the
// factored form of plane_terms.  The first sweep (A stage) is evaluated on the
// output tile grown by one cell on every side in x and y (34 pairs x 10 rows
// around the 32 x 8 pairs of the tile), from an input ring whose planes carry
// a halo of two; each plane of dE_(s+1) it completes goes into one of two
// shared-memory plane buffers, which the second sweep (B stage) reads one
// iteration later, so dE_(s+1) never leaves the SM.  352 threads: every
// thread but the last 12 owns a first-sweep pair, the first 256 also the
// second-sweep pair of the tile.  Iteration i: the A stage reads input plane
// z0-2+i and completes first-sweep plane z0+i-3; the B stage reads
// first-sweep plane z0+i-4 and completes output plane z0+i-5.  One barrier
// per iteration.  With UPD the second sweep also applies E^{n+1} = E^n + dE
// (E in place).
constexpr int FRW = 72;                // floats per row: column x0 + j at index j + 4, j in [-4, 67]
constexpr int FIR = 12, FAR = 10;      // rows of an input plane (y0-2..y0+9) and of a first-sweep plane (y0-1..y0+8)
constexpr int FIPL = FRW * FIR, FAPL = FRW * FAR;
constexpr int FNT = 352, FNA = 340, FNB = 256;
constexpr int FRS = 4;                 // input ring slots: one plane read, three in flight
constexpr int FNI = (FRW / 2) * FIR;   // pair copies per input plane and component (432)

template <bool UPD>
__global__ void __launch_bounds__(FNT, 2) k3_sweeps2f(Geo g, Coef3P c, const float *p0, const float *p1,
                                                     const float *p2, const float *i0, const float *i1,
                                                     const float *i2, float *o0, float *o1, float *o2) {
    using namespace pair2;
    extern __shared__ __align__(16) unsigned char m3raw[];
    float *ring = reinterpret_cast<float *>(m3raw);  // [FRS][3][FIPL] input planes, halo 2
    float *abuf = ring + FRS * 3 * FIPL;              // [2][3][FAPL] first-sweep planes, halo 1
    const float *in[3] = {i0, i1, i2};
    const float *dp[3] = {p0, p1, p2};
    float *out[3] = {o0, o1, o2};
    const int x0 = blockIdx.x * TX2, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    const int nin = z1 - z0 + 4;  // input planes z0-2 .. z1+1
    const int tid = threadIdx.x;
    const int64_t vol = (int64_t)g.nz * g.plane;
    // input copy items of this thread (pairs of columns, periodic wrap), and
    // the wrapped offset of the plane copied next
    int cs[2], co[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int q = tid + r * FNT;
        cs[r] = -1;
        co[r] = 0;
        if (q < FNI) {
            const int row = q / (FRW / 2), j = 2 * (q % (FRW / 2)) - 4;
            cs[r] = row * FRW + j + 4;
            co[r] = wrapm(y0 - 2 + row, g.ny) * (int)g.pitch + wrapm(x0 + j, g.nx);
        }
    }
    int64_t koff = (int64_t)wrapm(z0 - 2, g.nz) * g.plane;
    // copy group i: input plane z0-2+i (empty past the last)
    auto issue = [&](int i) {
        if (i < nin) {
            float *slot = ring + ((z0 - 2 + i) & (FRS - 1)) * 3 * FIPL;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (cs[r] < 0) continue;
                const int64_t go = koff + co[r];
#pragma unroll
                for (int q = 0; q < 3; ++q) cp_async_pair(slot + q * FIPL + cs[r], in[q] + go);
            }
            koff += g.plane;
            if (koff == vol) koff = 0;
        }
        cp_async_commit();
    };
    // first-sweep pair (A stage) and second-sweep pair (B stage) of this thread
    const bool hasA = tid < FNA, hasB = tid < FNB;
    const int pa = tid % 34 - 1, ra = tid / 34 - 1;  // pair -1..32, row -1..8
    const int pb = tid % 32, rb = tid / 32;          // pair 0..31, row 0..7
    const int cA = (ra + 2) * FRW + 2 * pa + 4;      // input-plane index of the A pair
    const int wA = (ra + 1) * FRW + 2 * pa + 4;      // first-sweep-plane index of the A pair
    const int cB = (rb + 1) * FRW + 2 * pb + 4;      // first-sweep-plane index of the B pair
    const bool outB = hasB && x0 + 2 * pb < g.nx && y0 + rb < g.ny;
    // own-pair offsets: A's dE' of its next plane (wrapped periodically: the
    // grown tile reaches planes z0-1 and z1), B's next output plane
    const int cellA = wrapm(y0 + ra, g.ny) * (int)g.pitch + wrapm(x0 + 2 * pa, g.nx);
    int64_t aoff = (int64_t)wrapm(z0 - 1, g.nz) * g.plane;
    int64_t bcell = (int64_t)z0 * g.plane + (int64_t)(y0 + rb) * g.pitch + (x0 + 2 * pb);
    f2 pa_d[3], pb_d[3], pb_e[3];  // dE' of A's next plane; dE' (and E^n) of B's next output
    auto load_a = [&]() {
#pragma unroll
        for (int q = 0; q < 3; ++q) pa_d[q] = __ldg(reinterpret_cast<const float2 *>(dp[q] + aoff + cellA));
        aoff += g.plane;
        if (aoff == vol) aoff = 0;
    };
    // B's output plane at offset `at` (bcell, or the plane after it)
    auto load_b = [&](bool ok, int64_t at) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            pb_d[q] = ok ? __ldg(reinterpret_cast<const float2 *>(dp[q] + at)) : mk(0.f, 0.f);
            if (UPD) pb_e[q] = ok ? *reinterpret_cast<const float2 *>(out[q] + at) : mk(0.f, 0.f);
        }
    };
#pragma unroll
    for (int i = 0; i < FRS - 1; ++i) issue(i);
    const f2 bxy6 = mul(c.bxy, c.c6);
    f2 ax_a = mk(0.f, 0.f), ax_b = ax_a, ay_a = ax_a, ay_b = ax_a, az_a = ax_a;  // A: partial planes o, o+1
    f2 bx_a = ax_a, bx_b = ax_a, by_a = ax_a, by_b = ax_a, bz_a = ax_a;          // B: the same
    for (int i = 0; i < nin + 1; ++i) {
        cp_async_wait<FRS - 2>();
        __syncthreads();
        issue(i + FRS - 1);
        // A stage: input plane z0-2+i; completes first-sweep plane z0+i-3 (i >= 2)
        if (hasA && i < nin) {
            if (i == 1) load_a();  // dE' of plane z0-1
            const float *pl = ring + ((z0 - 2 + i) & (FRS - 1)) * 3 * FIPL + cA;
            auto V = [&](int q, int dx, int dy) -> f2 {
                const float *row = pl + q * FIPL + dy * FRW;
                const f2 pr = *reinterpret_cast<const float2 *>(row);
                return dx == 0 ? pr : (dx > 0 ? mk(pr.y, row[2]) : mk(row[-1], pr.x));
            };
            const PlaneTerms t = plane_terms(V, c, bxy6);
            if (i >= 2) {
                float *dst = abuf + ((z0 + i - 3) & 1) * 3 * FAPL + wA;
                *reinterpret_cast<float2 *>(dst) = add(pa_d[0], add(ax_a, t.x1));
                *reinterpret_cast<float2 *>(dst + FAPL) = add(pa_d[1], add(ay_a, t.y1));
                *reinterpret_cast<float2 *>(dst + 2 * FAPL) = add(pa_d[2], add(az_a, t.zh));
                if (i + 1 < nin) load_a();  // dE' of plane z0+i-2, next iteration
            }
            ax_a = add(ax_b, t.x0);
            ax_b = t.xl;
            ay_a = add(ay_b, t.y0);
            ay_b = t.yl;
            az_a = t.zt;
        }
        // B stage: first-sweep plane z0+i-4 (i >= 3); completes output plane z0+i-5 (i >= 5)
        if (hasB && i >= 3) {
            if (i == 4) load_b(outB, bcell);  // output z0
            const float *pl = abuf + ((z0 + i - 4) & 1) * 3 * FAPL + cB;
            auto V = [&](int q, int dx, int dy) -> f2 {
                const float *row = pl + q * FAPL + dy * FRW;
                const f2 pr = *reinterpret_cast<const float2 *>(row);
                return dx == 0 ? pr : (dx > 0 ? mk(pr.y, row[2]) : mk(row[-1], pr.x));
            };
            const PlaneTerms t = plane_terms(V, c, bxy6);
            if (i >= 5) {
                f2 r[3] = {add(bx_a, t.x1), add(by_a, t.y1), add(bz_a, t.zh)};
                if (outB) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        r[q] = add(pb_d[q], r[q]);
                        if (UPD) r[q] = add(pb_e[q], r[q]);
                        *reinterpret_cast<float2 *>(out[q] + bcell) = r[q];
                    }
                }
                bcell += g.plane;
                load_b(outB && z0 + i - 4 < z1, bcell);  // output z0+i-4, next iteration
            }
            bx_a = add(bx_b, t.x0);
            bx_b = t.xl;
            by_a = add(by_b, t.y0);
            by_b = t.yl;
            bz_a = t.zt;
        }
    }
    cp_async_wait<0>();
}

inline dim3 grid3(const Geo &g) { return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + ZSEG - 1) / ZSEG); }

}  // namespace

bool march3d_supported(int dims, int passes) { return dims == 3 && passes >= 0 && passes <= 1; }

template <typename T, int N>
size_t ring_bytes() {
    return (size_t)RingDepth<T>::RS * N * PL * sizeof(T);
}
template <typename T>
size_t sweep_bytes() {
    return ring_bytes<T, 3>() + (size_t)RingDepth<T>::RS * 3 * NTH * sizeof(T);
}

template <typename T, int PASSES, bool HJ>
void run_source(const Geo &g, const Coef<T> &c, const T *const B[3], const T *const J[3], T *const out[3],
                cudaStream_t s) {
    constexpr int N = HJ ? 6 : 3;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k3_source<T, PASSES, HJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_bytes<T, N>());
        attr = true;
    }
    k3_source<T, PASSES, HJ><<<grid3(g), dim3(TX, TY), ring_bytes<T, N>(), s>>>(
        g, c, B[0], B[1], B[2], HJ ? J[0] : nullptr, HJ ? J[1] : nullptr, HJ ? J[2] : nullptr, out[0], out[1], out[2]);
}

bool pair_path(const Geo &g, float *) { return g.nx % 2 == 0 && g.pitch % 2 == 0; }

Coef3P coef3p(const Coef<float> &c) {
    auto pr = [](float v) { return make_float2(v, v); };
    return Coef3P{pr(c.ax), pr(c.ay), pr(c.az), pr(c.ayz), pr(c.azx), pr(c.axy), pr(c.byz), pr(c.bzx), pr(c.bxy),
                  pr(c.c6), pr(c.kx), pr(c.ky), pr(c.kz), pr(c.q), pr(c.q * (1.f / 64.f))};
}

constexpr int SRC_RS = 4;  // source ring slots (six components: 65 KB)

template <int PASSES, bool HJ>
void run_source2(const Geo &g, const Coef<float> &c, const float *const B[3], const float *const J[3],
                 float *const out[3], cudaStream_t s) {
    constexpr int N = HJ ? 6 : 3;
    constexpr size_t bytes = (size_t)SRC_RS * N * PL2 * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k3_source2<SRC_RS, PASSES, HJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        attr = true;
    }
    const dim3 grid((g.nx + TX2 - 1) / TX2, (g.ny + TY - 1) / TY, (g.nz + ZSEG - 1) / ZSEG);
    k3_source2<SRC_RS, PASSES, HJ><<<grid, dim3(TXP, TY), bytes, s>>>(
        g, coef3p(c), B[0], B[1], B[2], HJ ? J[0] : nullptr, HJ ? J[1] : nullptr, HJ ? J[2] : nullptr, out[0], out[1],
        out[2]);
}
bool pair_path(const Geo &, double *) { return false; }

template <bool UPD>
void run_sweep2(const Geo &g, const Coef<float> &c, const float *const dEp[3], const float *const in[3],
                float *const out[3], cudaStream_t s) {
    constexpr size_t bytes = (size_t)SWEEP_RS * 3 * PL2 * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k3_sweep2<UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        attr = true;
    }
    const Coef3P cp = coef3p(c);
    const dim3 grid((g.nx + TX2 - 1) / TX2, (g.ny + TY - 1) / TY, (g.nz + ZSEG - 1) / ZSEG);
    k3_sweep2<UPD><<<grid, dim3(TXP, TY), bytes, s>>>(g, cp, dEp[0], dEp[1], dEp[2], in[0], in[1], in[2], out[0],
                                                     out[1], out[2]);
}

template <bool UPD>
void run_sweeps2f(const Geo &g, const Coef<float> &c, const float *const dEp[3], const float *const in[3],
                  float *const out[3], cudaStream_t s) {
    constexpr size_t bytes = ((size_t)FRS * 3 * FIPL + (size_t)2 * 3 * FAPL) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k3_sweeps2f<UPD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        attr = true;
    }
    const dim3 grid((g.nx + TX2 - 1) / TX2, (g.ny + TY - 1) / TY, (g.nz + ZSEG - 1) / ZSEG);
    k3_sweeps2f<UPD><<<grid, FNT, bytes, s>>>(g, coef3p(c), dEp[0], dEp[1], dEp[2], in[0], in[1], in[2], out[0],
                                             out[1], out[2]);
}

template <typename T>
int launch_march3d_sweeps2(const Geo &g, const Coef<T> &c, const T *const dEp[3], const T *const in[3],
                           T *const out[3], cudaStream_t s, bool update) {
    if constexpr (std::is_same<T, float>::value) {
        if (pair_path(g, (float *)nullptr)) {
            if (update) run_sweeps2f<true>(g, c, dEp, in, out, s);
            else run_sweeps2f<false>(g, c, dEp, in, out, s);
            return 1;
        }
    }
    return 0;  // FP64, odd n_x or a small grid: the caller runs the sweeps one per pass
}

template <typename T>
int launch_march3d_source(const Geo &g, const Coef<T> &c, const T *const B[3], const T *const J[3], int passes,
                          T *const out[3], cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (pair_path(g, (float *)nullptr)) {
            if (!J || !J[0]) run_source2<0, false>(g, c, B, J, out, s);
            else if (passes == 1) run_source2<1, true>(g, c, B, J, out, s);
            else run_source2<0, true>(g, c, B, J, out, s);
            return 1;
        }
    }
    if (!J || !J[0]) run_source<T, 0, false>(g, c, B, J, out, s);
    else if (passes == 1) run_source<T, 1, true>(g, c, B, J, out, s);
    else run_source<T, 0, true>(g, c, B, J, out, s);
    return 1;
}

template <typename T>
int launch_march3d_faraday(const Geo &g, const Coef<T> &c, const T *const E[3], T *const B[3], cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        if (pair_path(g, (float *)nullptr)) {
            constexpr size_t bytes = (size_t)RingDepth<float>::RS * 3 * PL2 * sizeof(float);
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(k3_faraday2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
                attr = true;
            }
            const dim3 grid((g.nx + TX2 - 1) / TX2, (g.ny + TY - 1) / TY, (g.nz + ZSEG - 1) / ZSEG);
            k3_faraday2<<<grid, dim3(TXP, TY), bytes, s>>>(g, coef3p(c), E[0], E[1], E[2], B[0], B[1], B[2]);
            return 1;
        }
    }
    return 0;  // FP64 or odd n_x: the caller launches the one-thread-per-cell kernel
}

template <typename T>
int launch_march3d_sweep(const Geo &g, const Coef<T> &c, const T *const dEp[3], const T *const in[3], T *const out[3],
                         cudaStream_t s, bool update) {
    if constexpr (std::is_same<T, float>::value) {
        if (pair_path(g, (float *)nullptr)) {
            if (update) run_sweep2<true>(g, c, dEp, in, out, s);
            else run_sweep2<false>(g, c, dEp, in, out, s);
            return 1;
        }
    }
    if (update) return 0;  // the scalar sweep does not fuse the update: the caller launches it
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k3_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sweep_bytes<T>());
        attr = true;
    }
    k3_sweep<T><<<grid3(g), dim3(TX, TY), sweep_bytes<T>(), s>>>(g, c, dEp[0], dEp[1], dEp[2], in[0], in[1], in[2],
                                                                   out[0], out[1], out[2]);
    return 1;
}

#define FMX_M3_INST(T)                                                                                           \
    template int launch_march3d_source<T>(const Geo &, const Coef<T> &, const T *const[3], const T *const[3], int, \
                                          T *const[3], cudaStream_t);                                           \
    template int launch_march3d_sweep<T>(const Geo &, const Coef<T> &, const T *const[3], const T *const[3],       \
                                         T *const[3], cudaStream_t, bool);                                        \
    template int launch_march3d_faraday<T>(const Geo &, const Coef<T> &, const T *const[3], T *const[3], cudaStream_t); \
    template int launch_march3d_sweeps2<T>(const Geo &, const Coef<T> &, const T *const[3], const T *const[3],    \
                                           T *const[3], cudaStream_t, bool);
FMX_M3_INST(float)
FMX_M3_INST(double)
#undef FMX_M3_INST

}  // namespace fmx
