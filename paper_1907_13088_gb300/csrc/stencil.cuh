// Periodic stencil building blocks of the averaged-Yee step, shared by the
// staged kernels and the FP64 diagnostics.  Each helper reads through an
// accessor F (value at a shifted cell) and computes in the arithmetic type R.
//
//   Dbar_aa f = f[+1] - 2 f[0] + f[-1] along axis a;
//   alpha_a f = f + (1/6) Dbar_aa f, the (1/6, 2/3, 1/6) average of Sec. 2;
//   A (Eqs. matrixA_1st..matrixA_last):
//     A_aa = a_b Dbar_bb + a_c Dbar_cc + a_bc Dbar_bb Dbar_cc,
//     A_ab = b_ab Dbar_a Dbar_b (1 + Dbar_cc / 6),
//   with (a, b, c) a cyclic order of the axes;
//   source (Eqs. ampere_aux_x..z): dE'_a = k_b Dbar_b(alpha_c B_c)
//     - k_c Dbar_c(alpha_b B_b) - q j_a;
//   curl E of Faraday (Eqs. faraday_x..z): k_b Dbar_b E_c - k_c Dbar_c E_b.
// Axes >= DIM are inactive: their Dbar vanish and their alpha is 1.
#pragma once

#include "fmx_internal.h"

namespace fmx {

struct Pos {
    int i, j, k;
};

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Reads component array p (storage type S) at a periodic shift of a cell,
// converted to R.
template <typename S, typename R = S>
struct Field {
    const S *__restrict__ p;
    Geo g;
    __device__ __forceinline__ R operator()(Pos b, int dx, int dy, int dz) const {
        int x = wrapc(b.i + dx, g.nx), y = wrapc(b.j + dy, g.ny), z = wrapc(b.k + dz, g.nz);
        return (R)p[(int64_t)z * g.plane + (int64_t)y * g.pitch + x];
    }
};

__device__ __forceinline__ void unit(int a, int d, int &dx, int &dy, int &dz) {
    dx = a == 0 ? d : 0;
    dy = a == 1 ? d : 0;
    dz = a == 2 ? d : 0;
}

// f at base + o + d e_a
template <typename F>
__device__ __forceinline__ auto at_sh(const F &f, Pos b, const int o[3], int a, int d) {
    int dx, dy, dz;
    unit(a, d, dx, dy, dz);
    return f(b, o[0] + dx, o[1] + dy, o[2] + dz);
}

// Dbar_aa f at base + o
template <typename R, typename F>
__device__ __forceinline__ R d2(const F &f, Pos b, const int o[3], int a) {
    return at_sh(f, b, o, a, 1) - R(2) * at_sh(f, b, o, a, 0) + at_sh(f, b, o, a, -1);
}

// Dbar_aa Dbar_cc f at base
template <typename R, typename F>
__device__ __forceinline__ R d2d2(const F &f, Pos b, int a, int c) {
    int op[3] = {0, 0, 0}, o0[3] = {0, 0, 0}, om[3] = {0, 0, 0};
    op[c] = 1;
    om[c] = -1;
    return d2<R>(f, b, op, a) - R(2) * d2<R>(f, b, o0, a) + d2<R>(f, b, om, a);
}

template <typename T>
__device__ __forceinline__ T coef_diag(const Coef<T> &c, int a) {
    return a == 0 ? c.ax : (a == 1 ? c.ay : c.az);
}
// coefficient of Dbar_bbcc in A_aa (b, c the other two axes)
template <typename T>
__device__ __forceinline__ T coef_pair(const Coef<T> &c, int a) {
    return a == 0 ? c.ayz : (a == 1 ? c.azx : c.axy);
}
// coefficient of the cross element A_ab, indexed by the third axis
template <typename T>
__device__ __forceinline__ T coef_cross(const Coef<T> &c, int third) {
    return third == 0 ? c.byz : (third == 1 ? c.bzx : c.bxy);
}
template <typename T>
__device__ __forceinline__ T coef_k(const Coef<T> &c, int a) {
    return a == 0 ? c.kx : (a == 1 ? c.ky : c.kz);
}

// (A dE)_a at base.  E_b enters A_ab through Dbar_a (forward: the result sits
// half a cell off along a) Dbar_b (backward: E_b sits half a cell off along
// b) (1 + Dbar_cc/6), c the third axis.
template <typename R, int DIM, int A, typename F>
__device__ __forceinline__ R apply_a(const F f[3], Pos p, const Coef<R> &c) {
    constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
    constexpr bool aa = A < DIM, ab = B < DIM, ac = C < DIM;
    const int o0[3] = {0, 0, 0};
    R r = R(0);
    if (ab) r += coef_diag(c, B) * d2<R>(f[A], p, o0, B);
    if (ac) r += coef_diag(c, C) * d2<R>(f[A], p, o0, C);
    if (ab && ac) r += coef_pair(c, A) * d2d2<R>(f[A], p, B, C);
    if (aa && ab) {  // A_ab E_b, weight (1 + Dbar_cc/6)
        R w[4];
        const int sa[4] = {1, 1, 0, 0}, sb[4] = {0, -1, 0, -1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int o[3] = {0, 0, 0};
            o[A] = sa[q];
            o[B] = sb[q];
            R v = f[B](p, o[0], o[1], o[2]);
            if (ac) v += c.c6 * d2<R>(f[B], p, o, C);
            w[q] = v;
        }
        r += coef_cross(c, C) * (w[0] - w[1] - w[2] + w[3]);
    }
    if (aa && ac) {  // A_ac E_c, weight (1 + Dbar_bb/6)
        R w[4];
        const int sa[4] = {1, 1, 0, 0}, sc[4] = {0, -1, 0, -1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int o[3] = {0, 0, 0};
            o[A] = sa[q];
            o[C] = sc[q];
            R v = f[C](p, o[0], o[1], o[2]);
            if (ab) v += c.c6 * d2<R>(f[C], p, o, B);
            w[q] = v;
        }
        r += coef_cross(c, B) * (w[0] - w[1] - w[2] + w[3]);
    }
    return r;
}

// dE'_a without the current term: k_b Dbar_b(alpha_c B_c) - k_c Dbar_c(alpha_b B_b),
// both differences backward (B sits half a cell off along them).
template <typename R, int DIM, int A, typename F>
__device__ __forceinline__ R curl_alpha_b(const F b[3], Pos p, const Coef<R> &c) {
    constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
    constexpr bool ab = B < DIM, ac = C < DIM;
    R r = R(0);
    if (ab) {
        int o0[3] = {0, 0, 0}, om[3] = {0, 0, 0};
        om[B] = -1;
        R v0 = at_sh(b[C], p, o0, B, 0), v1 = at_sh(b[C], p, om, B, 0);
        if (ac) {
            v0 += c.c6 * d2<R>(b[C], p, o0, C);
            v1 += c.c6 * d2<R>(b[C], p, om, C);
        }
        r += coef_k(c, B) * (v0 - v1);
    }
    if (ac) {
        int o0[3] = {0, 0, 0}, om[3] = {0, 0, 0};
        om[C] = -1;
        R v0 = at_sh(b[B], p, o0, C, 0), v1 = at_sh(b[B], p, om, C, 0);
        if (ab) {
            v0 += c.c6 * d2<R>(b[B], p, o0, B);
            v1 += c.c6 * d2<R>(b[B], p, om, B);
        }
        r -= coef_k(c, C) * (v0 - v1);
    }
    return r;
}

// c dt (curl E)_a at a B_a position: k_b Dbar_b E_c - k_c Dbar_c E_b, both
// forward (E sits on integer positions along them).
template <typename R, int DIM, int A, typename F>
__device__ __forceinline__ R curl_e(const F e[3], Pos p, const Coef<R> &c) {
    constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
    const int o0[3] = {0, 0, 0};
    R r = R(0);
    if (B < DIM) r += coef_k(c, B) * (at_sh(e[C], p, o0, B, 1) - at_sh(e[C], p, o0, B, 0));
    if (C < DIM) r -= coef_k(c, C) * (at_sh(e[B], p, o0, C, 1) - at_sh(e[B], p, o0, C, 0));
    return r;
}

}  // namespace fmx
