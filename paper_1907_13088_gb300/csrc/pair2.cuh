// Packed FP32 pair arithmetic shared by the 2D polarisation kernels (the
// forward step in fused2d_pol.cu, its adjoint in adjoint2d.cu): a thread owns
// two adjacent columns and works on (column 2t, column 2t+1) pairs with the
// FP32x2 instructions.  Internal.
#pragma once

#include <cuda_runtime.h>

namespace fmx {
namespace pair2 {

typedef float2 f2;

__device__ __forceinline__ f2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f2 add(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 mul(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }

// coefficient pairs (both lanes equal), kept in the kernels' parameter space.
// qf = q / 4^(2p): the kernels apply the x and y binomials with their integer
// weights C(2p, k) and fold both normalisations into the current's factor
// (a power-of-two scaling, exact in FP32).
struct Coef2 {
    f2 kx, ky, qf, ax, ay, axy, bxy;
};

// binomial coefficient C(2P, k): p passes of (1, 2, 1) along one axis
__host__ __device__ constexpr int binom2(int P, int k) {
    int c = 1;
    for (int i = 0; i < k; ++i) c = c * (2 * P - i) / (i + 1);
    return c;
}

// compile-time pairs: -1, -2 and the 1/6 of alpha = 1 + Dbar^2 / 6 (the
// FP32 coefficient of the scheme: 1/6 rounded once, checked on the host)
__device__ __forceinline__ f2 m1() { return make_float2(-1.f, -1.f); }
__device__ __forceinline__ f2 m2() { return make_float2(-2.f, -2.f); }
__device__ __forceinline__ f2 c6() { return make_float2(1.f / 6.f, 1.f / 6.f); }
__device__ __forceinline__ f2 cst(int v) { return make_float2((float)v, (float)v); }

// unnormalised (2P+1)-tap binomial of v[0..2P] (pairs), symmetric taps folded
template <int P>
__device__ __forceinline__ f2 binom_taps(const f2 *v) {
    if constexpr (P == 0) {
        return v[0];
    } else {
        f2 acc = add(v[0], v[2 * P]);
#pragma unroll
        for (int k = 1; k < P; ++k) acc = __ffma2_rn(cst(binom2(P, k)), add(v[k], v[2 * P - k]), acc);
        return __ffma2_rn(cst(binom2(P, P)), v[P], acc);
    }
}

enum { TE = 0, TM = 1 };

// a hint: the line holding *p is fetched into L1 ahead of a later load of it
// (no register holds it; p must be an address the kernel may load)
__device__ __forceinline__ void prefetch_l1(const float *p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

}  // namespace pair2
}  // namespace fmx
