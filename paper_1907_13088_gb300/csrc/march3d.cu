// 3D z-marching kernels for the source (with the one-pass current filter) and
// the sweeps of Algorithm 1.  A CTA owns a TX x TY column tile and walks a
// segment of z planes; each input plane of the tile, with a one-cell halo in
// x and y, is loaded once into a 4-slot shared-memory ring, so that every
// stencil of the step (the A operator of Eqs. matrixA_1st..matrixA_last, the
// averaged curl of Eqs. ampere_aux_x..z, the 27-point binomial) reads its
// neighbours from shared memory.  One __syncthreads per plane: plane k+1 goes
// into slot (k+1) & 3 while slots (k-1..k+1) & 3 are read for plane k, and the
// slot written next, (k+2) & 3, is none of them.  The stencil arithmetic is
// the staged engine's (stencil.cuh), read through a ring accessor.
#include <cuda_runtime.h>

#include "fmx_internal.h"
#include "stencil.cuh"

namespace fmx {
namespace {

constexpr int TX = 32, TY = 8, NTH = TX * TY;  // tile and threads
constexpr int RW = TX + 2, RH = TY + 2, PL = RW * RH;  // a tile plane with its halo
constexpr int ZSEG = 32;                                // planes per CTA

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

// Loads of the tile's planes with their halo: a thread owns cells q = tid and
// q = tid + NTH (when < PL) of every plane; their in-plane offsets are fixed,
// so they are computed once.  fetch(k) reads plane k (periodic) of the N
// components into registers, commit(slot) stores them into the ring; the
// loop fetches plane k+2 while it computes plane k.
template <typename T, int N>
struct PlaneLoader {
    const T *src[N];
    int off0, off1;  // in-plane offsets of the thread's cells (off1 < 0: none)
    int q0, q1;
    T v0[N], v1[N];
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
    __device__ __forceinline__ void fetch(const Geo &g, int k) {
        const int64_t base = (int64_t)wrapm(k, g.nz) * g.plane;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            v0[c] = src[c][base + off0];
            if (q1 >= 0) v1[c] = src[c][base + off1];
        }
    }
    __device__ __forceinline__ void commit(T *ring, int slot) const {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            ring[(slot * N + c) * PL + q0] = v0[c];
            if (q1 >= 0) ring[(slot * N + c) * PL + q1] = v1[c];
        }
    }
};

template <typename T, int N>
__device__ __forceinline__ void ring_fields(Ring<T> f[N], const T *ring, int k) {
    const int cell = (threadIdx.y + 1) * RW + threadIdx.x + 1;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        f[c].base = ring + c * PL;
        f[c].sm1 = ((k - 1) & 3) * N * PL;
        f[c].s0 = (k & 3) * N * PL;
        f[c].sp1 = ((k + 1) & 3) * N * PL;
        f[c].cell = cell;
    }
}

// out = dEp + A in (one sweep of Algorithm 1), 3D.  (A register window of the
// 3 x 3 x 3 neighbourhood per component, read once per plane, was measured
// slower: 111 registers leave 2 CTAs per SM.)
template <typename T>
__global__ void __launch_bounds__(NTH) k3_sweep(Geo g, Coef<T> c, const T *p0, const T *p1, const T *p2,
                                                const T *i0, const T *i1, const T *i2, T *o0, T *o1, T *o2) {
    extern __shared__ __align__(16) unsigned char m3raw[];
    T *ring = reinterpret_cast<T *>(m3raw);  // [4][3][PL]
    const T *in[3] = {i0, i1, i2};
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    PlaneLoader<T, 3> ld;
    ld.init(in, g, x0, y0);
    ld.fetch(g, z0 - 1);
    ld.commit(ring, (z0 - 1) & 3);
    ld.fetch(g, z0);
    ld.commit(ring, z0 & 3);
    ld.fetch(g, z0 + 1);
    Pos p;
    p.i = x0 + threadIdx.x;
    p.j = y0 + threadIdx.y;
    const bool inside = p.i < g.nx && p.j < g.ny;
    for (int k = z0; k < z1; ++k) {
        ld.commit(ring, (k + 1) & 3);
        if (k + 1 < z1) ld.fetch(g, k + 2);
        __syncthreads();
        if (inside) {
            p.k = k;
            Ring<T> f[3];
            ring_fields<T, 3>(f, ring, k);
            const int64_t idx = (int64_t)k * g.plane + (int64_t)p.j * g.pitch + p.i;
            o0[idx] = p0[idx] + apply_a<T, 3, 0>(f, p, c);
            o1[idx] = p1[idx] + apply_a<T, 3, 1>(f, p, c);
            o2[idx] = p2[idx] + apply_a<T, 3, 2>(f, p, c);
        }
    }
}

// dE' = C_b (alpha B) - q F j, 3D, F = one (1/4, 1/2, 1/4) pass along each
// axis (PASSES = 1) or none (PASSES = 0); HJ: a current is bound
template <typename T, int PASSES, bool HJ>
__global__ void __launch_bounds__(NTH) k3_source(Geo g, Coef<T> c, const T *b0, const T *b1, const T *b2,
                                                 const T *j0, const T *j1, const T *j2, T *o0, T *o1, T *o2) {
    constexpr int N = HJ ? 6 : 3;
    extern __shared__ __align__(16) unsigned char m3raw[];
    T *ring = reinterpret_cast<T *>(m3raw);  // [4][N][PL]
    const T *src[6] = {b0, b1, b2, j0, j1, j2};
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * ZSEG, z1 = min(z0 + ZSEG, g.nz);
    PlaneLoader<T, N> ld;
    ld.init(src, g, x0, y0);
    ld.fetch(g, z0 - 1);
    ld.commit(ring, (z0 - 1) & 3);
    ld.fetch(g, z0);
    ld.commit(ring, z0 & 3);
    ld.fetch(g, z0 + 1);
    Pos p;
    p.i = x0 + threadIdx.x;
    p.j = y0 + threadIdx.y;
    const bool inside = p.i < g.nx && p.j < g.ny;
    for (int k = z0; k < z1; ++k) {
        ld.commit(ring, (k + 1) & 3);
        if (k + 1 < z1) ld.fetch(g, k + 2);
        __syncthreads();
        if (inside) {
            p.k = k;
            Ring<T> f[N];
            ring_fields<T, N>(f, ring, k);
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
}

inline dim3 grid3(const Geo &g) { return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (g.nz + ZSEG - 1) / ZSEG); }

}  // namespace

bool march3d_supported(int dims, int passes) { return dims == 3 && passes >= 0 && passes <= 1; }

template <typename T, int N>
size_t ring_bytes() {
    return (size_t)4 * N * PL * sizeof(T);
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

template <typename T>
int launch_march3d_source(const Geo &g, const Coef<T> &c, const T *const B[3], const T *const J[3], int passes,
                          T *const out[3], cudaStream_t s) {
    if (!J || !J[0]) run_source<T, 0, false>(g, c, B, J, out, s);
    else if (passes == 1) run_source<T, 1, true>(g, c, B, J, out, s);
    else run_source<T, 0, true>(g, c, B, J, out, s);
    return 1;
}

template <typename T>
int launch_march3d_sweep(const Geo &g, const Coef<T> &c, const T *const dEp[3], const T *const in[3], T *const out[3],
                         cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k3_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ring_bytes<T, 3>());
        attr = true;
    }
    k3_sweep<T><<<grid3(g), dim3(TX, TY), ring_bytes<T, 3>(), s>>>(g, c, dEp[0], dEp[1], dEp[2], in[0], in[1], in[2],
                                                                   out[0], out[1], out[2]);
    return 1;
}

#define FMX_M3_INST(T)                                                                                           \
    template int launch_march3d_source<T>(const Geo &, const Coef<T> &, const T *const[3], const T *const[3], int, \
                                          T *const[3], cudaStream_t);                                           \
    template int launch_march3d_sweep<T>(const Geo &, const Coef<T> &, const T *const[3], const T *const[3],       \
                                         T *const[3], cudaStream_t);
FMX_M3_INST(float)
FMX_M3_INST(double)
#undef FMX_M3_INST

}  // namespace fmx
