// NCI closed-form tools (Sec. 3, App. E): where a cold beam drifting along x
// at v -> c resonates with the grid's EM mode (Eqs. reson1, reson2), and the
// asymptotic growth rate there (Eq. NCI-growth-rate), on a k_x grid, FP64.
//
// For alias nu (Eq. aliasing_x) the beam line is omega = c k_x' with
// k_x' = k_x + 2 pi nu / dx, taken without time aliasing and only where
// |c k_x' dt| <= pi, the zone of the EM branch.  On that line Eq. reson1 is
//   [k_y]^2 / alpha_y = [omega]^2 / (alpha_t c^2) - [k_x]^2 / alpha_x =: R,
// and [k_y]^2 / alpha_y = (4 / dy^2) G(k_y dy / 2) with
// G(t) = sin^2 t / (1 - 2/3 sin^2 t) (Eq. G), increasing from 0 to 3 on
// [0, pi/2].  So the curve crosses k_x exactly when 0 <= R dy^2 / 4 <= 3, at
//   sin^2(k_y dy / 2) = g / (1 + 2g/3),  g = R dy^2 / 4,
// the k_y >= 0 branch (the mirror -k_y has the same growth rate).  The
// trivial meeting at omega = k = 0 (nu = 0, k_x = 0) is not a crossing.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "fmx.h"

namespace fmx {
void set_last_error(const char *msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 152 * 8;

struct NciCoef {
    double dx, dy, c, dt, omega_p;
    int l, nu_max, nkx;
    int64_t total;
};

__device__ __forceinline__ double ipow(double x, int n) {
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

__device__ __forceinline__ double sinc_half(double h) { return h == 0.0 ? 1.0 : sin(h) / h; }

// One thread per (nu, k_x) sample: row r = nu + nu_max of ky / gamma.
// Also folds the largest gamma into *gmax (its bit pattern: gamma >= 0, so
// unsigned order is numeric order).
__global__ void __launch_bounds__(kThreads) k_nci_resonance(NciCoef q, double *__restrict__ kx_out,
                                                            double *__restrict__ ky_out,
                                                            double *__restrict__ gamma_out,
                                                            unsigned long long *gmax) {
    const double kPi = 3.141592653589793238462643383279502884;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    unsigned long long best = 0ull;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < q.total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / q.nkx);
        const int i = (int)(t - (int64_t)r * q.nkx);
        const int nu = r - q.nu_max;
        const double kx = (2.0 * i + 1.0 - q.nkx) * kPi / ((double)q.nkx * q.dx);
        if (kx_out && r == 0) kx_out[i] = kx;
        const double kxp = kx + 2.0 * kPi * nu / q.dx;
        const double th = 0.5 * q.c * kxp * q.dt;  // omega dt / 2 on the beam line (Eq. reson2)
        double ky = nan, g = 0.0;
        if (kxp != 0.0 && fabs(2.0 * th) <= kPi) {  // omega = k = 0 meets trivially: no crossing
            double sth, cth, sxh, cxh;
            sincos(th, &sth, &cth);
            sincos(0.5 * kx * q.dx, &sxh, &cxh);
            const double x0 = sth / (0.5 * q.dt);                       // xi_0 = [omega]
            const double x1 = cth;                                      // xi_1
            const double x2 = 1.0 - (2.0 / 3.0) * sth * sth;            // xi_2 = alpha_t
            const double x3 = -(2.0 / 3.0) * q.dt * sth * cth;          // xi_3 = -dt sin(omega dt) / 3
            const double bx = sxh / (0.5 * q.dx);                       // [k]_x
            const double ax = 1.0 - (2.0 / 3.0) * sxh * sxh;            // alpha_x
            const double R = x0 * x0 / (x2 * q.c * q.c) - bx * bx / ax;
            const double gg = 0.25 * R * q.dy * q.dy;
            if (gg >= 0.0 && gg <= 3.0) {
                const double s2 = gg / (1.0 + (2.0 / 3.0) * gg);
                const double syh = sqrt(s2);
                const double hy = asin(syh);
                ky = 2.0 * hy / q.dy;
                const double by = syh / (0.5 * q.dy);                   // [k]_y
                const double ay = 1.0 - (2.0 / 3.0) * s2;               // alpha_y
                const double sgn = (nu & 1) ? -1.0 : 1.0;               // (-1)^nu
                // Eq. NCI-growth-rate with the momentum-conserving S factors
                const double shape = q.omega_p * ipow(sinc_half(0.5 * kxp * q.dx), q.l + 1) *
                                     ipow(sinc_half(hy), q.l + 1);
                const double num = q.c * q.c * by * ky * (ax * x0 * cth * sgn - x2 * q.c * bx);
                const double den = x0 * x0 * ax * ay * (2.0 * x1 - x3 * x0 / x2);
                g = 0.8660254037844386467637231707529362 * cbrt(shape * shape) * cbrt(fabs(num / den));
            }
        }
        ky_out[t] = ky;
        gamma_out[t] = g;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(g);
        if (g == g && bits > best) best = bits;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, best, o);
        best = v > best ? v : best;
    }
    if ((threadIdx.x & 31) == 0 && best && gmax) atomicMax(gmax, best);
}

// Lowest flat index whose gamma equals the maximum.
__global__ void __launch_bounds__(kThreads) k_nci_argmax(const double *__restrict__ gamma, int64_t total,
                                                         const unsigned long long *gmax,
                                                         unsigned long long *idx) {
    const unsigned long long m = *gmax;
    unsigned long long first = ~0ull;
    if (m) {
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x) {
            if ((unsigned long long)__double_as_longlong(gamma[t]) == m) {
                first = (unsigned long long)t;
                break;  // later t of this thread are larger
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_xor_sync(0xffffffffu, first, o);
        first = v < first ? v : first;
    }
    if ((threadIdx.x & 31) == 0 && first != ~0ull) atomicMin(idx, first);
}

// best = (gamma_max, k_x, k_y, nu) from the two reduction words it holds.
__global__ void k_nci_best(NciCoef q, const double *__restrict__ ky, double *best) {
    const double kPi = 3.141592653589793238462643383279502884;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const unsigned long long m = reinterpret_cast<const unsigned long long *>(best)[0];
    const unsigned long long t = reinterpret_cast<const unsigned long long *>(best)[1];
    if (!m || t == ~0ull) {
        best[0] = 0.0;
        best[1] = best[2] = best[3] = nan;
        return;
    }
    const int r = (int)(t / (unsigned long long)q.nkx);
    const int i = (int)(t - (unsigned long long)r * q.nkx);
    best[0] = __longlong_as_double((long long)m);
    best[1] = (2.0 * i + 1.0 - q.nkx) * kPi / ((double)q.nkx * q.dx);
    best[2] = ky[t];
    best[3] = (double)(r - q.nu_max);
}

fmx_status invalid(const char *msg) {
    fmx::set_last_error(msg);
    return FMX_EINVAL;
}

fmx_status cuda_error(cudaError_t e, const char *what) {
    char msg[256];
    snprintf(msg, sizeof(msg), "fmx_nci_resonance: %s: %s", what, cudaGetErrorString(e));
    fmx::set_last_error(msg);
    return FMX_ECUDA;
}

}  // namespace

extern "C" fmx_status fmx_nci_resonance(const fmx_nci_params *p, double *kx, double *ky, double *gamma,
                                        double *best, void *stream) {
    if (!p) return invalid("fmx_nci_resonance: params is NULL");
    if (!ky || !gamma) return invalid("fmx_nci_resonance: ky and gamma must be device arrays");
    if (!(p->dx > 0.0 && p->dy > 0.0 && p->c > 0.0) || !isfinite(p->dx) || !isfinite(p->dy) || !isfinite(p->c))
        return invalid("fmx_nci_resonance: dx, dy and c must be finite and > 0");
    if (!(p->courant > 0.0 && p->courant <= 1.0))
        return invalid("fmx_nci_resonance: courant must lie in (0, 1] (dt <= dt_CFL)");
    if (!(p->omega_p >= 0.0) || !isfinite(p->omega_p)) return invalid("fmx_nci_resonance: omega_p must be >= 0");
    if (p->shape_order < 0 || p->shape_order > FMX_NCI_MAX_SHAPE_ORDER)
        return invalid("fmx_nci_resonance: shape_order out of range");
    if (p->nu_max < 0 || p->nu_max > FMX_NCI_MAX_ALIAS) return invalid("fmx_nci_resonance: nu_max out of range");
    if (p->nkx < 1 || p->nkx > FMX_NCI_MAX_KX) return invalid("fmx_nci_resonance: nkx out of range");

    NciCoef q;
    q.dx = p->dx;
    q.dy = p->dy;
    q.c = p->c;
    q.dt = p->courant / (p->c * sqrt(1.0 / (p->dx * p->dx) + 1.0 / (p->dy * p->dy)));
    q.omega_p = p->omega_p;
    q.l = p->shape_order;
    q.nu_max = p->nu_max;
    q.nkx = p->nkx;
    q.total = (int64_t)(2 * p->nu_max + 1) * p->nkx;

    cudaStream_t s = (cudaStream_t)stream;
    const int64_t want = (q.total + kThreads - 1) / kThreads;
    const int blocks = (int)(want < kMaxBlocks ? want : kMaxBlocks);
    unsigned long long *words = reinterpret_cast<unsigned long long *>(best);
    cudaError_t e;
    if (best) {
        e = cudaMemsetAsync(words, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(words + 1, 0xff, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync");
    }
    k_nci_resonance<<<blocks, kThreads, 0, s>>>(q, kx, ky, gamma, best ? words : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "k_nci_resonance launch");
    if (best) {
        k_nci_argmax<<<blocks, kThreads, 0, s>>>(gamma, q.total, words, words + 1);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "k_nci_argmax launch");
        k_nci_best<<<1, 1, 0, s>>>(q, ky, best);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "k_nci_best launch");
    }
    return FMX_OK;
}
