// Internal declarations shared by the host API (fmx_api.cpp) and the CUDA
// kernels of the field advance.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fmx.h"

namespace fmx {

// Scalar factors of the step in the kernels' arithmetic type; same order and
// meaning as fmx_coefficients() (Eqs. ampere_aux_x..z, matrixA_1st..last).
template <typename T>
struct Coef {
    T kx, ky, kz;      // c dt / d_i
    T q;               // 4 pi dt
    T c6;              // 1/6: alpha = 1 + c6 Dbar^2
    T ax, ay, az;      // (sigma_i - 1)/6, coefficient of Dbar_ii
    T ayz, azx, axy;   // (sigma_i + sigma_j - 1)/36, coefficient of Dbar_iijj
    T byz, bzx, bxy;   // -sigma_ij/6, coefficient of Dbar_ij (1 + Dbar_kk/6)
};

struct Geo {
    int nx, ny, nz;
    int64_t pitch;   // elements per row
    int64_t plane;   // elements per z-plane = pitch * ny
};

// Device-side solver status; lives in the workspace.
struct DevStatus {
    double nrm2;     // ||dE'||^2 of the current solve
    double r2;       // last ||dE_(s+1) - dE_(s)||^2
    int count;       // sweeps done in the current solve
    int done;        // 1 when the current solve stopped
    int noconv;      // 1 when it stopped at m_max
    int err;         // latched device error (FMX_ETIMEOUT, ...)
    double cheb_rho; // Chebyshev mode: rho of the last sweep
    int steps;       // resident engine: steps completed by the last launch
    long long sweeps_total;  // resident engine: sweeps of all those steps
    // resident engine over several clusters: the grid barrier's arrival count
    // and generation, and the clusters' residual partials (two alternating sets)
    unsigned bar_count;
    unsigned bar_gen;
    double xpart[2][8];
};

// Chebyshev acceleration: M = 1 - A has its spectrum in [1 - hi, 1 - lo];
// theta, delta = centre and half-width, sig = theta / delta
struct ChebParams {
    double theta, delta, sig;
};

// Pointers of one staged step (all device).
template <typename T>
struct StagedPtrs {
    T *E[3];
    T *B[3];
    const T *J[3];    // raw current or nullptr
    T *jf[3];         // filtered current (workspace)
    T *tmp;           // one scratch component (workspace)
    T *dEp[3];        // dE' (workspace)
    T *dEa[3];        // sweep ping (workspace)
    T *dEb[3];        // sweep pong (workspace)
    double *partials; // FP64 block partial sums (workspace)
    DevStatus *st;    // status block (workspace)
};

// Number of FP64 partial slots the staged kernels need for a grid.
int64_t staged_partial_slots(const Geo &g);

// Launchers (staged.cu).  Each returns the number of kernels it enqueued.
template <typename T>
int launch_filter_pass(const Geo &g, int dims, const T *in, T *out, int axis, cudaStream_t s);

template <typename T>
int launch_staged_source(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p,
                         const T *const jsrc[3], cudaStream_t s, bool norm);

template <typename T>
int launch_staged_sweep(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p, const T *const in[3],
                        T *const out[3], bool resid, cudaStream_t s);

template <typename T>
int launch_resid_sweep(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p, cudaStream_t s);

int launch_resid_init(double *partials, int64_t nparts, DevStatus *st, cudaStream_t s);

// Chebyshev sweep s = st->count (x in dEp / dEa / dEb by the parity of s as in
// residual mode, the search direction d in jf, updated in place), then the
// single-block update (||d||^2, rho, count; stop test when resid)
template <typename T>
int launch_cheb_sweep(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &p, const ChebParams &cp,
                      cudaStream_t s);
int launch_cheb_update(double *partials, int64_t nparts, DevStatus *st, const ChebParams &cp, bool resid,
                       double tol2, int m_max, cudaStream_t s);
int launch_resid_update(double *partials, int64_t nparts, DevStatus *st, double tol2, int m_max, cudaStream_t s);

template <typename T>
int launch_update_e(const Geo &g, T *const E[3], const T *const dE[3], cudaStream_t s);

template <typename T>
int launch_update_e_resid(const Geo &g, const StagedPtrs<T> &p, cudaStream_t s);

template <typename T>
int launch_faraday(const Geo &g, int dims, const Coef<T> &c, T *const E[3], T *const B[3], cudaStream_t s);

// 3D z-marching kernels (march3d.cu): source with at most one binomial pass
// on the current fused in, and one sweep of Algorithm 1.
bool march3d_supported(int dims, int passes);
template <typename T>
int launch_march3d_source(const Geo &g, const Coef<T> &c, const T *const B[3], const T *const J[3], int passes,
                          T *const out[3], cudaStream_t s);
template <typename T>
int launch_march3d_sweep(const Geo &g, const Coef<T> &c, const T *const dEp[3], const T *const in[3], T *const out[3],
                         cudaStream_t s, bool update = false);
// Two sweeps of Algorithm 1 in one z-march pass (FP32 column pairs); with
// update the second applies E^{n+1} = E^n + dE into out.  Returns 0 (nothing
// launched) where that path does not apply.
template <typename T>
int launch_march3d_sweeps2(const Geo &g, const Coef<T> &c, const T *const dEp[3], const T *const in[3],
                           T *const out[3], cudaStream_t s, bool update);
// Faraday of the 3D FP32 column-pair path; returns 0 (nothing launched) where
// that path does not apply
template <typename T>
int launch_march3d_faraday(const Geo &g, const Coef<T> &c, const T *const E[3], T *const B[3], cudaStream_t s);

// Resident engine (resident.cu): nsteps whole steps in one launch of one
// thread-block cluster (grids small enough to stay in L2).  Algorithm 1 with
// m sweeps, or to the residual stop when resid; jpasses binomial passes on the
// current (once per launch, into P.jf).  Results in P.st (count = sweeps of
// the last step, steps, sweeps_total, noconv).  Returns 1, or -1 when the
// launch failed.
// Returns the clusters launched (one launch), or -1 when the launch failed.
// wait: the bounded software wait of a launch over several clusters (its
// limit in SM clock cycles; lost_arrival makes the wait expect one cluster
// more than exist, so that it must time out: a self-test of that path).
struct ResidentWait {
    long long limit_cycles;
    int lost_arrival;
};
template <typename T>
int launch_resident(const Geo &g, int dims, const Coef<T> &c, const StagedPtrs<T> &P, int nsteps, bool resid, int m,
                    double tol2, int m_max, int jpasses, const ResidentWait &wait, cudaStream_t s);
// clusters the resident engine launches for a grid of `cells` cells
template <typename T>
int resident_clusters(int dims, int64_t cells, bool lost_arrival);
// CTAs in the cluster the resident kernel launches with (16 where the device
// runs clusters of 16, else 8)
template <typename T>
int resident_cluster_size(int dims);

// Diagnostics (diag.cu): writes 6 FP64 values to out_dev (w_scheme sum,
// w_plain sum, divb max, divb sum sq, gauss max, gauss sum sq).
template <typename T>
int launch_diagnostics(const Geo &g, int dims, const Coef<double> &c, const double d[3], T *const E[3],
                       T *const B[3], double *partials, int64_t nparts, double *out_dev, cudaStream_t s);

// Adjoint step and Gaussian-envelope current (adjoint.cu).
template <typename T>
int launch_adj_source(const Geo &g, int dims, const Coef<T> &c, T *const Eb[3], T *const Bb[3], T *const u[3],
                      cudaStream_t s);
template <typename T>
int launch_adj_faraday(const Geo &g, int dims, const Coef<T> &c, T *const w[3], T *const Bb[3], cudaStream_t s);
template <typename T>
int launch_scale_copy(const Geo &g, T sc, T *const in[3], T *const out[3], cudaStream_t s);
// Gaussian-envelope current (device pointers into the grid's small region):
// amplitudes a_p = amp[p], or theta[p] sin(omega0 t + phi[p]) when amp is
// nullptr; for the projection, phi != nullptr and weights == nullptr make the
// weights sin(omega0 t + phi[p]).
struct GaussSrc {
    int np;
    const double *cxy, *amp, *theta, *phi;
    double omega0, t, width;
};
template <typename T>
int launch_gauss_source(const Geo &g, const GaussSrc &gs, T *const J[3], bool zero_xy, cudaStream_t s);
// partials: scratch of cap doubles; returns the launches or -1 when cap < np
template <typename T>
int launch_gauss_project(const Geo &g, const GaussSrc &gs, const T *f, double *partials, int64_t cap,
                         const double *weights, double *out, cudaStream_t s);

}  // namespace fmx
