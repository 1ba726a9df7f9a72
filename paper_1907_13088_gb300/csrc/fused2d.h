// Fused 2D step: one kernel launch advances (E^n, B^{n+1/2}) to
// (E^{n+1}, B^{n+3/2}) for the whole grid with the current filter, the
// source, m sweeps of Algorithm 1, the E update and the Faraday update kept
// on chip.  Internal; see fused2d.cu.
#pragma once

#include "fmx_internal.h"

namespace fmx {

template <typename T>
struct Fused2dArgs {
    const T *E[3];   // E^n
    const T *B[3];   // B^{n+1/2}
    const T *J[3];   // j^{n+1/2} or nullptr (vacuum)
    T *Eo[3];        // E^{n+1} (must not alias E)
    T *Bo[3];        // B^{n+3/2} (must not alias B)
    int m;           // sweeps of Algorithm 1
    int passes;      // binomial passes on the current (0 when J is nullptr)
};

// True when the fused kernel covers the problem (2D, fixed sweeps, current
// or no filter, instantiated sweep and pass counts).
bool fused2d_supported(const fmx_params *p);

// Enqueues one step; returns the number of kernels launched (1) or -1 when
// the (m, passes) pair is not instantiated.
template <typename T>
int launch_fused2d(const Geo &g, const Coef<T> &c, const Fused2dArgs<T> &a, cudaStream_t s);

// Launch geometry the fused kernel picks for a grid (for tests and the
// roofline bookkeeping): strip width, rows per segment, strips, segments,
// threads per block.
struct Fused2dShape {
    int threads, halo, width, rows, strips, segments;
};
template <typename T>
Fused2dShape fused2d_shape(const Geo &g, int m, int passes);

// FP32 path split by polarisation (fused2d_pol.cu): one TE and one TM launch
// per step, two columns per thread, packed FP32x2 arithmetic.  Needs an even
// n_x (column pairs never straddle the periodic seam).  Returns the number
// of kernels launched or -1.
bool fused2d_pol_supported(const Geo &g);
// s_tm: stream for the TM launch (nullptr: s); the caller orders the two
// seg_rows: rows per segment (0: one wave of CTAs at the measured occupancy)
int launch_fused2d_pol(const Geo &g, const Coef<float> &c, const Fused2dArgs<float> &a, cudaStream_t s,
                       cudaEvent_t *ev = nullptr, cudaStream_t s_tm = nullptr, int seg_rows = 0);
Fused2dShape fused2d_pol_shape(const Geo &g, int m, int passes, int seg_rows = 0);

// Fused 2D adjoint step (adjoint2d.cu), FP32, TE and TM kernels.  Maps
// (Ebar, Bbar) = dL/d(E^{n+1}, B^{n+3/2}) to dL/d(E^n, B^{n+1/2}) and writes
// dL/dj^{n+1/2} for the components whose Jbo pointer is set:
//   u = Ebar - C_b Bbar (the source curl without averaging), Ebar' = u,
//   w = sum_{s<=m} A^s u (the m sweeps of Algorithm 1; A is symmetric),
//   Bbar' = Bbar + S C_f w (the Faraday curl, alpha-averaged along each B
//   component's own axis), jbar = -4 pi dt F^p w (F symmetric).
template <typename T>
struct Adj2dArgs {
    const T *Eb[3];  // dL/dE^{n+1}
    const T *Bb[3];  // dL/dB^{n+3/2}
    T *Ebo[3];       // dL/dE^n (must not alias Eb or Bb)
    T *Bbo[3];       // dL/dB^{n+1/2} (must not alias Eb or Bb)
    T *Jbo[3];       // dL/dj^{n+1/2} per component, or nullptr
    int m;           // sweeps
    int passes;      // binomial passes of the current filter
    int l1pf;        // prefetch input rows into L1 (set by the launcher)
};
// Whether the 2D TE/TM kernels prefetch their input rows into L1: when a
// step's algorithmic bytes (60 per cell) exceed 1.5 times the L2 cache, so
// that the rows come from HBM (4096^2, m = 4, p = 3: +11%); below, with the
// fields in L2, the prefetches only cost issue slots (1024^2: -23%).
bool fused2d_l1_prefetch(const Geo &g);
// even nx, 32-bit element offsets; m <= 4, passes <= 3
bool adjoint2d_supported(const Geo &g, int m, int passes);
int launch_adjoint2d(const Geo &g, const Coef<float> &c, const Adj2dArgs<float> &a, cudaStream_t s, int seg_rows = 0);

// Batched step (fused2d.cu): independent FP32 grids advanced by one
// persistent launch per step over (grid, strip, segment) tiles.
struct BatchGrid {
    Geo g;
    Coef<float> c;
    const float *E[2][3];  // state sets; a step reads set `parity`, writes 1 - parity
    const float *B[2][3];
    const float *J[3];
    int W, L, nstrip;      // tile width (columns written), rows per segment, strips
};
struct BatchItem {
    int grid, strip, seg;
};
// Tile geometry and occupancy of the batched kernel for (m, passes, current);
// returns -1 when that combination is not instantiated.
int fused2d_batch_geometry(int m, int passes, bool hj, int *threads, int *halo, int *width, size_t *smem,
                           int *blocks_per_sm);
int launch_fused2d_batch(int m, int passes, bool hj, const BatchGrid *grids, const BatchItem *items, int nitems,
                         int parity, int nblocks, size_t smem, cudaStream_t s);
// The same on the polarisation-split column-pair kernels (fused2d_pol_batch.cu)
// for grids of the unlumped scheme: one launch runs the TE and the TM half of
// every item.  Items are wide tiles (the whole CTA, `width` columns written)
// followed by narrow tiles (half a CTA each, `width_narrow` columns, two per
// CTA, `narrow_bytes` of shared memory each).
int fused2d_pol_batch_geometry(int m, int passes, bool hj, int *threads, int *halo, int *width, size_t *smem,
                               int *blocks_per_sm, int *width_narrow, size_t *narrow_bytes);
int launch_fused2d_pol_batch(int m, int passes, bool hj, const BatchGrid *grids, const BatchItem *items, int nwide,
                             int nnarrow, int parity, int nblocks, size_t smem, size_t narrow_bytes, cudaStream_t s);

}  // namespace fmx
