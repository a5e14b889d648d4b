// eb_step.cuh -- argument blocks of the per-step kernels.  Not part of the ABI.
#pragma once

#include "eb_kernels.cuh"

template <typename T>
struct StepArgs {
  Dims D;
  StateIn<T> src;      // state the fluxes are computed from
  const T *base[5];    // state the update is added to; base[0] == nullptr: write dU itself
  T *out[5];
  double dt;
  T dtT;
  const int *kfast;
  GridDev G[4];
  unsigned *status;
  int copy_static;     // also write covered CVs and the w wall levels
  int tile_rows;       // rows of the bulk kernel's tiles (16, or 14 on the float path)
  int kcov_max;        // highest covered level + 1 over every grid and column
  // work split of the bulk kernel: CTA b marches the pieces boff[b] .. boff[b+1]-1
  // of bseg, each (tile, first level, end level, 0)
  const int4 *bseg;
  const int *boff;
  int bctas;
};

template <typename T>
struct WsrdArgs {
  Dims D;
  WsrdDev W;
  T *u;                // field on its grid, redistributed in place
  const double *refd;  // per-level reference profile of the field (stored values are u - refd) or nullptr
  T *dev;              // [nsmall] deviation sums D of the neighbourhood averages
  T *pval;             // [nsmall] field value at each neighbourhood's pivot
  T *sig;              // [3 * nsmall] limited slopes
  unsigned *status;
};

// the redistribution of all five fields in one pass: f[q] is field q, and
// its small CVs (affected CVs) are the work items off_small[q] .. off_small[q+1]-1
// (off_aff[q] ..) of each fused launch
template <typename T>
struct WsrdSet {
  WsrdArgs<T> f[5];
  long long off_small[6];
  long long off_aff[6];
};

template <typename T>
void launch_flux_update(const StepArgs<T> &A, cudaStream_t s);
template <typename T>
void launch_flux_fast(const StepArgs<T> &A, cudaStream_t s);   // static copy + bulk
template <typename T>
void launch_static_copy(const StepArgs<T> &A, cudaStream_t s);
template <typename T>
void launch_flux_bulk(const StepArgs<T> &A, cudaStream_t s);
template <typename T>
void launch_flux_band(const StepArgs<T> &A, cudaStream_t s);

template <typename T>
void launch_wsrd(const WsrdArgs<T> &R, cudaStream_t s);
template <typename T>
void launch_wsrd5(const WsrdSet<T> &S, cudaStream_t s);
// sources of the compressible system (eb_sources.cu): flags EB_SOURCE_*,
// per-level tables p0 and 1 / (rho0 theta0), scratch pp of one cell field
template <typename T>
void launch_sources(const StepArgs<T> &A, int flags, const T *p0, const T *irt0, T *pp, cudaStream_t s);

// One ensemble member in one step direction: the arguments of its flux
// update and of its five-field redistribution.
template <typename T>
struct EnsMember {
  StepArgs<T> A;
  WsrdSet<T> S;
};

// The persistent ensemble step (one cooperative launch per step).  Item
// counts of every phase are prefix sums over the members (nm + 1 entries);
// ctl[0..3] (zeroed before every launch) hold the barrier's arrival count and
// generation and the next bulk unit and face chunk to hand out; *fault (set
// only by the failure test) names a CTA + 1 that leaves before the first
// barrier.
template <typename T>
struct EnsembleArgs {
  const EnsMember<T> *m;
  int nm;
  const int2 *units;        // bulk work units (member, CTA group of its split), longest first
  int nunits;
  const long long *pre_stage, *pre_face, *pre_band, *pre_small, *pre_aff;
  unsigned *ctl;
  const int *fault;
  unsigned spin_limit;      // polls of a barrier wait before it gives up
  int faces_first;          // 1: face fluxes run in the first phase (no staged values)
};

// Launch attributes of the persistent kernel: CTAs that fit the device at
// once (the launch is cooperative), or 0 if the kernel cannot be used.
template <typename T>
int ensemble_kernel_ctas(bool vec, int info[3]);   // info: registers per thread, static and local bytes
template <typename T>
cudaError_t launch_ensemble_step(const EnsembleArgs<T> &E, bool vec, int ctas, cudaStream_t s);
