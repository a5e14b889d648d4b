// eb_handle.cuh -- the geometry handle and the host-side orchestration of
// one stage (flux divergence + redistribution), shared by the C ABI's
// translation units.  Not part of the ABI.
#pragma once

#include "eb_step.cuh"

#include <stdio.h>

#include <string>
#include <vector>

// message of the calling thread's last error (eb_last_error)
std::string &eb_error_slot();

namespace ebh {

inline eb_status fail(eb_status st, const char *fmt, const char *arg = nullptr) {
  char buf[512];
  snprintf(buf, sizeof(buf), fmt, arg ? arg : "");
  eb_error_slot() = buf;
  return st;
}

inline eb_status cuda_fail(cudaError_t e, const char *where) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  eb_error_slot() = buf;
  return e == cudaErrorMemoryAllocation ? EB_ERR_OOM : EB_ERR_CUDA;
}

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace ebh

#define CUDA_TRY(x, where)                                      \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) return ebh::cuda_fail(e_, where);    \
  } while (0)

// Work space of the projection (eb_project), allocated on its first use.
// One level of the projection's multigrid preconditioner (FP32): the cell
// grid coarsened 2^l times in every direction, face open fractions averaged
// over the fine faces a coarse face covers, 1 / delta^2 of the coarse spacing.
struct MgLevel {
  Dims D;
  float ix2 = 0, iy2 = 0, iz2 = 0;
  float *bx = nullptr, *by = nullptr, *bz = nullptr;   // low-face open fractions
  float *x = nullptr, *t = nullptr, *b = nullptr;      // correction, sweep target, right-hand side (coarse levels)
  int nb = 0;                                          // blocks of its kernels
};
constexpr int kMgMaxLevels = 16;

struct ProjWork {
  int precond = 0;             // 0: Jacobi, 1: multigrid V-cycle
  int nlev = 0;                // levels of the multigrid hierarchy (0: not built yet)
  MgLevel lev[kMgMaxLevels];
  bool ready = false;
  int nb = 0;                  // blocks of every projection kernel (fixed: deterministic sums)
  long long nact = 0;          // cells in the solve (diagonal > 0)
  double *bx = nullptr, *by = nullptr, *bz = nullptr;   // low-face open fractions of the c-cells
  double *ax = nullptr, *ay = nullptr, *az = nullptr;   // the same times 1 / delta^2 (the operator's coefficients)
  double *d = nullptr;         // diagonal of -L
  double *id = nullptr;        // its reciprocal (0 off the active cells): the Jacobi preconditioner
  double *rhs = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *x = nullptr;
  double *part = nullptr;      // partial sums, 8 slots of nb
  int *conv = nullptr;         // iteration count at convergence (0 = not yet)
  double *alpha = nullptr;     // c-cell volume fractions (warm-start input), on first use
  float *nin = nullptr, *nout = nullptr;   // network input (2 channels) and output, on first use
  double *host = nullptr;      // pinned copy of one slot of partial sums
};

struct eb_geom_s {
  eb_desc desc;
  Dims D;
  eb_precision prec;
  int device = 0;
  double *h = nullptr;
  int *kcov[4] = {}, *kreg[4] = {}, *kxt[4] = {};
  long long *roff[4] = {};
  int *kfast = nullptr;
  int4 *bseg = nullptr;   // bulk kernel work split
  int *boff = nullptr;
  int bctas = 0;
  int slab_levels = 0;    // slab height of the split (0: automatic)
  int plan_gen = 0;       // incremented whenever the split is rebuilt (its arrays move)
  int bulk_high = 0;      // 1: the bulk kernel runs on the high-priority stream
  int tile_rows = 16;     // rows of the bulk kernel's tiles (16, or 14 on the float path)
  int wsrd_side = 0;      // 1: the redistribution runs on the side stream (see stage)
  std::vector<int> kfast_host;
  int kcov_max = 0;
  GridDev G[4];
  WsrdDev W[4];
  // per-level reference profiles (zeros where none was given): rho0,
  // rho0*theta0, and the background momenta of rho*u and rho*v; states hold
  // each field minus its profile
  double *ref_d[4] = {nullptr, nullptr, nullptr, nullptr};
  float *ref_f[4] = {nullptr, nullptr, nullptr, nullptr};
  // per-level background values of the advected quantities, from the
  // profiles: theta0 = (rho0 theta0) / rho0, u_bg = ref_rhou / rho0,
  // v_bg = ref_rhov / rho0 (zero where rho0 is zero); the bulk kernel
  // advects deviations from them
  double *bg_d[3] = {nullptr, nullptr, nullptr};
  float *bg_f[3] = {nullptr, nullptr, nullptr};
  double *zero_d = nullptr;
  float *zero_f = nullptr;
  unsigned *status = nullptr;
  void *qhat = nullptr, *sig = nullptr, *pval = nullptr;
  long long max_small = 0;
  // scratch of the five-field redistribution pass (small CVs of all fields)
  void *qhat5 = nullptr, *sig5 = nullptr, *pval5 = nullptr;
  long long sum_small = 0;
  // the near-EB kernels run on the side stream and (bulk_high) the bulk
  // kernel on a stream of the highest priority, forked from and joined to the
  // caller's stream
  cudaStream_t side = nullptr, bulk = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join_bulk = nullptr;
  // scratch states for eb_step: 4 x 5 fields
  void *scr[4][5] = {};
  std::vector<void *> allocs;
  eb_geom_info_t info;
  bool has_ref = false;        // built with a reference profile
  bool has_wind_ref = false;   // a nonzero background momentum profile was set
  // sources of the compressible system (EB_SOURCE_* flags) and their
  // per-level tables: p0 = EOS of rho0 theta0, 1 / (rho0 theta0)
  int src_flags = 0;
  double *src_d[2] = {nullptr, nullptr};
  float *src_f[2] = {nullptr, nullptr};
  void *src_pp = nullptr;   // p' of every cell, scratch of the source pass
  ProjWork pw;

  template <typename P>
  cudaError_t alloc(P **p, long long count) {
    *p = nullptr;
    if (count < 1) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(P) * (size_t)count);
    if (e == cudaSuccess) {
      allocs.push_back((void *)*p);
      info.device_bytes += (int64_t)(sizeof(P) * count);
    }
    return e;
  }
  void release() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_join_bulk) cudaEventDestroy(ev_join_bulk);
    if (side) cudaStreamDestroy(side);
    if (bulk) cudaStreamDestroy(bulk);
    ev_fork = ev_join = ev_join_bulk = nullptr;
    side = bulk = nullptr;
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
    if (pw.host) cudaFreeHost(pw.host);
    pw = ProjWork();
    for (int g = 0; g < 4; ++g) free_wsrd(W[g]);
  }
};


// Projection of the face momenta of U (Sec. 2.2 anelastic constraint),
// implemented in eb_project.cu; phi0 may be NULL (zero start).
eb_status eb_project_impl(eb_geom g, void *const mom[3], double dt, double rtol, int maxit, const double *phi0,
                          double *phi_out, int *iters, double *relres, cudaStream_t s, bool correct);
// The projection's mean-free right-hand side D(m)/dt into g->pw.rhs and its
// RMS over the active cells (synchronises the stream).
eb_status eb_project_rhs(eb_geom g, void *const mom[3], double dt, double *rms, cudaStream_t s);

// (Re)build the bulk kernel's work split with slabs of slab_levels levels
// (0: automatic); the previous split is released.
eb_status eb_replan_bulk(eb_geom g, int slab_levels);

namespace ebh {

inline bool state_ok(const eb_state *U, size_t align) {
  if (!U) return false;
  const void *p[5] = {U->rho, U->rhotheta, U->rhou, U->rhov, U->rhow};
  for (const void *q : p)
    if (!q || ((uintptr_t)q % align)) return false;
  return true;
}

inline void **state_ptrs(const eb_state *U) { return (void **)&U->rho; }

template <typename T>
StepArgs<T> step_args(eb_geom g, void *const src[5], void *const base[5], void *const out[5], double dt, int copy) {
  StepArgs<T> A;
  A.D = g->D;
  for (int f = 0; f < 5; ++f) {
    A.src.f[f] = (const T *)src[f];
    A.base[f] = base ? (const T *)base[f] : nullptr;
    A.out[f] = (T *)out[f];
  }
  if (sizeof(T) == sizeof(double)) {
    A.src.ref_rho = (const T *)g->ref_d[0];
    A.src.ref_rt = (const T *)g->ref_d[1];
    A.src.ref_u = (const T *)g->ref_d[2];
    A.src.ref_v = (const T *)g->ref_d[3];
    A.src.bg_t = (const T *)g->bg_d[0];
    A.src.bg_u = (const T *)g->bg_d[1];
    A.src.bg_v = (const T *)g->bg_d[2];
  } else {
    A.src.ref_rho = (const T *)g->ref_f[0];
    A.src.ref_rt = (const T *)g->ref_f[1];
    A.src.ref_u = (const T *)g->ref_f[2];
    A.src.ref_v = (const T *)g->ref_f[3];
    A.src.bg_t = (const T *)g->bg_f[0];
    A.src.bg_u = (const T *)g->bg_f[1];
    A.src.bg_v = (const T *)g->bg_f[2];
  }
  A.dt = dt;
  A.dtT = (T)dt;
  A.kfast = g->kfast;
  A.bseg = g->bseg;
  A.boff = g->boff;
  A.bctas = g->bctas;
  for (int q = 0; q < 4; ++q) A.G[q] = g->G[q];
  A.status = g->status;
  A.copy_static = copy;
  A.tile_rows = g->tile_rows;
  A.kcov_max = g->kcov_max;
  return A;
}

template <typename T>
void wsrd_field(eb_geom g, int field, T *u, cudaStream_t s) {
  const int grid = field <= 1 ? 0 : field - 1;
  WsrdArgs<T> R;
  R.D = g->D;
  R.W = g->W[grid];
  R.u = u;
  R.refd = field <= 3 ? g->ref_d[field] : nullptr;
  R.dev = (T *)g->qhat;
  R.sig = (T *)g->sig;
  R.pval = (T *)g->pval;
  R.status = g->status;
  launch_wsrd(R, s);
}

// Flux divergence and provisional update.  The near-EB kernels and the bulk
// read the same input and write disjoint CVs, so they run side by side: the
// near-EB kernels on the handle's side stream, the bulk kernel either on the
// caller's stream (same priority: the scheduler interleaves the two) or on
// the handle's stream of the highest priority (its CTAs, one wave of two per
// SM, take their SMs first and the near-EB kernels fill the remaining SMs
// meanwhile and all of them afterwards; faster where the near-EB work is
// large).  eb_geom_tune times both.  after_band(side) launches work that
// follows the near-EB kernels on the side stream (the redistribution, when
// stage allows it); both streams are joined to the caller's stream at the
// end.
template <typename T, typename Side>
void flux_update(eb_geom g, const StepArgs<T> &A, cudaStream_t s, Side &&after_band) {
  cudaEventRecord(g->ev_fork, s);
  cudaStreamWaitEvent(g->side, g->ev_fork, 0);
  if (g->bulk_high) {
    cudaStreamWaitEvent(g->bulk, g->ev_fork, 0);
    launch_flux_fast(A, g->bulk);
    launch_flux_band(A, g->side);
    after_band(g->side);
    cudaEventRecord(g->ev_join_bulk, g->bulk);
    cudaStreamWaitEvent(s, g->ev_join_bulk, 0);
  } else {
    launch_flux_band(A, g->side);
    after_band(g->side);
    launch_flux_fast(A, s);
  }
  cudaEventRecord(g->ev_join, g->side);
  cudaStreamWaitEvent(s, g->ev_join, 0);
}

template <typename T>
void flux_update(eb_geom g, const StepArgs<T> &A, cudaStream_t s) {
  flux_update(g, A, s, [](cudaStream_t) {});
}

// Arguments of the redistribution of all five fields of the state out[].
template <typename T>
WsrdSet<T> wsrd_set(eb_geom g, void *const out[5]) {
  WsrdSet<T> S;
  long long os = 0, oa = 0;
  for (int f = 0; f < 5; ++f) {
    const int grid = f <= 1 ? 0 : f - 1;
    WsrdArgs<T> &R = S.f[f];
    R.D = g->D;
    R.W = g->W[grid];
    R.u = (T *)out[f];
    R.refd = f <= 3 ? g->ref_d[f] : nullptr;
    R.dev = (T *)g->qhat5 + os;
    R.pval = (T *)g->pval5 + os;
    R.sig = (T *)g->sig5 + 3 * os;
    R.status = g->status;
    S.off_small[f] = os;
    S.off_aff[f] = oa;
    os += g->W[grid].nsmall;
    oa += g->W[grid].naff;
  }
  S.off_small[5] = os;
  S.off_aff[5] = oa;
  return S;
}

// Redistribution of all five fields of a state in one pass of three kernels.
template <typename T>
void wsrd_all(eb_geom g, void *const out[5], cudaStream_t s) {
  launch_wsrd5(wsrd_set<T>(g, out), s);
}

// One stage: flux update, then redistribution.  When every CV the
// redistribution reads or writes is a near-EB CV (checked at set-up) and the
// caller allows it, it follows the near-EB kernels on the side stream, beside
// the bulk kernel; otherwise it follows the join.  (Ensembles keep it after
// the join: their members already fill the GPU side by side, and the longer
// branches cost more than the shorter critical path gains.)
template <typename T>
void stage(eb_geom g, void *const src[5], void *const base[5], void *const out[5], double dt, int copy,
           cudaStream_t s, bool wsrd_beside = true) {
  const StepArgs<T> A = step_args<T>(g, src, base, out, dt, copy);
  if (g->src_flags) {   // the sources follow the whole flux update; the redistribution follows them
    flux_update(g, A, s);
    const bool f64 = sizeof(T) == sizeof(double);
    launch_sources<T>(A, g->src_flags, f64 ? (const T *)g->src_d[0] : (const T *)g->src_f[0],
                      f64 ? (const T *)g->src_d[1] : (const T *)g->src_f[1], (T *)g->src_pp, s);
    wsrd_all<T>(g, out, s);
  } else if (g->wsrd_side && wsrd_beside) {
    flux_update(g, A, s, [&](cudaStream_t side) { wsrd_all<T>(g, out, side); });
  } else {
    flux_update(g, A, s);
    wsrd_all<T>(g, out, s);
  }
}

inline size_t field_count(const Dims &D, int f) { return (size_t)D.nxy * (D.nz + (f == 4 ? 1 : 0)); }

}  // namespace ebh
