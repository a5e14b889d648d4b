// eb_internal.cuh -- device data layout and shared device code of the EB
// library.  Not part of the ABI.
//
// Layout.  State fields are dense SoA arrays, x fastest.  Geometry is NOT
// dense: per grid and per column (i, j) only the levels kcov <= k < kxt carry
// an explicit record ("band"); levels below kcov are covered, levels at or
// above kxt are regular (full cell, open faces).  The band covers the cut CVs
// plus one level of the redistribution neighbourhoods above them.  A column's
// records are contiguous from roff[col].  kfast[col] is the first level from
// which every CV of every grid at that column is regular and every CV its
// flux stencils read holds fluid, so the bulk kernel needs no geometry at all
// there.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/eb.h"

// A kernel's dynamic shared-memory limit belongs to a device's context: it
// is set once per device (done: one bit per device index).
template <typename K>
inline void ebk_smem_limit(K *kernel, int bytes, unsigned long long &done) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(done & bit)) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    done |= bit;
  }
}

// SM count of the current device, queried once per device.
inline int ebk_sm_count() {
  static int count[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int &c = count[dev & 63];
  if (c < 1) {
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    if (c < 1) c = 1;
  }
  return c;
}

#define EBK_COVERED 0
#define EBK_REGULAR 1
#define EBK_CUT 2

// Records of one grid.
struct GridDev {
  int nzg;                 // nz, or nz + 1 for w
  int *kcov, *kxt;         // [ncol]
  long long *roff;         // [ncol + 1]
  long long nrec;
  // geometry, FP64, per record
  double *alpha, *cent, *beta, *fcent, *nrm, *aeb, *ebc;   // cent/beta/nrm/ebc: 3*nrec, fcent: 6*nrec
  uint8_t *flag;
  // float copies for the mixed path: alpha, beta[3], fcent[6]
  float *alpha_f, *beta_f, *fcent_f;
  // dense per-CV byte (nzg x ncol): bit 0 = holds fluid (alpha > 0),
  // bit 1 = has a band record, bits 2..4 = low x / y / z face open
  uint8_t *dflag;
  // provisional face fluxes of the near-EB path, dense (nzg x ncol) per
  // direction: fluxes of the advected value, and the mass flux (c grid only)
  void *fh[3], *fhm[3];
  // faces whose provisional flux the near-EB path needs, per direction
  unsigned *flist[3];
  long long nface[3];
  // per listed face, the geometry-only availability tests of its provisional
  // flux as bits (built once): bit 0, 1 the two momenta of the mass flux,
  // bits 2 + 2 (t + 2), 3 + 2 (t + 2) the two c-cells beside the grid CV t
  // steps along the face normal (t = -2 .. 1), bits 10, 11 the far CVs t = -2, 1
  uint16_t *fmask[3];
  // advected value of every CV some listed face's stencil reads (the CV's
  // theta or face velocity, 0 where it holds no fluid), formed once per step
  // (k_stage) into the dense array pv (levels below nst) from the list stlist
  unsigned *stlist;
  long long nstage;
  void *pv;
  int nst;
  // CVs the near-EB kernel updates (non-covered, prognostic, below kfast),
  // state indices in plane-major order
  unsigned *blist;
  long long nband;
  long long nband_rec;   // blist[0, nband_rec): cut CVs (rows below); the rest are regular
  // near-EB rows of the CVs with a record: dU of CV blist[t] is
  // sum over d of sum_{q = srow[3t+d]}^{srow[3t+d+1]-1} scoef[q] * fh[d][sidx[q]]
  // (fhm for the mass of the c grid); built once per geometry
  unsigned *srow;        // [3 * nband_rec + 1]
  unsigned *sidx;        // [nterm] face index into the staged arrays of direction d
  double *scoef;         // [nterm]
  float *scoef_f;        // [nterm] float copies (mixed path)
  uint8_t *stiny;        // [nband_rec] 1: tiny cut CV, whose row the mixed path sums in double
  long long nterm;
  // CVs of this grid that no flux kernel writes and a step passes through:
  // covered CVs, and on the w grid the two wall levels; state indices
  unsigned *slist;
  long long nstatic;
  // redistribution per record
  uint8_t *code;
  int *nnb;
  double *kappa, *omega, *vhat, *xhat;   // xhat: 3*nrec
};

// Quotient of a 32-bit unsigned n by a divisor d fixed on the host, with one
// high multiply: q = (umulhi(n, m) + n) >> s, where s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1 (the round-up multiplier of Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994);
// exact for every n < 2^32 with the 33-bit sum taken in 64 bits.
struct FastDiv {
  unsigned d = 1, m = 1, s = 0;
  __host__ void init(unsigned dd) {
    d = dd;
    s = 0;
    while ((1ull << s) < (unsigned long long)dd) ++s;
    m = (unsigned)((((1ull << s) - dd) << 32) / dd + 1);
  }
  __host__ __device__ inline unsigned div(unsigned n) const {
#ifdef __CUDA_ARCH__
    const unsigned hi = __umulhi(n, m);
#else
    const unsigned hi = (unsigned)(((unsigned long long)n * m) >> 32);
#endif
    return (unsigned)(((unsigned long long)hi + n) >> s);
  }
};

struct Dims {
  int nx, ny, nz;
  long long nxy;
  double dx, dy, dz;
  double idx, idy, idz;   // 1/dx, 1/dy, 1/dz (set on the host with the spacings)
  FastDiv fnx, fny, fnxy; // division by nx, ny, nx*ny (state indices are < 2^32)
};

// (i, j, k) of a state index c of any grid
__device__ inline void split_index(const Dims &D, unsigned c, int &i, int &j, int &k) {
  const unsigned kk = D.fnxy.div(c), col = c - kk * (unsigned)D.nxy;
  const unsigned jj = D.fnx.div(col);
  i = (int)(col - jj * (unsigned)D.nx);
  j = (int)jj;
  k = (int)kk;
}

// Periodic index for offsets of at most n from [0, n) (every stencil here
// reaches a few cells and n >= 4 ... the set-up code uses full modulo).
__host__ __device__ inline int wrapi(int a, int n) {
  return a < 0 ? a + n : (a >= n ? a - n : a);
}

__host__ __device__ inline int wrapmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__host__ __device__ inline int nzg_of(const Dims &D, int g) { return D.nz + (g == 3 ? 1 : 0); }

__device__ inline long long lin(const Dims &D, int i, int j, int k) {
  return (long long)wrapi(i, D.nx) + (long long)D.nx * ((long long)wrapi(j, D.ny) + (long long)D.ny * k);
}

// Classification of CV (i, j, k) of a grid: flag and record id (or -1).
struct CvInfo {
  int flag;
  long long rec;
};

__device__ inline CvInfo cv_info(const GridDev &G, const Dims &D, int i, int j, int k) {
  if (k < 0 || k >= G.nzg) return {EBK_COVERED, -1};
  int col = wrapi(i, D.nx) + D.nx * wrapi(j, D.ny);
  int kc = G.kcov[col];
  if (k < kc) return {EBK_COVERED, -1};
  if (k >= G.kxt[col]) return {EBK_REGULAR, -1};
  long long r = G.roff[col] + (k - kc);
  return {(int)G.flag[r], r};
}

// Status word bits latched by kernels.
#define EB_DEV_NUMERIC 1u
#define EB_DEV_TIMEOUT 2u

// ---------------------------------------------------------------------------
// Arithmetic shared by every kernel that evaluates a face flux, so that a
// face computed by two kernels (the bulk and the near-EB path) gets the same
// bits from both and the update stays exactly conservative.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline T eb_div(T a, T b) {
  return a / b;
}
template <>
__device__ inline float eb_div<float>(float a, float b) {
  return __fdividef(a, b);
}

// Third-order upwind face value (fourth-order centred plus hyperviscosity,
// Sec. 4.1): m > 0 uses (LL, L, R), m < 0 uses (L, R, RR); the centred
// second-order value where that far CV does not exist.
template <typename T>
__device__ inline T upwind_value(T m, T pLL, T pL, T pR, T pRR, bool hasLL, bool hasRR) {
  const T c2 = T(0.5) * (pL + pR);
  const T vp = hasLL ? fma(T(5), pL, fma(T(2), pR, -pLL)) * T(1.0 / 6.0) : c2;
  const T vn = hasRR ? fma(T(5), pR, fma(T(2), pL, -pRR)) * T(1.0 / 6.0) : c2;
  return m > T(0) ? vp : vn;
}

// ---------------------------------------------------------------------------
// State access
// ---------------------------------------------------------------------------
template <typename T>
struct StateIn {
  const T *f[5];             // rho, rho*theta, rho*u, rho*v, rho*w
  const T *ref_rho, *ref_rt; // per cell level, reference added back to rho and rho*theta
  const T *ref_u, *ref_v;    // per cell level, background momenta added back to rho*u and rho*v
  const T *bg_t, *bg_u, *bg_v; // per cell level, background theta, u, v (profile ratios)
};

template <typename T>
struct StateOut {
  T *f[5];
};

// ---------------------------------------------------------------------------
// Geometry lookups of the near-EB code: dense per-CV flag bytes and the
// geometry records of the cut band.
// ---------------------------------------------------------------------------
struct GeoBand {
  const GridDev *G;   // four grids
  __device__ inline uint8_t dense(const Dims &D, int g, int i, int j, int k) const {
    return G[g].dflag[(long long)wrapi(i, D.nx) + (long long)D.nx * wrapi(j, D.ny) + D.nxy * k];
  }
  __device__ inline long long record(const Dims &D, int g, int i, int j, int k) const {
    const int col = wrapi(i, D.nx) + D.nx * wrapi(j, D.ny);
    return G[g].roff[col] + (k - G[g].kcov[col]);
  }
  __device__ inline bool holds_fluid(const Dims &D, int g, int i, int j, int k) const {
    if (k < 0 || k >= nzg_of(D, g)) return false;
    return dense(D, g, i, j, k) & 1;
  }
  __device__ inline double alpha(const Dims &D, int g, int i, int j, int k) const {
    if (k < 0 || k >= nzg_of(D, g)) return 0.0;
    const uint8_t f = dense(D, g, i, j, k);
    if (!(f & 1)) return 0.0;
    if (!(f & 2)) return 1.0;
    return G[g].alpha[record(D, g, i, j, k)];
  }
  // area fraction of the low d-face of CV (i, j, k) of grid g (0 outside the
  // grid), from the double records or their float copies
  template <typename R>
  __device__ inline R beta(const Dims &D, int g, int d, int i, int j, int k) const {
    if (k < 0 || k >= nzg_of(D, g)) return R(0);
    const uint8_t f = dense(D, g, i, j, k);
    if (!(f & 2)) return (f & 1) ? R(1) : R(0);
    const long long r = (long long)d * G[g].nrec + record(D, g, i, j, k);
    if (sizeof(R) == sizeof(double)) return (R)G[g].beta[r];
    return (R)G[g].beta_f[r];
  }
  template <typename R>
  __device__ inline void fcent(const Dims &D, int g, int d, int i, int j, int k, R &ga, R &gb) const {
    ga = gb = R(0);
    if (k < 0 || k >= nzg_of(D, g)) return;
    if (!(dense(D, g, i, j, k) & 2)) return;
    const long long r = record(D, g, i, j, k);
    const long long a = (long long)(2 * d) * G[g].nrec + r, b = (long long)(2 * d + 1) * G[g].nrec + r;
    if (sizeof(R) == sizeof(double)) {
      ga = (R)G[g].fcent[a];
      gb = (R)G[g].fcent[b];
    } else {
      ga = (R)G[g].fcent_f[a];
      gb = (R)G[g].fcent_f[b];
    }
  }
};
