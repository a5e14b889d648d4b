// eb_project.cu -- the anelastic projection (Sec. 2.2, Algorithm 2 step 5)
// and the anelastic step.
//
// The constraint div(rho0 u) = 0 is imposed on the face momenta with the
// cut-cell divergence of the flux update,
//   D(m)_c = sum_d (beta_d,hi m_d,hi - beta_d,lo m_d,lo) / delta_d,
// beta the open fractions of the c-cell's faces (walls closed).  With the
// face gradient G(phi) = (phi_R - phi_L) / delta_d, the correction
// m <- m* - dt G(phi) removes the divergence when L phi = D(G(phi)) = D(m*)/dt.
// L is the beta-weighted 7-point operator: symmetric, negative semi-definite,
// null space the constants (the fluid above a height-function terrain is
// connected), so the mean of the right-hand side (rounding only) is removed
// and -L phi = -rhs is solved by Jacobi-preconditioned conjugate gradients
// in FP64 to a relative residual.
//
// Every kernel runs on a fixed grid of nb blocks with grid-stride loops and
// writes one partial sum per block; a consumer block adds the nb partials in
// a fixed order, so the solve is deterministic.  Convergence is detected on
// the device (the kernels of later iterations return at once) and read by
// the host every 32 iterations (every 4 with the multigrid preconditioner).
#include "eb_handle.cuh"

#include <math.h>

using namespace ebh;

namespace {

constexpr int PB = 256;   // threads per block of every projection kernel

enum { S_SUM = 0, S_BB = 1, S_PQ = 2, S_RR = 3, S_RZ0 = 4, S_RZ1 = 5, S_CNT = 6, S_TMP = 7 };

__device__ inline double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; thread 0 writes it to part[blockIdx.x].
__device__ inline void block_partial(double v, double *part) {
  __shared__ double s[PB / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < PB / 32 ? s[threadIdx.x] : 0.0;
    a = warp_sum(a);
    if (threadIdx.x == 0) part[blockIdx.x] = a;
  }
}

// Total of nb partial sums, the same bits in every block.
__device__ inline double total(const double *part, int nb) {
  __shared__ double t;
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int q = threadIdx.x; q < nb; q += 32) a += part[q];
    a = warp_sum(a);
    if (threadIdx.x == 0) t = a;
  }
  __syncthreads();
  return t;
}

struct Nbr {
  long long xm, xp, ym, yp;
  int k;
};

__device__ inline Nbr neighbours(const Dims &D, long long c) {
  int i, j, k;
  split_index(D, (unsigned)c, i, j, k);
  Nbr n;
  n.xm = i == 0 ? c + D.nx - 1 : c - 1;
  n.xp = i == D.nx - 1 ? c - (D.nx - 1) : c + 1;
  n.ym = j == 0 ? c + (long long)D.nx * (D.ny - 1) : c - D.nx;
  n.yp = j == D.ny - 1 ? c - (long long)D.nx * (D.ny - 1) : c + D.nx;
  n.k = k;
  return n;
}

struct Op {
  Dims D;
  const double *bx, *by, *bz, *d, *id;
  const double *ax, *ay, *az;   // open fractions times 1 / delta^2 (set-up)
  double ix2, iy2, iz2;   // 1 / delta^2
  // (-L p)_c for an active cell: one product and six fused multiply-adds
  // (FP64 arithmetic, not HBM, bounds this on the GPU)
  __device__ inline double apply(const double *p, long long c, const Nbr &n) const {
    const double azl = az[c];
    const double azh = n.k + 1 < D.nz ? az[c + D.nxy] : 0.0;
    double v = d[c] * p[c];
    v = fma(-ax[c], p[n.xm], v);
    v = fma(-ax[n.xp], p[n.xp], v);
    v = fma(-ay[c], p[n.ym], v);
    v = fma(-ay[n.yp], p[n.yp], v);
    if (azl > 0.0) v = fma(-azl, p[c - D.nxy], v);
    if (azh > 0.0) v = fma(-azh, p[c + D.nxy], v);
    return v;
  }
};

__global__ void k_recip(long long N, const double *d, double *id) {
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB)
    id[c] = d[c] > 0.0 ? 1.0 / d[c] : 0.0;
}

__global__ void k_scale(long long N, const double *b, double s, double *a) {
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) a[c] = b[c] * s;
}

__global__ void k_wall(Dims D, double *bz) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c < D.nxy) bz[c] = 0.0;   // z = 0 carries no flux
}

__global__ void k_diag(Op O, double *d, double *part) {
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  double cnt = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    const Nbr n = neighbours(D, c);
    const double bzh = n.k + 1 < D.nz ? O.bz[c + D.nxy] : 0.0;
    const double v = (O.bx[c] + O.bx[n.xp]) * O.ix2 + (O.by[c] + O.by[n.yp]) * O.iy2 + (O.bz[c] + bzh) * O.iz2;
    d[c] = v;
    cnt += v > 0.0 ? 1.0 : 0.0;
  }
  block_partial(cnt, part);
}

// rhs = D(m) / dt on the active cells
template <typename T>
__global__ void k_rhs(Op O, const T *mu, const T *mv, const T *mw, double idt, double *rhs, double *part) {
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  double sum = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    double v = 0.0;
    if (O.d[c] > 0.0) {
      const Nbr n = neighbours(D, c);
      const double bzh = n.k + 1 < D.nz ? O.bz[c + D.nxy] : 0.0;
      const double dx = O.bx[n.xp] * (double)mu[n.xp] - O.bx[c] * (double)mu[c];
      const double dy = O.by[n.yp] * (double)mv[n.yp] - O.by[c] * (double)mv[c];
      const double dz = bzh * (double)mw[c + D.nxy] - O.bz[c] * (double)mw[c];
      v = (dx * D.idx + dy * D.idy + dz * D.idz) * idt;
    }
    rhs[c] = v;
    sum += v;
  }
  block_partial(sum, part);
}

// remove the mean of the right-hand side over the active cells
__global__ void k_center(Op O, double *rhs, const double *psum, const double *pcnt, int nb, double *pbb) {
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  const double mean = total(psum, nb) / fmax(1.0, total(pcnt, nb));
  double bb = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    if (O.d[c] > 0.0) {
      const double v = rhs[c] - mean;
      rhs[c] = v;
      bb += v * v;
    }
  }
  block_partial(bb, pbb);
}

// r = -rhs - A x, z = r / d, p = z
__global__ void k_init(Op O, const double *x, const double *rhs, double *r, double *z, double *p, double *prz,
                       double *prr) {
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  double rz = 0.0, rr = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    double rv = 0.0, zv = 0.0;
    if (O.d[c] > 0.0) {
      rv = -rhs[c] - O.apply(x, c, neighbours(D, c));
      zv = rv * O.id[c];
    }
    r[c] = rv;
    z[c] = zv;
    p[c] = zv;
    rz += rv * zv;
    rr += rv * rv;
  }
  block_partial(rz, prz);
  __syncthreads();
  block_partial(rr, prr);
}

// q = A p
__global__ void k_apply(Op O, const double *p, double *q, double *ppq, const int *conv) {
  if (*conv) return;
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  double pq = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    double v = 0.0;
    if (O.d[c] > 0.0) v = O.apply(p, c, neighbours(D, c));
    q[c] = v;
    pq += p[c] * v;
  }
  block_partial(pq, ppq);
}

// alpha = rz / pq; x += alpha p; r -= alpha q; z = r / d (Jacobi; the
// multigrid preconditioner forms z and r.z afterwards)
template <bool JAC>
__global__ void k_update(Op O, double *x, const double *p, const double *q, double *r, double *z, const double *ppq,
                         const double *prz, double *prz_next, double *prr, int nb, const int *conv) {
  if (*conv) return;
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  const double alpha = total(prz, nb) / total(ppq, nb);
  double rz = 0.0, rr = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    if (O.d[c] > 0.0) {
      x[c] += alpha * p[c];
      const double rv = r[c] - alpha * q[c];
      r[c] = rv;
      if (JAC) {
        const double zv = rv * O.id[c];
        z[c] = zv;
        rz += rv * zv;
      }
      rr += rv * rv;
    }
  }
  if (JAC) {
    block_partial(rz, prz_next);
    __syncthreads();
  }
  block_partial(rr, prr);
}

// convergence test; else p = z + (rz_next / rz) p
__global__ void k_direction(Op O, double *p, const double *z, const double *prz, const double *prz_next,
                            const double *prr, int nb, double thr2, int it, int *conv) {
  if (*conv) return;
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  const double rr = total(prr, nb);
  if (rr <= thr2) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *conv = it + 1;
    return;
  }
  const double beta = total(prz_next, nb) / total(prz, nb);
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB)
    p[c] = z[c] + beta * p[c];
}

// m -= dt G(x) on the open faces
template <typename T>
__global__ void k_correct(Op O, const double *x, double dt, T *mu, T *mv, T *mw) {
  const Dims &D = O.D;
  const long long N = D.nxy * D.nz;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    const Nbr n = neighbours(D, c);
    if (O.bx[c] > 0.0) mu[c] = (T)((double)mu[c] - dt * (x[c] - x[n.xm]) * D.idx);
    if (O.by[c] > 0.0) mv[c] = (T)((double)mv[c] - dt * (x[c] - x[n.ym]) * D.idy);
    if (n.k >= 1 && O.bz[c] > 0.0) mw[c] = (T)((double)mw[c] - dt * (x[c] - x[c - D.nxy]) * D.idz);
  }
}

// ---------------------------------------------------------------------------
// Multigrid preconditioner (EB_PRECOND_MG): z = V(r), one V-cycle in FP32
// (FP64 arithmetic is scarce on this GPU; the outer conjugate gradients stay
// in FP64).  Damped Jacobi with the same weight and the same number of
// sweeps before and after the coarse correction (three on the finest grid,
// where they cut 18 iterations to 16 at rtol 1e-10 on the 192x192x96 random
// terrain for a shorter solve; two on the coarser grids), restriction = 1/8
// of the transpose of the injection
// prolongation, and a fixed number of Jacobi sweeps from zero on the
// coarsest grid: up to float rounding V is a fixed symmetric positive
// semi-definite operator, as conjugate gradients need.
// ---------------------------------------------------------------------------
// Jacobi weight: the rows of the operator have off-diagonal magnitudes
// summing to the diagonal, so the eigenvalues of D^-1 A lie in [0, 2] and any
// weight below 1 keeps the smoother convergent and the V-cycle definite; 0.9
// took the 192x192x96 random terrain's projection from 16 iterations (0.8) to
// 13 at rtol 1e-10, 0.95 back up to 17.
constexpr float MG_OMEGA = 0.9f;
// Jacobi sweeps from zero on the coarsest grid (even: the result ends in x).
// Any count gives a positive operator (the weight keeps 1 - w*lambda in
// (-1, 1]); on the 192x192x96 random terrain 8 to 64 sweeps all needed 13
// outer iterations, and fewer sweeps cost less (16: 7.6 ms, 64: 8.0 ms).
constexpr int MG_COARSE_SWEEPS = 16;

// the operator of one level: S = sum_f a_f x_nb (off-diagonal part) and the
// diagonal d = sum_f a_f, from the six face coefficients of cell c
struct Op32 {
  Dims D;
  const float *bx, *by, *bz;
  float ix2, iy2, iz2;
  __device__ inline void parts(const float *x, long long c, float &S, float &d) const {
    const Nbr n = neighbours(D, c);
    const float axl = bx[c] * ix2, axh = bx[n.xp] * ix2, ayl = by[c] * iy2, ayh = by[n.yp] * iy2;
    const float azl = bz[c] * iz2, azh = n.k + 1 < D.nz ? bz[c + D.nxy] * iz2 : 0.f;
    d = axl + axh + ayl + ayh + azl + azh;
    S = axl * x[n.xm] + axh * x[n.xp] + ayl * x[n.ym] + ayh * x[n.yp];
    if (azl > 0.f) S += azl * x[c - D.nxy];
    if (azh > 0.f) S += azh * x[c + D.nxy];
  }
  __device__ inline float diag(long long c) const {
    const Nbr n = neighbours(D, c);
    const float azh = n.k + 1 < D.nz ? bz[c + D.nxy] * iz2 : 0.f;
    return (bx[c] + bx[n.xp]) * ix2 + (by[c] + by[n.yp]) * iy2 + bz[c] * iz2 + azh;
  }
};

// level 0: float copies of the open fractions
__global__ void k_mg_copy(long long N, const double *bx, const double *by, const double *bz, float *fx, float *fy,
                          float *fz) {
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    fx[c] = (float)bx[c];
    fy[c] = (float)by[c];
    fz[c] = (float)bz[c];
  }
}

// coarse open fractions: the mean over the four fine faces a coarse face covers
__global__ void k_mg_coarsen(Op32 F, Dims C, float *bx, float *by, float *bz) {
  const long long N = C.nxy * C.nz;
  const long long sy = F.D.nx, sz = F.D.nxy;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    int I, J, K;
    split_index(C, (unsigned)c, I, J, K);
    const long long f = 2LL * I + sy * 2LL * J + sz * 2LL * K;
    bx[c] = 0.25f * (F.bx[f] + F.bx[f + sy] + F.bx[f + sz] + F.bx[f + sy + sz]);
    by[c] = 0.25f * (F.by[f] + F.by[f + 1] + F.by[f + sz] + F.by[f + 1 + sz]);
    bz[c] = 0.25f * (F.bz[f] + F.bz[f + 1] + F.bz[f + sy] + F.bz[f + 1 + sy]);
  }
}

// one damped Jacobi sweep, xout = (1 - w) xin + w (b + S(xin)) / d (xin = 0
// when first); B is the right-hand side's type (the FP64 residual on level
// 0).  FINAL: the finest level's last sweep, which writes the FP64 z and the
// block partials of r.z.
template <typename B, bool FINAL>
__global__ void k_mg_sweep(Op32 L, const float *xin, float *xout, double *zout, const B *b, int first, double *prz,
                           const int *conv) {
  if (*conv) return;
  const long long N = L.D.nxy * L.D.nz;
  double rz = 0.0;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    float v = 0.f;
    if (first) {
      const float d = L.diag(c);
      if (d > 0.f) v = MG_OMEGA * (float)b[c] / d;
    } else {
      float S, d;
      L.parts(xin, c, S, d);
      if (d > 0.f) v = (1.f - MG_OMEGA) * xin[c] + MG_OMEGA * ((float)b[c] + S) / d;
    }
    if (FINAL) {
      zout[c] = (double)v;
      rz += (double)b[c] * (double)v;
    } else {
      xout[c] = v;
    }
  }
  if (FINAL) block_partial(rz, prz);
}

// coarse right-hand side: the mean of the eight children's residuals b - A x
template <typename B>
__global__ void k_mg_restrict(Op32 F, const float *x, const B *b, Dims C, float *bc, const int *conv) {
  if (*conv) return;
  const long long N = C.nxy * C.nz;
  const long long sy = F.D.nx, sz = F.D.nxy;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    int I, J, K;
    split_index(C, (unsigned)c, I, J, K);
    const long long f0 = 2LL * I + sy * 2LL * J + sz * 2LL * K;
    float sum = 0.f;
    for (int q = 0; q < 8; ++q) {
      const long long f = f0 + (q & 1) + ((q >> 1) & 1) * sy + (q >> 2) * sz;
      float S, d;
      F.parts(x, f, S, d);
      if (d > 0.f) sum += (float)b[f] - d * x[f] + S;
    }
    bc[c] = 0.125f * sum;
  }
}

// x += the parent's coarse correction (injection), on active cells
__global__ void k_mg_prolong(Op32 F, Dims C, const float *xc, float *x, const int *conv) {
  if (*conv) return;
  const long long N = F.D.nxy * F.D.nz;
  for (long long c = blockIdx.x * (long long)PB + threadIdx.x; c < N; c += (long long)gridDim.x * PB) {
    if (F.diag(c) > 0.f) {
      int i, j, k;
      split_index(F.D, (unsigned)c, i, j, k);
      x[c] += xc[(i >> 1) + (long long)C.nx * ((j >> 1) + (long long)C.ny * (k >> 1))];
    }
  }
}

// the coarsest grid (at most MG_SMEM_CELLS cells): MG_COARSE_SWEEPS Jacobi
// sweeps from zero in one block, the grid held in shared memory
constexpr int MG_SMEM_CELLS = 1024;
__global__ void k_mg_coarsest_smem(Op32 L, const float *b, float *x, const int *conv) {
  if (*conv) return;
  __shared__ float sbx[MG_SMEM_CELLS], sby[MG_SMEM_CELLS], sbz[MG_SMEM_CELLS], sb[MG_SMEM_CELLS];
  __shared__ float sx[MG_SMEM_CELLS], st[MG_SMEM_CELLS];
  const int N = (int)(L.D.nxy * L.D.nz);
  for (int c = threadIdx.x; c < N; c += blockDim.x) {
    sbx[c] = L.bx[c];
    sby[c] = L.by[c];
    sbz[c] = L.bz[c];
    sb[c] = b[c];
  }
  __syncthreads();
  Op32 S = L;
  S.bx = sbx;
  S.by = sby;
  S.bz = sbz;
  for (int sw = 0; sw < MG_COARSE_SWEEPS; ++sw) {
    const float *in = (sw & 1) ? st : sx;
    float *out = (sw & 1) ? sx : st;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      float v = 0.f;
      if (sw == 0) {
        const float d = S.diag(c);
        if (d > 0.f) v = MG_OMEGA * sb[c] / d;
      } else {
        float Sv, d;
        S.parts(in, c, Sv, d);
        if (d > 0.f) v = (1.f - MG_OMEGA) * in[c] + MG_OMEGA * (sb[c] + Sv) / d;
      }
      out[c] = v;
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < N; c += blockDim.x) x[c] = sx[c];
}

// The lower part of the V-cycle (every level from lt down, each at most
// MG_LOWER_CELLS cells) in one block: the same sweeps, restrictions, coarsest
// sweeps and prolongations as the multi-block kernels, separated by block
// barriers instead of launches (these levels are launch-bound otherwise).
constexpr long long MG_LOWER_CELLS = 8192;
struct MgLower {
  Op32 L[kMgMaxLevels];
  float *x[kMgMaxLevels], *t[kMgMaxLevels], *b[kMgMaxLevels];
  int lt, top;
};

__device__ inline void lower_sweep(const Op32 &L, const float *xin, float *xout, const float *b, bool first) {
  const long long N = L.D.nxy * L.D.nz;
  for (long long c = threadIdx.x; c < N; c += blockDim.x) {
    float v = 0.f;
    if (first) {
      const float d = L.diag(c);
      if (d > 0.f) v = MG_OMEGA * b[c] / d;
    } else {
      float S, d;
      L.parts(xin, c, S, d);
      if (d > 0.f) v = (1.f - MG_OMEGA) * xin[c] + MG_OMEGA * (b[c] + S) / d;
    }
    xout[c] = v;
  }
  __syncthreads();
}

__global__ void k_mg_lower(const __grid_constant__ MgLower M, const int *conv) {
  if (*conv) return;
  for (int l = M.lt; l < M.top; ++l) {
    const Op32 &F = M.L[l];
    lower_sweep(F, nullptr, M.t[l], M.b[l], true);
    lower_sweep(F, M.t[l], M.x[l], M.b[l], false);
    const Dims &C = M.L[l + 1].D;
    const long long N = C.nxy * C.nz, sy = F.D.nx, sz = F.D.nxy;
    for (long long c = threadIdx.x; c < N; c += blockDim.x) {   // as k_mg_restrict
      int I, J, K;
      split_index(C, (unsigned)c, I, J, K);
      const long long f0 = 2LL * I + sy * 2LL * J + sz * 2LL * K;
      float sum = 0.f;
      for (int q = 0; q < 8; ++q) {
        const long long f = f0 + (q & 1) + ((q >> 1) & 1) * sy + (q >> 2) * sz;
        float S, d;
        F.parts(M.x[l], f, S, d);
        if (d > 0.f) sum += M.b[l][f] - d * M.x[l][f] + S;
      }
      M.b[l + 1][c] = 0.125f * sum;
    }
    __syncthreads();
  }
  const int top = M.top;
  for (int sw = 0; sw < MG_COARSE_SWEEPS; ++sw)   // coarsest sweeps; the result ends in x
    lower_sweep(M.L[top], (sw & 1) ? M.t[top] : M.x[top], (sw & 1) ? M.x[top] : M.t[top], M.b[top], sw == 0);
  for (int l = top - 1; l >= M.lt; --l) {
    const Op32 &F = M.L[l];
    const Dims &C = M.L[l + 1].D;
    const long long N = F.D.nxy * F.D.nz;
    for (long long c = threadIdx.x; c < N; c += blockDim.x) {   // as k_mg_prolong
      if (F.diag(c) > 0.f) {
        int i, j, k;
        split_index(F.D, (unsigned)c, i, j, k);
        M.x[l][c] += M.x[l + 1][(i >> 1) + (long long)C.nx * ((j >> 1) + (long long)C.ny * (k >> 1))];
      }
    }
    __syncthreads();
    lower_sweep(F, M.x[l], M.t[l], M.b[l], false);
    lower_sweep(F, M.t[l], M.x[l], M.b[l], false);
  }
}

Op32 level_op(const MgLevel &L) {
  Op32 O;
  O.D = L.D;
  O.bx = L.bx;
  O.by = L.by;
  O.bz = L.bz;
  O.ix2 = L.ix2;
  O.iy2 = L.iy2;
  O.iz2 = L.iz2;
  return O;
}

// sizes of the levels (level 0 = the cell grid); false if multigrid does not apply
bool mg_plan(const Dims &D, int dims[kMgMaxLevels][3], int &nlev) {
  int nx = D.nx, ny = D.ny, nz = D.nz;
  nlev = 0;
  dims[nlev][0] = nx, dims[nlev][1] = ny, dims[nlev][2] = nz, ++nlev;
  while (nlev < kMgMaxLevels && (long long)nx * ny * nz > 512 && nx % 2 == 0 && ny % 2 == 0 && nz % 2 == 0 &&
         nx >= 4 && ny >= 4 && nz >= 4) {
    nx /= 2, ny /= 2, nz /= 2;
    dims[nlev][0] = nx, dims[nlev][1] = ny, dims[nlev][2] = nz, ++nlev;
  }
  return nlev >= 2 && (long long)nx * ny * nz <= 32768;
}

Op make_op(eb_geom g) {
  Op O;
  O.D = g->D;
  O.bx = g->pw.bx;
  O.by = g->pw.by;
  O.bz = g->pw.bz;
  O.d = g->pw.d;
  O.id = g->pw.id;
  O.ax = g->pw.ax;
  O.ay = g->pw.ay;
  O.az = g->pw.az;
  O.ix2 = g->D.idx * g->D.idx;
  O.iy2 = g->D.idy * g->D.idy;
  O.iz2 = g->D.idz * g->D.idz;
  return O;
}

// work space and the fixed part of the operator, on the first call
eb_status setup(eb_geom g, cudaStream_t s) {
  ProjWork &w = g->pw;
  if (w.ready) return EB_OK;
  const Dims &D = g->D;
  const long long N = D.nxy * D.nz;
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev), "device");
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device");
  w.nb = (int)std::max(1LL, std::min<long long>(4LL * std::max(sms, 1), (N + PB - 1) / PB));
  for (double **a : {&w.bx, &w.by, &w.bz, &w.ax, &w.ay, &w.az, &w.d, &w.id, &w.rhs, &w.r, &w.z, &w.p, &w.q, &w.x})
    CUDA_TRY(g->alloc(a, N), "alloc projection work space");
  CUDA_TRY(g->alloc(&w.part, 8LL * w.nb), "alloc projection work space");
  CUDA_TRY(g->alloc(&w.conv, 1), "alloc projection work space");
  CUDA_TRY(cudaMallocHost(&w.host, sizeof(double) * (size_t)w.nb), "alloc pinned scratch");
  launch_export_geometry(g->h, D, 0, g->G[0], EB_X_BETA_X, w.bx, s);
  launch_export_geometry(g->h, D, 0, g->G[0], EB_X_BETA_Y, w.by, s);
  launch_export_geometry(g->h, D, 0, g->G[0], EB_X_BETA_Z, w.bz, s);
  k_wall<<<(unsigned)((D.nxy + 255) / 256), 256, 0, s>>>(D, w.bz);
  k_scale<<<w.nb, PB, 0, s>>>(N, w.bx, D.idx * D.idx, w.ax);
  k_scale<<<w.nb, PB, 0, s>>>(N, w.by, D.idy * D.idy, w.ay);
  k_scale<<<w.nb, PB, 0, s>>>(N, w.bz, D.idz * D.idz, w.az);
  k_diag<<<w.nb, PB, 0, s>>>(make_op(g), w.d, w.part + S_CNT * w.nb);
  k_recip<<<w.nb, PB, 0, s>>>(N, w.d, w.id);
  CUDA_TRY(cudaMemcpyAsync(w.host, w.part + S_CNT * w.nb, sizeof(double) * w.nb, cudaMemcpyDeviceToHost, s),
           "count active cells");
  CUDA_TRY(cudaStreamSynchronize(s), "count active cells");
  double cnt = 0.0;
  for (int q = 0; q < w.nb; ++q) cnt += w.host[q];
  w.nact = (long long)cnt;
  w.ready = true;
  return EB_OK;
}

// the multigrid hierarchy, on the first projection that uses it
eb_status mg_setup(eb_geom g, cudaStream_t s) {
  ProjWork &w = g->pw;
  if (w.nlev) return EB_OK;
  int dims[kMgMaxLevels][3], nlev = 0;
  if (!mg_plan(g->D, dims, nlev)) return fail(EB_ERR_INVALID_ARG, "grid cannot be coarsened for multigrid");
  const Op O0 = make_op(g);
  MgLevel &L0 = w.lev[0];
  L0.D = g->D;
  L0.ix2 = (float)O0.ix2, L0.iy2 = (float)O0.iy2, L0.iz2 = (float)O0.iz2;
  L0.nb = w.nb;
  const long long N0 = g->D.nxy * g->D.nz;
  for (float **a : {&L0.bx, &L0.by, &L0.bz, &L0.x, &L0.t}) CUDA_TRY(g->alloc(a, N0), "alloc multigrid level");
  k_mg_copy<<<L0.nb, PB, 0, s>>>(N0, w.bx, w.by, w.bz, L0.bx, L0.by, L0.bz);
  for (int l = 1; l < nlev; ++l) {
    MgLevel &L = w.lev[l];
    const MgLevel &F = w.lev[l - 1];
    Dims &C = L.D;
    C = F.D;
    C.nx = dims[l][0], C.ny = dims[l][1], C.nz = dims[l][2];
    C.nxy = (long long)C.nx * C.ny;
    C.dx = 2 * F.D.dx, C.dy = 2 * F.D.dy, C.dz = 2 * F.D.dz;
    C.idx = 0.5 * F.D.idx, C.idy = 0.5 * F.D.idy, C.idz = 0.5 * F.D.idz;
    C.fnx.init((unsigned)C.nx);
    C.fny.init((unsigned)C.ny);
    C.fnxy.init((unsigned)C.nxy);
    L.ix2 = 0.25f * F.ix2, L.iy2 = 0.25f * F.iy2, L.iz2 = 0.25f * F.iz2;
    const long long N = C.nxy * C.nz;
    L.nb = (int)std::max(1LL, std::min<long long>(w.nb, (N + PB - 1) / PB));
    for (float **a : {&L.bx, &L.by, &L.bz, &L.x, &L.t, &L.b}) CUDA_TRY(g->alloc(a, N), "alloc multigrid level");
    k_mg_coarsen<<<L.nb, PB, 0, s>>>(level_op(F), C, L.bx, L.by, L.bz);
  }
  CUDA_TRY(cudaGetLastError(), "multigrid set-up");
  w.nlev = nlev;
  return EB_OK;
}

// z = V(r) (FP64 in and out) and the partial sums of r.z into prz
void vcycle(eb_geom g, const double *r, double *z, double *prz, cudaStream_t s) {
  ProjWork &w = g->pw;
  const MgLevel *L = w.lev;
  const int top = w.nlev - 1;
  // levels lt .. top (at most MG_LOWER_CELLS cells each) run in one block; level 0 never does
  int lt = top;
  while (lt > 1 && L[lt - 1].D.nxy * L[lt - 1].D.nz <= MG_LOWER_CELLS) --lt;
  // level 0: right-hand side r (FP64)
  {
    const Op32 O = level_op(L[0]);
    k_mg_sweep<double, false><<<L[0].nb, PB, 0, s>>>(O, nullptr, L[0].x, nullptr, r, 1, nullptr, w.conv);
    k_mg_sweep<double, false><<<L[0].nb, PB, 0, s>>>(O, L[0].x, L[0].t, nullptr, r, 0, nullptr, w.conv);
    k_mg_sweep<double, false><<<L[0].nb, PB, 0, s>>>(O, L[0].t, L[0].x, nullptr, r, 0, nullptr, w.conv);
    k_mg_restrict<double><<<L[1].nb, PB, 0, s>>>(O, L[0].x, r, L[1].D, L[1].b, w.conv);
  }
  for (int l = 1; l < lt; ++l) {
    const Op32 O = level_op(L[l]);
    k_mg_sweep<float, false><<<L[l].nb, PB, 0, s>>>(O, nullptr, L[l].t, nullptr, L[l].b, 1, nullptr, w.conv);
    k_mg_sweep<float, false><<<L[l].nb, PB, 0, s>>>(O, L[l].t, L[l].x, nullptr, L[l].b, 0, nullptr, w.conv);
    k_mg_restrict<float><<<L[l + 1].nb, PB, 0, s>>>(O, L[l].x, L[l].b, L[l + 1].D, L[l + 1].b, w.conv);
  }
  if (lt == top && L[top].D.nxy * L[top].D.nz <= MG_SMEM_CELLS) {
    k_mg_coarsest_smem<<<1, 1024, 0, s>>>(level_op(L[top]), L[top].b, L[top].x, w.conv);
  } else {
    MgLower M;
    for (int l = lt; l <= top; ++l) {
      M.L[l] = level_op(L[l]);
      M.x[l] = L[l].x;
      M.t[l] = L[l].t;
      M.b[l] = L[l].b;
    }
    M.lt = lt;
    M.top = top;
    k_mg_lower<<<1, 1024, 0, s>>>(M, w.conv);
  }
  for (int l = lt - 1; l >= 1; --l) {
    const Op32 O = level_op(L[l]);
    k_mg_prolong<<<L[l].nb, PB, 0, s>>>(O, L[l + 1].D, L[l + 1].x, L[l].x, w.conv);
    k_mg_sweep<float, false><<<L[l].nb, PB, 0, s>>>(O, L[l].x, L[l].t, nullptr, L[l].b, 0, nullptr, w.conv);
    k_mg_sweep<float, false><<<L[l].nb, PB, 0, s>>>(O, L[l].t, L[l].x, nullptr, L[l].b, 0, nullptr, w.conv);
  }
  {
    const Op32 O = level_op(L[0]);
    k_mg_prolong<<<L[0].nb, PB, 0, s>>>(O, L[1].D, L[1].x, L[0].x, w.conv);
    k_mg_sweep<double, false><<<L[0].nb, PB, 0, s>>>(O, L[0].x, L[0].t, nullptr, r, 0, nullptr, w.conv);
    k_mg_sweep<double, false><<<L[0].nb, PB, 0, s>>>(O, L[0].t, L[0].x, nullptr, r, 0, nullptr, w.conv);
    k_mg_sweep<double, true><<<L[0].nb, PB, 0, s>>>(O, L[0].x, nullptr, z, r, 0, prz, w.conv);
  }
}

double host_total(eb_geom g, int slot, cudaStream_t s, cudaError_t &e) {
  ProjWork &w = g->pw;
  e = cudaMemcpyAsync(w.host, w.part + slot * w.nb, sizeof(double) * w.nb, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  double t = 0.0;
  for (int q = 0; q < w.nb; ++q) t += w.host[q];
  return t;
}

template <typename T>
void launch_rhs(eb_geom g, void *const mom[3], double dt, cudaStream_t s) {
  ProjWork &w = g->pw;
  k_rhs<T><<<w.nb, PB, 0, s>>>(make_op(g), (const T *)mom[0], (const T *)mom[1], (const T *)mom[2], 1.0 / dt, w.rhs,
                               w.part + S_SUM * w.nb);
}

template <typename T>
void launch_correct(eb_geom g, void *const mom[3], double dt, cudaStream_t s) {
  ProjWork &w = g->pw;
  k_correct<T><<<w.nb, PB, 0, s>>>(make_op(g), w.x, dt, (T *)mom[0], (T *)mom[1], (T *)mom[2]);
}

}  // namespace

eb_status eb_project_rhs(eb_geom g, void *const mom[3], double dt, double *rms, cudaStream_t s) {
  if (g->has_wind_ref)
    return fail(EB_ERR_STATE, "the projection needs full momenta: this handle has a background momentum profile");
  if (g->src_flags)
    return fail(EB_ERR_STATE, "the anelastic calls take no compressible sources: this handle has them switched on");
  eb_status st = setup(g, s);
  if (st != EB_OK) return st;
  ProjWork &w = g->pw;
  if (g->prec == EB_F64) launch_rhs<double>(g, mom, dt, s);
  else launch_rhs<float>(g, mom, dt, s);
  k_center<<<w.nb, PB, 0, s>>>(make_op(g), w.rhs, w.part + S_SUM * w.nb, w.part + S_CNT * w.nb, w.nb,
                               w.part + S_BB * w.nb);
  cudaError_t e = cudaSuccess;
  const double bb = host_total(g, S_BB, s, e);
  CUDA_TRY(e, "right-hand side");
  if (rms) *rms = w.nact > 0 ? sqrt(bb / (double)w.nact) : 0.0;
  return EB_OK;
}

eb_status eb_project_impl(eb_geom g, void *const mom[3], double dt, double rtol, int maxit, const double *phi0,
                          double *phi_out, int *iters, double *relres, cudaStream_t s, bool correct) {
  if (g->has_wind_ref)
    return fail(EB_ERR_STATE, "the projection needs full momenta: this handle has a background momentum profile");
  if (g->src_flags)
    return fail(EB_ERR_STATE, "the anelastic calls take no compressible sources: this handle has them switched on");
  eb_status st = setup(g, s);
  if (st != EB_OK) return st;
  ProjWork &w = g->pw;
  const Dims &D = g->D;
  const long long N = D.nxy * D.nz;
  const Op O = make_op(g);
  if (g->prec == EB_F64) launch_rhs<double>(g, mom, dt, s);
  else launch_rhs<float>(g, mom, dt, s);
  k_center<<<w.nb, PB, 0, s>>>(O, w.rhs, w.part + S_SUM * w.nb, w.part + S_CNT * w.nb, w.nb, w.part + S_BB * w.nb);
  if (phi0) CUDA_TRY(cudaMemcpyAsync(w.x, phi0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s), "initial guess");
  else CUDA_TRY(cudaMemsetAsync(w.x, 0, sizeof(double) * N, s), "initial guess");
  const bool mg = w.precond == EB_PRECOND_MG;
  if (mg) {
    st = mg_setup(g, s);
    if (st != EB_OK) return st;
  }
  CUDA_TRY(cudaMemsetAsync(w.conv, 0, sizeof(int), s), "reset");
  k_init<<<w.nb, PB, 0, s>>>(O, w.x, w.rhs, w.r, w.z, w.p, w.part + S_RZ0 * w.nb, w.part + S_RR * w.nb);
  if (mg) {   // z = V(r), p = z
    vcycle(g, w.r, w.z, w.part + S_RZ0 * w.nb, s);
    CUDA_TRY(cudaMemcpyAsync(w.p, w.z, sizeof(double) * N, cudaMemcpyDeviceToDevice, s), "search direction");
  }
  cudaError_t e = cudaSuccess;
  const double bb = host_total(g, S_BB, s, e);
  CUDA_TRY(e, "residual norm");
  const double rr0 = host_total(g, S_RR, s, e);
  CUDA_TRY(e, "residual norm");
  const double thr2 = rtol * rtol * bb;
  int it = 0;
  double rr = rr0;
  if (bb > 0.0 && rr0 > thr2) {
    int done = 0;
    for (it = 0; it < maxit; ++it) {
      double *prz = w.part + (it % 2 ? S_RZ1 : S_RZ0) * w.nb;
      double *prz_next = w.part + (it % 2 ? S_RZ0 : S_RZ1) * w.nb;
      k_apply<<<w.nb, PB, 0, s>>>(O, w.p, w.q, w.part + S_PQ * w.nb, w.conv);
      if (mg) {
        k_update<false><<<w.nb, PB, 0, s>>>(O, w.x, w.p, w.q, w.r, w.z, w.part + S_PQ * w.nb, prz, prz_next,
                                            w.part + S_RR * w.nb, w.nb, w.conv);
        vcycle(g, w.r, w.z, prz_next, s);
      } else {
        k_update<true><<<w.nb, PB, 0, s>>>(O, w.x, w.p, w.q, w.r, w.z, w.part + S_PQ * w.nb, prz, prz_next,
                                           w.part + S_RR * w.nb, w.nb, w.conv);
      }
      k_direction<<<w.nb, PB, 0, s>>>(O, w.p, w.z, prz, prz_next, w.part + S_RR * w.nb, w.nb, thr2, it, w.conv);
      // the host reads the convergence flag every few iterations (a V-cycle
      // iteration costs far more than a Jacobi one, so it looks sooner)
      if ((it + 1) % (mg ? 4 : 32) == 0 || it + 1 == maxit) {
        CUDA_TRY(cudaMemcpyAsync(&done, w.conv, sizeof(int), cudaMemcpyDeviceToHost, s), "convergence flag");
        CUDA_TRY(cudaStreamSynchronize(s), "convergence flag");
        if (done) break;
      }
    }
    it = done ? done : maxit;
    rr = host_total(g, S_RR, s, e);
    CUDA_TRY(e, "residual norm");
  }
  if (correct) {
    if (g->prec == EB_F64) launch_correct<double>(g, mom, dt, s);
    else launch_correct<float>(g, mom, dt, s);
  }
  if (phi_out) CUDA_TRY(cudaMemcpyAsync(phi_out, w.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s), "phi");
  CUDA_TRY(cudaGetLastError(), "projection");
  if (iters) *iters = it;
  if (relres) *relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
  return EB_OK;
}

extern "C" {

eb_status eb_project(eb_geom geom, eb_state *U, double dt, double rtol, int maxit, const double *phi0, double *phi,
                     int *iters, double *relres, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(U, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(EB_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(EB_ERR_INVALID_ARG, "rtol must lie in (0, 1)");
  if (maxit < 0) return fail(EB_ERR_INVALID_ARG, "maxit must be >= 0");
  if ((phi0 && ((uintptr_t)phi0 % 8)) || (phi && ((uintptr_t)phi % 8)))
    return fail(EB_ERR_INVALID_ARG, "phi pointer misaligned");
  void **u = state_ptrs(U);
  void *mom[3] = {u[2], u[3], u[4]};
  return eb_project_impl(geom, mom, dt, rtol, maxit, phi0, phi, iters, relres, as_stream(stream), true);
}

eb_status eb_project_set_preconditioner(eb_geom geom, int kind) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (kind != EB_PRECOND_JACOBI && kind != EB_PRECOND_MG) return fail(EB_ERR_INVALID_ARG, "unknown preconditioner");
  if (kind == EB_PRECOND_MG) {
    int dims[kMgMaxLevels][3], nlev = 0;
    if (!mg_plan(geom->D, dims, nlev))
      return fail(EB_ERR_INVALID_ARG,
                  "grid cannot be coarsened for multigrid (even sizes needed; coarsest grid <= 32768 cells)");
  }
  geom->pw.precond = kind;
  return EB_OK;
}

eb_status eb_anelastic_step(eb_geom geom, const eb_state *Un, eb_state *Unp1, double dt, int nsteps, double rtol,
                            int maxit, int *iters, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (!geom->has_ref) return fail(EB_ERR_STATE, "the anelastic step needs a handle built with a reference profile");
  if (geom->src_flags)
    return fail(EB_ERR_STATE, "the anelastic calls take no compressible sources: this handle has them switched on");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(Un, es) || !state_ok(Unp1, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(EB_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (nsteps < 1) return fail(EB_ERR_INVALID_ARG, "nsteps must be >= 1");
  if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(EB_ERR_INVALID_ARG, "rtol must lie in (0, 1)");
  if (maxit < 0) return fail(EB_ERR_INVALID_ARG, "maxit must be >= 0");
  void **u0 = state_ptrs(Un), **u1 = state_ptrs(Unp1);
  for (int f = 0; f < 5; ++f)
    for (int e = 0; e < 5; ++e) {
      const char *a = (const char *)u0[f], *b = (const char *)u1[e];
      if (a < b + field_count(geom->D, e) * es && b < a + field_count(geom->D, f) * es)
        return fail(EB_ERR_INVALID_ARG, "Un and Unp1 overlap");
    }
  cudaStream_t s = as_stream(stream);
  // scratch states: C, D alternate between steps, A holds the first stage
  for (int b = 0; b < 3; ++b)
    for (int f = 0; f < 5; ++f)
      if (!geom->scr[b][f]) {
        cudaError_t e = cudaMalloc(&geom->scr[b][f], field_count(geom->D, f) * es);
        if (e != cudaSuccess) return cuda_fail(e, "alloc step scratch");
        geom->allocs.push_back(geom->scr[b][f]);
      }
  void **C = geom->scr[0], **Dd = geom->scr[1], **A = geom->scr[2];
  void **cur = u0;
  for (int n = 0; n < nsteps; ++n) {
    void **dst = (n == nsteps - 1) ? u1 : (cur == C ? Dd : C);
    void **srcs[2] = {cur, A}, **outs[2] = {A, dst};
    const double frac[2] = {0.5, 1.0};
    for (int q = 0; q < 2; ++q) {
      if (geom->prec == EB_F64) stage<double>(geom, srcs[q], cur, outs[q], dt * frac[q], 1, s);
      else stage<float>(geom, srcs[q], cur, outs[q], dt * frac[q], 1, s);
      // the density stays at the reference: perturbation zero
      CUDA_TRY(cudaMemsetAsync(outs[q][0], 0, field_count(geom->D, 0) * es, s), "density");
      void *mom[3] = {outs[q][2], outs[q][3], outs[q][4]};
      int it = 0;
      const eb_status st =
          eb_project_impl(geom, mom, dt * frac[q], rtol, maxit, nullptr, nullptr, &it, nullptr, s, true);
      if (st != EB_OK) return st;
      if (iters) iters[2 * n + q] = it;
    }
    cur = dst;
  }
  CUDA_TRY(cudaGetLastError(), "anelastic step");
  return EB_OK;
}

}  // extern "C"
