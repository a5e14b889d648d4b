// eb_sources.cu -- the sources of the compressible system (Sec. 2.1, Eq.
// mom-comp) that eb_step adds to the flux divergence of every stage when the
// handle asks for them (eb_geom_set_sources):
//   -grad p' on the momentum grids, p' = p - p0(z) the perturbation pressure,
//            p from the equation of state p = P00 (R rho theta / P00)^gamma;
//   B = -rho' g on rho*w (buoyancy).
// Pressure and density live at cell centres; every momentum CV sits between
// the cell e_d back along its staggering axis d (a) and the cell of the same
// index (b): its source is -(p'_b - p'_a) / dx_d, and on w also
// -g (rho'_a + rho'_b) / 2.  A covered cell takes the other cell's value (no
// pressure force across a wall side).  The source enters the CV's dU as it
// stands, after the flux divergence and before the redistribution.
//
// States hold perturbations about the reference profiles, so
//   p' = p0(k) * expm1(gamma * log1p((rho theta)' / (rho0 theta0)(k)))
// (the deviation form of p - p0: the float path rounds p', not p ~ 1e5 Pa);
// p0(k) and 1 / (rho0 theta0)(k) are per-level tables built in double when
// the sources are switched on.  A first pass writes p' of every fluid cell
// (k_pressure), the second forms the sources (k_sources).
#include "eb_step.cuh"

namespace {

template <typename T>
struct SourceArgs {
  Dims D;
  const uint8_t *cflag;      // dense flags of the c grid (bit 0: holds fluid)
  const uint8_t *gflag[3];   // of the u, v, w grids
  const T *rho, *rt;         // rho', (rho theta)' of the stage's source state
  T *out[3];                 // rho*u, rho*v, rho*w of the stage's output
  const T *p0, *irt0;        // per level: p0, 1 / (rho0 theta0)
  T *pp;                     // p' of every fluid cell (written by k_pressure)
  T dt, gamma, grav, inv[3];
  int pressure, buoyancy;
  unsigned *status;
};

__device__ inline float log1p_t(float x) { return log1pf(x); }
__device__ inline double log1p_t(double x) { return log1p(x); }
__device__ inline float expm1_t(float x) { return expm1f(x); }
__device__ inline double expm1_t(double x) { return expm1(x); }

// p' of every cell that holds fluid, once per stage (the source pass reads
// each cell's value for up to six faces)
template <typename T>
__global__ void k_pressure(const __grid_constant__ SourceArgs<T> S) {
  const Dims &D = S.D;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= D.nxy * (long long)D.nz) return;
  if (!(S.cflag[t] & 1)) return;
  const int k = (int)D.fnxy.div((unsigned)t);
  S.pp[t] = S.p0[k] * expm1_t(S.gamma * log1p_t(S.rt[t] * S.irt0[k]));
}

// one thread per (i, j, k) position: the u and v CVs of level k (k < nz) and
// the w CV of face level k (0 < k < nz)
template <typename T>
__global__ void k_sources(const __grid_constant__ SourceArgs<T> S) {
  const Dims &D = S.D;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= D.nxy * (long long)(D.nz + 1)) return;
  int i, j, k;
  split_index(D, (unsigned)t, i, j, k);   // below 2^32 (checked when the handle is built)
  auto pprime = [&](long long c, int) -> T { return S.pp[c]; };
  const bool own = k < D.nz && (S.cflag[t] & 1);
  T p_own = T(0);
  if (own && S.pressure) p_own = pprime(t, k);
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (d < 2 ? k >= D.nz : (k == 0 || k >= D.nz)) continue;
    if (!(S.gflag[d][t] & 1)) continue;
    long long a;
    int ka = k;
    if (d == 0) a = (i == 0 ? D.nx - 1 : i - 1) + (long long)D.nx * j + D.nxy * k;
    else if (d == 1) a = i + (long long)D.nx * (j == 0 ? D.ny - 1 : j - 1) + D.nxy * k;
    else {
      a = t - D.nxy;
      ka = k - 1;
    }
    const bool fa = S.cflag[a] & 1;
    if (!fa && !own) continue;
    T s = T(0);
    if (S.pressure) {
      T pa = fa ? pprime(a, ka) : p_own;
      const T pb = own ? p_own : pa;
      s -= (pb - pa) * S.inv[d];
    }
    if (S.buoyancy && d == 2) {
      T ra = fa ? S.rho[a] : S.rho[t];
      const T rb = own ? S.rho[t] : ra;
      s -= S.grav * T(0.5) * (ra + rb);
    }
    const T v = S.out[d][t] + S.dt * s;
    S.out[d][t] = v;
    bad = bad || !isfinite(v);
  }
  if (bad) atomicOr(S.status, EB_DEV_NUMERIC);
}

}  // namespace

template <typename T>
void launch_sources(const StepArgs<T> &A, int flags, const T *p0, const T *irt0, T *pp, cudaStream_t s) {
  SourceArgs<T> S;
  S.D = A.D;
  S.cflag = A.G[0].dflag;
  for (int d = 0; d < 3; ++d) {
    S.gflag[d] = A.G[d + 1].dflag;
    S.out[d] = A.out[d + 2];
  }
  S.rho = A.src.f[0];
  S.rt = A.src.f[1];
  S.p0 = p0;
  S.irt0 = irt0;
  S.pp = pp;
  S.dt = A.dtT;
  S.gamma = (T)(EB_CP / (EB_CP - EB_RD));
  S.grav = (T)EB_GRAV;
  S.inv[0] = (T)A.D.idx;
  S.inv[1] = (T)A.D.idy;
  S.inv[2] = (T)A.D.idz;
  S.pressure = (flags & EB_SOURCE_PRESSURE) ? 1 : 0;
  S.buoyancy = (flags & EB_SOURCE_BUOYANCY) ? 1 : 0;
  S.status = A.status;
  if (S.pressure) {
    const long long nc = A.D.nxy * (long long)A.D.nz;
    k_pressure<T><<<(unsigned)((nc + 255) / 256), 256, 0, s>>>(S);
  }
  const long long n = A.D.nxy * (long long)(A.D.nz + 1);
  k_sources<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S);
}

template void launch_sources<float>(const StepArgs<float> &, int, const float *, const float *, float *,
                                    cudaStream_t);
template void launch_sources<double>(const StepArgs<double> &, int, const double *, const double *, double *,
                                     cudaStream_t);
