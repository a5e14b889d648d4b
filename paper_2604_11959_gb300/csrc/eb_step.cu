// eb_step.cu -- per-step kernels of the EB advance.
//
//   flux + update (Eqs. update-cc / update-fc, Sec. 4.1):
//     (the geometry-free bulk above each column's kfast level is in
//     eb_fast.cu)
//     k_stage        : (FP64 path) the advected value of every CV the face
//                      stencils read, once;
//     k_face_flux    : the provisional flux of every face the near-EB CVs
//                      read, once, with covered-neighbour fallbacks;
//     k_band         : the cut CVs below kfast (open-face fractions and
//                      fluxes interpolated to the cut-face centroids, as rows
//                      of coefficients built at set-up), then, in the same
//                      launch, the regular CVs below kfast (plain face
//                      differences).
//   weighted state redistribution (Sec. 5.1, Eqs. qhat_omega, qrecon,
//   final_update_omega), on compact lists built at set-up:
//     k_qhat  : neighbourhood averages of the small CVs;
//     k_sigma : least-squares slopes and the limiter, 8 lanes per small CV;
//     k_final : the final update of every CV the redistribution changes.
//
// Every kernel writes a disjoint set of CVs, so no atomics are needed and
// results are deterministic.
#include "eb_step.cuh"
#include "eb_bulk.cuh"

#include <math.h>

namespace {

template <typename T>
__device__ inline bool finite_val(T v) {
  return isfinite(v);
}

// Faces of the low side of CV (i,j,k) along d exist inside the domain?  The
// high z face of the top c, u, v CVs is the wall.
__device__ inline bool high_face_exists(const Dims &D, int g, int d, int k) {
  if (d != 2) return true;
  return g == 3 ? (k + 1 <= D.nz) : (k + 1 < D.nz);
}

// Flux through the centroid of the low d-face of CV (i,j,k): bilinear
// interpolation of the provisional fluxes of the face and of the neighbour
// faces toward which the centroid is offset (Sec. 4.1), read from the face
// arrays staged by k_face_flux.  An offset is dropped when a face it needs is
// closed or outside the domain.
__device__ inline bool face_usable_dense(const GeoBand &geo, const Dims &D, int g, int d, int i, int j, int k) {
  if (k < 0 || k >= nzg_of(D, g)) return false;
  if (g == 3 && d != 2 && (k < 1 || k > D.nz - 1)) return false;
  if (g != 3 && d == 2 && k == 0) return false;   // bottom wall faces carry no flux
  return (geo.dense(D, g, i, j, k) >> (2 + d)) & 1;
}

// The CV that owns a face (its low face): coordinates, state index, dense
// flag byte and record (-1 without one), looked up once.
struct FaceOwner {
  int i, j, k;
  long long c;
  uint8_t flag;
  long long rec;
};

__device__ inline FaceOwner face_owner(const GeoBand &geo, const Dims &D, int g, int i, int j, int k) {
  FaceOwner o{i, j, k, lin(D, i, j, k), 0, -1};
  if (k >= 0 && k < nzg_of(D, g)) {
    o.flag = geo.G[g].dflag[o.c];
    if (o.flag & 2) o.rec = geo.record(D, g, i, j, k);
  }
  return o;
}

// open area fraction of the owner's low d-face (float copies on the float path)
template <typename R>
__device__ inline R owner_beta(const GeoBand &geo, int g, int d, const FaceOwner &o) {
  if (o.rec < 0) return (o.flag & 1) ? R(1) : R(0);
  const long long r = (long long)d * geo.G[g].nrec + o.rec;
  if (sizeof(R) == sizeof(double)) return (R)geo.G[g].beta[r];
  return (R)geo.G[g].beta_f[r];
}

// (index, weight) terms of the flux through the centroid of the owner's low
// d-face (Sec. 4.1): the face itself and the neighbour faces of the bilinear
// interpolation toward the centroid; an offset is dropped when a face it
// needs is closed or outside the domain.  At most four terms.
__device__ inline int centroid_terms(const GeoBand &geo, const Dims &D, int g, int d, const FaceOwner &o,
                                     long long idx[4], double w[4]) {
  idx[0] = o.c;
  w[0] = 1.0;
  if (o.rec < 0) return 1;   // no record: open face, centroid at the centre
  const GridDev &G = geo.G[g];
  const double ga = G.fcent[(long long)(2 * d) * G.nrec + o.rec];
  const double gb = G.fcent[(long long)(2 * d + 1) * G.nrec + o.rec];
  if (ga == 0.0 && gb == 0.0) return 1;
  const int i = o.i, j = o.j, k = o.k;
  const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
  int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
  ea[ta] = ga >= 0.0 ? 1 : -1;
  eb[tb] = gb >= 0.0 ? 1 : -1;
  const bool ua = ga != 0.0 && face_usable_dense(geo, D, g, d, i + ea[0], j + ea[1], k + ea[2]);
  const bool ub = gb != 0.0 && face_usable_dense(geo, D, g, d, i + eb[0], j + eb[1], k + eb[2]);
  const bool uab = ga != 0.0 && gb != 0.0 &&
                   face_usable_dense(geo, D, g, d, i + ea[0] + eb[0], j + ea[1] + eb[1], k + ea[2] + eb[2]);
  const bool za = ga != 0.0 && (!ua || (gb != 0.0 && !uab));
  const bool zb = gb != 0.0 && (!ub || (ga != 0.0 && !uab));
  const double wa = za ? 0.0 : fabs(ga);
  const double wb = zb ? 0.0 : fabs(gb);
  if (wa == 0.0 && wb == 0.0) return 1;
  w[0] = (1.0 - wa) * (1.0 - wb);
  int n = 1;
  if (wa != 0.0) {
    idx[n] = lin(D, i + ea[0], j + ea[1], k + ea[2]);
    w[n++] = wa * (1.0 - wb);
  }
  if (wb != 0.0) {
    idx[n] = lin(D, i + eb[0], j + eb[1], k + eb[2]);
    w[n++] = wb * (1.0 - wa);
  }
  if (wa != 0.0 && wb != 0.0) {
    idx[n] = lin(D, i + ea[0] + eb[0], j + ea[1] + eb[1], k + ea[2] + eb[2]);
    w[n++] = wa * wb;
  }
  return n;
}

template <typename T>
__device__ inline void write_out(const StepArgs<T> &A, int f, long long c, T delta) {
  T v;
  if (A.base[0]) v = A.base[f][c] + A.dtT * delta;
  else v = delta;
  A.out[f][c] = v;
  if (!isfinite(v)) atomicOr(A.status, EB_DEV_NUMERIC);
}

template <typename T>
__device__ inline void write_out_d(const StepArgs<T> &A, int f, long long c, double delta) {
  T v;
  if (A.base[0]) v = A.base[f][c] + (T)(A.dt * delta);
  else v = (T)delta;
  A.out[f][c] = v;
  if (!isfinite(v)) atomicOr(A.status, EB_DEV_NUMERIC);
}

// Near-EB rows.  For a cut CV (it has a geometry record), the open area fractions,
// the centroid interpolation weights, 1 / dx_d and 1 / alpha depend on the
// geometry alone, so its dU of Eqs. update-cc / update-fc is a fixed linear
// combination of the staged face fluxes: each term of the low d-face enters
// with +beta w / (dx_d alpha), each term of the high d-face with
// -beta w / (dx_d alpha).  The rows are built once per geometry (a count pass,
// a scan, a fill pass) in double; every step applies them (k_band).
struct RowBuild {
  Dims D;
  GridDev G[4];
  int g;
  long long *cnt;
};

template <bool FILL>
__global__ void k_band_rows(RowBuild B) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int g = B.g;
  const GridDev &G = B.G[g];
  if (t >= G.nband_rec) return;
  GeoBand geo;
  geo.G = B.G;
  const Dims &D = B.D;
  int i, j, k;
  split_index(D, G.blist[t], i, j, k);
  const FaceOwner own = face_owner(geo, D, g, i, j, k);
  const double alpha = own.rec >= 0 ? G.alpha[own.rec] : 1.0;
  const double inv[3] = {D.idx, D.idy, D.idz};
  long long pos = FILL ? B.cnt[3 * t] : 0;
  for (int d = 0; d < 3; ++d) {
    const bool lo_wall = g != 3 && d == 2 && k == 0;
    const double bl = lo_wall ? 0.0 : owner_beta<double>(geo, g, d, own);
    const bool hx = high_face_exists(D, g, d, k);
    const FaceOwner hi = hx ? face_owner(geo, D, g, i + (d == 0), j + (d == 1), k + (d == 2))
                            : FaceOwner{i, j, k, own.c, 0, -1};
    const double bh = hx ? owner_beta<double>(geo, g, d, hi) : 0.0;
    int n = 0;
    for (int side = 0; side < 2; ++side) {
      const double b = side ? -bh : bl;
      if (b == 0.0) continue;
      long long idx[4];
      double w[4];
      const int m = centroid_terms(geo, D, g, d, side ? hi : own, idx, w);
      if (FILL) {
        for (int q = 0; q < m; ++q, ++pos) {
          const double coef = b * w[q] * inv[d] / alpha;
          G.sidx[pos] = (unsigned)idx[q];
          G.scoef[pos] = coef;
          G.scoef_f[pos] = (float)coef;
        }
      }
      n += m;
    }
    if (!FILL) B.cnt[3 * t + d] = n;
  }
  if (FILL) G.stiny[t] = (own.rec >= 0 && alpha < 1e-3) ? 1 : 0;
}

__global__ void k_rows_to_u32(const long long *src, long long n, unsigned *dst) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (unsigned)src[t];
}

// Phase A of the near-EB path: the provisional flux of every listed face,
// once (general geometry: covered-neighbour fallbacks, zero momentum of
// covered CVs).
// The provisional flux of Sec. 4.1 through the low Dd-face of CV c =
// (i, j, k) of grid G, with the availability rules of the general face flux
// (covered or absent CVs carry no momentum, the centred value replaces the
// third-order one when the far upstream CV is not available), written for
// one (grid, direction) pair at a time: every neighbour index is the face's
// own index plus a periodic offset computed once.
// index offset of a step s along direction dir from coordinate x (periodic in x, y)
__device__ inline long long step_off(const Dims &D, int dir, int x, int s) {
  if (dir == 2) return (long long)s * D.nxy;
  const int n = dir == 0 ? D.nx : D.ny;
  int t = x + s;
  t = t < 0 ? t + n : (t >= n ? t - n : t);
  return (long long)(t - x) * (dir == 0 ? 1 : D.nx);
}

// full momentum of face-grid G (1: rho*u, 2: rho*v, 3: rho*w) at state index
// idx on level k: the stored value plus the background profile (rho*w has none)
template <typename T, int G>
__device__ inline T momentum(const StateIn<T> &U, long long idx, int k) {
  if constexpr (G == 1) return U.f[2][idx] + U.ref_u[k];
  else if constexpr (G == 2) return U.f[3][idx] + U.ref_v[k];
  else if constexpr (G == 3) return U.f[4][idx];
  else return T(0);   // the c grid has no momentum of its own (never called)
}

// advected value of CV (i, j, k) of grid G (state index idx): theta on the c
// grid; on a face grid the momentum over the mean density of the non-covered
// c-cells beside the CV, 0 when both are covered (Sec. 4.1)
template <typename T, int G>
__device__ inline T cv_advected(const StepArgs<T> &A, long long idx, int i, int j, int k) {
  const Dims &D = A.D;
  auto rho = [&](long long q, int kk) -> T { return A.src.ref_rho[kk] + A.src.f[0][q]; };
  if (G == 0) return eb_div(A.src.ref_rt[k] + A.src.f[1][idx], rho(idx, k));
  constexpr int S = G - 1;
  const int crd[3] = {i, j, k};
  const long long ia = idx + step_off(D, S, crd[S], -1);
  const int ka = k - (S == 2 ? 1 : 0);
  auto fluid0 = [&](long long q, int kk) -> bool { return kk >= 0 && kk < D.nz && (A.G[0].dflag[q] & 1); };
  const bool a = fluid0(ia, ka), b = fluid0(idx, k);
  T rb;
  if (a && b) rb = T(0.5) * (rho(ia, ka) + rho(idx, k));
  else if (a) rb = rho(ia, ka);
  else if (b) rb = rho(idx, k);
  else return T(0);
  return eb_div(momentum<T, G>(A.src, idx, k), rb);
}

template <typename T, int G, int Dd, bool MASK>
__device__ inline unsigned face_flux_lean(const StepArgs<T> &A, long long c, int i, int j, int k, unsigned bits,
                                          T &fm, T &fp) {
  const Dims &D = A.D;
  constexpr int S = G - 1;      // stagger direction of a face grid (c grid: none)
  constexpr int MG = Dd + 1;    // momentum grid normal to the face
  const int crd[3] = {i, j, k};
  // index offset of a step s along direction dir from coordinate x (periodic in x, y)
  auto off = [&](int dir, int x, int s) -> long long {
    if (dir == 2) return (long long)s * D.nxy;
    const int n = dir == 0 ? D.nx : D.ny;
    int t = x + s;
    t = t < 0 ? t + n : (t >= n ? t - n : t);
    return (long long)(t - x) * (dir == 0 ? 1 : D.nx);
  };
  // availability test number n: evaluated from the dense flags when the
  // masks are built (MASK), read from the face's mask bits otherwise
  unsigned out = 0;
  auto fluid = [&](int n, int q, long long idx, int kk) -> bool {
    if (!MASK) return (bits >> n) & 1;
    const bool f = kk >= 0 && kk < nzg_of(D, q) && (A.G[q].dflag[idx] & 1);
    out |= (unsigned)f << n;
    return f;
  };
  // momentum of grid MG entering a mass flux (test n)
  auto mom = [&](int n, long long idx, int kk) -> T {
    if (MG == 3 && (kk <= 0 || kk >= D.nz)) return T(0);
    const bool f = fluid(n, MG, idx, kk);
    if (MASK) return T(0);
    return f ? momentum<T, MG>(A.src, idx, kk) : T(0);
  };
  auto rho = [&](long long idx, int kk) -> T { return A.src.ref_rho[kk] + A.src.f[0][idx]; };
  // advected value of the grid-G CV t steps along Dd from the face's CV
  auto advected = [&](int t) -> T {
    const long long idx = c + off(Dd, crd[Dd], t);
    const int kk = k + (Dd == 2 ? t : 0);
    if (G == 0) return MASK ? T(0) : eb_div(A.src.ref_rt[kk] + A.src.f[1][idx], rho(idx, kk));
    if (G == 3 && (kk <= 0 || kk >= D.nz)) return T(0);
    // the two c-cells beside the face-grid CV: one step back along S, and
    // itself (the CV's own coordinate along S, wrapped, when S is Dd)
    const int cs = S == Dd ? (S == 2 ? kk : wrapi(crd[S] + t, S == 0 ? D.nx : D.ny)) : crd[S];
    const long long ia = idx + off(S, cs, -1);
    const int ka = kk - (S == 2 ? 1 : 0);
    const bool a = fluid(2 + 2 * (t + 2), 0, ia, ka), b = fluid(3 + 2 * (t + 2), 0, idx, kk);
    if (MASK) return T(0);
    T rb;
    if (a && b) rb = T(0.5) * (rho(ia, ka) + rho(idx, kk));
    else if (a) rb = rho(ia, ka);
    else if (b) rb = rho(idx, kk);
    else return T(0);
    return eb_div(momentum<T, G>(A.src, idx, kk), rb);
  };
  auto cv_fluid = [&](int n, int t) -> bool {
    const long long idx = c + off(Dd, crd[Dd], t);
    return fluid(n, G, idx, k + (Dd == 2 ? t : 0));
  };
  if (MASK) {   // every test, whatever the flow direction
    if (G != 0) mom(0, c + off(G == MG ? Dd : S, crd[G == MG ? Dd : S], -1), k - ((G == MG ? Dd : S) == 2 ? 1 : 0));
    mom(1, c, k);
    for (int t = -2; t <= 1; ++t) advected(t);
    cv_fluid(10, -2);
    cv_fluid(11, 1);
    return out;
  }
  // mass flux
  if (G == 0) {
    fm = mom(1, c, k);
  } else if (G == MG) {
    fm = T(0.5) * (mom(0, c + off(Dd, crd[Dd], -1), k - (Dd == 2 ? 1 : 0)) + mom(1, c, k));
  } else {
    fm = T(0.5) * (mom(0, c + off(S, crd[S], -1), k - (S == 2 ? 1 : 0)) + mom(1, c, k));
  }
  fp = T(0);
  if (fm == T(0)) return 0;
  // FP64 path: advected values staged once per CV this step (k_stage; zero on
  // the w-grid wall levels, which are never staged), as FP64 divisions are
  // scarce on this GPU; the float path forms them here
  const T *PV = (const T *)A.G[G].pv;
  auto staged = [&](int t) -> T {
    if constexpr (sizeof(T) == sizeof(double)) return PV[c + off(Dd, crd[Dd], t)];
    else return advected(t);
  };
  const T pL = staged(-1), pR = staged(0);
  T val;
  if (fm > T(0)) {
    const bool has = cv_fluid(10, -2);
    const T pF = has ? staged(-2) : T(0);
    val = upwind_value(fm, pF, pL, pR, T(0), has, false);
  } else {
    const bool has = cv_fluid(11, 1);
    const T pF = has ? staged(1) : T(0);
    val = upwind_value(fm, T(0), pL, pR, pF, false, has);
  }
  fp = fm * val;
  return 0;
}

// list entry t of all faces -> (grid, direction, entry of that list)
template <typename T>
__device__ inline bool face_of(const StepArgs<T> &A, long long &t, int &g, int &d) {
  for (g = 0; g < 4; ++g) {
    for (d = 0; d < 3; ++d) {
      if (t < A.G[g].nface[d]) return true;
      t -= A.G[g].nface[d];
    }
  }
  return false;
}

template <typename T, bool MASK>
__device__ inline unsigned face_dispatch(const StepArgs<T> &A, int g, int d, unsigned c, unsigned bits, T &fm,
                                         T &fp) {
  int i, j, k;
  split_index(A.D, c, i, j, k);
  // one compiled copy per (grid, direction)
  switch (g * 3 + d) {
    case 0: return face_flux_lean<T, 0, 0, MASK>(A, c, i, j, k, bits, fm, fp);
    case 1: return face_flux_lean<T, 0, 1, MASK>(A, c, i, j, k, bits, fm, fp);
    case 2: return face_flux_lean<T, 0, 2, MASK>(A, c, i, j, k, bits, fm, fp);
    case 3: return face_flux_lean<T, 1, 0, MASK>(A, c, i, j, k, bits, fm, fp);
    case 4: return face_flux_lean<T, 1, 1, MASK>(A, c, i, j, k, bits, fm, fp);
    case 5: return face_flux_lean<T, 1, 2, MASK>(A, c, i, j, k, bits, fm, fp);
    case 6: return face_flux_lean<T, 2, 0, MASK>(A, c, i, j, k, bits, fm, fp);
    case 7: return face_flux_lean<T, 2, 1, MASK>(A, c, i, j, k, bits, fm, fp);
    case 8: return face_flux_lean<T, 2, 2, MASK>(A, c, i, j, k, bits, fm, fp);
    case 9: return face_flux_lean<T, 3, 0, MASK>(A, c, i, j, k, bits, fm, fp);
    case 10: return face_flux_lean<T, 3, 1, MASK>(A, c, i, j, k, bits, fm, fp);
    default: return face_flux_lean<T, 3, 2, MASK>(A, c, i, j, k, bits, fm, fp);
  }
}

// Set-up: the availability bits of every listed face.
__global__ void k_face_mask(StepArgs<float> A) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int g, d;
  if (!face_of(A, t, g, d)) return;
  float fm, fp;
  A.G[g].fmask[d][t] = (uint16_t)face_dispatch<float, true>(A, g, d, A.G[g].flist[d][t], 0u, fm, fp);
}

// the provisional flux of listed face t (all grids and directions in turn)
template <typename T>
__device__ inline void face_one(const StepArgs<T> &A, long long t) {
  int g, d;
  if (!face_of(A, t, g, d)) return;
  const unsigned c = A.G[g].flist[d][t];
  T fm, fp;
  face_dispatch<T, false>(A, g, d, c, A.G[g].fmask[d][t], fm, fp);
  ((T *)A.G[g].fh[d])[c] = fp;
  if (A.G[g].fhm[d]) ((T *)A.G[g].fhm[d])[c] = fm;
}

template <typename T>
__global__ void k_face_flux(StepArgs<T> A) {
  face_one(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Set-up: every CV of grid G a listed (G, Dd) face's stencil reads (t = -2 .. 1
// along the face normal; w-grid wall levels excluded: their value is 0).
template <int G, int Dd>
__device__ inline void stage_marks_one(const Dims &D, const GridDev *GG, unsigned c, uint8_t *const marks[4]) {
  int i, j, k;
  split_index(D, c, i, j, k);
  const int crd[3] = {i, j, k};
  for (int t = -2; t <= 1; ++t) {
    const int kk = k + (Dd == 2 ? t : 0);
    if (kk < 0 || kk >= GG[G].nst || kk >= nzg_of(D, G)) continue;
    if (G == 3 && (kk <= 0 || kk >= D.nz)) continue;
    marks[G][c + step_off(D, Dd, crd[Dd], t)] = 1;
  }
}

struct StageMarkArgs {
  Dims D;
  GridDev G[4];
  uint8_t *marks[4];
};

__global__ void k_stage_marks(StageMarkArgs M) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  int g = 0, d = 0;
  for (g = 0; g < 4; ++g) {
    for (d = 0; d < 3; ++d) {
      if (t < M.G[g].nface[d]) break;
      t -= M.G[g].nface[d];
    }
    if (d < 3) break;
  }
  if (g >= 4) return;
  const unsigned c = M.G[g].flist[d][t];
  switch (g * 3 + d) {
    case 0: stage_marks_one<0, 0>(M.D, M.G, c, M.marks); break;
    case 1: stage_marks_one<0, 1>(M.D, M.G, c, M.marks); break;
    case 2: stage_marks_one<0, 2>(M.D, M.G, c, M.marks); break;
    case 3: stage_marks_one<1, 0>(M.D, M.G, c, M.marks); break;
    case 4: stage_marks_one<1, 1>(M.D, M.G, c, M.marks); break;
    case 5: stage_marks_one<1, 2>(M.D, M.G, c, M.marks); break;
    case 6: stage_marks_one<2, 0>(M.D, M.G, c, M.marks); break;
    case 7: stage_marks_one<2, 1>(M.D, M.G, c, M.marks); break;
    case 8: stage_marks_one<2, 2>(M.D, M.G, c, M.marks); break;
    case 9: stage_marks_one<3, 0>(M.D, M.G, c, M.marks); break;
    case 10: stage_marks_one<3, 1>(M.D, M.G, c, M.marks); break;
    default: stage_marks_one<3, 2>(M.D, M.G, c, M.marks); break;
  }
}

// Phase A0: the advected value of every staged CV, once per step.
// the advected value of staged CV t (all grids in turn)
template <typename T>
__device__ inline void stage_one(const StepArgs<T> &A, long long t) {
  int g = 0;
  for (g = 0; g < 4; ++g) {
    if (t < A.G[g].nstage) break;
    t -= A.G[g].nstage;
  }
  if (g >= 4) return;
  const unsigned c = A.G[g].stlist[t];
  int i, j, k;
  split_index(A.D, c, i, j, k);
  T v;
  switch (g) {
    case 0: v = cv_advected<T, 0>(A, c, i, j, k); break;
    case 1: v = cv_advected<T, 1>(A, c, i, j, k); break;
    case 2: v = cv_advected<T, 2>(A, c, i, j, k); break;
    default: v = cv_advected<T, 3>(A, c, i, j, k); break;
  }
  ((T *)A.G[g].pv)[c] = v;
}

template <typename T>
__global__ void k_stage(StepArgs<T> A) {
  stage_one(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// Phase B: the divergence of every listed cut CV, from
// its precomputed row; the mixed path sums the rows of tiny cut CVs
// (alpha < 1e-3, whose coefficients carry 1 / alpha) in double.
template <typename T, typename R, typename C>
__device__ inline void apply_row(const StepArgs<T> &A, const GridDev &G, const C *coef, long long t, R &sm,
                                 R &sp) {
  sm = R(0);
  sp = R(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const T *FH = (const T *)G.fh[d];
    const T *FM = (const T *)G.fhm[d];
    const unsigned q1 = G.srow[3 * t + d + 1];
    unsigned q = G.srow[3 * t + d];
    // four terms at a time: their index, coefficient and flux loads are independent
    for (; q + 4 <= q1; q += 4) {
      unsigned f[4];
      R cq[4], h[4], m[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        f[e] = G.sidx[q + e];
        cq[e] = (R)coef[q + e];
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        h[e] = (R)FH[f[e]];
        m[e] = FM ? (R)FM[f[e]] : R(0);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        sp += cq[e] * h[e];
        sm += cq[e] * m[e];
      }
    }
    for (; q < q1; ++q) {
      const unsigned f = G.sidx[q];
      const R cq = (R)coef[q];
      sp += cq * (R)FH[f];
      if (FM) sm += cq * (R)FM[f];
    }
  }
}

// The other near-EB CVs are regular (with a geometry record or without):
// every face is open with its centroid at the face centre, so the divergence
// is the plain difference of the staged face fluxes.
template <typename T>
__device__ inline void regular_cv(const StepArgs<T> &A, long long t) {
  const Dims &D = A.D;
  int g = 0;
  for (g = 0; g < 4; ++g) {
    const long long n = A.G[g].nband - A.G[g].nband_rec;
    if (t < n) break;
    t -= n;
  }
  if (g >= 4) return;
  const unsigned c = A.G[g].blist[A.G[g].nband_rec + t];
  int i, j, k;
  split_index(D, c, i, j, k);
  const T inv[3] = {T(D.idx), T(D.idy), T(D.idz)};
  T sm = T(0), sp = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int di = d == 0, dj = d == 1, dk = d == 2;
    const T *FH = (const T *)A.G[g].fh[d];
    const T *FM = (const T *)A.G[g].fhm[d];
    const T bl = (g != 3 && d == 2 && k == 0) ? T(0) : T(1);
    const T bh = high_face_exists(D, g, d, k) ? T(1) : T(0);
    T ml = T(0), pl = T(0), mh = T(0), ph = T(0);
    if (bl > T(0)) {
      pl = FH[c];
      if (FM) ml = FM[c];
    }
    if (bh > T(0)) {
      const long long n = lin(D, i + di, j + dj, k + dk);
      ph = FH[n];
      if (FM) mh = FM[n];
    }
    sm += (bh * mh - bl * ml) * inv[d];
    sp += (bh * ph - bl * pl) * inv[d];
  }
  if (g == 0) {
    write_out(A, 0, c, -sm);
    write_out(A, 1, c, -sp);
  } else {
    write_out(A, g + 1, c, -sp);
  }
}

// the divergence and update of near-EB CV t: the cut CVs' rows first, then
// the regular near-EB CVs
template <typename T>
__device__ inline void band_one(const StepArgs<T> &A, long long t) {
  const long long nrec = A.G[0].nband_rec + A.G[1].nband_rec + A.G[2].nband_rec + A.G[3].nband_rec;
  if (t >= nrec) {   // the regular CVs follow the rows in the same launch
    regular_cv(A, t - nrec);
    return;
  }
  int g = 0;
  for (g = 0; g < 4; ++g) {
    if (t < A.G[g].nband_rec) break;
    t -= A.G[g].nband_rec;
  }
  if (g >= 4) return;
  const GridDev &G = A.G[g];
  const unsigned c = G.blist[t];
  if (sizeof(T) == sizeof(double) || G.stiny[t]) {
    double sm, sp;
    apply_row<T, double, double>(A, G, G.scoef, t, sm, sp);
    if (g == 0) {
      write_out_d(A, 0, c, sm);
      write_out_d(A, 1, c, sp);
    } else {
      write_out_d(A, g + 1, c, sp);
    }
  } else {
    T sm, sp;
    apply_row<T, T, float>(A, G, G.scoef_f, t, sm, sp);
    if (g == 0) {
      write_out(A, 0, c, sm);
      write_out(A, 1, c, sp);
    } else {
      write_out(A, g + 1, c, sp);
    }
  }
}

template <typename T>
__global__ void k_band(StepArgs<T> A) {
  band_one(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// redistribution
//
// A neighbourhood average is held as Qhat_r = Uhat[p_r] + D_r with its pivot
// p_r (set-up) and the deviation sum D_r = sum_{m != p} w_m (Uhat_m - Uhat_p)
// (Eq. qhat_omega, the weights sum to one).  Non-small CVs have p = itself,
// D = 0.  Every difference of averages is (Uhat[p_a] - Uhat[p_b]) + (D_a - D_b),
// so a tiny cell merged into one large neighbour (Qhat within ~alpha of that
// neighbour) keeps full relative accuracy in the limiter, and a uniform state
// is reproduced exactly.
// ---------------------------------------------------------------------------

// Uhat_a - Uhat_b of two CVs of the field (state indices), with the
// reference profile difference taken in double.
template <typename T>
__device__ inline T vdiff(const WsrdArgs<T> &R, long long a, long long b) {
  T d = R.u[a] - R.u[b];
  if (R.refd) {
    const unsigned ka = R.D.fnxy.div((unsigned)a), kb = R.D.fnxy.div((unsigned)b);
    if (ka != kb) d += (T)(R.refd[ka] - R.refd[kb]);
  }
  return d;
}

// The same difference from two values already read, located at a and b.
template <typename T>
__device__ inline T vdiff_vals(const WsrdArgs<T> &R, T va, long long a, T vb, long long b) {
  T d = va - vb;
  if (R.refd) {
    const unsigned ka = R.D.fnxy.div((unsigned)a), kb = R.D.fnxy.div((unsigned)b);
    if (ka != kb) d += (T)(R.refd[ka] - R.refd[kb]);
  }
  return d;
}

// A weight table in the state's precision (float copies on the mixed path).
template <typename T>
__device__ inline const T *tab(const double *d, const float *f);
template <>
__device__ inline const double *tab<double>(const double *d, const float *) {
  return d;
}
template <>
__device__ inline const float *tab<float>(const double *, const float *f) {
  return f;
}

// Kahan-compensated running sum in float; plain in double.
template <typename T>
struct CompSum {
  T s = T(0), c = T(0);
  __device__ inline void add(T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};
template <>
struct CompSum<double> {
  double s = 0.0, c = 0.0;
  __device__ inline void add(double x) { s += x; }
};

template <typename T>
__device__ inline void qhat_one(const WsrdArgs<T> &R, long long s) {
  const int n = R.W.s_nmem[s], p = R.W.s_piv[s];
  const long long lp = R.W.s_plin[s];
  CompSum<T> acc;
  for (int q = 0; q < n; ++q) {
    if (q == p) continue;
    acc.add(tab<T>(R.W.s_mw, R.W.s_mw_f)[8 * s + q] * vdiff(R, R.W.s_mlin[8 * s + q], lp));
  }
  R.dev[s] = acc.s;
  R.pval[s] = R.u[lp];   // snapshot: the final update overwrites the field in place
}

// One group of GS lanes per small CV (8 in the kernels: four CVs per warp):
// lanes walk the stencil, shuffles reduce the slope and the stencil's range
// of Qhat - Qhat_r; lane q evaluates the limiter at member q's centroid and a
// min-reduction combines them.  A group without a CV (valid false) takes part
// in the shuffles only.
template <typename T, int GS>
__device__ inline void sigma_one(const WsrdArgs<T> &R, long long s, int lane, bool valid) {
  static_assert(GS == 8 || GS == 16 || GS == 32, "lane groups of 8, 16 or 32 lanes");
  long long o0 = 0, o1 = 0, pr = 0;
  T dr = T(0);
  if (valid) {
    o0 = R.W.s_loff[s];
    o1 = R.W.s_loff[s + 1];
    pr = R.W.s_plin[s];
    dr = R.dev[s];
  }
  T sx = T(0), sy = T(0), sz = T(0), bmax = T(0), bmin = T(0);
#pragma unroll 2
  for (long long o = o0 + lane; o < o1; o += GS) {
    const int sid = R.W.l_sid[o];
    const long long pm = R.W.l_plin[o];
    const T dm = sid >= 0 ? R.dev[sid] : T(0);
    const T b = vdiff(R, pm, pr) + (dm - dr);
    const T *lc = tab<T>(R.W.l_c, R.W.l_c_f) + 3 * o;
    sx += lc[0] * b;
    sy += lc[1] * b;
    sz += lc[2] * b;
    bmax = b > bmax ? b : bmax;
    bmin = b < bmin ? b : bmin;
  }
  for (int off = GS / 2; off > 0; off >>= 1) {   // stays within the group
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
    sz += __shfl_xor_sync(0xffffffffu, sz, off);
    const T a = __shfl_xor_sync(0xffffffffu, bmax, off);
    const T c = __shfl_xor_sync(0xffffffffu, bmin, off);
    bmax = a > bmax ? a : bmax;
    bmin = c < bmin ? c : bmin;
  }
  T phi = T(1);
  if (o1 > o0 && lane < R.W.s_nmem[s]) {   // o1 > o0 only for a valid group
    const T *e = tab<T>(R.W.s_me, R.W.s_me_f) + 24 * s + 3 * lane;
    const T del = sx * e[0] + sy * e[1] + sz * e[2];
    T ph = T(1);
    if (del > T(0)) ph = bmax / del;
    else if (del < T(0)) ph = bmin / del;
    phi = ph < T(1) ? ph : T(1);   // a value that is not below 1 (or NaN) leaves phi at 1
  }
  for (int off = 4; off > 0; off >>= 1) {   // members are lanes 0 .. 7
    const T o = __shfl_xor_sync(0xffffffffu, phi, off);
    phi = o < phi ? o : phi;
  }
  if (lane != 0 || !valid) return;
  R.sig[3 * s] = sx * phi;
  R.sig[3 * s + 1] = sy * phi;
  R.sig[3 * s + 2] = sz * phi;
}

// U_i = P_i + sum_r (kappa_r / N_i) (q_r(x_i) - P_i), P_i = q_i(x_i) for a
// small CV and Uhat_i otherwise: Eq. final_update_omega with omega_i written
// as 1 - sum_r kappa_r / N_i.  Formed as an offset added to Uhat_i.
template <typename T>
__device__ inline void final_one(const WsrdArgs<T> &R, long long a) {
  const long long c = R.W.a_lin[a];
  const int sid = R.W.a_sid[a];
  // every value this thread reads besides its own CV comes from the
  // snapshots of k_qhat: other threads overwrite their CVs meanwhile
  const T ui = R.u[c];
  T si = T(0), di = T(0), pvi = ui;
  long long pi = c;
  if (sid >= 0) {
    const T *e = tab<T>(R.W.a_eself, R.W.a_eself_f) + 3 * a;
    si = R.sig[3 * sid] * e[0] + R.sig[3 * sid + 1] * e[1] + R.sig[3 * sid + 2] * e[2];
    pi = R.W.s_plin[sid];
    pvi = R.pval[sid];
    di = R.dev[sid];
  }
  CompSum<T> acc;
  for (long long o = R.W.a_woff[a]; o < R.W.a_woff[a + 1]; ++o) {
    const int r = R.W.w_sid[o];
    const T *e = tab<T>(R.W.w_e, R.W.w_e_f) + 3 * o;
    const long long pr = R.W.s_plin[r];
    const T sr = R.sig[3 * r] * e[0] + R.sig[3 * r + 1] * e[1] + R.sig[3 * r + 2] * e[2];
    const T diff = vdiff_vals(R, R.pval[r], pr, pvi, pi) + (R.dev[r] - di) + (sr - si);
    acc.add(tab<T>(R.W.w_k, R.W.w_k_f)[o] * diff);
  }
  // a small CV's result is anchored at its pivot value: its own provisional
  // value can be huge (tiny cell after the flux update) and must not be added
  // and subtracted again
  T v;
  if (sid >= 0) {
    T anchor = pvi;
    if (R.refd) {
      const unsigned kp = R.D.fnxy.div((unsigned)pi), kc = R.D.fnxy.div((unsigned)c);
      if (kp != kc) anchor += (T)(R.refd[kp] - R.refd[kc]);
    }
    v = anchor + ((di + si) + acc.s);
  } else {
    v = ui + acc.s;
  }
  R.u[c] = v;
  if (!finite_val(v)) atomicOr(R.status, EB_DEV_NUMERIC);
}

// one field
template <typename T>
__global__ void k_qhat(WsrdArgs<T> R) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < R.W.nsmall) qhat_one(R, s);
}
template <typename T>
__global__ void k_sigma(WsrdArgs<T> R) {
  const long long s = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 3;
  sigma_one<T, 8>(R, s, threadIdx.x & 7, s < R.W.nsmall);
}
template <typename T>
__global__ void k_final(WsrdArgs<T> R) {
  const long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (a < R.W.naff) final_one(R, a);
}

// all five fields in one launch: work item t belongs to the field f with
// off[f] <= t < off[f + 1]
__device__ inline int field_of(const long long off[6], long long t) {
  int f = 0;
  while (f < 4 && t >= off[f + 1]) ++f;
  return f;
}
template <typename T>
__global__ void k_qhat5(const __grid_constant__ WsrdSet<T> S) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= S.off_small[5]) return;
  const int f = field_of(S.off_small, t);
  qhat_one(S.f[f], t - S.off_small[f]);
}
template <typename T>
__global__ void k_sigma5(const __grid_constant__ WsrdSet<T> S) {
  const long long t = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 3;
  const bool valid = t < S.off_small[5];
  const int f = valid ? field_of(S.off_small, t) : 0;
  sigma_one<T, 8>(S.f[f], valid ? t - S.off_small[f] : 0, threadIdx.x & 7, valid);
}
template <typename T>
__global__ void k_final5(const __grid_constant__ WsrdSet<T> S) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= S.off_aff[5]) return;
  const int f = field_of(S.off_aff, t);
  final_one(S.f[f], t - S.off_aff[f]);
}


// ---------------------------------------------------------------------------
// persistent ensemble step: every phase of one step of every member in one
// cooperative launch, separated by grid-wide barriers whose waits are
// bounded (an expired wait latches EB_DEV_TIMEOUT in every member's status
// word and the CTA returns)
// ---------------------------------------------------------------------------

// member m of the item with global index t: pre[m] <= t < pre[m + 1]
__device__ inline int member_of(const long long *pre, int nm, long long t) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ inline void ens_timeout(const EnsembleArgs<T> &E) {
  for (int q = 0; q < E.nm; ++q) atomicOr(E.m[q].A.status, EB_DEV_TIMEOUT);
}

// Grid-wide barrier: every CTA arrives once; the last one to arrive resets
// the count and advances the generation.  A waiting CTA polls the
// generation at most spin_limit times (about a microsecond apart) and then
// gives up.  Returns whether every CTA arrived.
template <typename T>
__device__ bool ens_barrier(const EnsembleArgs<T> &E) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    volatile unsigned *gen = E.ctl + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(E.ctl, 1u) + 1u;
    int good = 1;
    if (arrived == gridDim.x) {
      atomicExch(E.ctl, 0u);
      __threadfence();
      atomicAdd(E.ctl + 1, 1u);
    } else {
      unsigned polls = 0;
      while (*gen == g) {
        if (++polls > E.spin_limit) {
          good = 0;
          ens_timeout(E);
          break;
        }
        __nanosleep(1000);
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// Items of a phase handed out in chunks of one warp: lane 0 takes the next
// chunk from the counter, the warp walks it.
template <typename F>
__device__ inline void warp_chunks(unsigned *counter, long long total, F &&fn) {
  const unsigned lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31u;
  for (;;) {
    unsigned c = 0;
    if (lane == 0) c = atomicAdd(counter, 1u);
    c = __shfl_sync(0xffffffffu, c, 0);
    const long long t = (long long)c * 32 + lane;
    if ((long long)c * 32 >= total) break;
    if (t < total) fn(t);
  }
}

// The bulk march keeps its carried state in registers here (no tensor
// memory): a cooperative launch may only hold as many CTAs as the driver
// counts co-resident, and it counts a CTA that allocates tensor memory as
// filling its SM.
template <typename T, int V>
__global__ void __launch_bounds__(bulk::BulkTile<T>::NT, (sizeof(T) == 4 ? 2 : 1))
    k_ensemble_step(const __grid_constant__ EnsembleArgs<T> E) {
  using P = typename bulk::PairOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  __shared__ unsigned tm_slot;
  __shared__ int s_unit;
  if (*E.fault == (int)blockIdx.x + 1) return;   // failure test: this CTA never arrives
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const long long gtid = (long long)blockIdx.x * bulk::BulkTile<T>::NT + tid;
  const long long nthreads = (long long)gridDim.x * bulk::BulkTile<T>::NT;
  const int nm = E.nm;

  // phase 1: the bulk kernel's units of every member, longest first, handed
  // out one per CTA; then (float path) the face fluxes in warp chunks
  const unsigned tbase = bulk::bulk_tmem_begin<T, false>(&tm_slot);
  for (;;) {
    if (tid == 0) s_unit = (int)atomicAdd(E.ctl + 2, 1u);
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u >= E.nunits) break;
    const int2 w = E.units[u];
    const StepArgs<T> &A = E.m[w.x].A;
    P bad = bulk::splat(T(0));
    for (int sgi = A.boff[w.y]; sgi < A.boff[w.y + 1]; ++sgi)
      bulk::bulk_march<T, V, false>(A, A.bseg[sgi], smem_bytes, tbase, bad);
    if (!(isfinite(bad.x) && isfinite(bad.y))) atomicOr(A.status, EB_DEV_NUMERIC);
  }
  bulk::bulk_tmem_end<T, false>(&tm_slot);
  for (long long t = gtid; t < E.pre_stage[nm]; t += nthreads) {
    const int q = member_of(E.pre_stage, nm, t);
    stage_one(E.m[q].A, t - E.pre_stage[q]);
  }
  if (E.faces_first)
    warp_chunks(E.ctl + 3, E.pre_face[nm], [&](long long t) {
      const int q = member_of(E.pre_face, nm, t);
      face_one(E.m[q].A, t - E.pre_face[q]);
    });
  if (!ens_barrier(E)) return;
  // phase 2 (double path): face fluxes from the staged values
  if (!E.faces_first) {
    for (long long t = gtid; t < E.pre_face[nm]; t += nthreads) {
      const int q = member_of(E.pre_face, nm, t);
      face_one(E.m[q].A, t - E.pre_face[q]);
    }
    if (!ens_barrier(E)) return;
  }
  // phase 3: near-EB divergence and update
  for (long long t = gtid; t < E.pre_band[nm]; t += nthreads) {
    const int q = member_of(E.pre_band, nm, t);
    band_one(E.m[q].A, t - E.pre_band[q]);
  }
  if (!ens_barrier(E)) return;
  // phases 4-6: redistribution of all five fields of every member
  for (long long t = gtid; t < E.pre_small[nm]; t += nthreads) {
    const int q = member_of(E.pre_small, nm, t);
    const WsrdSet<T> &S = E.m[q].S;
    const long long ts = t - E.pre_small[q];
    const int f = field_of(S.off_small, ts);
    qhat_one(S.f[f], ts - S.off_small[f]);
  }
  if (!ens_barrier(E)) return;
  {
    // 8 lanes per small CV; every lane of a warp takes part in each round
    const long long groups = E.pre_small[nm];
    const long long wbase = (gtid >> 5) * 4, wstep = (nthreads >> 5) * 4;
    for (long long b = wbase; b < groups; b += wstep) {
      const long long g = b + ((tid & 31) >> 3);
      const bool valid = g < groups;
      const int q = valid ? member_of(E.pre_small, nm, g) : 0;
      const WsrdSet<T> &S = E.m[q].S;
      const long long ts = valid ? g - E.pre_small[q] : 0;
      const int f = valid ? field_of(S.off_small, ts) : 0;
      sigma_one<T, 8>(S.f[f], valid ? ts - S.off_small[f] : 0, tid & 7, valid);
    }
  }
  if (!ens_barrier(E)) return;
  for (long long t = gtid; t < E.pre_aff[nm]; t += nthreads) {
    const int q = member_of(E.pre_aff, nm, t);
    const WsrdSet<T> &S = E.m[q].S;
    const long long ta = t - E.pre_aff[q];
    const int f = field_of(S.off_aff, ta);
    final_one(S.f[f], ta - S.off_aff[f]);
  }
}

template <typename T, int V>
int ensemble_ctas_v(int info[3]) {
  auto *k = k_ensemble_step<T, V>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bulk::BulkTile<T>::BYTES) !=
      cudaSuccess)
    return 0;
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, bulk::BulkTile<T>::NT, bulk::BulkTile<T>::BYTES) !=
      cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k) == cudaSuccess) {
    info[0] = fa.numRegs;
    info[1] = (int)fa.sharedSizeBytes;
    info[2] = (int)fa.localSizeBytes;
  }
  return per * sms;
}

template <typename T, int V>
cudaError_t launch_ensemble_v(const EnsembleArgs<T> &E, int ctas, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas, 1, 1);
  cfg.blockDim = dim3(bulk::BulkTile<T>::NPX, bulk::BulkTile<T>::TY, 1);
  cfg.dynamicSmemBytes = bulk::BulkTile<T>::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_ensemble_step<T, V>, E);
}
}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
template <typename T>
void launch_flux_band(const StepArgs<T> &A, cudaStream_t s) {
  long long nf = 0, nb = 0, nr = 0;
  for (int g = 0; g < 4; ++g) {
    nb += A.G[g].nband_rec;
    nr += A.G[g].nband - A.G[g].nband_rec;
    for (int d = 0; d < 3; ++d) nf += A.G[g].nface[d];
  }
  long long ns = 0;
  for (int g = 0; g < 4; ++g) ns += A.G[g].nstage;
  if (ns) k_stage<T><<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(A);
  if (nf) k_face_flux<T><<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(A);
  if (nb + nr) k_band<T><<<(unsigned)((nb + nr + 255) / 256), 256, 0, s>>>(A);
}

template <typename T>
void launch_flux_update(const StepArgs<T> &A, cudaStream_t s) {
  launch_flux_fast(A, s);
  launch_flux_band(A, s);
}

template <typename T>
void launch_wsrd(const WsrdArgs<T> &R, cudaStream_t s) {
  if (R.W.nsmall) {
    k_qhat<T><<<(unsigned)((R.W.nsmall + 127) / 128), 128, 0, s>>>(R);
    k_sigma<T><<<(unsigned)((R.W.nsmall * 8 + 255) / 256), 256, 0, s>>>(R);
  }
  if (R.W.naff) k_final<T><<<(unsigned)((R.W.naff + 127) / 128), 128, 0, s>>>(R);
}

template <typename T>
void launch_wsrd5(const WsrdSet<T> &S, cudaStream_t s) {
  if (S.off_small[5]) {
    k_qhat5<T><<<(unsigned)((S.off_small[5] + 127) / 128), 128, 0, s>>>(S);
    k_sigma5<T><<<(unsigned)((S.off_small[5] * 8 + 255) / 256), 256, 0, s>>>(S);
  }
  if (S.off_aff[5]) k_final5<T><<<(unsigned)((S.off_aff[5] + 127) / 128), 128, 0, s>>>(S);
}

void launch_band_rows(const Dims &D, const GridDev G[4], int g, bool fill, long long *cnt, cudaStream_t s) {
  if (G[g].nband_rec == 0) return;
  RowBuild B;
  B.D = D;
  for (int q = 0; q < 4; ++q) B.G[q] = G[q];
  B.g = g;
  B.cnt = cnt;
  const unsigned blocks = (unsigned)((G[g].nband_rec + 127) / 128);
  if (fill) k_band_rows<true><<<blocks, 128, 0, s>>>(B);
  else k_band_rows<false><<<blocks, 128, 0, s>>>(B);
}

void launch_face_masks(const Dims &D, const GridDev G[4], cudaStream_t s) {
  StepArgs<float> A{};
  A.D = D;
  long long nf = 0;
  for (int q = 0; q < 4; ++q) {
    A.G[q] = G[q];
    for (int d = 0; d < 3; ++d) nf += G[q].nface[d];
  }
  if (nf) k_face_mask<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(A);
}

void launch_stage_marks(const Dims &D, const GridDev G[4], uint8_t *const marks[4], cudaStream_t s) {
  StageMarkArgs M;
  M.D = D;
  long long nf = 0;
  for (int q = 0; q < 4; ++q) {
    M.G[q] = G[q];
    M.marks[q] = marks[q];
    for (int d = 0; d < 3; ++d) nf += G[q].nface[d];
  }
  if (nf) k_stage_marks<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(M);
}

void launch_rows_to_u32(const long long *src, long long n, unsigned *dst, cudaStream_t s) {
  if (n > 0) k_rows_to_u32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, dst);
}

template void launch_flux_update<double>(const StepArgs<double> &, cudaStream_t);
template void launch_wsrd5<double>(const WsrdSet<double> &, cudaStream_t);
template void launch_wsrd5<float>(const WsrdSet<float> &, cudaStream_t);
template void launch_flux_band<double>(const StepArgs<double> &, cudaStream_t);
template void launch_flux_band<float>(const StepArgs<float> &, cudaStream_t);
template void launch_flux_update<float>(const StepArgs<float> &, cudaStream_t);
template void launch_wsrd<double>(const WsrdArgs<double> &, cudaStream_t);
template void launch_wsrd<float>(const WsrdArgs<float> &, cudaStream_t);

template <typename T>
int ensemble_kernel_ctas(bool vec, int info[3]) {
  constexpr int V = 16 / sizeof(T);
  return vec ? ensemble_ctas_v<T, V>(info) : ensemble_ctas_v<T, 1>(info);
}

template <typename T>
cudaError_t launch_ensemble_step(const EnsembleArgs<T> &E, bool vec, int ctas, cudaStream_t s) {
  constexpr int V = 16 / sizeof(T);
  return vec ? launch_ensemble_v<T, V>(E, ctas, s) : launch_ensemble_v<T, 1>(E, ctas, s);
}

template int ensemble_kernel_ctas<float>(bool, int[3]);
template int ensemble_kernel_ctas<double>(bool, int[3]);
template cudaError_t launch_ensemble_step<float>(const EnsembleArgs<float> &, bool, int, cudaStream_t);
template cudaError_t launch_ensemble_step<double>(const EnsembleArgs<double> &, bool, int, cudaStream_t);
