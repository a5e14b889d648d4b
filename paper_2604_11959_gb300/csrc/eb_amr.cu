// eb_amr.cu -- two-level static refinement (Sec. 4.3): the coarse level of a
// refinement ratio of 2 in every direction, built from the fine level by
// merging its cells, and the restriction of a fine state to the coarse level.
//
// A coarse CV of any grid is a block of 2 x 2 x 2 cells of the fine c grid:
// cells 2I, 2I + 1 along x for the c grid and 2I - 1, 2I for the u grid (the
// right half of coarse cell I - 1 and the left half of cell I), likewise
// along y for v and along z for w; fine cells below the bottom or above the
// top of the domain hold no fluid and take no part in the class.  Merging:
//   volume fraction   the mean of the 8 fine ones, the centroid their
//                     volume-weighted mean position;
//   face fraction     the mean of the 4 fine faces on the coarse low face,
//                     the centroid their area-weighted mean position;
//   EB area           the sum of the fine ones (a quarter of it in units of
//                     the coarse dx dy), the centroid their area-weighted mean;
//   EB normal         the direction of the area-weighted sum of the fine EB
//                     normals: the boundary of the fluid in the CV is closed,
//                     so that sum is sum_d (open area of the high d-face - open
//                     area of the low d-face) e_d;
//   class             covered or regular when all its fine cells inside the
//                     domain are, else cut.
// Positions are offsets from the CV (or face) centre in grid units of its
// level: a fine cell's centre lies at -1/2 or +1/2 fine units from the coarse
// CV centre along each axis, and a fine unit is half a coarse one.
#include "eb_handle.cuh"

using namespace ebh;

namespace {

// the fine c-grid cell (i, j, k): class (-1 outside the domain in z) and, with
// V, its moments in the record layout of the geometry kernels (alpha, cent[3],
// beta[3], fcent[6], nrm[3], aeb, ebc[3])
struct FineC {
  Dims D;
  GridDev G;
};

template <bool V>
__device__ inline int fine_cell(const FineC &F, int i, int j, int k, double v[20]) {
  if (V)
    for (int q = 0; q < 20; ++q) v[q] = 0.0;
  if (k < 0 || k >= F.D.nz) return -1;
  const int col = wrapi(i, F.D.nx) + F.D.nx * wrapi(j, F.D.ny);
  const int kc = F.G.kcov[col], kx = F.G.kxt[col];
  if (k < kc) return EBK_COVERED;
  if (k >= kx) {
    if (V) v[0] = v[4] = v[5] = v[6] = 1.0;
    return EBK_REGULAR;
  }
  const long long r = F.G.roff[col] + (k - kc), n = F.G.nrec;
  if (V) {
    v[0] = F.G.alpha[r];
    for (int d = 0; d < 3; ++d) {
      v[1 + d] = F.G.cent[d * n + r];
      v[4 + d] = F.G.beta[d * n + r];
      v[13 + d] = F.G.nrm[d * n + r];
      v[17 + d] = F.G.ebc[d * n + r];
    }
    for (int q = 0; q < 6; ++q) v[7 + q] = F.G.fcent[q * n + r];
    v[16] = F.G.aeb[r];
  }
  return F.G.flag[r];
}

// the volume fraction (q = 0) or the low q-1 face fraction (q = 1..3) of
// fine cell (i, j, k) alone: 0 outside the domain or covered, 1 regular
__device__ inline double fine_frac(const FineC &F, int i, int j, int k, int q) {
  if (k < 0 || k >= F.D.nz) return 0.0;
  const int col = wrapi(i, F.D.nx) + F.D.nx * wrapi(j, F.D.ny);
  const int kc = F.G.kcov[col], kx = F.G.kxt[col];
  if (k < kc) return 0.0;
  if (k >= kx) return 1.0;
  const long long r = F.G.roff[col] + (k - kc);
  return q == 0 ? F.G.alpha[r] : F.G.beta[(q - 1) * F.G.nrec + r];
}

// open fraction of the low d-face of fine cell (i, j, k); the lid above the
// top is open, the floor below the bottom closed
__device__ inline double fine_low_face(const FineC &F, int i, int j, int k, int d) {
  if (k >= F.D.nz) return d == 2 ? 1.0 : 0.0;
  double v[20];
  if (fine_cell<true>(F, i, j, k, v) < 0) return 0.0;
  return v[4 + d];
}

// first fine cell of the block of coarse CV (I, J, K) of grid g
__device__ inline void block_origin(int g, int I, int J, int K, int f0[3]) {
  f0[0] = 2 * I - (g == 1);
  f0[1] = 2 * J - (g == 2);
  f0[2] = 2 * K - (g == 3);
}

__device__ inline int coarse_class(const FineC &F, int g, int I, int J, int K) {
  int f0[3];
  block_origin(g, I, J, K, f0);
  int nin = 0, ncov = 0, nreg = 0;
  double v[20];
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int cls = fine_cell<false>(F, f0[0] + a, f0[1] + b, f0[2] + c, v);
        if (cls < 0) continue;
        ++nin;
        ncov += cls == EBK_COVERED;
        nreg += cls == EBK_REGULAR;
      }
  return ncov == nin ? EBK_COVERED : (nreg == nin ? EBK_REGULAR : EBK_CUT);
}

__global__ void k_coarse_bounds(FineC F, Dims Dc, int g, int *kcov, int *kreg) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= Dc.nx * Dc.ny) return;
  const int I = col % Dc.nx, J = col / Dc.nx;
  const int nzg = nzg_of(Dc, g);
  int kc = 0;
  while (kc < nzg && coarse_class(F, g, I, J, kc) == EBK_COVERED) ++kc;
  int kr = nzg;
  while (kr > kc && coarse_class(F, g, I, J, kr - 1) == EBK_REGULAR) --kr;
  kcov[col] = kc;
  kreg[col] = kr;
}

// the merged moments of coarse CV (I, J, K) of grid g, record layout
__device__ inline void merge_cv(const FineC &F, const Dims &Dc, int g, int I, int J, int K, double out[20]) {
  int f0[3];
  block_origin(g, I, J, K, f0);
  double vol = 0, m[3] = {0, 0, 0}, eba = 0, eb[3] = {0, 0, 0};
  double fa[3] = {0, 0, 0}, f1[3] = {0, 0, 0}, f2[3] = {0, 0, 0}, fh[3] = {0, 0, 0};
  double v[20];
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        if (fine_cell<true>(F, f0[0] + a, f0[1] + b, f0[2] + c, v) < 0) continue;
        const int q[3] = {a, b, c};
        const double o[3] = {a - 0.5, b - 0.5, c - 0.5};
        vol += v[0];
        eba += v[16];
        for (int d = 0; d < 3; ++d) {
          m[d] += v[0] * (o[d] + v[1 + d]);
          eb[d] += v[16] * (o[d] + v[17 + d]);
        }
        for (int d = 0; d < 3; ++d) {
          if (q[d] != 0) continue;   // the fine cells on the coarse low d-face
          const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
          const double be = v[4 + d];
          fa[d] += be;
          f1[d] += be * (o[t1] + v[7 + 2 * d]);
          f2[d] += be * (o[t2] + v[8 + 2 * d]);
        }
      }
  // open areas of the coarse high faces: the low faces of the fine cells two
  // beyond the block's first along d
  for (int d = 0; d < 3; ++d)
    for (int u = 0; u < 2; ++u)
      for (int w = 0; w < 2; ++w) {
        int p[3] = {f0[0], f0[1], f0[2]};
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        p[d] += 2;
        p[t1] += u;
        p[t2] += w;
        fh[d] += fine_low_face(F, p[0], p[1], p[2], d);
      }
  const double Af[3] = {F.D.dy * F.D.dz, F.D.dx * F.D.dz, F.D.dx * F.D.dy};
  out[0] = vol / 8.0;
  double nv[3], nn = 0.0;
  for (int d = 0; d < 3; ++d) {
    out[1 + d] = vol > 0 ? 0.5 * m[d] / vol : 0.0;
    out[4 + d] = fa[d] / 4.0;
    out[7 + 2 * d] = fa[d] > 0 ? 0.5 * f1[d] / fa[d] : 0.0;
    out[8 + 2 * d] = fa[d] > 0 ? 0.5 * f2[d] / fa[d] : 0.0;
    out[17 + d] = eba > 0 ? 0.5 * eb[d] / eba : 0.0;
    nv[d] = (fh[d] - fa[d]) * Af[d];
    nn += nv[d] * nv[d];
  }
  nn = sqrt(nn);
  for (int d = 0; d < 3; ++d) out[13 + d] = (eba > 0 && nn > 0) ? nv[d] / nn : 0.0;
  out[16] = eba / 4.0;
}

__global__ void k_coarse_geometry(FineC F, Dims Dc, int g, GridDev G) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= Dc.nx * Dc.ny) return;
  const int I = col % Dc.nx, J = col / Dc.nx;
  const long long n = G.nrec;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    double v[20];
    merge_cv(F, Dc, g, I, J, k, v);
    G.flag[r] = (uint8_t)coarse_class(F, g, I, J, k);
    G.alpha[r] = v[0];
    for (int d = 0; d < 3; ++d) {
      G.cent[d * n + r] = v[1 + d];
      G.beta[d * n + r] = v[4 + d];
      G.nrm[d * n + r] = v[13 + d];
      G.ebc[d * n + r] = v[17 + d];
    }
    for (int q = 0; q < 6; ++q) G.fcent[q * n + r] = v[7 + q];
    G.aeb[r] = v[16];
    G.alpha_f[r] = (float)v[0];
    for (int d = 0; d < 3; ++d) G.beta_f[d * n + r] = (float)v[4 + d];
    for (int q = 0; q < 6; ++q) G.fcent_f[q * n + r] = (float)v[7 + q];
  }
}

__global__ void k_subsample_heights(const double *hf, Dims Df, double *hc, Dims Dc) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long n = (long long)(Dc.nx + 1) * (Dc.ny + 1);
  if (t >= n) return;
  const int I = (int)(t % (Dc.nx + 1)), J = (int)(t / (Dc.nx + 1));
  hc[t] = hf[(long long)(2 * J) * (Df.nx + 1) + 2 * I];
}

// Restriction: coarse value = (sum of w times fine value) / (sum of w), with
// w the fine volume fractions (c grid) or the fine low-face fractions of the
// 4 fine faces on the coarse face (face grids), in double; the states hold
// perturbations about per-level profiles of their own level (pf fine, pc
// coarse; zeros where none), so the profiles' weighted mean minus the coarse
// profile is added.  The fine handle may be an x-window of the fine level:
// its local column q is global fine column fx0 + q (mod nxg); coarse columns
// I0 .. I0 + ncols - 1 (mod the coarse nx) are restricted.  CVs without fine
// fluid or open area keep their value.
template <typename T>
struct RestrictArgs {
  FineC F;
  Dims Dc;
  const T *uf[5];
  T *uc[5];
  const double *pf[5], *pc[5];   // per-level profiles (nullptr: none)
  int fx0, nxg, I0, ncols;
};

template <typename T>
__global__ void k_restrict(const __grid_constant__ RestrictArgs<T> R, int f) {
  const Dims &Dc = R.Dc;
  const int g = f <= 1 ? 0 : f - 1;
  const long long plane = (long long)R.ncols * Dc.ny;
  const long long n = plane * nzg_of(Dc, g);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int K = (int)(t / plane);
  const long long c2 = t - (long long)K * plane;
  const int J = (int)(c2 / R.ncols), It = (int)(c2 - (long long)J * R.ncols);
  const int I = wrapi(R.I0 + It, Dc.nx);
  const long long tc = I + (long long)Dc.nx * J + Dc.nxy * K;
  const Dims &Df = R.F.D;
  auto local = [&](int gx) { return wrapi(gx - R.fx0, R.nxg); };   // fine global column -> the handle's column
  double w = 0.0, s = 0.0, sp = 0.0;
  if (g == 0) {
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const int i = local(2 * I + a), j = 2 * J + b, k = 2 * K + c;
          const double al = fine_frac(R.F, i, j, k, 0);
          const long long q = i + (long long)Df.nx * j + Df.nxy * k;
          w += al;
          s += al * (double)R.uf[f][q];
          if (R.pf[f]) sp += al * R.pf[f][k];
        }
  } else {
    const int d = g - 1;
    for (int y = 0; y < 2; ++y)
      for (int x = 0; x < 2; ++x) {
        int p[3] = {2 * I, 2 * J, 2 * K};
        const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        p[t1] += x;
        p[t2] += y;
        if (p[2] >= Df.nz) continue;   // the lid above the top: a wall of w
        p[0] = local(p[0]);
        const double be = fine_frac(R.F, p[0], p[1], p[2], 1 + d);
        const long long q = p[0] + (long long)Df.nx * p[1] + Df.nxy * p[2];
        w += be;
        s += be * (double)R.uf[f][q];
        if (R.pf[f]) sp += be * R.pf[f][p[2]];
      }
  }
  if (w > 0.0) {
    double val = s / w;
    if (R.pf[f]) val += sp / w;
    if (R.pc[f]) val -= R.pc[f][K];
    R.uc[f][tc] = (T)val;
  }
}

// Prolongation onto the fine handle's columns outside [lo, hi) (local
// indices): every fine CV takes the value of the coarse CV it lies in; a fine
// face of a face grid on a coarse face takes that face's value, one halfway
// between two coarse faces (odd fine index along the face's axis) their mean;
// full values (state plus profile) are interpolated, in double.
template <typename T>
struct ProlongArgs {
  Dims Df, Dc;
  const T *uc[5];
  T *uf[5];
  const double *pf[5], *pc[5];
  int fx0, nxg, lo, hi;
};

template <typename T>
__global__ void k_prolong(const __grid_constant__ ProlongArgs<T> P, int f) {
  const Dims &Df = P.Df, &Dc = P.Dc;
  const int g = f <= 1 ? 0 : f - 1;
  const long long n = Df.nxy * (long long)nzg_of(Df, g);
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int i, j, k;
  split_index(Df, (unsigned)t, i, j, k);
  if (i >= P.lo && i < P.hi) return;   // an owned column
  const int gi = wrapi(P.fx0 + i, P.nxg);
  int c[3] = {gi / 2, j / 2, k / 2};
  const int fc[3] = {gi, j, k};
  auto full = [&](int I, int J, int K) -> double {
    const double u = (double)P.uc[f][I + (long long)Dc.nx * J + Dc.nxy * K];
    return P.pc[f] ? u + P.pc[f][K] : u;
  };
  double val;
  const int d = g - 1;
  if (g == 0 || fc[d] % 2 == 0) {
    val = full(c[0], c[1], c[2]);
  } else {
    int e[3] = {c[0], c[1], c[2]};
    e[d] += 1;
    if (d == 0) e[0] = wrapi(e[0], Dc.nx);
    if (d == 1) e[1] = wrapi(e[1], Dc.ny);
    val = 0.5 * (full(c[0], c[1], c[2]) + full(e[0], e[1], e[2]));
  }
  if (P.pf[f]) val -= P.pf[f][k];
  P.uf[f][t] = (T)val;
}

}  // namespace

void launch_coarse_bounds(const Dims &Df, const GridDev &Gf, const Dims &Dc, int g, int *kcov, int *kreg,
                          cudaStream_t s) {
  FineC F{Df, Gf};
  k_coarse_bounds<<<(unsigned)((Dc.nxy + 127) / 128), 128, 0, s>>>(F, Dc, g, kcov, kreg);
}

void launch_coarse_geometry(const Dims &Df, const GridDev &Gf, const Dims &Dc, int g, const GridDev &Gc,
                            cudaStream_t s) {
  FineC F{Df, Gf};
  k_coarse_geometry<<<(unsigned)((Dc.nxy + 63) / 64), 64, 0, s>>>(F, Dc, g, Gc);
}

void launch_subsample_heights(const double *hf, const Dims &Df, double *hc, const Dims &Dc, cudaStream_t s) {
  const long long n = (long long)(Dc.nx + 1) * (Dc.ny + 1);
  k_subsample_heights<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(hf, Df, hc, Dc);
}

template <typename T>
static void restrict_t(eb_geom fine, eb_geom coarse, const eb_state *Uf, eb_state *Uc, int fx0, int lo, int hi,
                       cudaStream_t s) {
  RestrictArgs<T> R;
  R.F = FineC{fine->D, fine->G[0]};
  R.Dc = coarse->D;
  R.nxg = 2 * coarse->D.nx;
  R.fx0 = wrapi(fx0, R.nxg);
  R.I0 = wrapi(R.fx0 + lo, R.nxg) / 2;
  R.ncols = (hi - lo) / 2;
  void **uf = state_ptrs(Uf), **uc = state_ptrs(Uc);
  for (int f = 0; f < 5; ++f) {
    R.uf[f] = (const T *)uf[f];
    R.uc[f] = (T *)uc[f];
    R.pf[f] = f <= 3 ? fine->ref_d[f] : nullptr;
    R.pc[f] = f <= 3 ? coarse->ref_d[f] : nullptr;
  }
  for (int f = 0; f < 5; ++f) {
    const int g = f <= 1 ? 0 : f - 1;
    const long long n = (long long)R.ncols * coarse->D.ny * nzg_of(coarse->D, g);
    if (n > 0) k_restrict<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, f);
  }
}

template <typename T>
static void prolong_t(eb_geom coarse, const eb_state *Uc, eb_geom fine, eb_state *Uf, int fx0, int lo, int hi,
                      cudaStream_t s) {
  ProlongArgs<T> P;
  P.Df = fine->D;
  P.Dc = coarse->D;
  P.nxg = 2 * coarse->D.nx;
  P.fx0 = wrapi(fx0, P.nxg);
  P.lo = lo;
  P.hi = hi;
  void **uf = state_ptrs(Uf), **uc = state_ptrs(Uc);
  for (int f = 0; f < 5; ++f) {
    P.uc[f] = (const T *)uc[f];
    P.uf[f] = (T *)uf[f];
    P.pf[f] = f <= 3 ? fine->ref_d[f] : nullptr;
    P.pc[f] = f <= 3 ? coarse->ref_d[f] : nullptr;
  }
  for (int f = 0; f < 5; ++f) {
    const int g = f <= 1 ? 0 : f - 1;
    const long long n = fine->D.nxy * (long long)nzg_of(fine->D, g);
    k_prolong<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, f);
  }
}

// the fine handle is the coarse level's fine level over fine columns fx0 ..
// fx0 + nx - 1 (mod 2 nx_c), full y and z
static eb_status check_levels(eb_geom fine, eb_geom coarse, const eb_state *Uf, const eb_state *Uc, int lo, int hi) {
  if (!fine || !coarse) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (fine->D.ny != 2 * coarse->D.ny || fine->D.nz != 2 * coarse->D.nz || fine->D.nx > 2 * coarse->D.nx)
    return fail(EB_ERR_INVALID_ARG, "the fine handle must be an x-window of the coarse handle's fine level");
  if (fabs(2.0 * fine->D.dx - coarse->D.dx) > 1e-12 * coarse->D.dx ||
      fabs(2.0 * fine->D.dy - coarse->D.dy) > 1e-12 * coarse->D.dy ||
      fabs(2.0 * fine->D.dz - coarse->D.dz) > 1e-12 * coarse->D.dz)
    return fail(EB_ERR_INVALID_ARG, "the fine cells must be half the coarse ones");
  if (fine->prec != coarse->prec) return fail(EB_ERR_INVALID_ARG, "the handles differ in precision");
  if (lo < 0 || hi > fine->D.nx || lo > hi) return fail(EB_ERR_INVALID_ARG, "column range outside the fine handle");
  const size_t es = fine->prec == EB_F64 ? 8 : 4;
  if (!state_ok(Uf, es) || !state_ok(Uc, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  return EB_OK;
}

eb_status eb_restrict(eb_geom fine, eb_geom coarse, const eb_state *Uf, eb_state *Uc, int fine_x0, int lo, int hi,
                      void *stream) {
  eb_status st = check_levels(fine, coarse, Uf, Uc, lo, hi);
  if (st != EB_OK) return st;
  if ((lo % 2) || (hi % 2) || ((fine_x0 % 2 + 2) % 2))
    return fail(EB_ERR_INVALID_ARG, "restriction columns must start on even fine columns");
  cudaStream_t s = as_stream(stream);
  if (fine->prec == EB_F64) restrict_t<double>(fine, coarse, Uf, Uc, fine_x0, lo, hi, s);
  else restrict_t<float>(fine, coarse, Uf, Uc, fine_x0, lo, hi, s);
  CUDA_TRY(cudaGetLastError(), "restriction");
  return EB_OK;
}

eb_status eb_prolong(eb_geom coarse, const eb_state *Uc, eb_geom fine, eb_state *Uf, int fine_x0, int lo, int hi,
                     void *stream) {
  eb_status st = check_levels(fine, coarse, Uf, Uc, lo, hi);
  if (st != EB_OK) return st;
  cudaStream_t s = as_stream(stream);
  if (fine->prec == EB_F64) prolong_t<double>(coarse, Uc, fine, Uf, fine_x0, lo, hi, s);
  else prolong_t<float>(coarse, Uc, fine, Uf, fine_x0, lo, hi, s);
  CUDA_TRY(cudaGetLastError(), "prolongation");
  return EB_OK;
}
