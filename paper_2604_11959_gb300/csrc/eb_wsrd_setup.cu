// eb_wsrd_setup.cu -- one-time tables of weighted state redistribution
// (Sec. 5.1 of the paper): small CVs (V < V_target), their merging
// neighbourhoods M (first along the EB normal, then the next-largest normal
// component, then 2x2x2), kappa (Eq. kappa, capped at 1), N and omega
// (Eq. omega), the weighted neighbourhood volume and centroid (Eqs. nbhd_vol,
// centroid).  The paper notes all of this can be fixed when the EB is defined;
// so is the least-squares fit of the neighbourhood-average gradient, whose
// stencil and point positions depend on geometry only: each small CV stores
// one coefficient row per stencil point, and the per-step gradient is a dot
// product with Qhat differences.
//
// Everything is computed by gathering: a CV finds the neighbourhoods that
// hold it by reading the codes of its 26 neighbours, so no atomics are used
// and the tables are deterministic.  Lists are compacted with prefix sums in
// column order.
#include "eb_kernels.cuh"

#include <math.h>

namespace {

__constant__ int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ inline bool prognostic(const Dims &D, int g, int k) { return !(g == 3 && (k == 0 || k == D.nz)); }

struct View {
  bool active;
  double alpha;
  long long rec;
};

// A CV takes part in redistribution when it exists, is prognostic and holds
// fluid.
__device__ View view(const GridDev &G, const Dims &D, int g, int i, int j, int k) {
  if (k < 0 || k >= G.nzg || !prognostic(D, g, k)) return {false, 0.0, -1};
  const CvInfo c = cv_info(G, D, i, j, k);
  if (c.flag == EBK_COVERED) return {false, 0.0, -1};
  const double a = c.rec >= 0 ? G.alpha[c.rec] : 1.0;
  return {a > 0.0, a, c.rec};
}

__device__ inline double rec_or(const double *arr, long long r, double dflt) { return r >= 0 ? arr[r] : dflt; }

// Axis order by decreasing |n_d|; components within 1e-12 count as equal and
// the lower axis index wins.
__device__ void order_axes(const double n[3], int ax[3]) {
  const double tol = 1e-12;
  const double a[3] = {fabs(n[0]), fabs(n[1]), fabs(n[2])};
  int first = 2;
  for (int d = 2; d >= 0; --d) {
    bool beaten = false;
    for (int e = 0; e < 3; ++e)
      if (e != d && a[e] > a[d] + tol) beaten = true;
    if (!beaten) first = d;
  }
  const int r0 = first == 0 ? 1 : 0;
  const int r1 = first == 2 ? 1 : 2;
  ax[0] = first;
  if (a[r1] > a[r0] + tol) {
    ax[1] = r1;
    ax[2] = r0;
  } else {
    ax[1] = r0;
    ax[2] = r1;
  }
}

__device__ int perm_of(const int ax[3]) {
  for (int p = 0; p < 6; ++p)
    if (kPerm[p][0] == ax[0] && kPerm[p][1] == ax[1] && kPerm[p][2] == ax[2]) return p;
  return 0;
}

// Offsets of the candidates of growth level L, in growth order (self first).
__device__ int level_offsets(const int ax[3], const int s[3], int L, int off[8][3]) {
  for (int c = 0; c < 8; ++c) {
    off[c][0] = off[c][1] = off[c][2] = 0;
    if (c & 1) off[c][ax[0]] += s[ax[0]];
    if (c & 2) off[c][ax[1]] += s[ax[1]];
    if (c & 4) off[c][ax[2]] += s[ax[2]];
  }
  return L == 1 ? 2 : (L == 2 ? 4 : 8);
}

__device__ int unpack(int code, int off[8][3]) {
  const int c = code - 1;
  const int L = c % 3 + 1;
  const int sb = (c / 3) % 8, p = (c / 3) / 8;
  int ax[3], s[3];
  for (int d = 0; d < 3; ++d) {
    ax[d] = kPerm[p][d];
    s[d] = ((sb >> d) & 1) ? -1 : 1;
  }
  return level_offsets(ax, s, L, off);
}

// Active members of the neighbourhood of CV (i,j,k) with code `code`.
struct Members {
  int n;
  int off[8][3];
  View v[8];
};

__device__ void members_of(const GridDev &G, const Dims &D, int g, int i, int j, int k, int code, Members &M) {
  int off[8][3];
  const int cnt = unpack(code, off);
  M.n = 0;
  for (int c = 0; c < cnt; ++c) {
    const View v = view(G, D, g, i + off[c][0], j + off[c][1], k + off[c][2]);
    if (!v.active) continue;
    for (int d = 0; d < 3; ++d) M.off[M.n][d] = off[c][d];
    M.v[M.n] = v;
    ++M.n;
  }
}

// --- pass 1: small CVs, their codes and kappa --------------------------------
__global__ void k_codes(Dims D, int g, GridDev G, double vt) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  const long long n = G.nrec;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    G.code[r] = 0;
    G.kappa[r] = 0.0;
    const View me = view(G, D, g, i, j, k);
    if (!me.active || !(me.alpha < vt)) continue;
    const double nv[3] = {G.nrm[r], G.nrm[n + r], G.nrm[2 * n + r]};
    int ax[3], s[3], sb = 0;
    order_axes(nv, ax);
    for (int d = 0; d < 3; ++d) {
      s[d] = nv[d] < -1e-12 ? -1 : 1;   // components within 1e-12 of zero count as zero: +1
      if (s[d] < 0) sb |= 1 << d;
    }
    int L = 1;
    double sum = 0.0;
    for (L = 1; L <= 3; ++L) {
      int off[8][3];
      const int cnt = level_offsets(ax, s, L, off);
      sum = 0.0;
      for (int c = 1; c < cnt; ++c) {
        const View v = view(G, D, g, i + off[c][0], j + off[c][1], k + off[c][2]);
        if (v.active) sum += v.alpha;
      }
      if (!(me.alpha + sum < vt)) break;
    }
    if (L > 3) L = 3;
    G.code[r] = (uint8_t)(1 + (perm_of(ax) * 8 + sb) * 3 + (L - 1));
    const double kap = sum > 0.0 ? (vt - me.alpha) / sum : 0.0;
    G.kappa[r] = kap > 1.0 ? 1.0 : kap;
  }
}

// --- pass 2: N and omega, gathered from the 26 neighbours ---------------------
__global__ void k_nnb_omega(Dims D, int g, GridDev G) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    G.nnb[r] = 0;
    G.omega[r] = 0.0;
    if (!view(G, D, g, i, j, k).active) continue;
    int N = 1;
    double ks = 0.0;
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (!di && !dj && !dk) continue;
          const View o = view(G, D, g, i + di, j + dj, k + dk);
          if (!o.active || o.rec < 0 || G.code[o.rec] == 0) continue;
          int off[8][3];
          const int cnt = unpack(G.code[o.rec], off);
          for (int c = 1; c < cnt; ++c)
            if (off[c][0] == -di && off[c][1] == -dj && off[c][2] == -dk) {
              ++N;
              ks += G.kappa[o.rec];
            }
        }
    G.nnb[r] = N;
    G.omega[r] = 1.0 - ks / N;
  }
}

// --- pass 3: weighted volume and centroid ------------------------------------
__global__ void k_vhat_xhat(Dims D, int g, GridDev G) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  const long long n = G.nrec;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    G.vhat[r] = 0.0;
    G.xhat[r] = G.xhat[n + r] = G.xhat[2 * n + r] = 0.0;
    const View me = view(G, D, g, i, j, k);
    if (!me.active) continue;
    const double wv = G.omega[r] * me.alpha;
    double vh = wv;
    double xs[3] = {wv * G.cent[r], wv * G.cent[n + r], wv * G.cent[2 * n + r]};
    if (G.code[r]) {
      Members M;
      members_of(G, D, g, i, j, k, G.code[r], M);
      for (int q = 1; q < M.n; ++q) {
        const long long m = M.v[q].rec;
        const double w = G.kappa[r] * M.v[q].alpha / (m >= 0 ? G.nnb[m] : 1);
        vh += w;
        for (int d = 0; d < 3; ++d) xs[d] += w * (M.off[q][d] + rec_or(G.cent + d * n, m, 0.0));
      }
    }
    G.vhat[r] = vh;
    for (int d = 0; d < 3; ++d) G.xhat[d * n + r] = xs[d] / vh;
  }
}

// --- compaction flags ---------------------------------------------------------
__global__ void k_flags(Dims D, int g, GridDev G, long long *small_cnt, long long *aff_cnt) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    const bool act = view(G, D, g, i, j, k).active;
    small_cnt[r] = (act && G.code[r]) ? 1 : 0;
    aff_cnt[r] = (act && (G.code[r] || G.nnb[r] >= 2)) ? 1 : 0;
  }
}

__global__ void k_assign_small(Dims D, int g, GridDev G, const long long *small_id, WsrdDev W) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    const bool act = view(G, D, g, i, j, k).active;
    if (act && G.code[r]) {
      const long long s = small_id[r];
      W.sid[r] = (int)s;
      W.s_lin[s] = lin(D, i, j, k);
      W.s_rec[s] = r;
    } else {
      W.sid[r] = -1;
    }
  }
}

// Position of CV m (offset o from r) relative to r's neighbourhood centroid:
// o + xhat_m - xhat_r, xhat_m = CV centroid for non-small CVs.
__device__ inline void rel_pos(const GridDev &G, long long m, const int o[3], const double xr[3], double p[3]) {
  for (int d = 0; d < 3; ++d) p[d] = o[d] + rec_or(G.xhat + d * G.nrec, m, 0.0) - xr[d];
}

// Least-squares stencil of small CV r: the non-covered CVs of the box
// |o_d| <= w_d around it, w_d widened from 1 to 2 where the centroid spread
// along d is below half a cell.  Returns the point count, or 0 when the fit
// is rejected (spread still too small, fewer than 4 points, or a near
// singular normal matrix); M receives the normal matrix.
__device__ int lsq_stencil(const GridDev &G, const Dims &D, int g, int i, int j, int k, const double xr[3], int w[3],
                           double Mn[3][3]) {
  w[0] = w[1] = w[2] = 1;
  int cnt = 0;
  for (int pass = 0; pass < 2; ++pass) {
    double spread[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) Mn[a][b] = 0.0;
    cnt = 0;
    for (int dk = -w[2]; dk <= w[2]; ++dk)
      for (int dj = -w[1]; dj <= w[1]; ++dj)
        for (int di = -w[0]; di <= w[0]; ++di) {
          if (!di && !dj && !dk) continue;
          const View v = view(G, D, g, i + di, j + dj, k + dk);
          if (!v.active) continue;
          const int o[3] = {di, dj, dk};
          double p[3];
          rel_pos(G, v.rec, o, xr, p);
          for (int a = 0; a < 3; ++a) {
            spread[a] = fmax(spread[a], fabs(p[a]));
            for (int b = 0; b < 3; ++b) Mn[a][b] += p[a] * p[b];
          }
          ++cnt;
        }
    bool widen = false;
    for (int a = 0; a < 3; ++a)
      if (spread[a] < 0.5) {
        if (pass == 1) return 0;
        w[a] = 2;
        widen = true;
      }
    if (!widen) break;
  }
  if (cnt < 4) return 0;
  const double det = Mn[0][0] * (Mn[1][1] * Mn[2][2] - Mn[1][2] * Mn[2][1]) -
                     Mn[0][1] * (Mn[1][0] * Mn[2][2] - Mn[1][2] * Mn[2][0]) +
                     Mn[0][2] * (Mn[1][0] * Mn[2][1] - Mn[1][1] * Mn[2][0]);
  const double tr = (Mn[0][0] + Mn[1][1] + Mn[2][2]) / 3.0;
  if (!(det > 1e-12 * tr * tr * tr)) return 0;
  return cnt;
}

// x - xhat_r for a point x relative to r's centre, as sum_m w_m (x - x_m)
// over the members of M_r (weights of Eq. centroid, summing to one): exact
// to rounding even when xhat_r sits next to one member.
__device__ void from_xhat(const GridDev &G, const Dims &D, int g, int i, int j, int k, long long r, const double x[3],
                          double e[3]) {
  const long long n = G.nrec;
  e[0] = e[1] = e[2] = 0.0;
  if (!G.code[r]) {
    for (int d = 0; d < 3; ++d) e[d] = x[d] - G.cent[d * n + r];
    return;
  }
  Members M;
  members_of(G, D, g, i, j, k, G.code[r], M);
  for (int q = 0; q < M.n; ++q) {
    const long long m = M.v[q].rec;
    const double w = q == 0 ? G.omega[r] * M.v[0].alpha / G.vhat[r]
                            : G.kappa[r] * M.v[q].alpha / (m >= 0 ? G.nnb[m] : 1) / G.vhat[r];
    for (int d = 0; d < 3; ++d) e[d] += w * (x[d] - (M.off[q][d] + rec_or(G.cent + d * n, m, 0.0)));
  }
}

// Per small CV: members, Qhat weights, pivot, limiter points, stencil size.
__global__ void k_small_tables(Dims D, int g, GridDev G, WsrdDev W, double vt, long long *lsq_cnt) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= W.nsmall) return;
  const long long r = W.s_rec[s];
  const long long L = W.s_lin[s];
  const int i = (int)(L % D.nx), j = (int)((L / D.nx) % D.ny), k = (int)(L / D.nxy);
  const long long n = G.nrec;
  Members M;
  members_of(G, D, g, i, j, k, G.code[r], M);
  const double xr[3] = {G.xhat[r], G.xhat[n + r], G.xhat[2 * n + r]};
  const double vh = G.vhat[r];
  int piv = -1, big = 0;
  for (int q = 0; q < 8; ++q) {
    long long ml = -1;
    double w = 0.0, e[3] = {0, 0, 0};
    if (q < M.n) {
      const long long m = M.v[q].rec;
      ml = lin(D, i + M.off[q][0], j + M.off[q][1], k + M.off[q][2]);
      if (q == 0) w = G.omega[r] * M.v[0].alpha / vh;
      else w = G.kappa[r] * M.v[q].alpha / (m >= 0 ? G.nnb[m] : 1) / vh;
      double xq[3];
      for (int d = 0; d < 3; ++d) xq[d] = M.off[q][d] + rec_or(G.cent + d * n, m, 0.0);
      from_xhat(G, D, g, i, j, k, r, xq, e);
      if (piv < 0 && M.v[q].alpha >= vt) piv = q;
      if (M.v[q].alpha > M.v[big].alpha) big = q;
    }
    W.s_mlin[8 * s + q] = ml;
    W.s_mw[8 * s + q] = w;
    for (int d = 0; d < 3; ++d) W.s_me[24 * s + 3 * q + d] = e[d];
  }
  W.s_nmem[s] = M.n;
  W.s_piv[s] = piv >= 0 ? piv : big;
  int wd[3];
  double Mn[3][3];
  lsq_cnt[s] = M.n >= 2 ? lsq_stencil(G, D, g, i, j, k, xr, wd, Mn) : 0;
}

// Gradient coefficient rows c_m = (A^T A)^{-1} (x_m - xhat_r): the per-step
// gradient is sum_m c_m (Qhat_m - Qhat_r).
__global__ void k_lsq_fill(Dims D, int g, GridDev G, WsrdDev W) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= W.nsmall) return;
  const long long o0 = W.s_loff[s], o1 = W.s_loff[s + 1];
  if (o1 == o0) return;
  const long long r = W.s_rec[s];
  const long long L = W.s_lin[s];
  const int i = (int)(L % D.nx), j = (int)((L / D.nx) % D.ny), k = (int)(L / D.nxy);
  const long long n = G.nrec;
  const double xr[3] = {G.xhat[r], G.xhat[n + r], G.xhat[2 * n + r]};
  int w[3];
  double Mn[3][3];
  lsq_stencil(G, D, g, i, j, k, xr, w, Mn);
  const double det = Mn[0][0] * (Mn[1][1] * Mn[2][2] - Mn[1][2] * Mn[2][1]) -
                     Mn[0][1] * (Mn[1][0] * Mn[2][2] - Mn[1][2] * Mn[2][0]) +
                     Mn[0][2] * (Mn[1][0] * Mn[2][1] - Mn[1][1] * Mn[2][0]);
  double inv[3][3];
  inv[0][0] = (Mn[1][1] * Mn[2][2] - Mn[1][2] * Mn[2][1]) / det;
  inv[0][1] = (Mn[0][2] * Mn[2][1] - Mn[0][1] * Mn[2][2]) / det;
  inv[0][2] = (Mn[0][1] * Mn[1][2] - Mn[0][2] * Mn[1][1]) / det;
  inv[1][0] = (Mn[1][2] * Mn[2][0] - Mn[1][0] * Mn[2][2]) / det;
  inv[1][1] = (Mn[0][0] * Mn[2][2] - Mn[0][2] * Mn[2][0]) / det;
  inv[1][2] = (Mn[0][2] * Mn[1][0] - Mn[0][0] * Mn[1][2]) / det;
  inv[2][0] = (Mn[1][0] * Mn[2][1] - Mn[1][1] * Mn[2][0]) / det;
  inv[2][1] = (Mn[0][1] * Mn[2][0] - Mn[0][0] * Mn[2][1]) / det;
  inv[2][2] = (Mn[0][0] * Mn[1][1] - Mn[0][1] * Mn[1][0]) / det;
  long long o = o0;
  for (int dk = -w[2]; dk <= w[2]; ++dk)
    for (int dj = -w[1]; dj <= w[1]; ++dj)
      for (int di = -w[0]; di <= w[0]; ++di) {
        if (!di && !dj && !dk) continue;
        const View v = view(G, D, g, i + di, j + dj, k + dk);
        if (!v.active) continue;
        const int off[3] = {di, dj, dk};
        double p[3];
        rel_pos(G, v.rec, off, xr, p);
        W.l_lin[o] = lin(D, i + di, j + dj, k + dk);
        W.l_sid[o] = v.rec >= 0 ? W.sid[v.rec] : -1;
        for (int a = 0; a < 3; ++a) W.l_c[3 * o + a] = inv[a][0] * p[0] + inv[a][1] * p[1] + inv[a][2] * p[2];
        ++o;
      }
}

// Pivot state indices, looked up once here instead of twice per step.
__global__ void k_pivot_lin(WsrdDev W) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s < W.nsmall) W.s_plin[s] = W.s_mlin[8 * s + W.s_piv[s]];
}

__global__ void k_stencil_pivot_lin(WsrdDev W) {
  const long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (o < W.nlsq) W.l_plin[o] = W.l_sid[o] >= 0 ? W.s_plin[W.l_sid[o]] : W.l_lin[o];
}

// Per affected CV: its own small id and the neighbourhoods that hold it.
__global__ void k_aff_count(Dims D, int g, GridDev G, const long long *aff_id, WsrdDev W, long long *wcnt) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  const long long n = G.nrec;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    if (!view(G, D, g, i, j, k).active || !(G.code[r] || G.nnb[r] >= 2)) continue;
    const long long a = aff_id[r];
    W.a_lin[a] = lin(D, i, j, k);
    W.a_sid[a] = W.sid[r];
    double ee[3] = {0.0, 0.0, 0.0};
    if (G.code[r]) {
      const double xi[3] = {G.cent[r], G.cent[n + r], G.cent[2 * n + r]};
      from_xhat(G, D, g, i, j, k, r, xi, ee);
    }
    for (int d = 0; d < 3; ++d) W.a_eself[3 * a + d] = ee[d];
    wcnt[a] = G.nnb[r] - 1;
  }
}

__global__ void k_aff_fill(Dims D, int g, GridDev G, const long long *aff_id, WsrdDev W) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  const long long n = G.nrec;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    if (!view(G, D, g, i, j, k).active || !(G.code[r] || G.nnb[r] >= 2)) continue;
    const long long a = aff_id[r];
    long long o = W.a_woff[a];
    const double Ni = G.nnb[r];
    for (int dk = -1; dk <= 1; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          if (!di && !dj && !dk) continue;
          const View v = view(G, D, g, i + di, j + dj, k + dk);
          if (!v.active || v.rec < 0 || G.code[v.rec] == 0) continue;
          int off[8][3];
          const int cnt = unpack(G.code[v.rec], off);
          for (int c = 1; c < cnt; ++c)
            if (off[c][0] == -di && off[c][1] == -dj && off[c][2] == -dk) {
              const long long q = v.rec;
              W.w_sid[o] = W.sid[q];
              W.w_k[o] = G.kappa[q] / Ni;
              const double xi[3] = {-di + G.cent[r], -dj + G.cent[n + r], -dk + G.cent[2 * n + r]};
              double ee[3];
              from_xhat(G, D, g, i + di, j + dj, k + dk, q, xi, ee);
              for (int d = 0; d < 3; ++d) W.w_e[3 * o + d] = ee[d];
              ++o;
            }
        }
  }
}

__global__ void k_to_float(const double *src, float *dst, long long n) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) dst[t] = (float)src[t];
}

inline int cols_blocks(const Dims &D) { return (D.nx * D.ny + 127) / 128; }
inline int lin_blocks(long long n) { return (int)((n + 127) / 128); }

template <typename P>
cudaError_t dalloc(P **p, long long count) {
  *p = nullptr;
  if (count <= 0) count = 1;
  return cudaMalloc((void **)p, sizeof(P) * (size_t)count);
}

// Does a CV that the redistribution of grid g reads or writes lie outside the
// near-EB set (covered, a w wall level, or at or above kfast, where the bulk
// kernel writes it)?  One thread per table entry: pivots, members, LSQ
// stencil pivots, affected CVs.
__global__ void k_wsrd_reach(Dims D, int g, WsrdDev W, const int *kcov, const int *kfast, unsigned *far) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long c;
  if (t < W.nsmall) {
    c = W.s_plin[t];
  } else if ((t -= W.nsmall) < 8 * W.nsmall) {
    if (t % 8 >= W.s_nmem[t / 8]) return;
    c = W.s_mlin[t];
  } else if ((t -= 8 * W.nsmall) < W.nlsq) {
    c = W.l_plin[t];
  } else if ((t -= W.nlsq) < W.naff) {
    c = W.a_lin[t];
  } else {
    return;
  }
  const long long col = c % D.nxy;
  const int k = (int)(c / D.nxy);
  const bool wall = g == 3 && (k == 0 || k == D.nz);
  if (wall || k < kcov[col] || k >= kfast[col]) atomicOr(far, 1u);
}

}  // namespace

#define CK(x)                         \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

// Build the redistribution tables of grid g.  dev_tmp: device scratch of at
// least 3 * (G.nrec + 2) + 3 * (nrec/512 + 2) long longs.
cudaError_t build_wsrd(const Dims &D, int g, GridDev &G, const GridDev *all, double vt, WsrdDev &W,
                       cudaStream_t s, long long *dev_tmp) {
  (void)all;
  const int cb = cols_blocks(D);
  k_codes<<<cb, 128, 0, s>>>(D, g, G, vt);
  k_nnb_omega<<<cb, 128, 0, s>>>(D, g, G);
  k_vhat_xhat<<<cb, 128, 0, s>>>(D, g, G);
  CK(cudaGetLastError());
  const long long n = G.nrec;
  long long *small_id = dev_tmp, *aff_id = dev_tmp + (n + 1);
  long long *tot = dev_tmp + 2 * (n + 1);   // followed by scan scratch
  CK(cudaMemsetAsync(small_id, 0, sizeof(long long) * (n + 1), s));
  CK(cudaMemsetAsync(aff_id, 0, sizeof(long long) * (n + 1), s));
  k_flags<<<cb, 128, 0, s>>>(D, g, G, small_id, aff_id);
  long long h2[2];
  scan_exclusive(small_id, n, tot, s);
  CK(cudaMemcpyAsync(&h2[0], tot, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  scan_exclusive(aff_id, n, tot, s);
  CK(cudaMemcpyAsync(&h2[1], tot, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  W.nsmall = h2[0];
  W.naff = h2[1];
  CK(dalloc(&W.sid, n));
  CK(dalloc(&W.s_lin, W.nsmall));
  CK(dalloc(&W.s_rec, W.nsmall));
  CK(dalloc(&W.s_nmem, W.nsmall));
  CK(dalloc(&W.s_piv, W.nsmall));
  CK(dalloc(&W.s_mlin, 8 * W.nsmall));
  CK(dalloc(&W.s_mw, 8 * W.nsmall));
  CK(dalloc(&W.s_me, 24 * W.nsmall));
  CK(dalloc(&W.s_loff, W.nsmall + 1));
  CK(dalloc(&W.a_lin, W.naff));
  CK(dalloc(&W.a_sid, W.naff));
  CK(dalloc(&W.a_eself, 3 * W.naff));
  CK(dalloc(&W.a_woff, W.naff + 1));
  k_assign_small<<<cb, 128, 0, s>>>(D, g, G, small_id, W);
  // LSQ stencil sizes -> offsets
  CK(cudaMemsetAsync(W.s_loff, 0, sizeof(long long) * (W.nsmall + 1), s));
  if (W.nsmall) k_small_tables<<<lin_blocks(W.nsmall), 128, 0, s>>>(D, g, G, W, vt, W.s_loff);
  scan_exclusive(W.s_loff, W.nsmall + 1, tot, s);
  CK(cudaMemcpyAsync(&W.nlsq, tot, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(dalloc(&W.l_lin, W.nlsq));
  CK(dalloc(&W.l_sid, W.nlsq));
  CK(dalloc(&W.l_c, 3 * W.nlsq));
  if (W.nsmall) k_lsq_fill<<<lin_blocks(W.nsmall), 128, 0, s>>>(D, g, G, W);
  CK(dalloc(&W.s_plin, W.nsmall));
  CK(dalloc(&W.l_plin, W.nlsq));
  if (W.nsmall) k_pivot_lin<<<lin_blocks(W.nsmall), 128, 0, s>>>(W);
  if (W.nlsq) k_stencil_pivot_lin<<<lin_blocks(W.nlsq), 128, 0, s>>>(W);
  // affected CVs and their neighbourhood lists
  CK(cudaMemsetAsync(W.a_woff, 0, sizeof(long long) * (W.naff + 1), s));
  k_aff_count<<<cb, 128, 0, s>>>(D, g, G, aff_id, W, W.a_woff);
  scan_exclusive(W.a_woff, W.naff + 1, tot, s);
  CK(cudaMemcpyAsync(&W.nw, tot, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(dalloc(&W.w_sid, W.nw));
  CK(dalloc(&W.w_k, W.nw));
  CK(dalloc(&W.w_e, 3 * W.nw));
  k_aff_fill<<<cb, 128, 0, s>>>(D, g, G, aff_id, W);
  // float copies of the weight tables (mixed-precision path)
  const struct {
    const double *src;
    float **dst;
    long long n;
  } tabs[6] = {{W.s_mw, &W.s_mw_f, 8 * W.nsmall}, {W.s_me, &W.s_me_f, 24 * W.nsmall},
               {W.l_c, &W.l_c_f, 3 * W.nlsq},     {W.a_eself, &W.a_eself_f, 3 * W.naff},
               {W.w_k, &W.w_k_f, W.nw},           {W.w_e, &W.w_e_f, 3 * W.nw}};
  for (const auto &t : tabs) {
    CK(dalloc(t.dst, t.n));
    if (t.n > 0) k_to_float<<<lin_blocks(t.n), 128, 0, s>>>(t.src, *t.dst, t.n);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return cudaSuccess;
}

void free_wsrd(WsrdDev &W) {
  void *ptrs[] = {W.sid, W.s_lin, W.s_rec, W.s_nmem, W.s_piv, W.s_mlin, W.s_mw, W.s_me, W.s_loff, W.l_lin,
                  W.l_sid, W.l_c, W.a_lin, W.a_sid, W.a_eself, W.a_woff, W.w_sid, W.w_k, W.w_e,
                  W.s_mw_f, W.s_me_f, W.l_c_f, W.a_eself_f, W.w_k_f, W.w_e_f, W.s_plin, W.l_plin};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  W = WsrdDev();
}

void launch_wsrd_reach(const Dims &D, int g, const WsrdDev &W, const int *kcov, const int *kfast, unsigned *far,
                       cudaStream_t s) {
  const long long n = 9 * W.nsmall + W.nlsq + W.naff;
  if (n > 0) k_wsrd_reach<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(D, g, W, kcov, kfast, far);
}
