// eb_fast.cu -- the geometry-free bulk of the flux divergence and update
// (Eqs. update-cc / update-fc with alpha = beta = 1), for every CV at or
// above its column's kfast level, where every CV any flux stencil reads is a
// regular CV.
//
// Tiling.  A CTA owns a TX x TY tile of columns and marches up in z from the
// lowest kfast of its tile.  Shared memory holds a ring of four raw planes
// (k-1 .. k+2) of the five fields over the tile plus a halo (3 cells on the
// low sides, 2 on the high sides: the face velocity at the halo edge needs
// the density one cell further), and the primitive plane of level k
// (theta, u, v, w, halo 2) that the x and y upwind stencils read.  Each
// thread owns one column: its z stencils (levels k-2 .. k+2) live in
// registers, and the flux through the face above it is carried to the next
// level.  Every field is read from HBM once per level; halo reuse comes from
// shared memory and L2.
#include "eb_step.cuh"

#include <algorithm>

namespace {

template <typename T>
__device__ inline T divide(T a, T b) {
  return eb_div(a, b);
}

template <typename T>
__device__ inline T upwind_flux(T m, T pLL, T pL, T pR, T pRR, bool hasLL, bool hasRR) {
  return m * upwind_value(m, pLL, pL, pR, pRR, hasLL, hasRR);
}

template <typename T, int TX, int TY>
struct Tile {
  static constexpr int PX = TX + 5, PY = TY + 5, NP = PX * PY;   // raw planes
  static constexpr int QX = TX + 4, QY = TY + 4, NQ = QX * QY;   // primitive plane
  static constexpr int NT = TX * TY;
  static constexpr int RAW = 4 * 5 * NP;                           // ring of 4 planes x 5 fields
  static constexpr size_t BYTES = sizeof(T) * (size_t)(RAW + 4 * NQ);
  static constexpr int LOADS = (NP + NT - 1) / NT;
  static constexpr int PRIMS = (NQ + NT - 1) / NT;
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_fast_tiled(StepArgs<T> A) {
  using TL = Tile<T, TX, TY>;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  T *raw = reinterpret_cast<T *>(smem_bytes);
  T *prim = raw + TL::RAW;
  __shared__ int s_k0;
  const Dims &D = A.D;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int i = i0 + tx, j = j0 + ty;
  const bool inside = i < D.nx && j < D.ny;
  const int kf = inside ? A.kfast[i + D.nx * j] : D.nz;
  if (tid == 0) s_k0 = D.nz;
  __syncthreads();
  atomicMin(&s_k0, kf);
  __syncthreads();
  // this CTA's slab of levels: [max(tile's lowest kfast, chunk start), chunk end)
  const int k0 = max(s_k0, (int)blockIdx.z * A.kchunk);
  const int kend = min(D.nz, ((int)blockIdx.z + 1) * A.kchunk);
  if (k0 >= kend) return;

  // column offsets of the points this thread loads (fixed for the whole march)
  long long lcol[TL::LOADS];
  int lslot[TL::LOADS];
#pragma unroll
  for (int r = 0; r < TL::LOADS; ++r) {
    const int q = tid + r * TL::NT;
    lslot[r] = q < TL::NP ? q : -1;
    const int x = q % TL::PX - 3, y = q / TL::PX - 3;
    lcol[r] = (long long)wrapmod(i0 + x, D.nx) + (long long)D.nx * wrapmod(j0 + y, D.ny);
  }
  auto load_plane = [&](int L) {
    T *P = raw + (L & 3) * 5 * TL::NP;
    const bool live = L >= 0 && L < D.nz;
    const T rr = live ? A.src.ref_rho[L] : T(0);
    const T rt = live ? A.src.ref_rt[L] : T(0);
#pragma unroll
    for (int r = 0; r < TL::LOADS; ++r) {
      if (lslot[r] < 0) continue;
      T v0 = T(1), v1 = T(0), v2 = T(0), v3 = T(0), v4 = T(0);
      if (live) {
        const long long c = lcol[r] + D.nxy * L;
        v0 = rr + A.src.f[0][c];
        v1 = rt + A.src.f[1][c];
        v2 = A.src.f[2][c];
        v3 = A.src.f[3][c];
        v4 = L >= 1 ? A.src.f[4][c] : T(0);   // rho*w on the wall level 0 enters as zero
      }
      const int q = lslot[r];
      P[q] = v0;
      P[TL::NP + q] = v1;
      P[2 * TL::NP + q] = v2;
      P[3 * TL::NP + q] = v3;
      P[4 * TL::NP + q] = v4;
    }
  };
  // raw index of tile point (x, y)
  auto ri = [&](int x, int y) { return (y + 3) * TL::PX + (x + 3); };
  auto qi = [&](int x, int y) { return (y + 2) * TL::QX + (x + 2); };
  auto RAWV = [&](int L, int f, int x, int y) -> T { return raw[(L & 3) * 5 * TL::NP + f * TL::NP + ri(x, y)]; };

  // column primitives of plane L (theta, u, v, w), from the ring
  auto column_prims = [&](int L, T &th, T &u, T &v, T &w) {
    if (L < 0 || L >= D.nz) {
      th = u = v = T(0);
      w = T(0);   // w wall level nz (and beyond, where it is never used)
      return;
    }
    const T *P = raw + (L & 3) * 5 * TL::NP;
    const int p = ri(tx, ty);
    const T r = P[p];
    th = divide(P[TL::NP + p], r);
    u = divide(P[2 * TL::NP + p], T(0.5) * (P[p - 1] + r));
    v = divide(P[3 * TL::NP + p], T(0.5) * (P[p - TL::PX] + r));
    if (L == 0) {
      w = T(0);
    } else {
      const T *Pm = raw + ((L - 1) & 3) * 5 * TL::NP;
      w = divide(P[4 * TL::NP + p], T(0.5) * (Pm[p] + r));
    }
  };

  // ---- prologue: ring planes k0-3 .. k0+1, column window k0-2 .. k0+1
  T th[5], uu[5], vv[5], ww[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    load_plane(k0 - 3 + q);
    __syncthreads();
    if (q >= 1) column_prims(k0 - 3 + q, th[q - 1], uu[q - 1], vv[q - 1], ww[q - 1]);
    __syncthreads();
  }
  const T idx = T(1.0 / D.dx), idy = T(1.0 / D.dy), idz = T(1.0 / D.dz);
  const int nz = D.nz;
  // lower z face fluxes of level k0: c (mass, theta), u, v, w
  T zc_m, zc_t, zu, zv, zw;
  {
    const int k = k0;
    const T m = RAWV(k, 4, tx, ty);
    zc_m = m;
    zc_t = upwind_flux(m, th[0], th[1], th[2], th[3], true, k + 1 <= nz - 1);
    const T mu = T(0.5) * (RAWV(k, 4, tx - 1, ty) + m);
    zu = upwind_flux(mu, uu[0], uu[1], uu[2], uu[3], true, k + 1 <= nz - 1);
    const T mv = T(0.5) * (RAWV(k, 4, tx, ty - 1) + m);
    zv = upwind_flux(mv, vv[0], vv[1], vv[2], vv[3], true, k + 1 <= nz - 1);
    const T mw = T(0.5) * (RAWV(k - 1, 4, tx, ty) + m);
    zw = upwind_flux(mw, ww[0], ww[1], ww[2], ww[3], true, true);
  }

  for (int k = k0; k < kend; ++k) {
    // ---- stage plane k+2 and the primitive plane of level k
    __syncthreads();
    load_plane(k + 2);
    __syncthreads();
    column_prims(k + 2, th[4], uu[4], vv[4], ww[4]);
    if (k + 2 == nz) ww[4] = T(0);   // w wall level
    {
      const T *P = raw + (k & 3) * 5 * TL::NP;
      const T *Pm = raw + ((k - 1) & 3) * 5 * TL::NP;
#pragma unroll
      for (int r = 0; r < TL::PRIMS; ++r) {
        const int q = tid + r * TL::NT;
        if (q >= TL::NQ) continue;
        const int x = q % TL::QX - 2, y = q / TL::QX - 2;
        const int p = ri(x, y);
        const T rho = P[p];
        prim[q] = divide(P[TL::NP + p], rho);
        prim[TL::NQ + q] = divide(P[2 * TL::NP + p], T(0.5) * (P[p - 1] + rho));
        prim[2 * TL::NQ + q] = divide(P[3 * TL::NP + p], T(0.5) * (P[p - TL::PX] + rho));
        prim[3 * TL::NQ + q] = divide(P[4 * TL::NP + p], T(0.5) * (Pm[p] + rho));
      }
    }
    __syncthreads();
    const bool has1 = k + 1 <= nz - 1, has2 = k + 2 <= nz - 1;   // c, u, v levels above
    const T *TH = prim, *UP = prim + TL::NQ, *VP = prim + 2 * TL::NQ, *WP = prim + 3 * TL::NQ;
    if (inside && k >= kf) {
      const long long c = (long long)i + D.nx * ((long long)j + (long long)D.ny * k);
      // ---------------- c grid: rho and rho*theta
      {
        const T mxl = RAWV(k, 2, tx, ty), mxh = RAWV(k, 2, tx + 1, ty);
        const T fxl = upwind_flux(mxl, TH[qi(tx - 2, ty)], TH[qi(tx - 1, ty)], TH[qi(tx, ty)], TH[qi(tx + 1, ty)],
                                  true, true);
        const T fxh = upwind_flux(mxh, TH[qi(tx - 1, ty)], TH[qi(tx, ty)], TH[qi(tx + 1, ty)], TH[qi(tx + 2, ty)],
                                  true, true);
        const T myl = RAWV(k, 3, tx, ty), myh = RAWV(k, 3, tx, ty + 1);
        const T fyl = upwind_flux(myl, TH[qi(tx, ty - 2)], TH[qi(tx, ty - 1)], TH[qi(tx, ty)], TH[qi(tx, ty + 1)],
                                  true, true);
        const T fyh = upwind_flux(myh, TH[qi(tx, ty - 1)], TH[qi(tx, ty)], TH[qi(tx, ty + 1)], TH[qi(tx, ty + 2)],
                                  true, true);
        const T mzh = has1 ? RAWV(k + 1, 4, tx, ty) : T(0);
        const T fzh = upwind_flux(mzh, th[1], th[2], th[3], th[4], true, has2);
        const T dr = -((mxh - mxl) * idx + (myh - myl) * idy + (mzh - zc_m) * idz);
        const T dt_ = -((fxh - fxl) * idx + (fyh - fyl) * idy + (fzh - zc_t) * idz);
        const T o0 = A.base[0] ? A.base[0][c] + A.dtT * dr : dr;
        const T o1 = A.base[0] ? A.base[1][c] + A.dtT * dt_ : dt_;
        A.out[0][c] = o0;
        A.out[1][c] = o1;
        if (!(isfinite(o0) && isfinite(o1))) atomicOr(A.status, EB_DEV_NUMERIC);
        zc_m = mzh;
        zc_t = fzh;
      }
      // ---------------- u grid (x faces at cell centres, y and z faces on edges)
      {
        const T ul = RAWV(k, 2, tx - 1, ty), u0 = RAWV(k, 2, tx, ty), ur = RAWV(k, 2, tx + 1, ty);
        const T fxl = upwind_flux(T(0.5) * (ul + u0), UP[qi(tx - 2, ty)], UP[qi(tx - 1, ty)], UP[qi(tx, ty)],
                                  UP[qi(tx + 1, ty)], true, true);
        const T fxh = upwind_flux(T(0.5) * (u0 + ur), UP[qi(tx - 1, ty)], UP[qi(tx, ty)], UP[qi(tx + 1, ty)],
                                  UP[qi(tx + 2, ty)], true, true);
        const T myl = T(0.5) * (RAWV(k, 3, tx - 1, ty) + RAWV(k, 3, tx, ty));
        const T myh = T(0.5) * (RAWV(k, 3, tx - 1, ty + 1) + RAWV(k, 3, tx, ty + 1));
        const T fyl = upwind_flux(myl, UP[qi(tx, ty - 2)], UP[qi(tx, ty - 1)], UP[qi(tx, ty)], UP[qi(tx, ty + 1)],
                                  true, true);
        const T fyh = upwind_flux(myh, UP[qi(tx, ty - 1)], UP[qi(tx, ty)], UP[qi(tx, ty + 1)], UP[qi(tx, ty + 2)],
                                  true, true);
        const T mzh = has1 ? T(0.5) * (RAWV(k + 1, 4, tx - 1, ty) + RAWV(k + 1, 4, tx, ty)) : T(0);
        const T fzh = upwind_flux(mzh, uu[1], uu[2], uu[3], uu[4], true, has2);
        const T d = -((fxh - fxl) * idx + (fyh - fyl) * idy + (fzh - zu) * idz);
        const T o = A.base[0] ? A.base[2][c] + A.dtT * d : d;
        A.out[2][c] = o;
        if (!isfinite(o)) atomicOr(A.status, EB_DEV_NUMERIC);
        zu = fzh;
      }
      // ---------------- v grid
      {
        const T vl = RAWV(k, 3, tx, ty - 1), v0 = RAWV(k, 3, tx, ty), vr = RAWV(k, 3, tx, ty + 1);
        const T mxl = T(0.5) * (RAWV(k, 2, tx, ty - 1) + RAWV(k, 2, tx, ty));
        const T mxh = T(0.5) * (RAWV(k, 2, tx + 1, ty - 1) + RAWV(k, 2, tx + 1, ty));
        const T fxl = upwind_flux(mxl, VP[qi(tx - 2, ty)], VP[qi(tx - 1, ty)], VP[qi(tx, ty)], VP[qi(tx + 1, ty)],
                                  true, true);
        const T fxh = upwind_flux(mxh, VP[qi(tx - 1, ty)], VP[qi(tx, ty)], VP[qi(tx + 1, ty)], VP[qi(tx + 2, ty)],
                                  true, true);
        const T fyl = upwind_flux(T(0.5) * (vl + v0), VP[qi(tx, ty - 2)], VP[qi(tx, ty - 1)], VP[qi(tx, ty)],
                                  VP[qi(tx, ty + 1)], true, true);
        const T fyh = upwind_flux(T(0.5) * (v0 + vr), VP[qi(tx, ty - 1)], VP[qi(tx, ty)], VP[qi(tx, ty + 1)],
                                  VP[qi(tx, ty + 2)], true, true);
        const T mzh = has1 ? T(0.5) * (RAWV(k + 1, 4, tx, ty - 1) + RAWV(k + 1, 4, tx, ty)) : T(0);
        const T fzh = upwind_flux(mzh, vv[1], vv[2], vv[3], vv[4], true, has2);
        const T d = -((fxh - fxl) * idx + (fyh - fyl) * idy + (fzh - zv) * idz);
        const T o = A.base[0] ? A.base[3][c] + A.dtT * d : d;
        A.out[3][c] = o;
        if (!isfinite(o)) atomicOr(A.status, EB_DEV_NUMERIC);
        zv = fzh;
      }
      // ---------------- w grid (x and y faces on edges, z faces at cell centres)
      {
        const T mxl = T(0.5) * (RAWV(k - 1, 2, tx, ty) + RAWV(k, 2, tx, ty));
        const T mxh = T(0.5) * (RAWV(k - 1, 2, tx + 1, ty) + RAWV(k, 2, tx + 1, ty));
        const T fxl = upwind_flux(mxl, WP[qi(tx - 2, ty)], WP[qi(tx - 1, ty)], WP[qi(tx, ty)], WP[qi(tx + 1, ty)],
                                  true, true);
        const T fxh = upwind_flux(mxh, WP[qi(tx - 1, ty)], WP[qi(tx, ty)], WP[qi(tx + 1, ty)], WP[qi(tx + 2, ty)],
                                  true, true);
        const T myl = T(0.5) * (RAWV(k - 1, 3, tx, ty) + RAWV(k, 3, tx, ty));
        const T myh = T(0.5) * (RAWV(k - 1, 3, tx, ty + 1) + RAWV(k, 3, tx, ty + 1));
        const T fyl = upwind_flux(myl, WP[qi(tx, ty - 2)], WP[qi(tx, ty - 1)], WP[qi(tx, ty)], WP[qi(tx, ty + 1)],
                                  true, true);
        const T fyh = upwind_flux(myh, WP[qi(tx, ty - 1)], WP[qi(tx, ty)], WP[qi(tx, ty + 1)], WP[qi(tx, ty + 2)],
                                  true, true);
        const T w0 = RAWV(k, 4, tx, ty), w1 = has1 ? RAWV(k + 1, 4, tx, ty) : T(0);
        const T fzh = upwind_flux(T(0.5) * (w0 + w1), ww[1], ww[2], ww[3], ww[4], true, k + 2 <= nz);
        const T d = -((fxh - fxl) * idx + (fyh - fyl) * idy + (fzh - zw) * idz);
        const T o = A.base[0] ? A.base[4][c] + A.dtT * d : d;
        A.out[4][c] = o;
        if (!isfinite(o)) atomicOr(A.status, EB_DEV_NUMERIC);
        zw = fzh;
      }
    } else {
      // not yet at this column's fast level: keep the carried z fluxes current
      // (the c, u, v lower fluxes of level k+1 are the upper ones of level k)
      const T m = has1 ? RAWV(k + 1, 4, tx, ty) : T(0);
      zc_m = m;
      zc_t = upwind_flux(m, th[1], th[2], th[3], th[4], true, has2);
      zu = upwind_flux(has1 ? T(0.5) * (RAWV(k + 1, 4, tx - 1, ty) + m) : T(0), uu[1], uu[2], uu[3], uu[4], true,
                       has2);
      zv = upwind_flux(has1 ? T(0.5) * (RAWV(k + 1, 4, tx, ty - 1) + m) : T(0), vv[1], vv[2], vv[3], vv[4], true,
                       has2);
      zw = upwind_flux(T(0.5) * (RAWV(k, 4, tx, ty) + m), ww[1], ww[2], ww[3], ww[4], true, k + 2 <= nz);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      th[q] = th[q + 1];
      uu[q] = uu[q + 1];
      vv[q] = vv[q + 1];
      ww[q] = ww[q + 1];
    }
  }
}

// Pass-through of the CVs no kernel updates: covered CVs and the two wall
// levels of rho*w (or zeros when dU itself is written).
template <typename T>
__global__ void k_static(StepArgs<T> A) {
  const Dims &D = A.D;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= D.nx || j >= D.ny) return;
  const int col = i + D.nx * j;
  auto put = [&](int f, long long c) { A.out[f][c] = A.base[0] ? A.base[f][c] : T(0); };
  const long long c = lin(D, i, j, k);
  if (k < A.G[0].kcov[col]) {
    put(0, c);
    put(1, c);
  }
  if (k < A.G[1].kcov[col]) put(2, c);
  if (k < A.G[2].kcov[col]) put(3, c);
  if (k < A.G[3].kcov[col] || k == 0) put(4, c);
  if (k == D.nz - 1) put(4, lin(D, i, j, D.nz));
}

constexpr int FTX = 32, FTY = 8;

}  // namespace

template <typename T>
void launch_flux_fast(const StepArgs<T> &A, cudaStream_t s) {
  const Dims &D = A.D;
  if (A.copy_static) {
    dim3 blk(32, 8, 1), grd((D.nx + 31) / 32, (D.ny + 7) / 8, D.nz);
    k_static<T><<<grd, blk, 0, s>>>(A);
  }
  using TL = Tile<T, FTX, FTY>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_fast_tiled<T, FTX, FTY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::BYTES);
    attr_set = true;
  }
  // split the z march into slabs so that the grid fills the GPU for about
  // three waves of resident CTAs (slabs of at least 16 levels)
  const long long tiles = (long long)((D.nx + FTX - 1) / FTX) * ((D.ny + FTY - 1) / FTY);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long slots = (long long)(sms > 0 ? sms : 148) * 4;
  int nch = (int)((3 * slots + tiles - 1) / tiles);
  nch = std::max(1, std::min(nch, D.nz / 16));
  StepArgs<T> B = A;
  B.kchunk = (D.nz + nch - 1) / nch;
  dim3 blk(FTX, FTY, 1), grd((D.nx + FTX - 1) / FTX, (D.ny + FTY - 1) / FTY, nch);
  k_fast_tiled<T, FTX, FTY><<<grd, blk, TL::BYTES, s>>>(B);
}

template void launch_flux_fast<double>(const StepArgs<double> &, cudaStream_t);
template void launch_flux_fast<float>(const StepArgs<float> &, cudaStream_t);
