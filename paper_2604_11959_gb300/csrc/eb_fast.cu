// eb_fast.cu -- the bulk kernel (the march itself is in eb_bulk.cuh), the
// pass-through of covered CVs, the work split of the bulk kernel and the
// launchers.
#include "eb_bulk.cuh"

#include <algorithm>
#include <vector>

namespace {

using namespace bulk;

// One CTA marches the pieces boff[b] .. boff[b+1]-1 of the work split
// (tiles of TYV rows).  The float path is held to EB_BULK_MAXNREG registers
// per thread (96: the fewest without spills), so that beside its two CTAs per
// SM (2 x 256 x 96 of the 65536 registers) the near-EB kernels' blocks still
// find registers on the same SM and run beside the march.
#ifndef EB_BULK_MAXNREG
#define EB_BULK_MAXNREG 96
#endif
template <typename T, int V, int TYV>
__global__ void __launch_bounds__(BulkTile<T, TYV>::NT, (sizeof(T) == 4 ? 2 : 1))
    __maxnreg__(sizeof(T) == 4 ? EB_BULK_MAXNREG : 255) k_fast_tiled(StepArgs<T> A) {
  using P = typename PairOf<T>::type;
  extern __shared__ __align__(16) unsigned char smem_bytes[];
  __shared__ unsigned tm_slot;
  const unsigned tbase = bulk_tmem_begin<T>(&tm_slot);
  P bad = splat(T(0));   // becomes NaN once any written value is not finite
  for (int sgi = A.boff[blockIdx.x]; sgi < A.boff[blockIdx.x + 1]; ++sgi)
    bulk_march<T, V, bulk_tmem_default<T>(), TYV>(A, A.bseg[sgi], smem_bytes, tbase, bad);
  bulk_tmem_end<T>(&tm_slot);
  if (!(isfinite(bad.x) && isfinite(bad.y))) atomicOr(A.status, EB_DEV_NUMERIC);
}

// Pass-through of the CVs no kernel updates (covered CVs and the two wall
// levels of rho*w; zeros when dU itself is written), from per-grid lists
// built at set-up: one thread per listed CV.
// one grid's list per block range (bstart[q] .. bstart[q + 1] - 1); each
// thread copies up to four listed CVs, their loads issued together
struct StaticBlocks {
  unsigned bstart[5];
};
constexpr int STATIC_PER_THREAD = 4;

template <typename T>
__global__ void k_static(StepArgs<T> A, StaticBlocks SB) {
  int q = 0;
  while (q < 3 && blockIdx.x >= SB.bstart[q + 1]) ++q;
  const long long n = A.G[q].nstatic;
  const long long t0 = (long long)(blockIdx.x - SB.bstart[q]) * blockDim.x * STATIC_PER_THREAD + threadIdx.x;
  const unsigned *L = A.G[q].slist;
  const int f0 = q == 0 ? 0 : q + 1, nf = q == 0 ? 2 : 1;
  unsigned c[STATIC_PER_THREAD];
#pragma unroll
  for (int e = 0; e < STATIC_PER_THREAD; ++e) {
    const long long t = t0 + (long long)e * blockDim.x;
    c[e] = t < n ? L[t] : 0xffffffffu;
  }
  for (int f = f0; f < f0 + nf; ++f) {
    T v[STATIC_PER_THREAD];
#pragma unroll
    for (int e = 0; e < STATIC_PER_THREAD; ++e)
      v[e] = (c[e] != 0xffffffffu && A.base[0]) ? A.base[f][c[e]] : T(0);
#pragma unroll
    for (int e = 0; e < STATIC_PER_THREAD; ++e)
      if (c[e] != 0xffffffffu) A.out[f][c[e]] = v[e];
  }
}

template <typename T, int V, int TYV>
void set_smem_attr() {
  static unsigned long long done = 0;
  ebk_smem_limit(k_fast_tiled<T, V, TYV>, (int)BulkTile<T, TYV>::BYTES, done);
}

template <typename T, int V, int TYV>
void launch_bulk(const StepArgs<T> &A, cudaStream_t s) {
  using TL = BulkTile<T, TYV>;
  if (A.bctas < 1) return;
  set_smem_attr<T, V, TYV>();
  k_fast_tiled<T, V, TYV><<<A.bctas, dim3(TL::NPX, TL::TY, 1), TL::BYTES, s>>>(A);
}

template <typename T>
int resident_ctas_per_sm() {
  constexpr int V = 16 / sizeof(T);
  set_smem_attr<T, V, 16>();   // every variant set here, outside any graph capture
  set_smem_attr<T, 1, 16>();
  if constexpr (sizeof(T) == sizeof(float)) {
    set_smem_attr<T, V, 14>();
    set_smem_attr<T, 1, 14>();
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fast_tiled<T, V, 16>, BulkTile<T>::NT,
                                                    BulkTile<T>::BYTES) != cudaSuccess ||
      n < 1)
    n = 1;
  return n;
}

}  // namespace

cudaError_t bulk_plan(const Dims &D, const int *kfast_host, bool f64, int slab_levels, int tile_rows,
                      std::vector<int> &seg, std::vector<int> &off) {
  const int TX = BulkTile<float>::TX, TY = tile_rows;
  const int tx = (D.nx + TX - 1) / TX, ty = (D.ny + TY - 1) / TY;
  const long long ntile = (long long)tx * ty;
  std::vector<int> kb(ntile, D.nz);
  for (int j = 0; j < D.ny; ++j)
    for (int i = 0; i < D.nx; ++i) {
      int &v = kb[(i / TX) + (long long)tx * (j / TY)];
      v = std::min(v, kfast_host[i + (long long)D.nx * j]);
    }
  long long W = 0;
  for (long long t = 0; t < ntile; ++t) W += std::max(0, D.nz - kb[t]);
  seg.clear();
  off.assign(1, 0);
  if (W == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long slots = (long long)std::max(sms, 1) * (f64 ? resident_ctas_per_sm<double>()
                                                              : resident_ctas_per_sm<float>());
  // Lockstep slabs: every tile is cut at the same levels, and the pieces are
  // launched slab by slab from the top, so CTAs of neighbouring tiles march
  // the same levels at the same time and read each other's halo from L2.
  // Slabs of slab_levels levels, or (0) of at least 16 levels sized for
  // about three waves of CTAs; the short pieces of the lowest slabs come last.
  const long long Lc = slab_levels > 0 ? (long long)slab_levels : std::max(16LL, (W + 3 * slots - 1) / (3 * slots));
  const int nslab = (int)((D.nz + Lc - 1) / Lc);
  for (int sl = nslab - 1; sl >= 0; --sl) {
    const int za = (int)(sl * Lc), zb = (int)std::min<long long>(D.nz, (sl + 1) * Lc);
    for (long long t = 0; t < ntile; ++t) {
      const int a = std::max(za, kb[t]);
      if (a >= zb) continue;
      seg.push_back((int)t);
      seg.push_back(a);
      seg.push_back(zb);
      seg.push_back(0);
      off.push_back((int)(seg.size() / 4));
    }
  }
  return cudaGetLastError();
}

template <typename T>
void launch_flux_bulk(const StepArgs<T> &A, cudaStream_t s);

template <typename T>
void launch_static_copy(const StepArgs<T> &A, cudaStream_t s) {
  const Dims &D = A.D;
  if (A.copy_static) {
    StaticBlocks SB;
    SB.bstart[0] = 0;
    for (int q = 0; q < 4; ++q)
      SB.bstart[q + 1] = SB.bstart[q] + (unsigned)((A.G[q].nstatic + 256 * STATIC_PER_THREAD - 1) /
                                                   (256 * STATIC_PER_THREAD));
    if (SB.bstart[4] > 0) k_static<T><<<SB.bstart[4], 256, 0, s>>>(A, SB);
  }
}

template <typename T>
void launch_flux_fast(const StepArgs<T> &A, cudaStream_t s) {
  launch_static_copy(A, s);
  launch_flux_bulk(A, s);
}

template <typename T>
void launch_flux_bulk(const StepArgs<T> &A, cudaStream_t s) {
  const Dims &D = A.D;
  // 16-byte copies and pair stores need every row of every field to start on
  // a 16-byte boundary: nx a multiple of the copy width and aligned pointers
  constexpr int V = 16 / sizeof(T);
  bool vec = D.nx % V == 0;
  for (int f = 0; f < 5; ++f) {
    vec = vec && ((uintptr_t)A.src.f[f] % 16 == 0) && ((uintptr_t)A.out[f] % 16 == 0);
    if (A.base[0]) vec = vec && ((uintptr_t)A.base[f] % 16 == 0);
  }
  if constexpr (sizeof(T) == sizeof(float)) {   // 14-row tiles on the float path only
    if (A.tile_rows == 14) {
      if (vec) launch_bulk<T, V, 14>(A, s);
      else launch_bulk<T, 1, 14>(A, s);
      return;
    }
  }
  if (vec) launch_bulk<T, V, 16>(A, s);
  else launch_bulk<T, 1, 16>(A, s);
}

template void launch_flux_fast<double>(const StepArgs<double> &, cudaStream_t);
template void launch_flux_fast<float>(const StepArgs<float> &, cudaStream_t);
template void launch_static_copy<double>(const StepArgs<double> &, cudaStream_t);
template void launch_static_copy<float>(const StepArgs<float> &, cudaStream_t);
template void launch_flux_bulk<double>(const StepArgs<double> &, cudaStream_t);
template void launch_flux_bulk<float>(const StepArgs<float> &, cudaStream_t);
