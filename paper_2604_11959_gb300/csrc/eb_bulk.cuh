// eb_bulk.cuh -- the geometry-free bulk march of the flux divergence and
// update (Eqs. update-cc / update-fc with alpha = beta = 1), shared by the
// bulk kernel (eb_fast.cu) and the persistent ensemble kernel (eb_step.cu).
//
// (Eqs. update-cc / update-fc with alpha = beta = 1), for every CV at or
// above its column's kfast level, where every CV any flux stencil reads is a
// regular CV.
//
// Work split.  The domain is cut into tiles of TX x TY columns; a tile's work
// is the levels from its lowest kfast to the top, cut into slabs at the same
// levels for every tile.  One CTA marches one (tile, slab) piece; the pieces
// are launched slab by slab so that neighbouring tiles march the same levels
// at the same time and their halo reads hit L2 (built once per geometry on
// the host).
//
// One march over levels [kb, ke) of a tile.  Each thread owns two adjacent
// columns (x = 2t, 2t + 1 of the tile) and processes them as a pair: float2
// shared-memory and global accesses and, on the float path, the packed
// FP32x2 arithmetic of sm_100+ (__ffma2_rn / __fadd2_rn / __fmul2_rn).  Per
// level p of the march (the level whose primitives are formed):
//   phase 1: the primitive plane of level p (theta, u, v, w; halo 2) from
//            raw planes p and p - 1 (shared ring of five raw levels, filled
//            by asynchronous 16-byte copies two levels ahead);
//   barrier; the raw plane of level p + 2 is requested;
//   phase 2a: the x / y face fluxes of level p of the four advected
//            quantities, once per face, into shared face planes;
//   barrier;
//   phase 2b: the x / y part of each CV's divergence at level p (kept for
//            two levels), the z flux through the top of level k = p - 2 from
//            a window of the thread's own columns (levels p - 3 .. p), and
//            the update of level k.
// On the float path the window, the two pending x / y parts and the carried
// bottom z fluxes (58 words per thread) live in tensor memory between the
// levels that use them: shared memory is full with the ring, and in
// registers they would hold 58 of the 128 a thread has at two CTAs per SM
// through every phase.  Each level stores its new window level and x / y
// part and reloads the rest in one batch before the z step (tcgen05.st /
// tcgen05.ld, 32x32b shapes: TMEM lane = the thread's lane).  The double
// path keeps them in registers.
// Every field is read from HBM once per level (halo re-reads hit L2) and
// written once.  Advective face fluxes carry a factor 6 that the divergence
// removes with 1/(6 dx).
#pragma once

#include "eb_step.cuh"

#include <type_traits>

namespace bulk {

// ---- asynchronous global -> shared copies ---------------------------------
__device__ inline unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int BYTES>
__device__ inline void copy_async(void *dst, const void *src) {
  const size_t g = __cvta_generic_to_global(src);
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(g) : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(dst)), "l"(g), "n"(BYTES)
                 : "memory");
  }
}
__device__ inline void copy_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void copy_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ---- tensor memory as per-thread storage (float path) -----------------------
// The z window of a thread's own columns, the carried x / y divergence parts
// and the carried bottom z fluxes live in tensor memory between the levels
// that use them: TMEM lane = the thread's lane in its warp's lane quarter,
// 64 columns per warp (two warps per quarter).
__device__ inline void tm_alloc(unsigned *dst, unsigned ncols) {   // one whole warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ inline void tm_dealloc(unsigned taddr, unsigned ncols) {   // one whole warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ inline void tm_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ inline void tm_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ inline void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
__device__ inline void tm_st8(unsigned taddr, float2 a, float2 b, float2 c, float2 d) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
               "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(b.x)),
               "r"(__float_as_uint(b.y)), "r"(__float_as_uint(c.x)), "r"(__float_as_uint(c.y)),
               "r"(__float_as_uint(d.x)), "r"(__float_as_uint(d.y))
               : "memory");
}
__device__ inline void tm_st2(unsigned taddr, float2 a) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};\n" ::"r"(taddr), "r"(__float_as_uint(a.x)),
               "r"(__float_as_uint(a.y))
               : "memory");
}
// window levels at a0, a1, a2 (8 words each), x / y parts at aq (8), bottom
// fluxes at az (10): after any pending stores, loaded and waited for
__device__ inline void tm_load_z(unsigned a0, unsigned a1, unsigned a2, unsigned aq, unsigned az, unsigned o[42]) {
  asm volatile(
      "tcgen05.wait::st.sync.aligned;\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%42];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%43];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16, %17, %18, %19, %20, %21, %22, %23}, [%44];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%24, %25, %26, %27, %28, %29, %30, %31}, [%45];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%32, %33, %34, %35, %36, %37, %38, %39}, [%46];\n"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%40, %41}, [%47];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]),
        "=r"(o[7]), "=r"(o[8]), "=r"(o[9]), "=r"(o[10]), "=r"(o[11]), "=r"(o[12]), "=r"(o[13]),
        "=r"(o[14]), "=r"(o[15]), "=r"(o[16]), "=r"(o[17]), "=r"(o[18]), "=r"(o[19]), "=r"(o[20]),
        "=r"(o[21]), "=r"(o[22]), "=r"(o[23]), "=r"(o[24]), "=r"(o[25]), "=r"(o[26]), "=r"(o[27]),
        "=r"(o[28]), "=r"(o[29]), "=r"(o[30]), "=r"(o[31]), "=r"(o[32]), "=r"(o[33]), "=r"(o[34]),
        "=r"(o[35]), "=r"(o[36]), "=r"(o[37]), "=r"(o[38]), "=r"(o[39]), "=r"(o[40]), "=r"(o[41])
      : "r"(a0), "r"(a1), "r"(a2), "r"(aq), "r"(az), "r"(az + 8u)
      : "memory");
}
__device__ inline float2 w2(const unsigned *o, int q) {
  return make_float2(__uint_as_float(o[q]), __uint_as_float(o[q + 1]));
}

// ---- pairs of adjacent columns ----------------------------------------------
template <typename T>
struct PairOf;
template <>
struct PairOf<float> {
  using type = float2;
};
template <>
struct PairOf<double> {
  using type = double2;
};

__device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
template <typename T>
__device__ inline typename PairOf<T>::type splat(T a) {
  return mk(a, a);
}

// correctly rounded elementwise operations (packed on the float path)
__device__ inline float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ inline double2 padd(double2 a, double2 b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
__device__ inline float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ inline double2 pmul(double2 a, double2 b) { return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)); }
__device__ inline float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ inline double2 pfma(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
// a - b, rounded once (the product -1 * b is exact)
__device__ inline float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ inline double2 psub(double2 a, double2 b) { return make_double2(__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)); }
// elementwise reciprocal: the fast approximate one on the float path
__device__ inline float2 prcp(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
__device__ inline double2 prcp(double2 a) { return make_double2(1.0 / a.x, 1.0 / a.y); }
template <typename P>
__device__ inline P psel_pos(P m, P a, P b) {   // a where m > 0, else b
  return mk(m.x > 0 ? a.x : b.x, m.y > 0 ? a.y : b.y);
}

__device__ inline float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ inline double2 ld2(const double *p) { return *reinterpret_cast<const double2 *>(p); }
__device__ inline void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ inline void st2(double *p, double2 v) { *reinterpret_cast<double2 *>(p) = v; }

// 6 * m * (third-order upwind face value) for two faces, each between b and
// c with far values a (low side) and d (high side): m > 0 takes
// (5b + 2c - a), m < 0 takes (5c + 2b - d), or the centred 3(b + c) when the
// far high CV does not exist (Sec. 4.1).
template <typename P>
__device__ inline P flux6(P m, P a, P b, P c, P d, bool has_d = true) {
  using T = decltype(m.x);
  const P two = splat(T(2)), five = splat(T(5)), mone = splat(T(-1));
  const P vp = pfma(b, five, pfma(a, mone, pmul(c, two)));
  const P vn = has_d ? pfma(c, five, pfma(d, mone, pmul(b, two))) : pmul(padd(b, c), splat(T(3)));
  return pmul(m, psel_pos(m, vp, vn));
}

// Tile of the bulk march: TX x TY columns (TY = 16, or 14 so that a 256-row
// domain cuts into 19 tile rows and two slabs of 152 tiles fill every SM
// with two CTAs).
template <typename T, int TY_ = 16>
struct BulkTile {
  static constexpr int TX = 32, TY = TY_;    // columns and rows of a tile
  static constexpr int NPX = TX / 2;         // column pairs per row (threads per row)
  static constexpr int NT = NPX * TY;        // threads
  static constexpr int HX = 4;               // raw halo in x on both sides (16-byte aligned rows)
  static constexpr int PX = TX + 2 * HX;     // raw row: x = -4 .. TX + 3
  static constexpr int PY = TY + 5;          // raw rows: y = -3 .. TY + 1
  static constexpr int NP = PX * PY;         // one raw plane of one field
  static constexpr int SLOTS = 5;            // raw levels p - 2 .. p + 2
  static constexpr int QX = TX + 4;          // primitive row: x = -2 .. TX + 1
  static constexpr int QY = TY + 4;          // primitive rows: y = -2 .. TY + 1
  static constexpr int NQ = QX * QY;
  static constexpr int NQP = NQ / 2;         // primitive pairs
  static constexpr int FXW = NPX + 1;        // x faces at even x = 0, 2, .., TX of a row
  static constexpr int NFX = FXW * TY, NFY = TX * (TY + 1);
  static constexpr int RAW = SLOTS * 5 * NP;
  static constexpr int PRIM = 4 * NQ;
  static constexpr size_t BYTES = sizeof(T) * (size_t)(RAW + PRIM + 4 * NFX + 4 * NFY);
  static constexpr int QR = (NQP + NT - 1) / NT;   // primitive pairs per thread
  __device__ static constexpr int ri(int x, int y) { return (y + 3) * PX + (x + HX); }
  __device__ static constexpr int qi(int x, int y) { return (y + 2) * QX + (x + 2); }
};

// V elements per asynchronous copy: 16 bytes when every row of every field
// starts on a 16-byte boundary (then pairs are also stored as one access),
// else one element.
// Where a thread's carried state lives between the levels that use it:
// tensor memory on the float path of the bulk kernel, registers otherwise
// (the double path, and every path inside a cooperative launch, whose
// co-residency check counts a CTA that allocates tensor memory as filling
// its SM).  The arithmetic is the same either way.
template <typename T>
__host__ __device__ constexpr bool bulk_tmem_default() {
  return sizeof(T) == sizeof(float);
}

// Tensor memory of a CTA for the carried state: 128 columns allocated by
// warp 0; returns this thread's base address (lane = the thread's lane in
// its warp's quarter, 64 columns per warp).  Without TM nothing is
// allocated.
template <typename T, bool TM = bulk_tmem_default<T>()>
__device__ inline unsigned bulk_tmem_begin(unsigned *slot) {
  if constexpr (TM) {
    const int tid = threadIdx.y * BulkTile<T>::NPX + threadIdx.x;
    if (tid < 32) tm_alloc(slot, 128u);
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    return *slot + ((unsigned)(32 * ((tid >> 5) & 3)) << 16) + 64u * (unsigned)(tid >> 7);
  } else {
    return 0u;
  }
}

// Releases what bulk_tmem_begin allocated (every thread of the CTA calls it).
template <typename T, bool TM = bulk_tmem_default<T>()>
__device__ inline void bulk_tmem_end(unsigned *slot) {
  if constexpr (TM) {
    const int tid = threadIdx.y * BulkTile<T>::NPX + threadIdx.x;
    tm_wait_st();
    tm_fence_before();
    __syncthreads();
    tm_fence_after();
    if (tid < 32) tm_dealloc(*slot, 128u);
  }
}

// One march of the CTA over the levels [sg.y, sg.z) of tile sg.x (tiles of
// TYV rows).  smem_bytes holds BulkTile<T, TYV>::BYTES of dynamic shared
// memory, tbase is this thread's
// tensor-memory base (bulk_tmem_begin), and bad turns NaN when a written
// value is not finite.  Every thread of the CTA calls it.
template <typename T, int V, bool TM = bulk_tmem_default<T>(), int TYV = 16>
__device__ __forceinline__ void bulk_march(const StepArgs<T> &A, const int4 sg, unsigned char *smem_bytes,
                                           const unsigned tbase, typename PairOf<T>::type &bad) {
  using TL = BulkTile<T, TYV>;
  using P = typename PairOf<T>::type;
  constexpr int TX = TL::TX, TY = TL::TY, NPX = TL::NPX, NT = TL::NT, PX = TL::PX, NP = TL::NP, QX = TL::QX,
                NQ = TL::NQ;
  constexpr int GX = PX / V, NPOS = GX * TL::PY, CR = (NPOS + NT - 1) / NT;
  constexpr int CB = (int)(V * sizeof(T));
  constexpr bool PAIRIO = V > 1;
  static_assert(PX % V == 0, "raw rows must split into whole copies");
  static_assert(NPX >= TY, "one row of threads computes the faces on the high x edge");
  T *raw = reinterpret_cast<T *>(smem_bytes);
  T *prim = raw + TL::RAW;
  T *FX = prim + TL::PRIM;
  T *FY = FX + 4 * TL::NFX;

  const Dims &D = A.D;
  const int nz = D.nz;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * NPX + tx;
  const int tiles_x = (D.nx + TX - 1) / TX;
  const T idx = T(D.idx), idy = T(D.idy), idz = T(D.idz);
  const T idx6 = T(D.idx / 6.0), idy6 = T(D.idy / 6.0), idz6 = T(D.idz / 6.0);
  const P half = splat(T(0.5)), zero = splat(T(0));
  const bool same_base = A.base[0] != nullptr && A.base[0] == A.src.f[0] && A.base[1] == A.src.f[1] &&
                         A.base[2] == A.src.f[2] && A.base[3] == A.src.f[3] && A.base[4] == A.src.f[4];
  const int self = TL::ri(2 * tx, ty);

  auto RAWP = [&](int L) -> const T * { return raw + (L % TL::SLOTS) * 5 * NP; };


  const int tile = sg.x, kbeg = sg.y, kend = sg.z;   // kbeg >= 3 (kfast >= 3)
  const int i0 = (tile % tiles_x) * TX, j0 = (tile / tiles_x) * TY;
  const int i = i0 + 2 * tx, j = j0 + ty;
  const bool jin = j < D.ny;
  const int kfx = (jin && i < D.nx) ? A.kfast[i + D.nx * j] : nz;
  const int kfy = (jin && i + 1 < D.nx) ? A.kfast[i + 1 + D.nx * j] : nz;

  // copy plan: raw-plane positions this thread requests every level
  int cpos_s[CR], cpos_g[CR];
#pragma unroll
  for (int r = 0; r < CR; ++r) {
    const int q = tid + r * NT;
    cpos_s[r] = -1;
    cpos_g[r] = 0;
    if (q < NPOS) {
      const int row = q / GX, gx = q % GX;
      const int x = wrapmod(i0 - TL::HX + gx * V, D.nx), y = wrapmod(j0 - 3 + row, D.ny);
      cpos_s[r] = row * PX + gx * V;
      cpos_g[r] = x + D.nx * y;
    }
  }
  auto request = [&](int L) {
    if (L >= 0 && L < nz) {
      T *Pl = raw + (L % TL::SLOTS) * 5 * NP;
      const long long off = D.nxy * L;
#pragma unroll
      for (int r = 0; r < CR; ++r) {
        if (cpos_s[r] < 0) continue;
#pragma unroll
        for (int f = 0; f < 5; ++f) copy_async<CB>(Pl + f * NP + cpos_s[r], A.src.f[f] + off + cpos_g[r]);
      }
    }
    copy_commit();
  };
  // primitive pairs of this thread: raw index (the pair's shared index is 2q)
  int qraw[TL::QR];
#pragma unroll
  for (int r = 0; r < TL::QR; ++r) {
    const int q = tid + r * NT;
    qraw[r] = q < TL::NQP ? TL::ri(2 * (q % (QX / 2)) - 2, q / (QX / 2) - 2) : -1;
  }

  // face fluxes (x 6) through the low x and y faces of the column pair at
  // even tile x, row y of level p, all four grids: each momentum and
  // primitive value is read from shared memory once
  auto faces = [&](const T *Rk, const T *Rkm, int x, int y, T ru, T rv, T rum, T rvm, P fxo[4], P fyo[4]) {
    const int c = TL::ri(x, y);
    const T *U = Rk + 2 * NP, *Vv = Rk + 3 * NP;
    const P pru = splat(ru), prv = splat(rv);
    const P uc = padd(ld2(U + c), pru), ul = padd(ld2(U + c - 2), pru), ud = padd(ld2(U + c - PX), pru),
            ub = padd(ld2(Rkm + 2 * NP + c), splat(rum));
    const P vc = padd(ld2(Vv + c), prv), vl = padd(ld2(Vv + c - 2), prv), vd = padd(ld2(Vv + c - PX), prv),
            vkm = padd(ld2(Rkm + 3 * NP + c), splat(rvm));
    const P mx[4] = {uc, pmul(padd(mk(ul.y, uc.x), uc), half), pmul(padd(ud, uc), half), pmul(padd(ub, uc), half)};
    const P my[4] = {vc, pmul(padd(mk(vl.y, vc.x), vc), half), pmul(padd(vd, vc), half), pmul(padd(vkm, vc), half)};
#pragma unroll
    for (int G = 0; G < 4; ++G) {
      const T *Q = prim + G * NQ + TL::qi(x, y);
      const P pc = ld2(Q), pl = ld2(Q - 2), pr = ld2(Q + 2);
      fxo[G] = flux6(mx[G], pl, mk(pl.y, pc.x), pc, mk(pc.y, pr.x));
      fyo[G] = flux6(my[G], ld2(Q - 2 * QX), ld2(Q - QX), pc, ld2(Q + QX));
    }
  };
  // per-level profiles: stored with four zero levels on both sides, so the
  // levels -4 .. nz + 3 the march touches read without bounds checks
  auto ref_r = [&](int L) -> T { return A.src.ref_rho[L]; };
  auto ref_u = [&](int L) -> T { return A.src.ref_u[L]; };
  auto ref_v = [&](int L) -> T { return A.src.ref_v[L]; };
  auto bg = [&](const T *b, int L) -> T { return b[L]; };
  const int p0 = kbeg - 2, p1 = kend + 1;
  T rr_m = ref_r(p0 - 1), rr_p = ref_r(p0);
  T ru_m = ref_u(p0 - 1), ru_p = ref_u(p0), rv_m = ref_v(p0 - 1), rv_p = ref_v(p0);
  T bt_p = bg(A.src.bg_t, p0), bu_p = bg(A.src.bg_u, p0), bv_p = bg(A.src.bg_v, p0);

  // prologue: raw levels p0 - 1, p0 landed, p0 + 1 in flight
  request(p0 - 1);
  request(p0);
  request(p0 + 1);
  copy_wait<1>();
  __syncthreads();

  // own-column primitive window (levels p - 3 .. p), carried bottom fluxes,
  // and the x / y divergence parts of levels p - 2, p - 1
  P th[4], uu[4], vv[4], ww[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) th[q] = uu[q] = vv[q] = ww[q] = zero;
  P zc_m = zero, zc_t = zero, zu = zero, zv = zero, zw = zero;
  P q0[4], q1[4];
#pragma unroll
  for (int G = 0; G < 4; ++G) q0[G] = q1[G] = zero;
  long long cidx = (long long)i + (long long)D.nx * ((long long)j + (long long)D.ny * (p0 - 2));

  for (int p = p0; p <= p1; ++p, cidx += D.nxy) {
    const int k = p - 2;
    const T rr_n = ref_r(p + 1), ru_n = ref_u(p + 1), rv_n = ref_v(p + 1);
    const T bt_n = bg(A.src.bg_t, p + 1), bu_n = bg(A.src.bg_u, p + 1), bv_n = bg(A.src.bg_v, p + 1);
    // ---- phase 1: primitive plane of level p
    if (p < nz) {
      const T *R = RAWP(p), *Rm = RAWP(p - 1);
      const P rrp = splat(rr_p);
#pragma unroll
      for (int r = 0; r < TL::QR; ++r) {
        const int c = qraw[r];
        if (c < 0) continue;
        T *Q = prim + 2 * (tid + r * NT);
        // deviations from the level's background values: theta - theta0 =
        // (rho*theta' - theta0 rho') / rho and u - u_bg = (rho*u' - u_bg
        // rhobar') / rhobar, all from stored perturbations, so the
        // rounding scales with the deviation; w has no background
        const P rp = ld2(R + c);
        const P rho = padd(rp, rrp);
        const P rbx = pmul(padd(mk(R[c - 1], rp.x), rp), half);
        const P rby = pmul(padd(ld2(R + c - PX), rp), half);
        const P rhob = padd(ld2(Rm + c), splat(rr_m));
        st2(Q, pmul(pfma(splat(-bt_p), rp, ld2(R + NP + c)), prcp(rho)));
        st2(Q + NQ, pmul(pfma(splat(-bu_p), rbx, ld2(R + 2 * NP + c)), prcp(padd(rbx, rrp))));
        st2(Q + 2 * NQ, pmul(pfma(splat(-bv_p), rby, ld2(R + 3 * NP + c)), prcp(padd(rby, rrp))));
        st2(Q + 3 * NQ, pmul(ld2(R + 4 * NP + c), prcp(pmul(padd(rhob, rho), half))));
      }
    }
    __syncthreads();
    request(p + 2 <= p1 ? p + 2 : -1);

    // ---- phase 2a: own window; x / y faces of level p
    // (on the tensor-memory path the own values of level p stay in registers
    // for the z step: after the barrier below, other warps may already be
    // writing the primitive plane of level p + 1)
    P a0 = zero, a1 = zero, a2 = zero, a3 = zero;   // above the top: zeros (w wall level nz)
    if constexpr (TM) {
      if (p < nz) {   // full values: the z fluxes cross levels of different backgrounds
        const T *Q = prim + TL::qi(2 * tx, ty);
        a0 = padd(ld2(Q), splat(bt_p));
        a1 = padd(ld2(Q + NQ), splat(bu_p));
        a2 = padd(ld2(Q + 2 * NQ), splat(bv_p));
        a3 = ld2(Q + 3 * NQ);
      }
      __syncwarp();
      tm_st8(tbase + 8u * (unsigned)(p & 3), a0, a1, a2, a3);
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        th[q] = th[q + 1];
        uu[q] = uu[q + 1];
        vv[q] = vv[q + 1];
        ww[q] = ww[q + 1];
      }
      if (p < nz) {   // full values: the z fluxes cross levels of different backgrounds
        const T *Q = prim + TL::qi(2 * tx, ty);
        th[3] = padd(ld2(Q), splat(bt_p));
        uu[3] = padd(ld2(Q + NQ), splat(bu_p));
        vv[3] = padd(ld2(Q + 2 * NQ), splat(bv_p));
        ww[3] = ld2(Q + 3 * NQ);
      } else {
        th[3] = uu[3] = vv[3] = ww[3] = zero;   // above the top; w wall level nz
      }
    }
    const bool face_level = p >= kbeg && p < kend;
    P fx[4], fy[4];
    if (face_level) {
      const T *Rk = RAWP(p), *Rkm = RAWP(p - 1);
      faces(Rk, Rkm, 2 * tx, ty, ru_p, rv_p, ru_m, rv_m, fx, fy);
#pragma unroll
      for (int G = 0; G < 4; ++G) {
        FX[G * TL::NFX + ty * TL::FXW + tx] = fx[G].x;
        st2(FY + G * TL::NFY + ty * TX + 2 * tx, fy[G]);
      }
      if (ty <= 1) {   // faces on the high y edge of the tile: row ty takes grids 2 ty, 2 ty + 1
        const int G0 = 2 * ty;
        const int c = TL::ri(2 * tx, TY);
        const T *Vv = Rk + 3 * NP;
        const P prv = splat(rv_p);
        const P vc = padd(ld2(Vv + c), prv);
        const P mA = ty ? pmul(padd(padd(ld2(Vv + c - PX), prv), vc), half) : vc;
        const P mB =
            pmul(padd(ty ? padd(ld2(Rkm + 3 * NP + c), splat(rv_m)) : mk(Vv[c - 1] + rv_p, vc.x), vc), half);
        const T *Q = prim + G0 * NQ + TL::qi(2 * tx, TY);
        const P fA = flux6(mA, ld2(Q - 2 * QX), ld2(Q - QX), ld2(Q), ld2(Q + QX));
        Q += NQ;
        const P fB = flux6(mB, ld2(Q - 2 * QX), ld2(Q - QX), ld2(Q), ld2(Q + QX));
        st2(FY + G0 * TL::NFY + TY * TX + 2 * tx, fA);
        st2(FY + (G0 + 1) * TL::NFY + TY * TX + 2 * tx, fB);
      } else if (ty >= TY - 2 && tx < TY) {   // faces on the high x edge of the tile (row tx): two grids per row
        const int hi = ty - (TY - 2), G0 = 2 * hi;
        const int c = TL::ri(TX, tx);
        const T *U = Rk + 2 * NP;
        const T u0 = U[c] + ru_p;
        const T mA = hi ? T(0.5) * ((U[c - PX] + ru_p) + u0) : u0;
        const T mB = T(0.5) * ((hi ? Rkm[2 * NP + c] + ru_m : U[c - 1] + ru_p) + u0);
        const T *Q = prim + G0 * NQ + TL::qi(TX, tx);
        FX[G0 * TL::NFX + tx * TL::FXW + NPX] =
            flux6(splat(mA), splat(Q[-2]), splat(Q[-1]), splat(Q[0]), splat(Q[1])).x;
        Q += NQ;
        FX[(G0 + 1) * TL::NFX + tx * TL::FXW + NPX] =
            flux6(splat(mB), splat(Q[-2]), splat(Q[-1]), splat(Q[0]), splat(Q[1])).x;
      }
    }
    copy_wait<1>();   // raw p + 1 landed (this thread's copies)
    __syncthreads();

    // ---- phase 2b: x / y divergence of level p; z flux and update of level k
    P sxy[4];
    if (face_level) {
      const P ix = splat(idx6), iy = splat(idy6);
#pragma unroll
      for (int G = 0; G < 4; ++G) {
        const P dfx = psub(mk(fx[G].y, FX[G * TL::NFX + ty * TL::FXW + tx + 1]), fx[G]);
        const P dfy = psub(ld2(FY + G * TL::NFY + (ty + 1) * TX + 2 * tx), fy[G]);
        sxy[G] = pfma(dfx, ix, pmul(dfy, iy));
      }
      // the background part of the face values: bg times the x / y mass
      // divergence of each grid's CV, from differences of the stored
      // momenta of level p (the profiles cancel within a level)
      {
        const T *Rk = RAWP(p);
        const T *U = Rk + 2 * NP + self, *Vv = Rk + 3 * NP + self;
        const P u0 = ld2(U), u1 = mk(u0.y, U[2]), um = mk(U[-1], u0.x), ud0 = ld2(U - PX);
        const P ud1 = mk(ud0.y, U[2 - PX]);
        const P v0 = ld2(Vv), vu = ld2(Vv + PX), vd = ld2(Vv - PX);
        const P vl = mk(Vv[-1], v0.x), vul = mk(Vv[PX - 1], vu.x);
        const P jx = splat(idx), jy = splat(idy), hx = splat(T(0.5) * idx), hy = splat(T(0.5) * idy);
        // c grid: faces of the cell carry rho*u, rho*v themselves
        const P mc = pfma(psub(u1, u0), jx, pmul(psub(vu, v0), jy));
        // u grid: x faces at cell centres (means along x), y faces at edges (means along x of rho*v)
        const P mu = pfma(psub(u1, um), hx, pmul(psub(padd(vul, vu), padd(vl, v0)), hy));
        // v grid: x faces at edges (means along y of rho*u), y faces at cell centres
        const P mv = pfma(psub(padd(ud1, u1), padd(ud0, u0)), hx, pmul(psub(vu, vd), hy));
        sxy[0] = pfma(splat(bt_p), mc, sxy[0]);
        sxy[1] = pfma(splat(bu_p), mu, sxy[1]);
        sxy[2] = pfma(splat(bv_p), mv, sxy[2]);
      }
    } else {
#pragma unroll
      for (int G = 0; G < 4; ++G) sxy[G] = zero;
    }
    auto zstep = [&](auto H2) {
      // flux through the top of level k: masses from rho*w of levels k, k + 1
      constexpr bool has2 = decltype(H2)::value;
      const bool has1 = has2 || k + 1 <= nz - 1;
      const T *Rk = RAWP(k);
      const T *W1 = RAWP(k + 1) + 4 * NP;
      const P m = has1 ? ld2(W1 + self) : zero;
      const P mu = has1 ? pmul(padd(mk(W1[self - 1], m.x), m), half) : zero;
      const P mv = has1 ? pmul(padd(ld2(W1 + self - PX), m), half) : zero;
      const P mw = pmul(padd(ld2(Rk + 4 * NP + self), m), half);
      const P fzc = flux6(m, th[0], th[1], th[2], th[3], has2);
      const P fzu = flux6(mu, uu[0], uu[1], uu[2], uu[3], has2);
      const P fzv = flux6(mv, vv[0], vv[1], vv[2], vv[3], has2);
      const P fzw = flux6(mw, ww[0], ww[1], ww[2], ww[3], has2 || k + 2 <= nz);
      if (k >= kbeg && (k >= kfx || k >= kfy)) {
        const T *U = Rk + 2 * NP, *Vv = Rk + 3 * NP;
        const P uc = ld2(U + self);
        const P dmx = psub(mk(uc.y, U[self + 2]), uc);
        const P dmy = psub(ld2(Vv + self + PX), ld2(Vv + self));
        const P iz6 = splat(-idz6);
        P d[5];
        d[0] = pfma(dmx, splat(-idx), pfma(dmy, splat(-idy), pmul(psub(m, zc_m), splat(-idz))));
        d[1] = pfma(psub(fzc, zc_t), iz6, pmul(q0[0], splat(T(-1))));
        d[2] = pfma(psub(fzu, zu), iz6, pmul(q0[1], splat(T(-1))));
        d[3] = pfma(psub(fzv, zv), iz6, pmul(q0[2], splat(T(-1))));
        d[4] = pfma(psub(fzw, zw), iz6, pmul(q0[3], splat(T(-1))));
        const bool both = k >= kfx && k >= kfy;
        const P dtp = splat(A.dtT);
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          P o;
          if (same_base) {
            o = pfma(d[f], dtp, ld2(Rk + f * NP + self));
          } else if (A.base[0]) {
            const T *b = A.base[f] + cidx;   // element-wise: the pair may end past the last column
            o = pfma(d[f], dtp, PAIRIO ? ld2(b) : mk(k >= kfx ? b[0] : T(0), k >= kfy ? b[1] : T(0)));
          } else {
            o = d[f];
          }
          T *dst = A.out[f] + cidx;
          if (both) {
            if (PAIRIO) st2(dst, o);
            else {
              dst[0] = o.x;
              dst[1] = o.y;
            }
            bad = pfma(o, zero, bad);
          } else if (k >= kfx) {
            dst[0] = o.x;
            bad.x = fma(o.x, T(0), bad.x);
          } else {
            dst[1] = o.y;
            bad.y = fma(o.y, T(0), bad.y);
          }
        }
      }
      zc_m = m;
      zc_t = fzc;
      zu = fzu;
      zv = fzv;
      zw = fzw;
    };
    // below the top two levels the far high CV of every z stencil exists:
    // a copy of the z step without the run-time fallback selects
    if (k >= kbeg - 1) {
      if constexpr (TM) {
        unsigned o[42];
        __syncwarp();
        tm_load_z(tbase + 8u * (unsigned)((p + 1) & 3), tbase + 8u * (unsigned)((p + 2) & 3),
                  tbase + 8u * (unsigned)((p + 3) & 3), tbase + 32u + 8u * (unsigned)(p & 1), tbase + 48u, o);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          th[q] = w2(o, 8 * q);
          uu[q] = w2(o, 8 * q + 2);
          vv[q] = w2(o, 8 * q + 4);
          ww[q] = w2(o, 8 * q + 6);
        }
#pragma unroll
        for (int G = 0; G < 4; ++G) q0[G] = w2(o, 24 + 2 * G);
        zc_m = w2(o, 32);
        zc_t = w2(o, 34);
        zu = w2(o, 36);
        zv = w2(o, 38);
        zw = w2(o, 40);
        th[3] = a0;
        uu[3] = a1;
        vv[3] = a2;
        ww[3] = a3;
      }
      if (k + 2 <= nz - 1) zstep(std::true_type());
      else zstep(std::false_type());
      if constexpr (TM) {
        __syncwarp();
        tm_st8(tbase + 48u, zc_m, zc_t, zu, zv);
        tm_st2(tbase + 56u, zw);
      }
    }
    if constexpr (TM) {
      __syncwarp();
      tm_st8(tbase + 32u + 8u * (unsigned)(p & 1), sxy[0], sxy[1], sxy[2], sxy[3]);
    } else {
#pragma unroll
      for (int G = 0; G < 4; ++G) {
        q0[G] = q1[G];
        q1[G] = sxy[G];
      }
    }
    rr_m = rr_p;
    rr_p = rr_n;
    bt_p = bt_n;
    bu_p = bu_n;
    bv_p = bv_n;
    ru_m = ru_p;
    ru_p = ru_n;
    rv_m = rv_p;
    rv_p = rv_n;
  }
  copy_wait<0>();
  __syncthreads();   // the next march reuses the shared ring
}

}  // namespace bulk
