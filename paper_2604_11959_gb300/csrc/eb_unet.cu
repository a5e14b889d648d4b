// eb_unet.cu -- the warm-start network of the anelastic projection: a
// three-level 3D U-Net (channels 16 / 32 / 64, 3x3x3 convolutions with zero
// padding, 2x2x2 average pooling, 2x nearest upsampling, concatenated skips,
// 1x1 head), trained and run by the kernels below.
//
// Precision: BF16 weights (a copy of the FP32 master weights that Adam
// updates), FP32 activations, gradients and accumulation.
// Parameters are one flat vector: per layer, weights [cout][cin][k^3] then
// biases [cout].  Activations are [channels][nz][ny][nx].
//
// Convolutions run on the fifth-generation tensor cores (tcgen05.mma, BF16
// operands in shared memory, FP32 accumulators in tensor memory) as implicit
// GEMMs, with FP32 activations and gradients split into BF16 hi + lo so that
// the products keep FP32-level accuracy: the forward pass and the input
// gradient (the same convolution on the output gradient with the weights
// transposed and flipped; rows = voxels, columns = output channels, K =
// input channels x taps) and the weight gradient (rows = taps x input
// channels, columns = output channels, K = voxels).
#include "eb_handle.cuh"
#include "eb_umma.cuh"

#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

using namespace ebh;

namespace {

struct LayerSpec {
  int cin, cout, k;
};
constexpr LayerSpec kLayers[11] = {{2, 16, 3},  {16, 16, 3}, {16, 32, 3}, {32, 32, 3}, {32, 64, 3}, {64, 64, 3},
                                   {96, 32, 3}, {32, 32, 3}, {48, 16, 3}, {16, 16, 3}, {16, 1, 1}};

long long layer_w(int l) { return (long long)kLayers[l].cout * kLayers[l].cin * kLayers[l].k * kLayers[l].k * kLayers[l].k; }
long long total_params() {
  long long n = 0;
  for (int l = 0; l < 11; ++l) n += layer_w(l) + kLayers[l].cout;
  return n;
}

struct Vol {
  int nx, ny, nz;
  __host__ __device__ long long n() const { return (long long)nx * ny * nz; }
};


// ---- tensor-core convolution (forward and input gradient) ------------------
// The convolution as an implicit GEMM on the fifth-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulators in tensor memory).  A CTA
// owns 8 x 16 voxels (x, y) on TZ consecutive z-levels.  Per z-level the
// GEMM has M = 128 rows (row m = voxel (m % 8, m / 8) of the tile), N = the
// output channels (NP: 16 ... 96) and K = the input channels, 16 per chunk;
// the 27 taps add 27 products into the same accumulator.  Each tap's A
// operand is read in place from the chunk's halo: the halo holds, per group
// of 8 channels, one 16-byte row per voxel (x fastest), so the 8 voxels of a
// core matrix are 8 consecutive rows wherever the tap puts them, the next y
// row is 10 rows (160 bytes) on and the second group of 8 channels one plane
// on.  The FP32 inputs are split into BF16 hi + lo (v = hi + lo to about
// 2^-17 relative) and both parts are multiplied by the BF16 weights, so the
// products keep FP32-level accuracy.  The weights come prepacked per chunk
// as [tap][channel group][output channel][8 channels] (k_pack_all), one
// contiguous copy.  One thread issues the 54 TZ products of a chunk and
// commits them to an mbarrier; every thread waits (bounded) before the
// chunk's shared memory is refilled and before the accumulators are read.
template <int NP, int TZ>
struct ConvTile {
  static constexpr int HX = 10, HY = 18, HZ = TZ + 2;   // halo of the 8 x 16 x TZ tile
  static constexpr int HV = HX * HY * HZ;
  static constexpr int PLANE = HV * 16;                // bytes of one 8-channel group
  static constexpr int ACT = 2 * PLANE;                // hi (or lo) of a 16-channel chunk
  static constexpr int WB = 27 * 2 * NP * 16;          // the chunk's weights
  static constexpr int SMEM = 2 * ACT + WB;
  static constexpr int COLS = TZ * NP;
  static constexpr uint32_t TCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static_assert(NP % 16 == 0 && NP >= 16 && NP <= 256, "M = 128 products need N a multiple of 16 up to 256");
  static_assert(TZ % 2 == 0 && COLS <= 256, "two warp quads share the z-levels; two CTAs per SM share TMEM");
};

constexpr long long kWaitCycles = 2000000000LL;   // about one second at the maximum SM clock

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

template <int NP, int TZ, bool MASK>
__global__ void __launch_bounds__(256, 2) k_conv3_umma(const float *in, int cin, const __nv_bfloat16 *Wp,
                                                       const float *bias, float *out, int cout, Vol V, int relu,
                                                       const float *mask, int *err, int skip_commit) {
  using G = ConvTile<NP, TZ>;
  extern __shared__ __align__(16) unsigned char cv_smem[];
  __shared__ uint32_t tbase;
  __shared__ __align__(8) uint64_t mbar;
  unsigned char *s_hi = cv_smem, *s_lo = cv_smem + G::ACT, *s_w = cv_smem + 2 * G::ACT;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntx = (V.nx + 7) / 8, nty = (V.ny + 15) / 16, ntz = (V.nz + TZ - 1) / TZ;
  const int ntiles = ntx * nty * ntz, nch = (cin + 15) / 16;
  const long long N = V.n();
  if (warp == 0) umma::alloc(&tbase, G::TCOLS);
  if (tid == 0) umma::bar_init(&mbar, 1);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tm = tbase;
  // The CTA walks the (tile, chunk) steps i of its tiles blockIdx.x,
  // blockIdx.x + gridDim.x, ..., chunks innermost.  A thread owns the halo
  // items q = tid + 256 k (8 channels of one halo voxel each); their values
  // for step i + 1 are loaded into registers right after step i's products
  // are issued and stored (as hi and lo rows) once those products are done.
  constexpr int ITEMS = 2 * G::HV, IS = (ITEMS + 255) / 256;
  const int mine = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nsteps = mine * nch;
  float pv[IS][8];
  auto tile_of = [&](int i) { return (int)blockIdx.x + (i / nch) * (int)gridDim.x; };
  auto load_step = [&](int i) {
    const int tile = tile_of(i), c0 = (i % nch) * 16;
    const int x0 = (tile % ntx) * 8, y0 = ((tile / ntx) % nty) * 16, z0 = (tile / (ntx * nty)) * TZ;
#pragma unroll
    for (int k = 0; k < IS; ++k) {
      const int q = tid + 256 * k;
      const int kg = q / G::HV, h = q - kg * G::HV;
      const int hx = h % G::HX, hy = (h / G::HX) % G::HY, hz = h / (G::HX * G::HY);
      const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
      const bool inside = q < ITEMS && x >= 0 && x < V.nx && y >= 0 && y < V.ny && z >= 0 && z < V.nz;
      const float *src = in + ((long long)z * V.ny + y) * V.nx + x;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int c = c0 + kg * 8 + j;
        pv[k][j] = inside && c < cin ? src[(long long)c * N] : 0.f;
      }
    }
  };
  auto store_step = [&]() {
#pragma unroll
    for (int k = 0; k < IS; ++k) {
      const int q = tid + 256 * k;
      if (q >= ITEMS) break;
      const int kg = q / G::HV, h = q - kg * G::HV;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(pv[k][j]), h1 = __float2bfloat16_rn(pv[k][j + 1]);
        hw[j / 2] = pack_bf16(h0, h1);
        lw[j / 2] = pack_bf16(__float2bfloat16_rn(pv[k][j] - __bfloat162float(h0)),
                              __float2bfloat16_rn(pv[k][j + 1] - __bfloat162float(h1)));
      }
      *reinterpret_cast<uint4 *>(s_hi + kg * G::PLANE + h * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(s_lo + kg * G::PLANE + h * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  };
  // the accumulators of a finished tile: warps w and w + 4 read TMEM lanes
  // 32 (w % 4) ... (row m = this lane), one half of the z-levels each
  auto epilogue = [&](int tile) {
    const int x0 = (tile % ntx) * 8, y0 = ((tile / ntx) % nty) * 16, z0 = (tile / (ntx * nty)) * TZ;
    const int quad = warp & 3, half = warp >> 2;
    const int m = 32 * quad + lane;
    const int x = x0 + (m & 7), y = y0 + (m >> 3);
    const bool xy = x < V.nx && y < V.ny;
#pragma unroll
    for (int r = 0; r < TZ / 2; ++r) {
      const int rz = half * (TZ / 2) + r, z = z0 + rz;
      const long long vox = ((long long)z * V.ny + y) * V.nx + x;
      const bool live = xy && z < V.nz;
#pragma unroll
      for (int cc = 0; cc < NP; cc += 16) {
        // the mask values first (all 16 loads in flight), then the accumulators
        float mk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          mk[j] = MASK && live && cc + j < cout ? __ldg(mask + (long long)(cc + j) * N + vox) : 1.f;
        float v[16];
        umma::ld16(tm + ((uint32_t)(32 * quad) << 16) + (uint32_t)(rz * NP + cc), v);
        if (live) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int co = cc + j;
            if (co < cout) {
              float o = v[j] + (bias ? bias[co] : 0.f);
              if (relu) o = fmaxf(o, 0.f);
              if (MASK && !(mk[j] > 0.f)) o = 0.f;   // ReLU backward of the input
              out[(long long)co * N + vox] = o;
            }
          }
        }
      }
    }
  };
  bool ok = true;
  int i = 0;
  if (nsteps > 0) load_step(0);
  for (; i < nsteps; ++i) {
    const int ch = i % nch;
    if (i > 0) {   // step i - 1's products read the buffers refilled below
      ok = umma::bar_wait(&mbar, (uint32_t)((i - 1) & 1), kWaitCycles);
      ok = __syncthreads_and(ok) != 0;
      if (!ok) break;
      umma::fence_after();
      if (ch == 0) {   // step i - 1 finished a tile
        epilogue(tile_of(i - 1));
        umma::fence_before();
      }
    }
    store_step();
    if (nch > 1 || i == 0) {   // the chunk's weights (once, when there is one chunk)
      const uint4 *wsrc = reinterpret_cast<const uint4 *>(Wp) + (long long)ch * (G::WB / 16);
      for (int q = tid; q < G::WB / 16; q += 256) reinterpret_cast<uint4 *>(s_w)[q] = wsrc[q];
    }
    umma::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      // the start address sits in the low bits of a descriptor (shared
      // addresses / 16 < 2^14, so no carry): each tap adds its offset / 16
      umma::fence_after();
      constexpr uint32_t idesc = umma::idesc_bf16(128, NP);
      const uint64_t ahi = umma::sdesc(umma::smem_u32(s_hi), G::PLANE, G::HX * 16);
      const uint64_t alo = umma::sdesc(umma::smem_u32(s_lo), G::PLANE, G::HX * 16);
      const uint64_t bw = umma::sdesc(umma::smem_u32(s_w), NP * 16, 128);
#pragma unroll
      for (int rz = 0; rz < TZ; ++rz)
#pragma unroll
        for (int a = 0; a < 27; ++a) {
          const int dz = a / 9, dy = (a / 3) % 3, dx = a % 3;
          const uint64_t off = (uint64_t)(((rz + dz) * G::HY + dy) * G::HX + dx);   // 16-byte rows
          const uint64_t bo = (uint64_t)(a * 2 * NP);
          const uint32_t d = tm + (uint32_t)(rz * NP);
          umma::mma_bf16(d, ahi + off, bw + bo, idesc, (ch > 0 || a > 0) ? 1u : 0u);
          umma::mma_bf16(d, alo + off, bw + bo, idesc, 1u);
        }
      if (!(skip_commit && i == 0)) umma::commit(&mbar);   // skipped only by the failure test
    }
    if (i + 1 < nsteps) load_step(i + 1);
  }
  if (ok && nsteps > 0) {
    ok = umma::bar_wait(&mbar, (uint32_t)((nsteps - 1) & 1), kWaitCycles);
    ok = __syncthreads_and(ok) != 0;
    umma::fence_after();
    if (ok) epilogue(tile_of(nsteps - 1));
  }
  if (!ok) {
    // the last products may still be running: give them another bounded
    // wait before the tensor memory is released
    umma::bar_wait(&mbar, (uint32_t)((i - 1) & 1), kWaitCycles);
    if (tid == 0) atomicExch(err, 1);
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::dealloc(tm, G::TCOLS);
}

// 1x1 head: out[v] = b + sum_ci W[ci] in[ci][v]
__global__ void k_head(const float *in, int cin, const __nv_bfloat16 *W, const float *bias, float *out, long long N) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= N) return;
  float a = bias[0];
  for (int c = 0; c < cin; ++c) a = fmaf(__bfloat162float(W[c]), in[c * N + v], a);
  out[v] = a;
}

// head backward: dIn[ci][v] = W[ci] dy[v] where the head's (ReLU) input post[ci][v] > 0, else 0
__global__ void k_head_bwd(const float *dy, const __nv_bfloat16 *W, int cin, const float *post, float *din,
                           long long N) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= N) return;
  const float g = dy[v];
  for (int c = 0; c < cin; ++c) din[c * N + v] = post[c * N + v] > 0.f ? __bfloat162float(W[c]) * g : 0.f;
}

// sum over voxels of a[c][v] * b[v] (b may be NULL: plain sum) into out[c]
__global__ void k_chan_dot(const float *a, const float *b, int C, long long N, float *out) {
  const int c = blockIdx.y;
  float s = 0.f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
    s += a[c * N + v] * (b ? b[v] : 1.f);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? w[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out + c, s);
  }
}

// The weights of a convolution prepacked for k_conv3_umma: Wp[chunk][tap]
// [group][n][j] = the weight from input channel 16 chunk + 8 group + j to
// output channel n at that tap, zero beyond the channel counts.  flip = 0:
// the layer itself (n = output channel, W[n][c][a]); flip = 1: its input
// gradient, the convolution with transposed and flipped weights (n = the
// layer's input channel, c its output channel: W[c][n][26 - a]).
__device__ inline void pack_elem(const __nv_bfloat16 *W, int cout, int cin, int flip, int NP, __nv_bfloat16 *Wp,
                                 long long q) {
  const int j = (int)(q % 8), n = (int)((q / 8) % NP), kg = (int)((q / (8 * NP)) % 2);
  const int a = (int)((q / (16LL * NP)) % 27), chunk = (int)(q / (16LL * NP * 27));
  const int c = chunk * 16 + kg * 8 + j;
  __nv_bfloat16 w = __float2bfloat16_rn(0.f);
  if (!flip) {
    if (n < cout && c < cin) w = W[((long long)n * cin + c) * 27 + a];
  } else {
    if (n < cin && c < cout) w = W[((long long)c * cin + n) * 27 + (26 - a)];
  }
  Wp[q] = w;
}

// Every convolution's packed weights in one launch (after each change of
// the weights): job j packs the layer at w_off[j] into dst_off[j], its
// elements numbered start[j] ... start[j + 1] - 1 of the launch.
struct PackJobs {
  int n;
  long long start[20], w_off[19], dst_off[19];
  int cout[19], cin[19], flip[19], NP[19];
};

__global__ void k_pack_all(const __nv_bfloat16 *pb, __nv_bfloat16 *wp, PackJobs J) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= J.start[J.n]) return;
  int j = 0;
  while (q >= J.start[j + 1]) ++j;
  pack_elem(pb + J.w_off[j], J.cout[j], J.cin[j], J.flip[j], J.NP[j], wp + J.dst_off[j], q - J.start[j]);
}

// Weight gradient on the fifth-generation tensor cores.  For a chunk of 16
// input channels and one tap offset dz, dW[co][ci][a] = sum over voxels v of
// in[ci][v + a] dout[co][v] is a GEMM with rows m = (dy, dx, ci) (9 x 16 = 144
// rows, two M = 128 products), columns = the output channels (NP) and K = the
// voxels, 16 per product (two x-rows of 8).  The halo of a tile of 8 x 8 x 2
// voxels is held as rows of 8 x-voxels, ordered [z][y][dx copy][channel], the
// copy dx starting dx - 1 voxels from the tile: along one (z, y) the 48 rows
// (dx, ci) follow each other and the next y row continues them, so the rows
// (dy, dx, ci) of every tap of a dz are one run of 16-byte rows at a constant
// 128-byte stride per 8 rows, and the second x-row of a product is 48 rows
// (768 bytes) on.  The output gradient is held as rows of 8 x-voxels ordered
// [z][y][output channel].  Both operands are split into BF16 hi + lo and
// multiplied as hi.hi + hi.lo + lo.hi (relative error about 2^-16).  A CTA
// walks tiles blockIdx.x, blockIdx.x + gridDim.x, ..., adds every tile into
// its tensor-memory accumulators (DZN offsets dz x 2 row blocks x NP
// columns) and adds them to dW once, atomically, at the end.
template <int NP>
struct WgTile {
  static constexpr int TX = 8, TY = 8, TZ = 2, HY = TY + 2, HZ = TZ + 2, CI = 16;
  static constexpr int DZN = NP >= 64 ? 1 : 3;         // dz offsets per CTA (tensor-memory columns)
  static constexpr int ROWS = 9 * CI, NM = 2;          // used rows, M = 128 blocks
  static constexpr int PAD = NM * 128 - ROWS;          // rows the second block reads past the taps
  static constexpr int IN_ROWS = HZ * HY * 3 * CI + PAD;
  static constexpr int IN_B = IN_ROWS * 16;            // hi (or lo) of the input halo
  static constexpr int DO_B = TZ * TY * NP * 16;       // hi (or lo) of the output gradient
  static constexpr int SMEM = 2 * IN_B + 2 * DO_B;
  static constexpr int COLS = DZN * NM * NP;
  static constexpr uint32_t TCOLS = COLS <= 32 ? 32 : COLS <= 64 ? 64 : COLS <= 128 ? 128 : COLS <= 256 ? 256 : 512;
  static constexpr int STEPS = TZ * TY / 2;            // K = 16 products per tile
  static_assert(COLS <= 256, "two CTAs per SM share the tensor memory");
};

template <int NP>
__global__ void __launch_bounds__(256, 2) k_conv3_wgrad_umma(const float *in, int cin, const float *dout, int cout,
                                                             Vol V, float *dW, float *dB, int *err, int vec) {
  using G = WgTile<NP>;
  extern __shared__ __align__(16) unsigned char wg_smem[];
  __shared__ uint32_t tbase;
  __shared__ __align__(8) uint64_t mbar;
  unsigned char *i_hi = wg_smem, *i_lo = wg_smem + G::IN_B;
  unsigned char *d_hi = wg_smem + 2 * G::IN_B, *d_lo = d_hi + G::DO_B;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntx = (V.nx + G::TX - 1) / G::TX, nty = (V.ny + G::TY - 1) / G::TY, ntz = (V.nz + G::TZ - 1) / G::TZ;
  const int ntiles = ntx * nty * ntz;
  const int dz0 = blockIdx.y * G::DZN, c0 = blockIdx.z * G::CI;
  const long long N = V.n();
  if (warp == 0) umma::alloc(&tbase, G::TCOLS);
  if (tid == 0) umma::bar_init(&mbar, 1);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tm = tbase;
  // Each thread owns up to IS input rows (q = tid + 256 k) and DS output-
  // gradient rows of every tile.  Their values are loaded into registers for
  // the next tile right after the current tile's products are issued, so
  // that the loads run while the tensor core works; they are converted and
  // stored once those products have finished reading the buffers.
  constexpr int IT = G::HZ * G::HY * G::CI, IS = (IT + 255) / 256;
  constexpr int DI = G::TZ * G::TY * NP, DS = DI / 256;
  static_assert(DI % 256 == 0, "whole output-gradient rows per thread");
  float pin[IS][10], pdo[DS][8], bsum[DS];
#pragma unroll
  for (int k = 0; k < DS; ++k) bsum[k] = 0.f;
  auto load_tile = [&](int tile) {
    const int x0 = (tile % ntx) * G::TX, y0 = ((tile / ntx) % nty) * G::TY, z0 = (tile / (ntx * nty)) * G::TZ;
#pragma unroll
    for (int k = 0; k < IS; ++k) {
      const int q = tid + 256 * k;
      const int ci = q % G::CI, hy = (q / G::CI) % G::HY, hz = q / (G::CI * G::HY);
      const int y = y0 + hy - 1, z = z0 + hz - 1, c = c0 + ci;
      const bool row = q < IT && c < cin && y >= 0 && y < V.ny && z >= 0 && z < V.nz;
      const float *src = in + (long long)c * N + ((long long)z * V.ny + y) * V.nx;
      if (vec) {   // rows of a multiple of 4 values, 16-byte aligned: x0 - 4 ... x0 + 11 in four float4
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 *s4 = reinterpret_cast<const float4 *>(src + x0);
        const float4 a = row && x0 >= 4 ? __ldg(s4 - 1) : z4;
        const float4 b = row ? __ldg(s4) : z4;
        const float4 c4 = row && x0 + 4 < V.nx ? __ldg(s4 + 1) : z4;
        const float4 d = row && x0 + 8 < V.nx ? __ldg(s4 + 2) : z4;
        pin[k][0] = a.w;
        pin[k][1] = b.x, pin[k][2] = b.y, pin[k][3] = b.z, pin[k][4] = b.w;
        pin[k][5] = c4.x, pin[k][6] = c4.y, pin[k][7] = c4.z, pin[k][8] = c4.w;
        pin[k][9] = d.x;
      } else {
#pragma unroll
        for (int e = 0; e < 10; ++e) {
          const int x = x0 - 1 + e;
          pin[k][e] = row && x >= 0 && x < V.nx ? src[x] : 0.f;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < DS; ++k) {
      const int q = tid + 256 * k;
      const int co = q % NP, vy = (q / NP) % G::TY, vz = q / (NP * G::TY);
      const int y = y0 + vy, z = z0 + vz;
      const bool row = co < cout && y < V.ny && z < V.nz;
      const float *src = dout + (long long)co * N + ((long long)z * V.ny + y) * V.nx;
      if (vec) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 *s4 = reinterpret_cast<const float4 *>(src + x0);
        const float4 b = row ? __ldg(s4) : z4;
        const float4 c4 = row && x0 + 4 < V.nx ? __ldg(s4 + 1) : z4;
        pdo[k][0] = b.x, pdo[k][1] = b.y, pdo[k][2] = b.z, pdo[k][3] = b.w;
        pdo[k][4] = c4.x, pdo[k][5] = c4.y, pdo[k][6] = c4.z, pdo[k][7] = c4.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) pdo[k][e] = row && x0 + e < V.nx ? src[x0 + e] : 0.f;
      }
    }
  };
  auto store_tile = [&]() {
#pragma unroll
    for (int k = 0; k < IS; ++k) {
      const int q = tid + 256 * k;
      if (q >= IT) break;
      const int ci = q % G::CI, hzy = q / G::CI;   // hz * HY + hy
      __nv_bfloat16 h[10], l[10];
#pragma unroll
      for (int e = 0; e < 10; ++e) {
        h[e] = __float2bfloat16_rn(pin[k][e]);
        l[e] = __float2bfloat16_rn(pin[k][e] - __bfloat162float(h[e]));
      }
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {   // the copy dx starts dx - 1 voxels from the tile
        const int r = (hzy * 3 + dx) * G::CI + ci;
        *reinterpret_cast<uint4 *>(i_hi + r * 16) =
            make_uint4(pack_bf16(h[dx], h[dx + 1]), pack_bf16(h[dx + 2], h[dx + 3]),
                       pack_bf16(h[dx + 4], h[dx + 5]), pack_bf16(h[dx + 6], h[dx + 7]));
        *reinterpret_cast<uint4 *>(i_lo + r * 16) =
            make_uint4(pack_bf16(l[dx], l[dx + 1]), pack_bf16(l[dx + 2], l[dx + 3]),
                       pack_bf16(l[dx + 4], l[dx + 5]), pack_bf16(l[dx + 6], l[dx + 7]));
      }
    }
#pragma unroll
    for (int k = 0; k < DS; ++k) {
      const int q = tid + 256 * k;
      if (dB && blockIdx.y == 0 && blockIdx.z == 0) {   // bias gradient: once per tile (first dz set, chunk)
        float r = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) r += pdo[k][e];
        bsum[k] += r;
      }
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(pdo[k][e]), h1 = __float2bfloat16_rn(pdo[k][e + 1]);
        hw[e / 2] = pack_bf16(h0, h1);
        lw[e / 2] = pack_bf16(__float2bfloat16_rn(pdo[k][e] - __bfloat162float(h0)),
                              __float2bfloat16_rn(pdo[k][e + 1] - __bfloat162float(h1)));
      }
      *reinterpret_cast<uint4 *>(d_hi + q * 16) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4 *>(d_lo + q * 16) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
  };
  bool ok = true;
  int it = 0;
  if ((int)blockIdx.x < ntiles) load_tile(blockIdx.x);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    if (it > 0) {   // the previous tile's products read the buffers refilled below
      ok = umma::bar_wait(&mbar, (uint32_t)((it - 1) & 1), kWaitCycles);
      ok = __syncthreads_and(ok) != 0;
      if (!ok) break;
    }
    store_tile();
    umma::fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      // descriptors advance by their start address / 16 (one 16-byte row)
      umma::fence_after();
      constexpr uint32_t idesc = umma::idesc_bf16(128, NP);
      const uint64_t arow0 = (uint64_t)(dz0 * G::HY * 3 * G::CI);
      const uint64_t ah = umma::sdesc(umma::smem_u32(i_hi), 3 * G::CI * 16, 128) + arow0;
      const uint64_t al = umma::sdesc(umma::smem_u32(i_lo), 3 * G::CI * 16, 128) + arow0;
      const uint64_t bh = umma::sdesc(umma::smem_u32(d_hi), NP * 16, 128);
      const uint64_t bl = umma::sdesc(umma::smem_u32(d_lo), NP * 16, 128);
#pragma unroll
      for (int s = 0; s < G::STEPS; ++s) {
        const int vz = s / (G::TY / 2), vy = 2 * (s % (G::TY / 2));
        const uint64_t bo = (uint64_t)((vz * G::TY + vy) * NP);
#pragma unroll
        for (int dzi = 0; dzi < G::DZN; ++dzi)
#pragma unroll
          for (int j = 0; j < G::NM; ++j) {
            const uint64_t ao = (uint64_t)(((vz + dzi) * G::HY + vy) * 3 * G::CI + j * 128);
            const uint32_t d = tm + (uint32_t)((dzi * G::NM + j) * NP);
            umma::mma_bf16(d, ah + ao, bh + bo, idesc, (it > 0 || s > 0) ? 1u : 0u);
            umma::mma_bf16(d, ah + ao, bl + bo, idesc, 1u);
            umma::mma_bf16(d, al + ao, bh + bo, idesc, 1u);
          }
      }
      umma::commit(&mbar);
    }
    if (tile + (int)gridDim.x < ntiles) load_tile(tile + gridDim.x);
  }
  if (ok && it > 0) {
    ok = umma::bar_wait(&mbar, (uint32_t)((it - 1) & 1), kWaitCycles);
    ok = __syncthreads_and(ok) != 0;
  }
  umma::fence_after();
  if (ok && it > 0) {
    // warps w and w + 4 read TMEM lanes 32 (w % 4) ...; the two warp quads
    // take alternate accumulators
    const int quad = warp & 3, half = warp >> 2, m = 32 * quad + lane;
    for (int acc = half; acc < G::DZN * G::NM; acc += 2) {
      const int dzi = acc / G::NM, j = acc % G::NM, r = j * 128 + m;
      const int dy = r / (3 * G::CI), dx = (r / G::CI) % 3, ci = c0 + r % G::CI;
      const bool live = r < G::ROWS && ci < cin;
      const int a = (dz0 + dzi) * 9 + dy * 3 + dx;
#pragma unroll
      for (int cc = 0; cc < NP; cc += 16) {
        float v[16];
        umma::ld16(tm + ((uint32_t)(32 * quad) << 16) + (uint32_t)(acc * NP + cc), v);
        if (live) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (cc + q < cout) atomicAdd(dW + ((long long)(cc + q) * cin + ci) * 27 + a, v[q]);
        }
      }
    }
  } else if (!ok) {
    umma::bar_wait(&mbar, (uint32_t)((it - 1) & 1), kWaitCycles);
    if (tid == 0) atomicExch(err, 1);
  }
  if (dB && blockIdx.y == 0 && blockIdx.z == 0) {
#pragma unroll
    for (int k = 0; k < DS; ++k) {
      const int co = (tid + 256 * k) % NP;
      if (co < cout) atomicAdd(dB + co, bsum[k]);
    }
  }
  umma::fence_before();
  __syncthreads();
  if (warp == 0) umma::dealloc(tm, G::TCOLS);
}

// The pooling and upsampling kernels take one channel per blockIdx.y and a
// voxel of it per thread, with 32-bit index arithmetic (a network's volumes
// hold fewer than 2^31 values per channel; eb_unet_create checks).

// 2x2x2 average pool: out (C, V/2) from in (C, V)
__global__ void k_pool(const float *in, Vol V, float *out) {
  const unsigned hx = V.nx / 2, hy = V.ny / 2, hn = hx * hy * (unsigned)(V.nz / 2);
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= hn) return;
  const unsigned x = r % hx, t = r / hx, y = t % hy, z = t / hy;
  const unsigned nx = V.nx, nxy = nx * V.ny;
  const float *src = in + (size_t)blockIdx.y * nxy * V.nz + (2 * z) * nxy + (2 * y) * nx + 2 * x;
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 8; ++a) s += src[(a >> 2) * nxy + ((a >> 1) & 1) * nx + (a & 1)];
  out[(size_t)blockIdx.y * hn + r] = s * 0.125f;
}

// din (C, V) += pool backward of dout (C, V/2), then zeroed where post (C, V)
// (the ReLU output the gradient belongs to) is not positive
__global__ void k_pool_bwd_add(const float *dout, Vol V, const float *post, float *din) {
  const unsigned n = (unsigned)V.nx * V.ny * V.nz;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const unsigned x = r % V.nx, t = r / V.nx, y = t % V.ny, z = t / V.ny;
  const unsigned hx = V.nx / 2, hy = V.ny / 2, hn = hx * hy * (unsigned)(V.nz / 2);
  const size_t q = (size_t)blockIdx.y * n + r;
  const float g = din[q] + 0.125f * dout[(size_t)blockIdx.y * hn + ((z / 2) * hy + y / 2) * hx + x / 2];
  din[q] = post[q] > 0.f ? g : 0.f;
}

// out (C, V) = nearest upsampling of in (C, V/2)
__global__ void k_up(const float *in, Vol V, float *out) {
  const unsigned n = (unsigned)V.nx * V.ny * V.nz;
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const unsigned x = r % V.nx, t = r / V.nx, y = t % V.ny, z = t / V.ny;
  const unsigned hx = V.nx / 2, hy = V.ny / 2, hn = hx * hy * (unsigned)(V.nz / 2);
  out[(size_t)blockIdx.y * n + r] = in[(size_t)blockIdx.y * hn + ((z / 2) * hy + y / 2) * hx + x / 2];
}

// din (C, V/2) = upsampling backward of dout (C, V): sum of the 8 children,
// zeroed where post (C, V/2) (the ReLU output upsampled) is not positive
__global__ void k_up_bwd(const float *dout, Vol V, const float *post, float *din) {
  const unsigned hx = V.nx / 2, hy = V.ny / 2, hn = hx * hy * (unsigned)(V.nz / 2);
  const unsigned r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= hn) return;
  const unsigned x = r % hx, t = r / hx, y = t % hy, z = t / hy;
  const unsigned nx = V.nx, nxy = nx * V.ny;
  const float *src = dout + (size_t)blockIdx.y * nxy * V.nz + (2 * z) * nxy + (2 * y) * nx + 2 * x;
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < 8; ++a) s += src[(a >> 2) * nxy + ((a >> 1) & 1) * nx + (a & 1)];
  const size_t q = (size_t)blockIdx.y * hn + r;
  din[q] = post[q] > 0.f ? s : 0.f;
}

// masked half mean-square loss: dy = mask (y - t) / sum(mask); loss sums
// (cnt: the number of voxels the mask selects)
__global__ void k_loss(const float *y, const float *t, const float *mask, long long N, const float *cnt, float *dy,
                       float *loss) {
  const float inv_n = 1.f / fmaxf(*cnt, 1.f);
  float s = 0.f;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x) {
    const float e = mask[v] > 0.f ? y[v] - t[v] : 0.f;
    dy[v] = e * inv_n;
    s += 0.5f * e * e * inv_n;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? w[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(loss, s);
  }
}

__global__ void k_adam(float *p, float *m, float *v, const float *g, __nv_bfloat16 *pb, long long n, float lr,
                       float c1, float c2) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float gq = g[q];
  const float mq = 0.9f * m[q] + 0.1f * gq;
  const float vq = 0.999f * v[q] + 0.001f * gq * gq;
  m[q] = mq;
  v[q] = vq;
  const float pq = p[q] - lr * (mq * c1) / (sqrtf(vq * c2) + 1e-8f);
  p[q] = pq;
  pb[q] = __float2bfloat16_rn(pq);
}

__global__ void k_to_bf16(const float *p, __nv_bfloat16 *pb, long long n) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) pb[q] = __float2bfloat16_rn(p[q]);
}

inline unsigned nblk(long long n, int b = 256) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct eb_unet_s {
  Vol V[3];
  long long np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16 *pb = nullptr, *wp = nullptr;   // working weights, one convolution's packed weights
  int *err = nullptr;                            // set when a bounded device wait expired
  int fault = 0;                                 // failure test: the next convolution skips its commit
  long long wp_off[10][2];                       // packed weights: forward, input gradient
  long long off_w[11], off_b[11];
  // activations (forward) and their gradients
  float *e1a, *e1, *p1, *e2a, *e2, *p2, *ba, *bt, *c2, *d2a, *d2, *c1, *d1a, *d1, *y;
  float *ge1a, *ge1, *gp1, *ge2a, *ge2, *gp2, *gba, *gbt, *gc2, *gd2a, *gd2, *gc1, *gd1a, *gd1, *gy;
  float *loss = nullptr;
  bool grads = false;
  int t = 0;   // Adam steps taken
  std::vector<void *> allocs;
  template <typename P>
  cudaError_t alloc(P **q, long long n) {
    cudaError_t e = cudaMalloc((void **)q, sizeof(P) * (size_t)std::max(1LL, n));
    if (e == cudaSuccess) allocs.push_back(*q);
    return e;
  }
  void release() {
    for (void *q : allocs) cudaFree(q);
    allocs.clear();
  }
};

namespace {

// packed weights of one convolution: chunks x 27 taps x 2 groups x NP x 8
long long packed_size(int cin, int cout) { return (long long)((cin + 15) / 16) * 27 * 2 * ((cout + 15) / 16 * 16) * 8; }

template <int NP, int TZ, bool MASK>
void conv3_umma_launch(const float *in, int cin, const __nv_bfloat16 *Wp, const float *bias, float *out, int cout,
                       const Vol &V, bool relu, const float *mask, int *err, int skip_commit, cudaStream_t s) {
  using G = ConvTile<NP, TZ>;
  static unsigned long long attr = 0;
  ebk_smem_limit(k_conv3_umma<NP, TZ, MASK>, G::SMEM, attr);
  const int sms = ebk_sm_count();
  const int tiles = ((V.nx + 7) / 8) * ((V.ny + 15) / 16) * ((V.nz + TZ - 1) / TZ);
  const int grid = std::max(1, std::min(tiles, 2 * sms));   // persistent: two CTAs per SM walk the tiles
  k_conv3_umma<NP, TZ, MASK><<<grid, 256, G::SMEM, s>>>(in, cin, Wp, bias, out, cout, V, relu ? 1 : 0, mask, err,
                                                    skip_commit);
}

// out (cout, V) = conv of in (cin, V) with the packed weights Wp (a layer's
// own, or its transposed and flipped ones for an input gradient); mask:
// where not NULL, out is zeroed wherever mask (cout, V) is not positive (the
// ReLU backward of the layer below)
void conv3_tc(eb_unet u, const float *in, int cin, const __nv_bfloat16 *Wp, const float *bias, float *out, int cout,
              const Vol &V, bool relu, const float *mask, cudaStream_t s) {
  const int NP = (cout + 15) / 16 * 16;
  const int skip = u->fault;   // the failure test: one launch never signals its products' completion
  u->fault = 0;
  // the combinations the network uses: forward passes without a mask, input
  // gradients with one where a ReLU lies below the layer
  if (mask) {
    switch (NP) {
      case 16: conv3_umma_launch<16, 2, true>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
      case 32: conv3_umma_launch<32, 2, true>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
      default: conv3_umma_launch<64, 2, true>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
    }
  } else {
    switch (NP) {
      case 16: conv3_umma_launch<16, 2, false>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
      case 32: conv3_umma_launch<32, 2, false>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
      case 48: conv3_umma_launch<48, 2, false>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
      case 64: conv3_umma_launch<64, 2, false>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
      default: conv3_umma_launch<96, 2, false>(in, cin, Wp, bias, out, cout, V, relu, mask, u->err, skip, s); break;
    }
  }
}

void conv3(eb_unet u, int l, const float *in, float *out, const Vol &V, bool relu, cudaStream_t s) {
  const LayerSpec &L = kLayers[l];
  conv3_tc(u, in, L.cin, u->wp + u->wp_off[l][0], u->p + u->off_b[l], out, L.cout, V, relu, nullptr, s);
}

// the input gradients that carry a ReLU mask (layers 1, 3, 5, 7, 9) have 16,
// 32 or 64 output channels: the masked kernels instantiated above
static_assert(kLayers[1].cin == 16 && kLayers[3].cin == 32 && kLayers[5].cin == 64 && kLayers[7].cin == 32 &&
                  kLayers[9].cin == 16,
              "masked input gradients need 16, 32 or 64 channels");

// input gradient of layer l: din = conv of dout with flipped, transposed W,
// zeroed where mask (the layer's ReLU input, when there is one) is not positive
void conv3_dgrad(eb_unet u, int l, const float *dout, float *din, const float *mask, const Vol &V, cudaStream_t s) {
  const LayerSpec &L = kLayers[l];
  conv3_tc(u, dout, L.cout, u->wp + u->wp_off[l][1], nullptr, din, L.cin, V, false, mask, s);
}

// every convolution's packed weights from the BF16 working weights
void pack_weights(eb_unet u, cudaStream_t s) {
  PackJobs J{};
  for (int l = 0; l < 10; ++l)
    for (int dir = 0; dir < (l == 0 ? 1 : 2); ++dir) {
      const LayerSpec &L = kLayers[l];
      const int j = J.n++;
      J.w_off[j] = u->off_w[l];
      J.dst_off[j] = u->wp_off[l][dir];
      J.cout[j] = L.cout;
      J.cin[j] = L.cin;
      J.flip[j] = dir;
      J.NP[j] = ((dir ? L.cin : L.cout) + 15) / 16 * 16;
      J.start[j + 1] = J.start[j] + (dir ? packed_size(L.cout, L.cin) : packed_size(L.cin, L.cout));
    }
  k_pack_all<<<nblk(J.start[J.n]), 256, 0, s>>>(u->pb, u->wp, J);
}

template <int NP>
void conv3_wgrad_launch(const float *in, int cin, const float *dout, int cout, const Vol &V, float *dW, float *dB,
                        int *err, cudaStream_t s) {
  using G = WgTile<NP>;
  static unsigned long long attr = 0;
  ebk_smem_limit(k_conv3_wgrad_umma<NP>, G::SMEM, attr);
  const int sms = ebk_sm_count();
  const int ntiles = ((V.nx + G::TX - 1) / G::TX) * ((V.ny + G::TY - 1) / G::TY) * ((V.nz + G::TZ - 1) / G::TZ);
  const int gy = 3 / G::DZN, gz = (cin + G::CI - 1) / G::CI;
  const int gx = std::max(1, std::min(ntiles, 2 * sms / (gy * gz)));   // two CTAs per SM, each over many tiles
  // float4 loads where every row starts on a 16-byte boundary
  const int vec = V.nx % 4 == 0 && (uintptr_t)in % 16 == 0 && (uintptr_t)dout % 16 == 0;
  k_conv3_wgrad_umma<NP><<<dim3(gx, gy, gz), 256, G::SMEM, s>>>(in, cin, dout, cout, V, dW, dB, err, vec);
}

void conv3_wgrad(eb_unet u, int l, const float *in, const float *dout, const Vol &V, cudaStream_t s) {
  const LayerSpec &L = kLayers[l];
  float *dW = u->g + u->off_w[l], *dB = u->g + u->off_b[l];   // the bias gradient rides along
  if (L.cout <= 16) conv3_wgrad_launch<16>(in, L.cin, dout, L.cout, V, dW, dB, u->err, s);
  else if (L.cout <= 32) conv3_wgrad_launch<32>(in, L.cin, dout, L.cout, V, dW, dB, u->err, s);
  else conv3_wgrad_launch<64>(in, L.cin, dout, L.cout, V, dW, dB, u->err, s);
}

void forward(eb_unet u, const float *x, cudaStream_t s) {
  const Vol &V0 = u->V[0], &V1 = u->V[1], &V2 = u->V[2];
  conv3(u, 0, x, u->e1a, V0, true, s);
  conv3(u, 1, u->e1a, u->e1, V0, true, s);
  k_pool<<<dim3(nblk(V1.n()), 16), 256, 0, s>>>(u->e1, V0, u->p1);
  conv3(u, 2, u->p1, u->e2a, V1, true, s);
  conv3(u, 3, u->e2a, u->e2, V1, true, s);
  k_pool<<<dim3(nblk(V2.n()), 32), 256, 0, s>>>(u->e2, V1, u->p2);
  conv3(u, 4, u->p2, u->ba, V2, true, s);
  conv3(u, 5, u->ba, u->bt, V2, true, s);
  k_up<<<dim3(nblk(V1.n()), 64), 256, 0, s>>>(u->bt, V1, u->c2);
  cudaMemcpyAsync(u->c2 + 64 * V1.n(), u->e2, sizeof(float) * 32 * V1.n(), cudaMemcpyDeviceToDevice, s);
  conv3(u, 6, u->c2, u->d2a, V1, true, s);
  conv3(u, 7, u->d2a, u->d2, V1, true, s);
  k_up<<<dim3(nblk(V0.n()), 32), 256, 0, s>>>(u->d2, V0, u->c1);
  cudaMemcpyAsync(u->c1 + 32 * V0.n(), u->e1, sizeof(float) * 16 * V0.n(), cudaMemcpyDeviceToDevice, s);
  conv3(u, 8, u->c1, u->d1a, V0, true, s);
  conv3(u, 9, u->d1a, u->d1, V0, true, s);
  k_head<<<nblk(V0.n()), 256, 0, s>>>(u->d1, 16, u->pb + u->off_w[10], u->p + u->off_b[10], u->y, V0.n());
}

// gradient of the masked loss into u->g (zeroed first); loss into u->loss
void backward(eb_unet u, const float *x, cudaStream_t s) {
  const Vol &V0 = u->V[0], &V1 = u->V[1], &V2 = u->V[2];
  const long long n0 = V0.n(), n1 = V1.n(), n2 = V2.n();
  cudaMemsetAsync(u->g, 0, sizeof(float) * u->np, s);
  // head
  k_chan_dot<<<dim3(64, 16), 256, 0, s>>>(u->d1, u->gy, 16, n0, u->g + u->off_w[10]);
  k_chan_dot<<<dim3(64, 1), 256, 0, s>>>(u->gy, nullptr, 1, n0, u->g + u->off_b[10]);
  k_head_bwd<<<nblk(n0), 256, 0, s>>>(u->gy, u->pb + u->off_w[10], 16, u->d1, u->gd1, n0);
  conv3_wgrad(u, 9, u->d1a, u->gd1, V0, s);
  conv3_dgrad(u, 9, u->gd1, u->gd1a, u->d1a, V0, s);
  conv3_wgrad(u, 8, u->c1, u->gd1a, V0, s);
  conv3_dgrad(u, 8, u->gd1a, u->gc1, nullptr, V0, s);
  k_up_bwd<<<dim3(nblk(n1), 32), 256, 0, s>>>(u->gc1, V0, u->d2, u->gd2);
  cudaMemcpyAsync(u->ge1, u->gc1 + 32 * n0, sizeof(float) * 16 * n0, cudaMemcpyDeviceToDevice, s);
  conv3_wgrad(u, 7, u->d2a, u->gd2, V1, s);
  conv3_dgrad(u, 7, u->gd2, u->gd2a, u->d2a, V1, s);
  conv3_wgrad(u, 6, u->c2, u->gd2a, V1, s);
  conv3_dgrad(u, 6, u->gd2a, u->gc2, nullptr, V1, s);
  k_up_bwd<<<dim3(nblk(n2), 64), 256, 0, s>>>(u->gc2, V1, u->bt, u->gbt);
  cudaMemcpyAsync(u->ge2, u->gc2 + 64 * n1, sizeof(float) * 32 * n1, cudaMemcpyDeviceToDevice, s);
  conv3_wgrad(u, 5, u->ba, u->gbt, V2, s);
  conv3_dgrad(u, 5, u->gbt, u->gba, u->ba, V2, s);
  conv3_wgrad(u, 4, u->p2, u->gba, V2, s);
  conv3_dgrad(u, 4, u->gba, u->gp2, nullptr, V2, s);
  k_pool_bwd_add<<<dim3(nblk(n1), 32), 256, 0, s>>>(u->gp2, V1, u->e2, u->ge2);
  conv3_wgrad(u, 3, u->e2a, u->ge2, V1, s);
  conv3_dgrad(u, 3, u->ge2, u->ge2a, u->e2a, V1, s);
  conv3_wgrad(u, 2, u->p1, u->ge2a, V1, s);
  conv3_dgrad(u, 2, u->ge2a, u->gp1, nullptr, V1, s);
  k_pool_bwd_add<<<dim3(nblk(n0), 16), 256, 0, s>>>(u->gp1, V0, u->e1, u->ge1);
  conv3_wgrad(u, 1, u->e1a, u->ge1, V0, s);
  conv3_dgrad(u, 1, u->ge1, u->ge1a, u->e1a, V0, s);
  conv3_wgrad(u, 0, x, u->ge1a, V0, s);
}

eb_status ensure_grads(eb_unet u) {
  if (u->grads) return EB_OK;
  const long long n0 = u->V[0].n(), n1 = u->V[1].n(), n2 = u->V[2].n();
  struct {
    float **q;
    long long n;
  } b[] = {{&u->ge1a, 16 * n0}, {&u->ge1, 16 * n0}, {&u->gp1, 16 * n1}, {&u->ge2a, 32 * n1}, {&u->ge2, 32 * n1},
           {&u->gp2, 32 * n2},  {&u->gba, 64 * n2},  {&u->gbt, 64 * n2}, {&u->gc2, 96 * n1},  {&u->gd2a, 32 * n1},
           {&u->gd2, 32 * n1},  {&u->gc1, 48 * n0},  {&u->gd1a, 16 * n0}, {&u->gd1, 16 * n0}, {&u->gy, n0}};
  for (auto &e : b) CUDA_TRY(u->alloc(e.q, e.n), "alloc network gradients");
  CUDA_TRY(u->alloc(&u->g, u->np), "alloc network gradients");
  CUDA_TRY(u->alloc(&u->m, u->np), "alloc optimiser state");
  CUDA_TRY(u->alloc(&u->v, u->np), "alloc optimiser state");
  CUDA_TRY(cudaMemset(u->m, 0, sizeof(float) * u->np), "optimiser state");
  CUDA_TRY(cudaMemset(u->v, 0, sizeof(float) * u->np), "optimiser state");
  CUDA_TRY(u->alloc(&u->loss, 2), "alloc loss");   // loss, mask count
  u->grads = true;
  return EB_OK;
}

eb_status loss_and_backward(eb_unet u, const float *x, const float *target, const float *mask, float *loss,
                            cudaStream_t s) {
  eb_status st = ensure_grads(u);
  if (st != EB_OK) return st;
  const long long n0 = u->V[0].n();
  forward(u, x, s);
  CUDA_TRY(cudaMemsetAsync(u->loss, 0, 2 * sizeof(float), s), "loss");
  k_chan_dot<<<dim3(64, 1), 256, 0, s>>>(mask, nullptr, 1, n0, u->loss + 1);   // voxels the mask selects
  k_loss<<<256, 256, 0, s>>>(u->y, target, mask, n0, u->loss + 1, u->gy, u->loss);
  backward(u, x, s);
  if (loss) {
    CUDA_TRY(cudaMemcpyAsync(loss, u->loss, sizeof(float), cudaMemcpyDeviceToHost, s), "read loss");
    CUDA_TRY(cudaStreamSynchronize(s), "read loss");
  }
  return EB_OK;
}

// after the device has finished: EB_ERR_TIMEOUT (and the flag cleared) when
// a convolution gave up waiting for its tensor-core products
eb_status take_error(eb_unet u) {
  int h = 0;
  CUDA_TRY(cudaMemcpy(&h, u->err, sizeof(int), cudaMemcpyDeviceToHost), "network status");
  if (!h) return EB_OK;
  CUDA_TRY(cudaMemset(u->err, 0, sizeof(int)), "network status");
  return fail(EB_ERR_TIMEOUT, "a convolution's bounded wait for its tensor-core products expired");
}

}  // namespace

extern "C" {

int64_t eb_unet_num_params(void) { return total_params(); }

eb_status eb_unet_inject_wait_fault(eb_unet u) {
  if (!u) return fail(EB_ERR_INVALID_ARG, "NULL network");
  u->fault = 1;
  return EB_OK;
}

eb_status eb_unet_sync_status(eb_unet u) {
  if (!u) return fail(EB_ERR_INVALID_ARG, "NULL network");
  CUDA_TRY(cudaDeviceSynchronize(), "network status");
  return take_error(u);
}

eb_status eb_unet_create(int nx, int ny, int nz, eb_unet *out) {
  if (!out) return fail(EB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4)
    return fail(EB_ERR_INVALID_ARG, "nx, ny, nz must be multiples of 4 (two 2x poolings), at least 4");
  if ((long long)nx * ny * nz >= (1LL << 31)) return fail(EB_ERR_INVALID_ARG, "grid too large: 2^31 voxels or more");
  eb_unet u = new eb_unet_s();
  u->V[0] = {nx, ny, nz};
  u->V[1] = {nx / 2, ny / 2, nz / 2};
  u->V[2] = {nx / 4, ny / 4, nz / 4};
  u->np = total_params();
  long long o = 0;
  long long wpn = 0;
  for (int l = 0; l < 11; ++l) {
    u->off_w[l] = o;
    o += layer_w(l);
    u->off_b[l] = o;
    o += kLayers[l].cout;
    if (kLayers[l].k == 3) {
      u->wp_off[l][0] = wpn;
      wpn += packed_size(kLayers[l].cin, kLayers[l].cout);
      u->wp_off[l][1] = wpn;
      wpn += packed_size(kLayers[l].cout, kLayers[l].cin);
    }
  }
  const long long n0 = u->V[0].n(), n1 = u->V[1].n(), n2 = u->V[2].n();
  struct {
    float **q;
    long long n;
  } b[] = {{&u->e1a, 16 * n0}, {&u->e1, 16 * n0}, {&u->p1, 16 * n1}, {&u->e2a, 32 * n1}, {&u->e2, 32 * n1},
           {&u->p2, 32 * n2},  {&u->ba, 64 * n2},  {&u->bt, 64 * n2}, {&u->c2, 96 * n1},  {&u->d2a, 32 * n1},
           {&u->d2, 32 * n1},  {&u->c1, 48 * n0},  {&u->d1a, 16 * n0}, {&u->d1, 16 * n0}, {&u->y, n0}};
  cudaError_t e = cudaSuccess;
  for (auto &x : b)
    if (e == cudaSuccess) e = u->alloc(x.q, x.n);
  if (e == cudaSuccess) e = u->alloc(&u->p, u->np);
  if (e == cudaSuccess) e = u->alloc(&u->pb, u->np);
  if (e == cudaSuccess) e = u->alloc(&u->wp, wpn);
  if (e == cudaSuccess) e = cudaMemset(u->wp, 0, sizeof(__nv_bfloat16) * wpn);   // the packed zero weights
  if (e == cudaSuccess) e = u->alloc(&u->err, 1);
  if (e == cudaSuccess) e = cudaMemset(u->err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(u->p, 0, sizeof(float) * u->np);
  if (e == cudaSuccess) e = cudaMemset(u->pb, 0, sizeof(__nv_bfloat16) * u->np);
  if (e != cudaSuccess) {
    u->release();
    delete u;
    return cuda_fail(e, "network buffers");
  }
  *out = u;
  return EB_OK;
}

eb_status eb_unet_destroy(eb_unet u) {
  if (!u) return EB_OK;
  cudaDeviceSynchronize();
  u->release();
  delete u;
  return EB_OK;
}

eb_status eb_unet_set_params(eb_unet u, const float *host, int64_t n) {
  if (!u || !host) return fail(EB_ERR_INVALID_ARG, "NULL network or parameters");
  if (n != u->np) return fail(EB_ERR_INVALID_ARG, "wrong parameter count");
  CUDA_TRY(cudaMemcpy(u->p, host, sizeof(float) * n, cudaMemcpyHostToDevice), "set parameters");
  k_to_bf16<<<nblk(n), 256>>>(u->p, u->pb, n);
  pack_weights(u, 0);
  CUDA_TRY(cudaGetLastError(), "set parameters");
  if (u->grads) {
    CUDA_TRY(cudaMemset(u->m, 0, sizeof(float) * n), "optimiser state");
    CUDA_TRY(cudaMemset(u->v, 0, sizeof(float) * n), "optimiser state");
  }
  u->t = 0;
  CUDA_TRY(cudaDeviceSynchronize(), "set parameters");
  return EB_OK;
}

eb_status eb_unet_get_params(eb_unet u, float *host, int64_t n) {
  if (!u || !host) return fail(EB_ERR_INVALID_ARG, "NULL network or parameters");
  if (n != u->np) return fail(EB_ERR_INVALID_ARG, "wrong parameter count");
  CUDA_TRY(cudaMemcpy(host, u->p, sizeof(float) * n, cudaMemcpyDeviceToHost), "get parameters");
  return take_error(u);
}

eb_status eb_unet_forward(eb_unet u, const float *in, float *out, void *stream) {
  if (!u || !in || !out) return fail(EB_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = as_stream(stream);
  forward(u, in, s);
  CUDA_TRY(cudaMemcpyAsync(out, u->y, sizeof(float) * u->V[0].n(), cudaMemcpyDeviceToDevice, s), "output");
  CUDA_TRY(cudaGetLastError(), "network forward");
  return EB_OK;
}

eb_status eb_unet_gradient(eb_unet u, const float *in, const float *target, const float *mask, float *loss,
                           float *grad_host, void *stream) {
  if (!u || !in || !target || !mask) return fail(EB_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = as_stream(stream);
  eb_status st = loss_and_backward(u, in, target, mask, loss, s);
  if (st != EB_OK) return st;
  if (grad_host) {
    CUDA_TRY(cudaMemcpyAsync(grad_host, u->g, sizeof(float) * u->np, cudaMemcpyDeviceToHost, s), "gradient");
    CUDA_TRY(cudaStreamSynchronize(s), "gradient");
  }
  CUDA_TRY(cudaGetLastError(), "network gradient");
  if (loss || grad_host) return take_error(u);
  return EB_OK;
}

eb_status eb_unet_train_step(eb_unet u, const float *in, const float *target, const float *mask, float lr,
                             float *loss, void *stream) {
  if (!u || !in || !target || !mask) return fail(EB_ERR_INVALID_ARG, "NULL argument");
  if (!(lr > 0.f)) return fail(EB_ERR_INVALID_ARG, "lr must be > 0");
  cudaStream_t s = as_stream(stream);
  eb_status st = loss_and_backward(u, in, target, mask, loss, s);
  if (st != EB_OK) return st;
  u->t += 1;
  const float c1 = (float)(1.0 / (1.0 - pow(0.9, u->t))), c2 = (float)(1.0 / (1.0 - pow(0.999, u->t)));
  k_adam<<<nblk(u->np), 256, 0, s>>>(u->p, u->m, u->v, u->g, u->pb, u->np, lr, c1, c2);
  pack_weights(u, s);
  CUDA_TRY(cudaGetLastError(), "network update");
  return EB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// the network as the projection's initial guess
// ---------------------------------------------------------------------------
namespace {

// input channels [rhs / rms, alpha] and the mask of the cells in the solve
__global__ void k_net_input(const double *rhs, const double *alpha, const double *d, double inv_rms, long long N,
                            float *in, float *mask) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= N) return;
  const bool act = d[v] > 0.0;
  in[v] = act ? (float)(rhs[v] * inv_rms) : 0.f;
  in[N + v] = (float)alpha[v];
  if (mask) mask[v] = act ? 1.f : 0.f;
}

__global__ void k_sum_active(const double *x, const double *d, long long N, double *out) {
  double s = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N; v += (long long)gridDim.x * blockDim.x)
    if (d[v] > 0.0) s += x[v];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double w[32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? w[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, s);
  }
}

// training target: the mean-free solution over its normalisation
__global__ void k_net_target(const double *phi, const double *d, double mean, double inv_norm, long long N,
                             float *t) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v < N) t[v] = d[v] > 0.0 ? (float)((phi[v] - mean) * inv_norm) : 0.f;
}

// initial guess from the network output
__global__ void k_net_phi0(const float *y, const double *d, double norm, long long N, double *phi0) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v < N) phi0[v] = d[v] > 0.0 ? (double)y[v] * norm : 0.0;
}

eb_status warm_inputs(eb_geom g, const eb_state *U, double dt, double *rms, cudaStream_t s) {
  void **u = state_ptrs(U);
  void *mom[3] = {u[2], u[3], u[4]};
  eb_status st = eb_project_rhs(g, mom, dt, rms, s);
  if (st != EB_OK) return st;
  ProjWork &w = g->pw;
  const long long N = g->D.nxy * g->D.nz;
  if (!w.alpha) {
    CUDA_TRY(g->alloc(&w.alpha, N), "alloc volume fractions");
    launch_export_geometry(g->h, g->D, 0, g->G[0], EB_X_ALPHA, w.alpha, s);
  }
  if (!w.nin) CUDA_TRY(g->alloc(&w.nin, 2 * N), "alloc network input");
  return EB_OK;
}

bool same_grid(eb_geom g, eb_unet net) {
  return net->V[0].nx == g->D.nx && net->V[0].ny == g->D.ny && net->V[0].nz == g->D.nz;
}

}  // namespace

extern "C" {

eb_status eb_project_sample(eb_geom geom, const eb_state *U, double dt, double rtol, int maxit, double scale, float *in,
                            float *target, float *mask, int *iters, void *stream) {
  if (!geom || !in || !target || !mask) return fail(EB_ERR_INVALID_ARG, "NULL argument");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(U, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !(scale > 0.0)) return fail(EB_ERR_INVALID_ARG, "dt and scale must be > 0");
  cudaStream_t s = as_stream(stream);
  double rms = 0.0;
  eb_status st = warm_inputs(geom, U, dt, &rms, s);
  if (st != EB_OK) return st;
  if (!(rms > 0.0)) return fail(EB_ERR_STATE, "the momenta are already divergence-free");
  ProjWork &w = geom->pw;
  const Dims &D = geom->D;
  const long long N = D.nxy * D.nz;
  k_net_input<<<nblk(N), 256, 0, s>>>(w.rhs, w.alpha, w.d, 1.0 / rms, N, in, mask);
  void **u = state_ptrs(U);
  void *mom[3] = {u[2], u[3], u[4]};
  st = eb_project_impl(geom, mom, dt, rtol, maxit, nullptr, nullptr, iters, nullptr, s, false);
  if (st != EB_OK) return st;
  double *sum = w.part;   // a free slot of the projection's partial sums
  CUDA_TRY(cudaMemsetAsync(sum, 0, sizeof(double), s), "solution mean");
  k_sum_active<<<256, 256, 0, s>>>(w.x, w.d, N, sum);
  double h = 0.0;
  CUDA_TRY(cudaMemcpyAsync(&h, sum, sizeof(double), cudaMemcpyDeviceToHost, s), "solution mean");
  CUDA_TRY(cudaStreamSynchronize(s), "solution mean");
  const double mean = w.nact > 0 ? h / (double)w.nact : 0.0;
  k_net_target<<<nblk(N), 256, 0, s>>>(w.x, w.d, mean, 1.0 / (rms * D.dx * D.dx * scale), N, target);
  CUDA_TRY(cudaGetLastError(), "training sample");
  return EB_OK;
}

eb_status eb_project_warm(eb_geom geom, eb_unet net, eb_state *U, double dt, double rtol, int maxit, double scale,
                          int *iters, double *relres, void *stream) {
  if (!geom || !net) return fail(EB_ERR_INVALID_ARG, "NULL handle or network");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(U, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !isfinite(dt) || !(scale > 0.0)) return fail(EB_ERR_INVALID_ARG, "dt and scale must be > 0");
  if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(EB_ERR_INVALID_ARG, "rtol must lie in (0, 1)");
  if (!same_grid(geom, net)) return fail(EB_ERR_INVALID_ARG, "the network was created for another grid");
  cudaStream_t s = as_stream(stream);
  double rms = 0.0;
  eb_status st = warm_inputs(geom, U, dt, &rms, s);
  if (st != EB_OK) return st;
  ProjWork &w = geom->pw;
  const Dims &D = geom->D;
  const long long N = D.nxy * D.nz;
  const double *phi0 = nullptr;
  if (rms > 0.0) {
    k_net_input<<<nblk(N), 256, 0, s>>>(w.rhs, w.alpha, w.d, 1.0 / rms, N, w.nin, nullptr);
    forward(net, w.nin, s);
    k_net_phi0<<<nblk(N), 256, 0, s>>>(net->y, w.d, rms * D.dx * D.dx * scale, N, w.z);
    phi0 = w.z;   // copied into the solution vector before the solver touches z
  }
  void **u = state_ptrs(U);
  void *mom[3] = {u[2], u[3], u[4]};
  return eb_project_impl(geom, mom, dt, rtol, maxit, phi0, nullptr, iters, relres, s, true);
}

}  // extern "C"
