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
// Convolutions run on the tensor cores (mma.sync, BF16 operands, FP32
// accumulation) as implicit GEMMs, with the FP32 activations split into BF16
// hi + lo so that the products keep FP32-level accuracy: the forward pass
// (rows = voxels, columns = output channels, K = input channels x taps), the
// input gradient (the same kernel on the output gradient with the weights
// transposed and flipped) and the weight gradient (rows = output channels,
// columns = input channels, K = voxels, per tap; tiles add their sums
// atomically).
#include "eb_handle.cuh"

#include <cuda_bf16.h>
#include <math.h>

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

constexpr int TX = 16, TY = 8, TZ = 2;   // voxel tile of the weight gradient
constexpr int HXn = TX + 2, HYn = TY + 2, HZn = TZ + 2, HN = HXn * HYn * HZn;

// ---- tensor-core convolution (forward and input gradient) ------------------
// The same convolution as an implicit GEMM on the tensor cores (mma.sync,
// BF16 operands, FP32 accumulation): rows = 16 voxels along x (one warp per
// row; a CTA covers 16 x 8 x 1 voxels), columns = 32 output channels (four
// 8-wide tiles), K = 16 input channels per tap, 27 taps.  The FP32 inputs
// are split into BF16 hi + lo (v = hi + lo to about 2^-17 relative) and both
// parts are multiplied by the BF16 weights, so the products keep FP32-level
// accuracy.  Shared memory holds the 16-channel halo (channels fastest, a
// pitch of 24 halfwords: conflict-free 32-bit fragment loads) and the chunk's
// weights [tap][output channel][input channel].
constexpr int TC_CH = 16, TC_P = 24, TC_RZ = 2;   // channels per K chunk, channel pitch, z rows per warp
constexpr int TC_HX = 18, TC_HY = 10, TC_HZ = TC_RZ + 2, TC_HN = TC_HX * TC_HY * TC_HZ;
template <int NT>
constexpr size_t tc_smem() {
  return (size_t)(2 * TC_HN * TC_P + 27 * NT * 8 * TC_P) * sizeof(__nv_bfloat16);
}

__device__ inline void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// NT 8-wide tiles of output channels per CTA (8 NT channels); a CTA covers
// 16 x 8 x TC_RZ voxels, warp w the rows y0 + w, z0 .. z0 + TC_RZ - 1
template <int NT>
__global__ void __launch_bounds__(256) k_conv3_tc(const float *in, int cin, const __nv_bfloat16 *W, const float *bias,
                                                  float *out, int cout, Vol V, int relu) {
  constexpr int NCO = NT * 8;
  extern __shared__ __align__(16) unsigned char tc_smem[];
  __nv_bfloat16 *s_hi = reinterpret_cast<__nv_bfloat16 *>(tc_smem);
  __nv_bfloat16 *s_lo = s_hi + TC_HN * TC_P;
  __nv_bfloat16 *s_w = s_lo + TC_HN * TC_P;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ntx = (V.nx + 15) / 16, nty = (V.ny + 7) / 8;
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * 16, y0 = ((tile / ntx) % nty) * 8, z0 = (tile / (ntx * nty)) * TC_RZ;
  const int co0 = blockIdx.y * NCO;
  const long long N = V.n();
  float acc[TC_RZ][NT][4];
#pragma unroll
  for (int rz = 0; rz < TC_RZ; ++rz)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[rz][nt][e] = 0.f;
  for (int c0 = 0; c0 < cin; c0 += TC_CH) {
    __syncthreads();
    for (int q = threadIdx.x; q < TC_CH * TC_HN; q += blockDim.x) {
      const int c = q / TC_HN, h = q % TC_HN;
      const int hx = h % TC_HX, hy = (h / TC_HX) % TC_HY, hz = h / (TC_HX * TC_HY);
      const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
      float v = 0.f;
      if (c0 + c < cin && x >= 0 && x < V.nx && y >= 0 && y < V.ny && z >= 0 && z < V.nz)
        v = in[(long long)(c0 + c) * N + ((long long)z * V.ny + y) * V.nx + x];
      const __nv_bfloat16 hi = __float2bfloat16_rn(v);
      s_hi[h * TC_P + c] = hi;
      s_lo[h * TC_P + c] = __float2bfloat16_rn(v - __bfloat162float(hi));
    }
    for (int q = threadIdx.x; q < 27 * NCO * TC_CH; q += blockDim.x) {
      const int a = q % 27, r = q / 27, c = r % TC_CH, co = r / TC_CH;   // consecutive threads: consecutive taps
      __nv_bfloat16 w = __float2bfloat16_rn(0.f);
      if (co0 + co < cout && c0 + c < cin) w = W[((long long)(co0 + co) * cin + c0 + c) * 27 + a];
      s_w[(a * NCO + co) * TC_P + c] = w;
    }
    __syncthreads();
    for (int a = 0; a < 27; ++a) {
      const int dz = a / 9, dy = (a / 3) % 3, dx = a % 3;
      unsigned b[NT][2];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const unsigned *pb = reinterpret_cast<const unsigned *>(s_w + (a * NCO + nt * 8 + g) * TC_P + 2 * t);
        b[nt][0] = pb[0];
        b[nt][1] = pb[4];
      }
#pragma unroll
      for (int rz = 0; rz < TC_RZ; ++rz) {
        const int h0 = ((rz + dz) * TC_HY + (warp + dy)) * TC_HX + dx;   // halo voxel of row 0
        const unsigned *ph = reinterpret_cast<const unsigned *>(s_hi + (h0 + g) * TC_P + 2 * t);
        const unsigned *ph8 = reinterpret_cast<const unsigned *>(s_hi + (h0 + g + 8) * TC_P + 2 * t);
        const unsigned *pl = reinterpret_cast<const unsigned *>(s_lo + (h0 + g) * TC_P + 2 * t);
        const unsigned *pl8 = reinterpret_cast<const unsigned *>(s_lo + (h0 + g + 8) * TC_P + 2 * t);
        const unsigned ahi[4] = {ph[0], ph8[0], ph[4], ph8[4]};
        const unsigned alo[4] = {pl[0], pl8[0], pl[4], pl8[4]};
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          mma_bf16(acc[rz][nt], ahi, b[nt]);
          mma_bf16(acc[rz][nt], alo, b[nt]);
        }
      }
    }
  }
  const int y = y0 + warp;
  if (y >= V.ny) return;
#pragma unroll
  for (int rz = 0; rz < TC_RZ; ++rz) {
    const int z = z0 + rz;
    if (z >= V.nz) break;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int x = x0 + g + (e >= 2 ? 8 : 0), co = co0 + nt * 8 + 2 * t + (e & 1);
        if (x >= V.nx || co >= cout) continue;
        float r = acc[rz][nt][e] + (bias ? bias[co] : 0.f);
        if (relu) r = fmaxf(r, 0.f);
        out[(long long)co * N + ((long long)z * V.ny + y) * V.nx + x] = r;
      }
  }
}

// 1x1 head: out[v] = b + sum_ci W[ci] in[ci][v]
__global__ void k_head(const float *in, int cin, const __nv_bfloat16 *W, const float *bias, float *out, long long N) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= N) return;
  float a = bias[0];
  for (int c = 0; c < cin; ++c) a = fmaf(__bfloat162float(W[c]), in[c * N + v], a);
  out[v] = a;
}

// head backward: dIn[ci][v] = W[ci] dy[v]
__global__ void k_head_bwd(const float *dy, const __nv_bfloat16 *W, int cin, float *din, long long N) {
  const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (v >= N) return;
  const float g = dy[v];
  for (int c = 0; c < cin; ++c) din[c * N + v] = __bfloat162float(W[c]) * g;
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

// W' = transposed and flipped W: W'[ci][co][26 - a] = W[co][ci][a]
__global__ void k_flip(const __nv_bfloat16 *W, int cout, int cin, __nv_bfloat16 *Wt) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)cout * cin * 27) return;
  const int a = q % 27, ci = (q / 27) % cin, co = q / (27LL * cin);
  Wt[((long long)ci * cout + co) * 27 + (26 - a)] = W[q];
}

// Weight gradient on the tensor cores: per tap a, dW[co][ci][a] += sum over
// the tile's voxels of dOut[co][v] in[ci][v + a] -- a GEMM with rows = 16
// output channels, columns = 16 input channels (two 8-wide tiles), K = the
// 16 x 8 x 2 voxels of a tile (16 per step, one x-row).  Both operands are
// split into BF16 hi + lo and multiplied as hi.hi + hi.lo + lo.hi (relative
// error about 2^-16).  Warp w takes taps w, w + 8, w + 16, w + 24.  The input
// halo is held twice, the second copy shifted by one voxel along x, so that
// the voxel pairs of the x-shift dx = 1 start on a 32-bit boundary.  Row
// pitches (264 and 728 halfwords) keep the fragment loads conflict-free.
// Each tile adds its sums atomically.
constexpr int WG_DP = 264, WG_IP = 728, WG_C = 16;
constexpr size_t WG_SMEM = (size_t)(2 * WG_C * WG_DP + 4 * WG_C * WG_IP) * sizeof(__nv_bfloat16);

__global__ void __launch_bounds__(256) k_conv3_wgrad_tc(const float *in, int cin, const float *dout, int cout,
                                                        Vol V, float *dW) {
  extern __shared__ __align__(16) unsigned char wg_smem[];
  __nv_bfloat16 *d_hi = reinterpret_cast<__nv_bfloat16 *>(wg_smem);
  __nv_bfloat16 *d_lo = d_hi + WG_C * WG_DP;
  __nv_bfloat16 *i0h = d_lo + WG_C * WG_DP, *i0l = i0h + WG_C * WG_IP;
  __nv_bfloat16 *i1h = i0l + WG_C * WG_IP, *i1l = i1h + WG_C * WG_IP;
  const int ntx = (V.nx + TX - 1) / TX, nty = (V.ny + TY - 1) / TY;
  const int tile = blockIdx.x;
  const int x0 = (tile % ntx) * TX, y0 = ((tile / ntx) % nty) * TY, z0 = (tile / (ntx * nty)) * TZ;
  const int co0 = blockIdx.y * WG_C, ci0 = blockIdx.z * WG_C;
  const long long N = V.n();
  constexpr int NV = TX * TY * TZ;   // 256 voxels
  for (int q = threadIdx.x; q < WG_C * HN; q += blockDim.x) {
    const int c = q / HN, h = q % HN;
    const int hx = h % HXn, hy = (h / HXn) % HYn, hz = h / (HXn * HYn);
    const int x = x0 + hx - 1, y = y0 + hy - 1, z = z0 + hz - 1;
    float v = 0.f;
    if (ci0 + c < cin && x >= 0 && x < V.nx && y >= 0 && y < V.ny && z >= 0 && z < V.nz)
      v = in[(long long)(ci0 + c) * N + ((long long)z * V.ny + y) * V.nx + x];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v), lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    i0h[c * WG_IP + h] = hi;
    i0l[c * WG_IP + h] = lo;
    if (h >= 1) {   // shifted copy: i1[h - 1] = i0[h]
      i1h[c * WG_IP + h - 1] = hi;
      i1l[c * WG_IP + h - 1] = lo;
    }
    if (h == HN - 1) {
      i1h[c * WG_IP + h] = __float2bfloat16_rn(0.f);
      i1l[c * WG_IP + h] = __float2bfloat16_rn(0.f);
    }
  }
  for (int q = threadIdx.x; q < WG_C * NV; q += blockDim.x) {
    const int co = q / NV, r = q % NV;
    const int x = x0 + r % TX, y = y0 + (r / TX) % TY, z = z0 + r / (TX * TY);
    float v = 0.f;
    if (co0 + co < cout && x < V.nx && y < V.ny && z < V.nz)
      v = dout[(long long)(co0 + co) * N + ((long long)z * V.ny + y) * V.nx + x];
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    d_hi[co * WG_DP + r] = hi;
    d_lo[co * WG_DP + r] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[4][2][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[j][nt][e] = 0.f;
  auto u32 = [](const __nv_bfloat16 *p) { return *reinterpret_cast<const unsigned *>(p); };
  for (int row = 0; row < TY * TZ; ++row) {   // K steps: one x-row of 16 voxels each
    const int ty = row % TY, tz = row / TY, kb = row * TX;
    const unsigned ahi[4] = {u32(d_hi + g * WG_DP + kb + 2 * t), u32(d_hi + (g + 8) * WG_DP + kb + 2 * t),
                             u32(d_hi + g * WG_DP + kb + 2 * t + 8), u32(d_hi + (g + 8) * WG_DP + kb + 2 * t + 8)};
    const unsigned alo[4] = {u32(d_lo + g * WG_DP + kb + 2 * t), u32(d_lo + (g + 8) * WG_DP + kb + 2 * t),
                             u32(d_lo + g * WG_DP + kb + 2 * t + 8), u32(d_lo + (g + 8) * WG_DP + kb + 2 * t + 8)};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int a = warp + 8 * j;
      if (a >= 27) break;
      const int dz = a / 9, dy = (a / 3) % 3, dx = a % 3;
      const int base = ((tz + dz) * HYn + (ty + dy)) * HXn;
      const __nv_bfloat16 *bh = dx == 1 ? i1h : i0h, *bl = dx == 1 ? i1l : i0l;
      const int off = base + 2 * t + (dx == 2 ? 2 : 0);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int ci = nt * 8 + g;
        const unsigned bhi[2] = {u32(bh + ci * WG_IP + off), u32(bh + ci * WG_IP + off + 8)};
        const unsigned blo[2] = {u32(bl + ci * WG_IP + off), u32(bl + ci * WG_IP + off + 8)};
        mma_bf16(acc[j][nt], ahi, bhi);
        mma_bf16(acc[j][nt], ahi, blo);
        mma_bf16(acc[j][nt], alo, bhi);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int a = warp + 8 * j;
    if (a >= 27) break;
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int co = co0 + g + (e >= 2 ? 8 : 0), ci = ci0 + nt * 8 + 2 * t + (e & 1);
        if (co < cout && ci < cin) atomicAdd(dW + ((long long)co * cin + ci) * 27 + a, acc[j][nt][e]);
      }
  }
}

__global__ void k_relu_mask(float *d, const float *post, long long n) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n && !(post[q] > 0.f)) d[q] = 0.f;
}

// 2x2x2 average pool: out (C, V/2) from in (C, V)
__global__ void k_pool(const float *in, Vol V, int C, float *out) {
  const Vol H{V.nx / 2, V.ny / 2, V.nz / 2};
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)C * H.n()) return;
  const long long c = q / H.n(), r = q % H.n();
  const int x = r % H.nx, y = (r / H.nx) % H.ny, z = r / ((long long)H.nx * H.ny);
  float s = 0.f;
  for (int a = 0; a < 8; ++a)
    s += in[c * V.n() + ((long long)(2 * z + (a >> 2)) * V.ny + 2 * y + ((a >> 1) & 1)) * V.nx + 2 * x + (a & 1)];
  out[q] = s * 0.125f;
}

// din (C, V) += pool backward of dout (C, V/2)
__global__ void k_pool_bwd_add(const float *dout, Vol V, int C, float *din) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)C * V.n()) return;
  const long long c = q / V.n(), r = q % V.n();
  const int x = r % V.nx, y = (r / V.nx) % V.ny, z = r / ((long long)V.nx * V.ny);
  const Vol H{V.nx / 2, V.ny / 2, V.nz / 2};
  din[q] += 0.125f * dout[c * H.n() + ((long long)(z / 2) * H.ny + y / 2) * H.nx + x / 2];
}

// out (C, V) = nearest upsampling of in (C, V/2), written at channel offset
__global__ void k_up(const float *in, Vol V, int C, float *out) {
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)C * V.n()) return;
  const long long c = q / V.n(), r = q % V.n();
  const int x = r % V.nx, y = (r / V.nx) % V.ny, z = r / ((long long)V.nx * V.ny);
  const Vol H{V.nx / 2, V.ny / 2, V.nz / 2};
  out[q] = in[c * H.n() + ((long long)(z / 2) * H.ny + y / 2) * H.nx + x / 2];
}

// din (C, V/2) = upsampling backward of dout (C, V): sum of the 8 children
__global__ void k_up_bwd(const float *dout, Vol V, int C, float *din) {
  const Vol H{V.nx / 2, V.ny / 2, V.nz / 2};
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= (long long)C * H.n()) return;
  const long long c = q / H.n(), r = q % H.n();
  const int x = r % H.nx, y = (r / H.nx) % H.ny, z = r / ((long long)H.nx * H.ny);
  float s = 0.f;
  for (int a = 0; a < 8; ++a)
    s += dout[c * V.n() + ((long long)(2 * z + (a >> 2)) * V.ny + 2 * y + ((a >> 1) & 1)) * V.nx + 2 * x + (a & 1)];
  din[q] = s;
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
  __nv_bfloat16 *pb = nullptr, *wt = nullptr;   // working weights, transposed scratch
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

// the tensor-core convolution on a volume: 16 x 8 x 4 voxel tiles, 8 NT output
// channels per CTA with NT = 1, 2 or 4 from the number of output channels
template <int NT>
void conv3_tc_nt(const float *in, int cin, const __nv_bfloat16 *W, const float *bias, float *out, int cout,
                 const Vol &V, bool relu, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv3_tc<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem<NT>());
    attr = true;
  }
  const unsigned tiles = (unsigned)(((V.nx + 15) / 16) * ((V.ny + 7) / 8) * ((V.nz + TC_RZ - 1) / TC_RZ));
  k_conv3_tc<NT><<<dim3(tiles, (cout + NT * 8 - 1) / (NT * 8)), 256, tc_smem<NT>(), s>>>(in, cin, W, bias, out,
                                                                                        cout, V, relu ? 1 : 0);
}

void conv3_tc(const float *in, int cin, const __nv_bfloat16 *W, const float *bias, float *out, int cout,
              const Vol &V, bool relu, cudaStream_t s) {
  if (cout <= 8) conv3_tc_nt<1>(in, cin, W, bias, out, cout, V, relu, s);
  else if (cout <= 16) conv3_tc_nt<2>(in, cin, W, bias, out, cout, V, relu, s);
  else conv3_tc_nt<4>(in, cin, W, bias, out, cout, V, relu, s);
}

void conv3(eb_unet u, int l, const float *in, float *out, const Vol &V, bool relu, cudaStream_t s) {
  const LayerSpec &L = kLayers[l];
  conv3_tc(in, L.cin, u->pb + u->off_w[l], u->p + u->off_b[l], out, L.cout, V, relu, s);
}

// input gradient of layer l: din = conv of dout with flipped, transposed W
void conv3_dgrad(eb_unet u, int l, const float *dout, float *din, const Vol &V, cudaStream_t s) {
  const LayerSpec &L = kLayers[l];
  k_flip<<<nblk(layer_w(l)), 256, 0, s>>>(u->pb + u->off_w[l], L.cout, L.cin, u->wt);
  conv3_tc(dout, L.cout, u->wt, nullptr, din, L.cin, V, false, s);
}

void conv3_wgrad(eb_unet u, int l, const float *in, const float *dout, const Vol &V, cudaStream_t s) {
  const LayerSpec &L = kLayers[l];
  const unsigned tiles = (unsigned)(((V.nx + TX - 1) / TX) * ((V.ny + TY - 1) / TY) * ((V.nz + TZ - 1) / TZ));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_conv3_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM);
    attr = true;
  }
  k_conv3_wgrad_tc<<<dim3(tiles, (L.cout + WG_C - 1) / WG_C, (L.cin + WG_C - 1) / WG_C), 256, WG_SMEM, s>>>(
      in, L.cin, dout, L.cout, V, u->g + u->off_w[l]);
  k_chan_dot<<<dim3(64, L.cout), 256, 0, s>>>(dout, nullptr, L.cout, V.n(), u->g + u->off_b[l]);
}

void forward(eb_unet u, const float *x, cudaStream_t s) {
  const Vol &V0 = u->V[0], &V1 = u->V[1], &V2 = u->V[2];
  conv3(u, 0, x, u->e1a, V0, true, s);
  conv3(u, 1, u->e1a, u->e1, V0, true, s);
  k_pool<<<nblk(16 * V1.n()), 256, 0, s>>>(u->e1, V0, 16, u->p1);
  conv3(u, 2, u->p1, u->e2a, V1, true, s);
  conv3(u, 3, u->e2a, u->e2, V1, true, s);
  k_pool<<<nblk(32 * V2.n()), 256, 0, s>>>(u->e2, V1, 32, u->p2);
  conv3(u, 4, u->p2, u->ba, V2, true, s);
  conv3(u, 5, u->ba, u->bt, V2, true, s);
  k_up<<<nblk(64 * V1.n()), 256, 0, s>>>(u->bt, V1, 64, u->c2);
  cudaMemcpyAsync(u->c2 + 64 * V1.n(), u->e2, sizeof(float) * 32 * V1.n(), cudaMemcpyDeviceToDevice, s);
  conv3(u, 6, u->c2, u->d2a, V1, true, s);
  conv3(u, 7, u->d2a, u->d2, V1, true, s);
  k_up<<<nblk(32 * V0.n()), 256, 0, s>>>(u->d2, V0, 32, u->c1);
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
  k_head_bwd<<<nblk(n0), 256, 0, s>>>(u->gy, u->pb + u->off_w[10], 16, u->gd1, n0);
  k_relu_mask<<<nblk(16 * n0), 256, 0, s>>>(u->gd1, u->d1, 16 * n0);
  conv3_wgrad(u, 9, u->d1a, u->gd1, V0, s);
  conv3_dgrad(u, 9, u->gd1, u->gd1a, V0, s);
  k_relu_mask<<<nblk(16 * n0), 256, 0, s>>>(u->gd1a, u->d1a, 16 * n0);
  conv3_wgrad(u, 8, u->c1, u->gd1a, V0, s);
  conv3_dgrad(u, 8, u->gd1a, u->gc1, V0, s);
  k_up_bwd<<<nblk(32 * n1), 256, 0, s>>>(u->gc1, V0, 32, u->gd2);
  cudaMemcpyAsync(u->ge1, u->gc1 + 32 * n0, sizeof(float) * 16 * n0, cudaMemcpyDeviceToDevice, s);
  k_relu_mask<<<nblk(32 * n1), 256, 0, s>>>(u->gd2, u->d2, 32 * n1);
  conv3_wgrad(u, 7, u->d2a, u->gd2, V1, s);
  conv3_dgrad(u, 7, u->gd2, u->gd2a, V1, s);
  k_relu_mask<<<nblk(32 * n1), 256, 0, s>>>(u->gd2a, u->d2a, 32 * n1);
  conv3_wgrad(u, 6, u->c2, u->gd2a, V1, s);
  conv3_dgrad(u, 6, u->gd2a, u->gc2, V1, s);
  k_up_bwd<<<nblk(64 * n2), 256, 0, s>>>(u->gc2, V1, 64, u->gbt);
  cudaMemcpyAsync(u->ge2, u->gc2 + 64 * n1, sizeof(float) * 32 * n1, cudaMemcpyDeviceToDevice, s);
  k_relu_mask<<<nblk(64 * n2), 256, 0, s>>>(u->gbt, u->bt, 64 * n2);
  conv3_wgrad(u, 5, u->ba, u->gbt, V2, s);
  conv3_dgrad(u, 5, u->gbt, u->gba, V2, s);
  k_relu_mask<<<nblk(64 * n2), 256, 0, s>>>(u->gba, u->ba, 64 * n2);
  conv3_wgrad(u, 4, u->p2, u->gba, V2, s);
  conv3_dgrad(u, 4, u->gba, u->gp2, V2, s);
  k_pool_bwd_add<<<nblk(32 * n1), 256, 0, s>>>(u->gp2, V1, 32, u->ge2);
  k_relu_mask<<<nblk(32 * n1), 256, 0, s>>>(u->ge2, u->e2, 32 * n1);
  conv3_wgrad(u, 3, u->e2a, u->ge2, V1, s);
  conv3_dgrad(u, 3, u->ge2, u->ge2a, V1, s);
  k_relu_mask<<<nblk(32 * n1), 256, 0, s>>>(u->ge2a, u->e2a, 32 * n1);
  conv3_wgrad(u, 2, u->p1, u->ge2a, V1, s);
  conv3_dgrad(u, 2, u->ge2a, u->gp1, V1, s);
  k_pool_bwd_add<<<nblk(16 * n0), 256, 0, s>>>(u->gp1, V0, 16, u->ge1);
  k_relu_mask<<<nblk(16 * n0), 256, 0, s>>>(u->ge1, u->e1, 16 * n0);
  conv3_wgrad(u, 1, u->e1a, u->ge1, V0, s);
  conv3_dgrad(u, 1, u->ge1, u->ge1a, V0, s);
  k_relu_mask<<<nblk(16 * n0), 256, 0, s>>>(u->ge1a, u->e1a, 16 * n0);
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

}  // namespace

extern "C" {

int64_t eb_unet_num_params(void) { return total_params(); }

eb_status eb_unet_create(int nx, int ny, int nz, eb_unet *out) {
  if (!out) return fail(EB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4)
    return fail(EB_ERR_INVALID_ARG, "nx, ny, nz must be multiples of 4 (two 2x poolings), at least 4");
  eb_unet u = new eb_unet_s();
  u->V[0] = {nx, ny, nz};
  u->V[1] = {nx / 2, ny / 2, nz / 2};
  u->V[2] = {nx / 4, ny / 4, nz / 4};
  u->np = total_params();
  long long o = 0;
  long long wmax = 0;
  for (int l = 0; l < 11; ++l) {
    u->off_w[l] = o;
    o += layer_w(l);
    u->off_b[l] = o;
    o += kLayers[l].cout;
    wmax = std::max(wmax, layer_w(l));
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
  if (e == cudaSuccess) e = u->alloc(&u->wt, wmax);
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
  return EB_OK;
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
