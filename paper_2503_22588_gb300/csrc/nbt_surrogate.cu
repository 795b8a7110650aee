// nbt_surrogate.cu -- the learned IG surrogate: crops, network, training.
//
// The paper has no learned component.  The surrogate predicts the mean ray
// IG of a perspective (Section III's g_P, scaled) from a view-aligned
// occupancy crop and the pose, so that only the most promising candidates
// are raycast exactly.
//
// Network (all layers on the tcgen05 GEMM of nbt_tc.cuh, BF16 operands and
// activations, FP32 accumulation and FP32 master weights):
//   crop 32^3 x 8 (one-hot unknown / free / occupied in channels 0..2)
//   conv 3^3 8->16 s2, conv 16->32 s2, conv 32->64 s2, conv 64->64 s1 (ReLU)
//   flatten 4^3 x 64 = 4096 | 8 pose features -> fc 4104->128 (ReLU) -> fc 128->1
// Convolutions are implicit GEMMs: a loader gathers the im2col tile of the
// stage straight from the NDHWC activations into shared memory (nothing is
// materialised in HBM).  Backward: input gradients are GEMMs over a
// transposed-convolution loader (ReLU mask fused in the epilogue); weight
// gradients are split-K GEMMs whose loaders transpose 16-byte activation
// vectors into K-major stage rows, reduced over the splits in a fixed order.

#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "nbt_internal.cuh"
#include "nbt_tc.cuh"

namespace nbt {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kCrop = 32;
constexpr int kC0 = 8;
constexpr int kFeat = 8;
constexpr int kFlat = 4096;
constexpr int kFcIn = kFlat + kFeat;  // 4104
constexpr int kHid = 128;
constexpr int kLayers = 4;
struct LayerDims {
  int cin, cout, stride, din, dout;
};
constexpr LayerDims kL[kLayers] = {{8, 16, 2, 32, 16}, {16, 32, 2, 16, 8}, {32, 64, 2, 8, 4}, {64, 64, 1, 4, 4}};
// (the device-side weight copy kernel repeats these channel counts as literals)
constexpr int kSplitBytes = 64 << 20;  // split-K partials (weight gradients, fc1)
constexpr int kFc1Splits = 4;            // fc1: 32 row tiles of a 4096 batch x 4 K splits = 128 CTAs
// The splits launch_gemm makes of fc1's K stages of 64 (it rounds to whole stages per split).
constexpr int fc1_splits() {
  constexpr int stages = (kFcIn + 63) / 64, per = (stages + kFc1Splits - 1) / kFc1Splits;
  return (stages + per - 1) / per;
}
static_assert((int64_t)kFc1Splits * 4096 * kHid * 4 <= kSplitBytes, "fc1 partials of the largest batch");

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// Parameter vector (FP32): per conv layer W [cout][27 cin], b [cout]; then
// F1 [128][4104], g1 [128], f2 [128], g2 [1].
struct ParamLayout {
  int64_t w[kLayers], b[kLayers], f1, g1, f2, g2, total;
};
constexpr ParamLayout make_layout() {
  ParamLayout p{};
  int64_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    p.w[l] = o;
    o += (int64_t)kL[l].cout * 27 * kL[l].cin;
    p.b[l] = o;
    o += kL[l].cout;
  }
  p.f1 = o;
  o += (int64_t)kHid * kFcIn;
  p.g1 = o;
  o += kHid;
  p.f2 = o;
  o += kHid;
  p.g2 = o;
  o += 1;
  p.total = o;
  return p;
}
constexpr ParamLayout kP = make_layout();
// scalar copies for device code (arrays of a host constexpr are not visible there)
constexpr int64_t kW0 = kP.w[0], kW1 = kP.w[1], kW2 = kP.w[2], kW3 = kP.w[3];
constexpr int64_t kB0 = kP.b[0], kB1 = kP.b[1], kB2 = kP.b[2], kB3 = kP.b[3];

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

// ---------------------------------------------------------------------------
// Loaders
// ---------------------------------------------------------------------------

// Row-major K-major BF16 matrix [rows, K], row stride ld elements.
struct MatLoader {
  static constexpr bool kAsync = true;
  const bf16 *p;
  int rows, K, ld;
  __device__ __forceinline__ const void *src(int r, int kc) const {
    const int k = kc * 8;
    return (r >= rows || k >= K) ? nullptr : (const void *)(p + (size_t)r * ld + k);
  }
  __device__ __forceinline__ const void *base() const { return p; }
};

// Implicit im2col of a 3^3 convolution (padding 1): row m = output voxel
// (b, oz, oy, ox), K index = tap * cin + ci with tap = (dz*3 + dy)*3 + dx.
struct ConvFwdLoader {
  static constexpr bool kAsync = true;
  const bf16 *x;
  int M, D, stride, sh_do, sh_cg, cin;
  __device__ __forceinline__ const void *src(int m, int kc) const {
    if (m >= M) return nullptr;
    const int tap = kc >> sh_cg;
    if (tap >= 27) return nullptr;
    const int cg = kc & ((1 << sh_cg) - 1);
    const int dmask = (1 << sh_do) - 1;
    const int ox = m & dmask, oy = (m >> sh_do) & dmask, oz = (m >> (2 * sh_do)) & dmask, b = m >> (3 * sh_do);
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int iz = oz * stride + dz - 1, iy = oy * stride + dy - 1, ix = ox * stride + dx - 1;
    if ((unsigned)iz >= (unsigned)D || (unsigned)iy >= (unsigned)D || (unsigned)ix >= (unsigned)D) return nullptr;
    return x + ((((size_t)b * D + iz) * D + iy) * D + ix) * cin + cg * 8;
  }
  __device__ __forceinline__ const void *base() const { return x; }
};

// Implicit im2col of the transposed convolution giving the input gradient:
// row m = input voxel i, K index = tap * cout + co; the output voxel that
// tap d reads i from is o = (i + 1 - d) / s when that is integral and in
// range (forward: i = o*s + d - 1).
struct ConvBwdDataLoader {
  static constexpr bool kAsync = true;
  const bf16 *dy;
  int M, Di, Do, sh_s, sh_di, sh_cg, cout;
  __device__ __forceinline__ const void *src(int m, int kc) const {
    if (m >= M) return nullptr;
    const int tap = kc >> sh_cg;
    if (tap >= 27) return nullptr;
    const int cg = kc & ((1 << sh_cg) - 1);
    const int dmask = (1 << sh_di) - 1;
    const int ix = m & dmask, iy = (m >> sh_di) & dmask, iz = (m >> (2 * sh_di)) & dmask, b = m >> (3 * sh_di);
    const int dz = tap / 9, dy_ = (tap / 3) % 3, dx = tap % 3;
    const int tz = iz + 1 - dz, ty = iy + 1 - dy_, tx = ix + 1 - dx;
    const int smask = (1 << sh_s) - 1;
    if (tz < 0 || ty < 0 || tx < 0 || (tz & smask) || (ty & smask) || (tx & smask)) return nullptr;
    const int oz = tz >> sh_s, oy = ty >> sh_s, ox = tx >> sh_s;
    if (oz >= Do || oy >= Do || ox >= Do) return nullptr;
    return dy + ((((size_t)b * Do + oz) * Do + oy) * Do + ox) * cout + cg * 8;
  }
  __device__ __forceinline__ const void *base() const { return dy; }
};

// Weight gradient, operand A: rows = (tap, ci) (27 cin of them), K = output
// voxels m.  Each thread loads the 8 channels of one input voxel (16 bytes)
// and writes them transposed into 8 stage rows at K position m.
struct WgradColLoader {
  static constexpr bool kAsync = false;
  const bf16 *x;
  int Mout, D, stride, sh_do, cin;
  template <int ROWS>
  __device__ __forceinline__ void fill(uint8_t *s, int row0, int kc0, int tid) const {
    const int groups = ROWS / 8;  // 8-channel groups in the tile: (tap_local, cg)
    const int cgn = cin / 8;
    const int dmask = (1 << sh_do) - 1;
    for (int it = tid; it < 64 * groups; it += tc::kThreads) {
      const int mm = it & 63, g = it >> 6;
      const int r = g * 8;  // first stage row of this group
      const int row = row0 + r;
      const int tap = row / cin, cg = (row % cin) >> 3;
      const int m = kc0 * 8 + mm;
      uint4 v = zero4();
      if (tap < 27 && m < Mout) {
        const int ox = m & dmask, oy = (m >> sh_do) & dmask, oz = (m >> (2 * sh_do)) & dmask, b = m >> (3 * sh_do);
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const int iz = oz * stride + dz - 1, iy = oy * stride + dy - 1, ix = ox * stride + dx - 1;
        if ((unsigned)iz < (unsigned)D && (unsigned)iy < (unsigned)D && (unsigned)ix < (unsigned)D)
          v = __ldg((const uint4 *)(x + ((((size_t)b * D + iz) * D + iy) * D + ix) * cin + cg * 8));
      }
      (void)cgn;
      const uint16_t *e = (const uint16_t *)&v;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        *(uint16_t *)(s + tc::stage_off(r + k, mm >> 3, ROWS) + (mm & 7) * 2) = e[k];
    }
  }
};

// Weight gradient, operand B: rows = output channels co, K = output voxels
// m, from the NDHWC output gradient (16-byte vectors transposed into rows).
struct WgradDyLoader {
  static constexpr bool kAsync = false;
  const bf16 *dy;
  int Mout, cout;
  template <int ROWS>
  __device__ __forceinline__ void fill(uint8_t *s, int row0, int kc0, int tid) const {
    const int groups = ROWS / 8;
    for (int it = tid; it < 64 * groups; it += tc::kThreads) {
      const int mm = it & 63, g = it >> 6;
      const int r = g * 8;
      const int co = row0 + r;
      const int m = kc0 * 8 + mm;
      uint4 v = zero4();
      if (co < cout && m < Mout) v = __ldg((const uint4 *)(dy + (size_t)m * cout + co));
      const uint16_t *e = (const uint16_t *)&v;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        *(uint16_t *)(s + tc::stage_off(r + k, mm >> 3, ROWS) + (mm & 7) * 2) = e[k];
    }
  }
};

// ---------------------------------------------------------------------------
// Epilogues
// ---------------------------------------------------------------------------

// out[m * ld + n] = bf16(max(v + bias[n], 0)) for n < N.
struct EpiBiasRelu {
  bf16 *out;
  const float *bias;
  int N, ld;
  __device__ __forceinline__ void row(int m, int n, const float v[16], int) const {
    bf16 *d = out + (size_t)m * ld + n;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (n + i < N) d[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[n + i], 0.0f));
  }
};

// Last conv layer: its 64 output voxels of sample b = m / 64 go to the
// first 4096 columns of row b of the fully connected input X.
struct EpiConvToFlat {
  bf16 *x;
  const float *bias;
  __device__ __forceinline__ void row(int m, int n, const float v[16], int) const {
    bf16 *d = x + (size_t)(m >> 6) * kFcIn + (m & 63) * 64 + n;
#pragma unroll
    for (int i = 0; i < 16; ++i) d[i] = __float2bfloat16_rn(fmaxf(v[i] + bias[n + i], 0.0f));
  }
};

// FP32 store (split-K partials use plane z of size planes).
struct EpiF32 {
  float *out;
  int N, ld;
  int64_t plane;
  __device__ __forceinline__ void row(int m, int n, const float v[16], int z) const {
    float *d = out + z * plane + (size_t)m * ld + n;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (n + i < N) d[i] = v[i];
  }
};

// Input gradient with the ReLU mask of the layer input fused:
// out[m * ld + n] = bf16(v * [act[m * lda + n] > 0]) for n < N.
struct EpiMaskRelu {
  bf16 *out;
  const bf16 *act;
  int N, ld, lda;
  __device__ __forceinline__ void row(int m, int n, const float v[16], int) const {
    bf16 *d = out + (size_t)m * ld + n;
    const bf16 *a = act + (size_t)m * lda + n;
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (n + i < N) d[i] = __float2bfloat16_rn(__bfloat162float(a[i]) > 0.0f ? v[i] : 0.0f);
  }
};

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------

// Frustum crop (same FP32 operation order as the reference): sample (i, j,
// k) on the ray through pixel centre (i, j) of a 32 x 32 image of the field
// of view, at depth fraction (k + 1/2) / 32; one-hot class of the voxel that
// holds it, zero outside the map.  One thread per sample.
struct CropConst {
  float x0, xs, y0, ys, zc, inv_s, ox, oy, oz, ext_x, ext_y, ext_z;
  float occ_thr, free_thr;
};

// LINEAR: linear x-fastest layout, element index (z ny + y) nx + x computed
// instead of read from the offset tables.  Launched with 256 threads.
template <int KIND, bool LINEAR>
__global__ void __launch_bounds__(256) crop_kernel(DevMap m, CropConst cc, const float *__restrict__ poses, int64_t n,
                                                   uint8_t *__restrict__ crops, bf16 *__restrict__ feats) {
  // one CTA per perspective: the rotation is formed once, then every sample
  // of the crop uses it (same operations, same order as per sample)
  __shared__ float s_r[9], s_o[3], s_pz[7];
  const float org[3] = {cc.ox, cc.oy, cc.oz};
  for (int64_t v = blockIdx.x; v < n; v += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < 7; ++q) s_pz[q] = __ldg(poses + v * 7 + q);
      float r[9];
      quat_rot_f32(s_pz + 3, r);
#pragma unroll
      for (int q = 0; q < 9; ++q) s_r[q] = r[q];
#pragma unroll
      for (int a = 0; a < 3; ++a) s_o[a] = fmul(fsub(s_pz[a], org[a]), cc.inv_s);
    }
    __syncthreads();
    float r[9], o[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) r[q] = s_r[q];
#pragma unroll
    for (int a = 0; a < 3; ++a) o[a] = s_o[a];
    const int dims[3] = {m.nx, m.ny, m.nz};
    uint8_t *cv = crops + v * (int64_t)(kCrop * kCrop * kCrop);
    // Sample (i, j, k) of cell i + 32 j + 1024 k.  With 256 threads a thread
    // keeps the four samples i = 4 (tid % 8) .. 4 (tid % 8) + 3 of row j =
    // tid / 8 for every k, so the factors that depend on i, j or k alone are
    // formed once and the row's four codes leave in one 32-bit store; each
    // sample still runs the same operations in the same order.
    const int i0 = (threadIdx.x & 7) * 4, j = threadIdx.x >> 3;
    float cxq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cxq[q] = fadd(cc.x0, fmul((float)(i0 + q), cc.xs));
    const float cy = fadd(cc.y0, fmul((float)j, cc.ys));
    uint32_t *cw = (uint32_t *)(cv + j * 32 + i0);
    for (int k = 0; k < kCrop; ++k) {
      const float fr = fmul(fadd((float)k, 0.5f), 0.03125f);  // (k + 1/2) / 32, exact
      const float py = fmul(cy, fr), pz = fmul(cc.zc, fr);
      float ry[3], rz[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ry[a] = fmul(r[3 * a + 1], py);
        rz[a] = fmul(r[3 * a + 2], pz);
      }
      uint32_t word = 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float px = fmul(cxq[q], fr);
        int idx[3];
        bool inside = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float w = fadd(fadd(fmul(r[3 * a], px), ry[a]), rz[a]);
          const float qa = fadd(o[a], fmul(w, cc.inv_s));
          const float fl = floorf(qa);
          inside = inside && fl >= 0.0f && fl < (float)dims[a];
          idx[a] = inside ? (int)fl : 0;
        }
        uint32_t cls = 3u;  // 3 = outside: no channel set
        if (inside) {
          const int32_t off = LINEAR ? (idx[2] * m.ny + idx[1]) * m.nx + idx[0]
                                     : m.tab[idx[0]] + m.tab[m.nx + idx[1]] + m.tab[m.nx + m.ny + idx[2]];
          if (KIND == PAYLOAD_GAIN_F32) {
            const float pv = __ldg((const float *)m.payload + off);
            cls = pv > cc.occ_thr ? 2u : (pv < cc.free_thr ? 1u : 0u);
          } else if (KIND == PAYLOAD_U8) {
            const uint32_t st = __ldg((const uint8_t *)m.payload + off);
            cls = st >= 2u ? 2u : st;
          } else {
            const uint32_t byte = __ldg((const uint8_t *)m.payload + (off >> 2));
            const uint32_t st = (byte >> ((off & 3) << 1)) & 3u;
            cls = st >= 2u ? 2u : st;
          }
        }
        // code: 0 outside the map, else 1 + class (unknown, free, occupied)
        word |= (cls < 3u ? cls + 1u : 0u) << (8 * q);
      }
      cw[k * 256] = word;  // cells k * 1024 + j * 32 + i0 .. i0 + 3
    }
    if (threadIdx.x == 0) {
      const float ext[3] = {cc.ext_x, cc.ext_y, cc.ext_z};
#pragma unroll
      for (int a = 0; a < 3; ++a) feats[v * kFeat + a] = __float2bfloat16_rn(__fdiv_rn(fsub(s_pz[a], org[a]), ext[a]));
#pragma unroll
      for (int a = 0; a < 4; ++a) feats[v * kFeat + 3 + a] = __float2bfloat16_rn(s_pz[3 + a]);
      feats[v * kFeat + 7] = __float2bfloat16_rn(1.0f);
    }
  }
}

// Layer 0 sees one-hot crops, so it needs no multiplications: output
// channel co of an output voxel is b0[co] plus, over the 27 taps, the weight
// W0[co][tap][class] of the class of the tap's input sample (a sample
// outside the map, or a tap in the zero padding, adds nothing); then ReLU.
// The [tap][code][channel] table of BF16-rounded weights sits in shared
// memory (code 0, outside the map, is a zero row).
constexpr int kCodes = 4;
constexpr int kC1 = 16;      // layer 0 output channels
constexpr int kRowPad = 20;  // table row stride in floats: the four class rows of a tap fall in different banks

__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

__global__ void __launch_bounds__(256) conv0_lookup_kernel(const uint8_t *__restrict__ codes, const bf16 *__restrict__ w0,
                                                           const float *__restrict__ b0, int64_t n_views,
                                                           bf16 *__restrict__ act0) {
  __shared__ __align__(16) float tab[27 * kCodes * kRowPad];
  __shared__ __align__(16) uint8_t s_code[kCrop * kCrop * kCrop];
  __shared__ __align__(16) float bias[kC1];
  for (int e = threadIdx.x; e < 27 * kCodes * kC1; e += blockDim.x) {
    const int co = e % kC1, code = (e / kC1) % kCodes, tap = e / (kC1 * kCodes);
    tab[(tap * kCodes + code) * kRowPad + co] =
        code == 0 ? 0.0f : __bfloat162float(w0[co * (27 * kC0) + tap * kC0 + (code - 1)]);
  }
  if (threadIdx.x < kC1) bias[threadIdx.x] = b0[threadIdx.x];
  constexpr int kIn = kCrop * kCrop * kCrop, kOut = 16 * 16 * 16;
  for (int64_t v = blockIdx.x; v < n_views; v += gridDim.x) {
    __syncthreads();
    const uint4 *src = (const uint4 *)(codes + v * (int64_t)kIn);
    for (int e = threadIdx.x; e < kIn / 16; e += blockDim.x) ((uint4 *)s_code)[e] = src[e];
    __syncthreads();
    for (int cell = threadIdx.x; cell < kOut; cell += blockDim.x) {
      const int ox = cell & 15, oy = (cell >> 4) & 15, oz = cell >> 8;
      unsigned long long acc[kC1 / 2];
#pragma unroll
      for (int q = 0; q < kC1 / 2; ++q) acc[q] = ((const unsigned long long *)bias)[q];
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
        const int iz = 2 * oz + dz - 1;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const int iy = 2 * oy + dy - 1;
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const int ix = 2 * ox + dx - 1;
            const bool in = iz >= 0 && iz < kCrop && iy >= 0 && iy < kCrop && ix >= 0 && ix < kCrop;
            const int code = in ? s_code[(iz * kCrop + iy) * kCrop + ix] : 0;
            const float4 *row = (const float4 *)(tab + ((dz * 9 + dy * 3 + dx) * kCodes + code) * kRowPad);
#pragma unroll
            for (int q = 0; q < kC1 / 4; ++q) {
              const float4 w = row[q];
              const ulonglong2 wp = *(const ulonglong2 *)&w;
              acc[2 * q] = add_f32x2(acc[2 * q], wp.x);
              acc[2 * q + 1] = add_f32x2(acc[2 * q + 1], wp.y);
            }
          }
        }
      }
      uint4 out[2];
      uint32_t *u = (uint32_t *)out;
#pragma unroll
      for (int q = 0; q < kC1 / 2; ++q) {
        const float2 f = *(const float2 *)&acc[q];
        const __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(f.x, 0.0f), fmaxf(f.y, 0.0f));
        u[q] = *(const uint32_t *)&h;
      }
      uint4 *dst = (uint4 *)(act0 + (v * (int64_t)kOut + cell) * kC1);
      dst[0] = out[0];
      dst[1] = out[1];
    }
  }
}

// ---------------------------------------------------------------------------
// Layers 0 and 1 fused for inference: one CTA of 17 warps per crop at a
// time (persistent, one CTA per SM), both layers on tcgen05 with the A
// operands in tensor memory; only layer 1's output goes to global memory.
//
// Layer 0 as a GEMM over one-hot inputs: rows = output voxels (16^3 per
// crop, 32 tiles of 128), K = 28 taps x 4 slots (tap 27 and slot 3 are
// zero), slot s of a tap = 1.0 where the tap's input class code is s + 1;
// B = W0 on the three class channels (shared memory).  The crop's codes are
// repacked to 2 bits (one 64-bit word per x-row); the three codes a tap row
// needs (x = 2 ox - 1 .. 2 ox + 1) come out of one shift, and a 16-byte
// chunk of A (two taps) is one entry of a 16-entry table indexed by the two
// codes, stored by the row's own thread into its TMEM lane (tcgen05.st).
// Four A tiles in flight.  Bias and ReLU in the epilogue, which writes the
// layer-0 activation into shared memory as [channel group 0..1][z][y][x']
// 16-byte vectors with x' = (x & 1) * 8 + x / 2: the stride-2 reads of
// layer 1 then hit consecutive vectors.
// Layer 1: rows = 8^3 output voxels (4 tiles of 128), K = 27 taps x 16
// channels (padded to 2 stages of 224: each barrier round trip between the
// builders and the MMA warp costs more than the 14 MMAs of a stage), both in
// flight: each A chunk is
// read from the shared layer-0 activation (per-row offset plus per-chunk
// offset, zero where the tap falls in the padding: a 3-bit mask test) and
// stored into TMEM; W1 stays resident in shared memory.  TMEM: layer-0
// accumulators in 8 slots of 16 columns (0-127), layer 1 in 4 x 32
// (128-255), A stages from column 256.  Every mbarrier wait is bounded.
// ---------------------------------------------------------------------------
namespace fz {
constexpr int kThreads = 512;                  // builder threads (plus one MMA warp)
constexpr int kK0 = 112;                       // layer-0 K: 28 taps x 4 slots
constexpr int kTiles0 = 32;                    // 16^3 / 128
constexpr int kTiles1 = 4;                     // 8^3 / 128
constexpr int kChunksS1 = 28;                  // 16-byte A chunks per row in a layer-1 K stage (K = 224)
constexpr int kStages1 = 56 / kChunksS1;       // layer-1 K stages per tile (K = 27 taps x 16, padded to 448)
static_assert(56 % kChunksS1 == 0 && kChunksS1 % 2 == 0, "layer-1 stages");
constexpr int kBuf0 = 4;                       // layer-0 A tiles in flight (56 TMEM columns each)
constexpr int kBuf1 = 2;                       // layer-1 A stages in flight (112 TMEM columns each)
constexpr uint32_t kColA = 256;                // TMEM columns 0-127: layer-0 accumulators, 128-255: layer 1
constexpr uint32_t kColsA0 = kK0 / 2, kColsA1 = 4 * kChunksS1;
constexpr int kOffCodes = 0;                   // 32 x 32 x-rows x 8 B
constexpr int kOffAct0 = kOffCodes + 8192;     // 2 x 16^3 x 16 B
constexpr int kOffW0 = kOffAct0 + 131072;      // 7 K16 blocks x 16 rows x 32 B
constexpr int kOffW1 = kOffW0 + 3584;          // 28 K16 blocks x 32 rows x 32 B
constexpr int kOffLut = kOffW1 + 28672;
constexpr int kOffTap = kOffLut + 256;         // 64 x (offset, mask) for layer-1 chunks
constexpr int kSmem = kOffTap + 512;           // 172,288 B
constexpr uint32_t kTmemCols = 512;
static_assert(kColA + kBuf0 * kColsA0 <= kTmemCols && kColA + kBuf1 * kColsA1 <= kTmemCols, "TMEM budget");

// One-hot slots of class code c (0: none) as four BF16 values.
__host__ __device__ constexpr uint64_t onehot4(uint32_t c) { return (0x3F80ull << (16u * c)) >> 16; }


// Chunks [C0, C1) of this thread's layer-0 A row (output voxel (ox, oy,
// oz)), i.e. taps 2 C0 .. 2 C1 - 1: per tap row (dz, dy) the codes of x =
// 2 ox - 1 .. 2 ox + 1 at bits 0, 2, 4 of one word (x = -1 and rows outside
// the crop read as 0), then one table entry per pair of taps, stored into
// TMEM columns 4 kc .. 4 kc + 3 of the row's lane (trow: the tile's first
// column, the warp's lane quarter).
template <int C0, int C1>
__device__ __forceinline__ void build0(const uint64_t *codes, const uint4 *lut, uint32_t trow, int ox, int oy,
                                       int oz) {
  constexpr int n = 2 * (C1 - C0);
  uint32_t cd[n];
  uint32_t rowv = 0u;
  int row = -1;
#pragma unroll
  for (int i = 0; i < n; ++i) {
    const int tap = 2 * C0 + i;
    if (tap >= 27) {
      cd[i] = 0u;
      continue;
    }
    const int rw = tap / 3;  // (dz, dy) row, compile-time
    if (rw != row) {
      const int iz = 2 * oz + rw / 3 - 1, iy = 2 * oy + rw % 3 - 1;
      const uint64_t R = (iz | iy) < 0 ? 0ull : codes[iz * 32 + iy];  // upper bounds always hold
      rowv = ox == 0 ? (uint32_t)R << 2 : (uint32_t)(R >> (4 * ox - 2));
      row = rw;
    }
    cd[i] = (rowv >> (2 * (tap % 3))) & 3u;
  }
#pragma unroll
  for (int j = 0; j < C1 - C0; ++j) tc::tmem_st4(trow + 4u * (C0 + j), lut[cd[2 * j] | (cd[2 * j + 1] << 2)]);
}
}  // namespace fz

// Bounded wait that gives up at once when another warp already timed out
// (abort flag in shared memory); a timeout sets the flag.
__device__ __forceinline__ bool wait_abortable(uint64_t *bar, uint32_t par, volatile int *abort) {
  const uint64_t t0 = tc::globaltimer();
  while (!tc::mbar_try_wait(bar, par)) {
    if (*abort) return false;
    if (tc::globaltimer() - t0 > tc::c_wait_ns) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

// Warps 0-15 build the A stages (and read the accumulators back); warp 16
// waits for each stage to be complete, issues its MMAs and commits them.
// A stage is complete when all 512 builder threads have arrived on its
// "full" barrier (each after its own TMEM stores have completed); the
// commit arrives on its "empty" barrier, which the builders wait for before
// refilling the buffer or reading the accumulator.  No CTA-wide barrier
// inside the crop loop: the builders run up to four layer-0 tiles / two
// layer-1 stages ahead of the tensor core.
__global__ void __launch_bounds__(fz::kThreads + 32, 1)
    conv01_kernel(const uint8_t *__restrict__ codes, const bf16 *__restrict__ wb, const float *__restrict__ params,
                  int64_t n_views, bf16 *__restrict__ act1, int *err) {
  using namespace fz;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  __shared__ uint64_t full0[kBuf0], empty0[kBuf0], full1[kBuf1], empty1[kBuf1], bsync;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ float bias0[16], bias1[32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint64_t *codes64 = (uint64_t *)(sm + kOffCodes);
  uint8_t *act0 = sm + kOffAct0;
  uint8_t *w0s = sm + kOffW0, *w1s = sm + kOffW1;
  uint4 *lut = (uint4 *)(sm + kOffLut);
  int2 *tapinfo = (int2 *)(sm + kOffTap);
  volatile int *abort = &abort_flag;

  // resident operands: W0 on the class channels (K = 4 tap + slot), W1, biases, tables
  for (int e = tid; e < 16 * kK0; e += blockDim.x) {
    const int co = e / kK0, k = e % kK0, tap = k >> 2, sl = k & 3;
    const bf16 v = (tap < 27 && sl < 3) ? wb[kW0 + co * (27 * kC0) + tap * kC0 + sl] : __float2bfloat16(0.0f);
    const int kc = k >> 3;
    *(bf16 *)(w0s + (kc >> 1) * (16 * 32) + (co >> 3) * 256 + (kc & 1) * 128 + (co & 7) * 16 + (k & 7) * 2) = v;
  }
  for (int e = tid; e < 32 * 448; e += blockDim.x) {
    const int co = e / 448, k = e % 448;
    const bf16 v = k < 27 * 16 ? wb[kW1 + co * (27 * 16) + k] : __float2bfloat16(0.0f);
    const int kc = k >> 3;
    *(bf16 *)(w1s + (kc >> 1) * (32 * 32) + (co >> 3) * 256 + (kc & 1) * 128 + (co & 7) * 16 + (k & 7) * 2) = v;
  }
  if (tid < 16) {
    const uint64_t a = onehot4(tid & 3), b = onehot4(tid >> 2);
    lut[tid] = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    bias0[tid] = params[kB0 + tid];
  }
  if (tid < 32) bias1[tid] = params[kB1 + tid];
  if (tid < 64) {
    // layer-1 chunk kc = 2 tap + channel group: act0 offset relative to the
    // output voxel's own, and which low-side paddings it falls into
    const int kc = tid, tap = kc >> 1, cg = kc & 1;
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int xoff = dx == 0 ? 7 : (dx == 1 ? 0 : 8);
    const int off = cg * 65536 + (dz - 1) * 4096 + (dy - 1) * 256 + xoff * 16;
    const int mask = kc < 54 ? ((dx == 0) | ((dy == 0) << 1) | ((dz == 0) << 2)) : 8;
    tapinfo[kc] = make_int2(off, mask);
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) {
    for (int i = 0; i < kBuf0; ++i) {
      tc::mbar_init(&full0[i], kThreads);
      tc::mbar_init(&empty0[i], 1);
    }
    for (int i = 0; i < kBuf1; ++i) {
      tc::mbar_init(&full1[i], kThreads);
      tc::mbar_init(&empty1[i], 1);
    }
    tc::mbar_init(&bsync, kThreads);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_smem_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == kThreads / 32) {
    // ---- MMA warp: lane 0 issues, the whole warp follows the same waits ----
    constexpr uint32_t idesc0 = tc::idesc_bf16(128, 16);
    constexpr uint32_t idesc1 = tc::idesc_bf16(128, 32);
    // descriptors built once; a byte offset o moves the start address field
    // by o / 16 (no carry out of its 14 bits: shared memory is < 256 KB)
    const uint64_t w0_d = tc::sdesc(tc::smem_u32(w0s), 128, 256);
    const uint64_t w1_d = tc::sdesc(tc::smem_u32(w1s), 128, 256);
    uint32_t g0 = 0, g1 = 0;
    bool ok = true;
    uint64_t *last_bar = nullptr;  // the last commit (it covers every earlier MMA)
    uint32_t last_par = 0;
    for (int64_t view = blockIdx.x; view < n_views && ok; view += gridDim.x) {
      for (int t = 0; t < kTiles0 && ok; ++t) {
        const uint32_t g = g0 + (uint32_t)t, b = g % kBuf0;
        ok = __all_sync(0xffffffffu, wait_abortable(&full0[b], (g / kBuf0) & 1u, abort)) != 0;
        if (ok && lane == 0) {
          tc::fence_after_sync();
          const uint32_t a0 = tmem + kColA + b * kColsA0;
          const uint32_t d = tmem + (uint32_t)((t & 7) * 16);
#pragma unroll
          for (int kk = 0; kk < kK0 / 16; ++kk)
            tc::mma_bf16_ta(d, a0 + 8u * kk, w0_d + kk * (16 * 32 / 16), idesc0, kk > 0 ? 1u : 0u);
          tc::mma_commit(&empty0[b]);
        }
        if (ok) {
          last_bar = &empty0[b];
          last_par = (g / kBuf0) & 1u;
        }
        __syncwarp();
      }
      g0 += kTiles0;
      for (int s = 0; s < kTiles1 * kStages1 && ok; ++s) {
        const int mt = s / kStages1, ks = s % kStages1;
        const uint32_t g = g1 + (uint32_t)s, b = g % kBuf1;
        ok = __all_sync(0xffffffffu, wait_abortable(&full1[b], (g / kBuf1) & 1u, abort)) != 0;
        if (ok && lane == 0) {
          tc::fence_after_sync();
          const uint32_t a0 = tmem + kColA + b * kColsA1;
          const uint64_t b0 = w1_d + ks * (kChunksS1 / 2 * 32 * 32 / 16);
          const uint32_t d = tmem + 128u + (uint32_t)(mt * 32);
#pragma unroll
          for (int kk = 0; kk < kChunksS1 / 2; ++kk)
            tc::mma_bf16_ta(d, a0 + 8u * kk, b0 + kk * (32 * 32 / 16), idesc1, (ks | kk) != 0 ? 1u : 0u);
          tc::mma_commit(&empty1[b]);
        }
        if (ok) {
          last_bar = &empty1[b];
          last_par = (g / kBuf1) & 1u;
        }
        __syncwarp();
      }
      g1 += kTiles1 * kStages1;
    }
    // before TMEM is freed: the last commit done (bounded, whatever the abort flag says)
    if (last_bar) {
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(last_bar, last_par) && tc::globaltimer() - t0 < tc::c_wait_ns) {
      }
    }
  } else {
    // ---- builder warps ----
    const int quarter = warp & 3, part = warp >> 2;  // TMEM lane quarter; quarter of the row's chunks / columns
    const int r = quarter * 32 + lane;               // A row (TMEM lane) of this thread
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    uint32_t g0 = 0, g1 = 0, nb = 0;
    bool ok = true;
    auto wait_warp = [&](uint64_t *bar, uint32_t par) {
      return __all_sync(0xffffffffu, wait_abortable(bar, par, abort)) != 0;
    };
    // all builders reach this point (bounded)
    auto builders_sync = [&]() {
      tc::fence_before_sync();
      mbar_arrive(&bsync);
      const bool r_ok = __all_sync(0xffffffffu, wait_abortable(&bsync, nb & 1u, abort)) != 0;
      ++nb;
      tc::fence_after_sync();
      return r_ok;
    };
    // publish this thread's TMEM stage stores (and earlier accumulator reads) to the MMA warp
    auto publish = [&](uint64_t *bar) {
      tc::tmem_wait_st();
      tc::fence_before_sync();
      mbar_arrive(bar);
    };
    // layer-0 epilogue of tile t (slot t & 7): 4 channels per thread, bias, ReLU, BF16 into act0
    auto epi0 = [&](int t) {
      tc::fence_after_sync();
      float v[4];
      tc::tmem_ld4(tmem + lane_base + (uint32_t)((t & 7) * 16 + part * 4), v);
      const int cell = t * 128 + r;
      const int ox = cell & 15, oy = (cell >> 4) & 15, oz = cell >> 8;
      const __nv_bfloat162 h0 = __floats2bfloat162_rn(fmaxf(v[0] + bias0[part * 4], 0.0f),
                                                      fmaxf(v[1] + bias0[part * 4 + 1], 0.0f));
      const __nv_bfloat162 h1 = __floats2bfloat162_rn(fmaxf(v[2] + bias0[part * 4 + 2], 0.0f),
                                                      fmaxf(v[3] + bias0[part * 4 + 3], 0.0f));
      const int xp = (ox & 1) * 8 + (ox >> 1);
      *(uint2 *)(act0 + ((((part >> 1) * 16 + oz) * 16 + oy) * 16 + xp) * 16 + (part & 1) * 8) =
          make_uint2(*(const uint32_t *)&h0, *(const uint32_t *)&h1);
    };

    for (int64_t view = blockIdx.x; view < n_views && ok; view += gridDim.x) {
      // codes of this crop, 2 bits each: 16 codes (16 bytes) -> 32 bits
      {
        const uint4 *src = (const uint4 *)(codes + view * (int64_t)(kCrop * kCrop * kCrop));
        for (int c = tid; c < 2048; c += kThreads) {
          const uint4 v = __ldg(src + c);
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
          uint32_t p = 0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t b = (w[q] & 3u) | ((w[q] >> 6) & 0xCu) | ((w[q] >> 12) & 0x30u) | ((w[q] >> 18) & 0xC0u);
            p |= b << (8 * q);
          }
          ((uint32_t *)codes64)[c] = p;
        }
      }
      ok = builders_sync();  // codes complete
      // ---- layer 0: 32 tiles of 128 output voxels, four A tiles in flight ----
      // Tile t's A buffer was last used by tile t - 4, whose MMAs precede
      // those of tile t - 2, awaited for its epilogue; at a crop's first
      // tiles the previous crop's MMAs are all done.
      const int ox0 = r & 15;  // the same for every tile
      for (int t = 0; t < kTiles0 && ok; ++t) {
        const uint32_t g = g0 + (uint32_t)t, b = g % kBuf0;
        if (t >= 2) {
          const uint32_t ge = g - 2u;
          ok = wait_warp(&empty0[ge % kBuf0], (ge / kBuf0) & 1u);  // tile t - 2 done: accumulator ready
          if (!ok) break;
          epi0(t - 2);
        }
        const int oy = (8 * t + (r >> 4)) & 15, oz = t >> 1;
        const uint32_t trow = tmem + lane_base + kColA + b * kColsA0;
        switch (part) {  // chunks 0-3, 4-7, 8-10, 11-13
          case 0: build0<0, 4>(codes64, lut, trow, ox0, oy, oz); break;
          case 1: build0<4, 8>(codes64, lut, trow, ox0, oy, oz); break;
          case 2: build0<8, 11>(codes64, lut, trow, ox0, oy, oz); break;
          default: build0<11, 14>(codes64, lut, trow, ox0, oy, oz); break;
        }
        publish(&full0[b]);
      }
      if (!ok) break;
      {
        const uint32_t g = g0 + kTiles0 - 1;
        ok = wait_warp(&empty0[g % kBuf0], (g / kBuf0) & 1u);  // the last tile's commit covers every layer-0 MMA
      }
      if (!ok) break;
      epi0(kTiles0 - 2);
      epi0(kTiles0 - 1);
      g0 += kTiles0;
      ok = builders_sync();  // act0 complete
      if (!ok) break;
      // ---- layer 1: 4 M tiles x 2 K stages, both in flight ----
      {
        const int jj = tid >> 7;  // this thread's chunks of a stage: jj, jj + 4, ... (warp-uniform)
        const int ox = r & 7, oy = (r >> 3) & 7, ozl = r >> 6;
        for (int s = 0; s < kTiles1 * kStages1 && ok; ++s) {
          const int mt = s / kStages1, ks = s % kStages1;
          const uint32_t g = g1 + (uint32_t)s, b = g % kBuf1;
          if (s >= kBuf1) {
            ok = wait_warp(&empty1[b], ((g - kBuf1) / kBuf1) & 1u);
            if (!ok) break;
          }
          const int oz = 2 * mt + ozl;
          const int base = oz * 8192 + oy * 512 + ox * 16;
          const int low = (ox == 0) | ((oy == 0) << 1) | ((oz == 0) << 2) | 8;
          const uint32_t trow = tmem + lane_base + kColA + b * kColsA1;
#pragma unroll
          for (int j = jj; j < kChunksS1; j += 4) {
            const int2 ti = tapinfo[ks * kChunksS1 + j];
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if ((low & ti.y) == 0) v = *(const uint4 *)(act0 + base + ti.x);
            tc::tmem_st4(trow + 4u * j, v);
          }
          publish(&full1[b]);
        }
      }
      if (!ok) break;
      {
        const uint32_t g = g1 + kTiles1 * kStages1 - 1;
        ok = wait_warp(&empty1[g % kBuf1], (g / kBuf1) & 1u);  // every layer-1 MMA done, every stage built
      }
      if (!ok) break;
      g1 += kTiles1 * kStages1;
      tc::fence_after_sync();
      for (int mt = 0; mt < kTiles1; ++mt) {
        float v[8];
        tc::tmem_ld8(tmem + lane_base + 128u + (uint32_t)(mt * 32 + part * 8), v);
        const int o = mt * 128 + r;
        uint32_t u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const __nv_bfloat162 hh = __floats2bfloat162_rn(fmaxf(v[2 * q] + bias1[part * 8 + 2 * q], 0.0f),
                                                          fmaxf(v[2 * q + 1] + bias1[part * 8 + 2 * q + 1], 0.0f));
          u[q] = *(const uint32_t *)&hh;
        }
        *(uint4 *)(act1 + ((size_t)view * 512 + o) * 32 + part * 8) = make_uint4(u[0], u[1], u[2], u[3]);
      }
    }
    if (!ok) *abort = 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*abort && tid == 0) atomicExch(err, 1);
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Layers 2 and 3 (both 4^3 outputs per crop, 64 channels): a 128-row tile is
// exactly two crops, so the tile's whole input (two crops' activations:
// 2 x 32 KB for layer 2, 2 x 8 KB for layer 3) is staged in shared memory
// once and the im2col stages are copied shared -> shared instead of
// gathering each input vector up to 27 times from L2.  Same K order, same
// MMA sequence and same epilogues as the generic implicit GEMM, so the
// outputs are bit-identical.  Two persistent CTAs per SM, each 8 builder
// warps (A from the staged input into TMEM, B = the weight stage into
// shared memory by cp.async) and one MMA warp, two stages of K = 128 in
// flight on full/empty mbarriers (wider stages, fewer barrier round trips:
// 2.777 M against 2.758 M views/s with four stages of 64); the next tile's
// input is staged while the current tile's last MMAs run.
// ---------------------------------------------------------------------------
namespace c23 {
constexpr int kBuilders = 256;                   // builder threads (plus one MMA warp); two CTAs per SM
constexpr int kParts = kBuilders / 128;          // builders per tile row
constexpr int kSC = 16;                          // 16-byte K chunks per stage row (K = 128 per stage)
constexpr int kBuf = 2;                          // stages in flight
constexpr int kStageB = 64 * kSC * 16;           // weights per stage (A stages live in TMEM)
constexpr int kMaxIn = 2 * 8 * 8 * 8 * 32 * 2;   // two crops of layer 2's input: 64 KB
constexpr int kOffIn = 0;
constexpr int kOffStage = kOffIn + kMaxIn;
constexpr int kOffTap = kOffStage + kBuf * kStageB;
constexpr int kSmem = kOffTap + 256 * 8;         // 100,352 B
constexpr uint32_t kColA = 64, kColsA = 4 * kSC;  // TMEM: accumulator in columns 0-63, A stages after it
constexpr uint32_t kTmemCols = 256;
static_assert(kColA + kBuf * kColsA <= kTmemCols && kSC % 2 == 0 && kSC <= 32, "conv23 stages");

template <int L>
struct Geo;
template <>
struct Geo<2> {
  static constexpr int din = 8, stride = 2, cin = 32, cg = 4, stages = (27 * cg + kSC - 1) / kSC;
};
template <>
struct Geo<3> {
  static constexpr int din = 4, stride = 1, cin = 64, cg = 8, stages = (27 * cg + kSC - 1) / kSC;
};
}  // namespace c23

template <int L>
__global__ void __launch_bounds__(c23::kBuilders + 32, 2)
    conv23_kernel(const bf16 *__restrict__ in, const bf16 *__restrict__ w, const float *__restrict__ bias,
                  int64_t n_views, bf16 *__restrict__ out, int *err) {
  using namespace c23;
  using G = Geo<L>;
  constexpr int kIn = G::din * G::din * G::din * G::cin * 2;  // bytes of one crop's input
  constexpr int kK = 27 * G::cin;                               // weight row length
  constexpr int kChunks = 27 * G::cg;                           // real 16-byte chunks of a row
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t *sm = (uint8_t *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  __shared__ uint64_t full[kBuf], empty[kBuf], bsync;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ float sbias[64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *sin = sm + kOffIn, *stg = sm + kOffStage;
  int2 *tapinfo = (int2 *)(sm + kOffTap);
  volatile int *abort = &abort_flag;
  const int64_t n_tiles = (n_views + 1) / 2;

  if (tid < 64) sbias[tid] = bias[tid];
  static_assert(G::stages * kSC <= 256, "tap table");
  for (int kc = tid; kc < G::stages * kSC; kc += blockDim.x) {
    // chunk kc = tap * cg + channel group: input offset relative to the output
    // voxel's own, and the padding cases it falls into (bit 6: past K)
    const int tap = kc / G::cg, cgi = kc % G::cg;
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int off = (((dz - 1) * G::din + (dy - 1)) * G::din + (dx - 1)) * G::cin * 2 + cgi * 16;
    int mask = (dx == 0) | ((dy == 0) << 1) | ((dz == 0) << 2);
    if (G::stride == 1) mask |= ((dx == 2) << 3) | ((dy == 2) << 4) | ((dz == 2) << 5);
    tapinfo[kc] = make_int2(off, kc < kChunks ? mask : 64);
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, kTmemCols);
  if (tid == 0) {
    for (int i = 0; i < kBuf; ++i) {
      tc::mbar_init(&full[i], kBuilders);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_init(&bsync, kBuilders);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;

  if (warp == kBuilders / 32) {
    // ---- MMA warp ----
    constexpr uint32_t idesc = tc::idesc_bf16(128, 64);
    const uint64_t stg_d = tc::sdesc(tc::smem_u32(stg), 128, 256);
    uint32_t g = 0;
    bool ok = true;
    uint64_t *last_bar = nullptr;
    uint32_t last_par = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
      for (int ks = 0; ks < G::stages && ok; ++ks, ++g) {
        const uint32_t b = g % kBuf;
        ok = __all_sync(0xffffffffu, wait_abortable(&full[b], (g / kBuf) & 1u, abort)) != 0;
        if (ok && lane == 0) {
          tc::fence_after_sync();
          const uint64_t b0 = stg_d + (b * kStageB >> 4);
          const uint32_t a0 = tmem + kColA + b * kColsA;
#pragma unroll
          for (int kk = 0; kk < kSC / 2; ++kk)
            tc::mma_bf16_ta(tmem, a0 + 8u * kk, b0 + kk * (64 * 32 / 16), idesc, (ks | kk) != 0 ? 1u : 0u);
          tc::mma_commit(&empty[b]);
        }
        if (ok) {
          last_bar = &empty[b];
          last_par = (g / kBuf) & 1u;
        }
        __syncwarp();
      }
    }
    if (last_bar) {  // before TMEM is freed (bounded)
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(last_bar, last_par) && tc::globaltimer() - t0 < tc::c_wait_ns) {
      }
    }
  } else {
    // ---- builder warps ----
    const int quarter = warp & 3, part = warp >> 2;
    const int r = quarter * 32 + lane;  // tile row = TMEM lane of this thread
    const int crop = r >> 6, o = r & 63, ox = o & 3, oy = (o >> 2) & 3, oz = o >> 4;
    const int base = crop * kIn + ((G::stride * oz * G::din + G::stride * oy) * G::din + G::stride * ox) * G::cin * 2;
    int rowmask = (ox == 0) | ((oy == 0) << 1) | ((oz == 0) << 2) | 64;
    if (G::stride == 1) rowmask |= ((ox == 3) << 3) | ((oy == 3) << 4) | ((oz == 3) << 5);
    const int jj = tid >> 7;  // A chunks jj, jj + kParts, ... of a stage (warp-uniform)
    uint32_t g = 0, nb = 0;
    bool ok = true;
    auto wait_warp = [&](uint64_t *bar, uint32_t par) {
      return __all_sync(0xffffffffu, wait_abortable(bar, par, abort)) != 0;
    };
    auto builders_sync = [&]() {
      tc::fence_before_sync();
      mbar_arrive(&bsync);
      const bool r_ok = __all_sync(0xffffffffu, wait_abortable(&bsync, nb & 1u, abort)) != 0;
      ++nb;
      tc::fence_after_sync();
      return r_ok;
    };
    // the tile's two crops (the second may be past the batch: zeros)
    auto stage_input = [&](int64_t tile) {
      const uint32_t dst = tc::smem_u32(sin);
      for (int c = tid; c < 2 * kIn / 16; c += kBuilders) {
        const int64_t v = 2 * tile + (c * 16) / kIn;
        const bool valid = v < n_views;
        const uint8_t *src = (const uint8_t *)in + (valid ? (2 * tile * (int64_t)kIn + (int64_t)c * 16) : 0);
        tc::cp_async16(dst + c * 16, src, valid);
      }
      tc::cp_async_commit();
    };
    int64_t tile = blockIdx.x;
    if (tile < n_tiles) stage_input(tile);
    for (; tile < n_tiles && ok; tile += gridDim.x) {
      tc::cp_async_wait<0>();
      ok = builders_sync();  // this tile's input staged
      if (!ok) break;
      for (int ks = 0; ks < G::stages && ok; ++ks, ++g) {
        const uint32_t b = g % kBuf;
        if (g >= kBuf) {
          ok = wait_warp(&empty[b], ((g - kBuf) / kBuf) & 1u);
          if (!ok) break;
        }
        uint8_t *sb = stg + b * kStageB;
        const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16) + kColA + b * kColsA;
#pragma unroll
        for (int i = 0; i < 64 * kSC / kBuilders; ++i) {  // B: weight rows 0..63, K chunks kSC ks ..
          const int c = tid + kBuilders * i, br = c / kSC, bj = c % kSC;
          const int kc = ks * kSC + bj;
          const bool valid = kc < kChunks;
          const bf16 *src = w + (valid ? (size_t)br * kK + kc * 8 : 0);
          tc::cp_async16(tc::smem_u32(sb + (bj >> 1) * (64 * 32) + (br >> 3) * 256 + (bj & 1) * 128 + (br & 7) * 16),
                         src, valid);
        }
        tc::cp_async_commit();
#pragma unroll
        for (int i = 0; i < kSC / kParts; ++i) {  // A: im2col from the staged input
          const int j = jj + kParts * i;
          const int2 ti = tapinfo[ks * kSC + j];
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if ((rowmask & ti.y) == 0) v = *(const uint4 *)(sin + base + ti.x);
          tc::tmem_st4(trow + 4u * j, v);
        }
        tc::cp_async_wait<0>();
        tc::tmem_wait_st();
        tc::fence_smem_async();
        tc::fence_before_sync();
        mbar_arrive(&full[b]);
      }
      if (!ok) break;
      // every stage of this tile built: stage the next tile's input meanwhile
      const int64_t next = tile + gridDim.x;
      ok = builders_sync();  // all builders are done reading this tile's input
      if (!ok) break;
      if (next < n_tiles) stage_input(next);
      {
        const uint32_t gl = g - 1;
        ok = wait_warp(&empty[gl % kBuf], (gl / kBuf) & 1u);  // the tile's last commit covers all its MMAs
      }
      if (!ok) break;
      tc::fence_after_sync();
      const int64_t m = 2 * tile * 64 + r;
#pragma unroll
      for (int h = 0; h < 64 / kParts / 16; ++h) {  // columns n0 .. n0 + 15 of this row
        const int n0 = part * (64 / kParts) + 16 * h;
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)n0, v);
        if (m < n_views * 64) {
          uint32_t u[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const __nv_bfloat162 hh = __floats2bfloat162_rn(fmaxf(v[2 * q] + sbias[n0 + 2 * q], 0.0f),
                                                            fmaxf(v[2 * q + 1] + sbias[n0 + 2 * q + 1], 0.0f));
            u[q] = *(const uint32_t *)&hh;
          }
          bf16 *d = L == 2 ? out + m * 64 + n0 : out + (m >> 6) * kFcIn + (m & 63) * 64 + n0;
          ((uint4 *)d)[0] = make_uint4(u[0], u[1], u[2], u[3]);
          ((uint4 *)d)[1] = make_uint4(u[4], u[5], u[6], u[7]);
        }
      }
      tc::fence_before_sync();  // accumulator read before the next tile's MMAs (ordered by the full barriers)
    }
    tc::cp_async_wait<0>();
    if (!ok) *abort = 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (*abort && tid == 0) atomicExch(err, 1);
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Layer 0 weight gradient on one-hot crops: dW0[co][tap][class] is the sum
// of dy[o][co] over the output voxels o whose tap input has that class.  CTA
// c reduces output voxels [c chunk, (c + 1) chunk) in order into
// part[c][tap][class][co]; conv0_wgrad_reduce_kernel adds the chunks in
// order (deterministic).
constexpr int kW0Sub = 128;   // output voxels staged in shared memory at a time

__global__ void __launch_bounds__(256) conv0_wgrad_kernel(const uint8_t *__restrict__ codes,
                                                          const bf16 *__restrict__ dy, int64_t n_out, int64_t chunk,
                                                          float *__restrict__ part) {
  __shared__ uint8_t s_code[kW0Sub][28];
  __shared__ float s_dy[kW0Sub][kC1];
  const int64_t o0 = blockIdx.x * chunk, o1 = min(n_out, o0 + chunk);
  float acc[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};   // pairs (tap, co) = threadIdx.x, + 256
  for (int64_t b = o0; b < o1; b += kW0Sub) {
    const int nb = (int)min((int64_t)kW0Sub, o1 - b);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * 27; e += blockDim.x) {
      const int k = e / 27, tap = e % 27;
      const int64_t o = b + k;
      const int cell = (int)(o & 4095);
      const int ox = cell & 15, oy = (cell >> 4) & 15, oz = cell >> 8;
      const int iz = 2 * oz + tap / 9 - 1, iy = 2 * oy + (tap / 3) % 3 - 1, ix = 2 * ox + tap % 3 - 1;
      const bool in = iz >= 0 && iz < kCrop && iy >= 0 && iy < kCrop && ix >= 0 && ix < kCrop;
      s_code[k][tap] = in ? codes[(o >> 12) * (int64_t)(kCrop * kCrop * kCrop) + (iz * kCrop + iy) * kCrop + ix] : 0;
    }
    for (int e = threadIdx.x; e < nb * kC1; e += blockDim.x) s_dy[e / kC1][e % kC1] = __bfloat162float(dy[b * kC1 + e]);
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int pidx = threadIdx.x + 256 * h;
      if (pidx < 27 * kC1) {
        const int tap = pidx / kC1, co = pidx % kC1;
        for (int k = 0; k < nb; ++k) {
          const int code = s_code[k][tap];
          const float g = s_dy[k][co];
          acc[h][0] += code == 1 ? g : 0.0f;
          acc[h][1] += code == 2 ? g : 0.0f;
          acc[h][2] += code == 3 ? g : 0.0f;
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int pidx = threadIdx.x + 256 * h;
    if (pidx < 27 * kC1) {
      const int tap = pidx / kC1, co = pidx % kC1;
#pragma unroll
      for (int c = 0; c < 3; ++c) part[((int64_t)blockIdx.x * 27 * 3 + tap * 3 + c) * kC1 + co] = acc[h][c];
    }
  }
}

__global__ void conv0_wgrad_reduce_kernel(const float *__restrict__ part, int chunks, float *__restrict__ dw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;   // e = co * 27 * kC0 + tap * kC0 + c
  if (e >= kC1 * 27 * kC0) return;
  const int co = e / (27 * kC0), tap = (e / kC0) % 27, c = e % kC0;
  float acc = 0.0f;
  if (c < 3)
    for (int z = 0; z < chunks; ++z) acc += part[((int64_t)z * 27 * 3 + tap * 3 + c) * kC1 + co];
  dw[e] = acc;
}

// X[:, 4096:4104] = feats.
__global__ void put_feats_kernel(const bf16 *__restrict__ feats, bf16 *__restrict__ x, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * kFeat) x[(size_t)(t / kFeat) * kFcIn + kFlat + t % kFeat] = feats[t];
}

// y[b] = h1[b] . f2 + g2 (one warp per sample, fixed shuffle tree).
__global__ void fc2_forward_kernel(const bf16 *__restrict__ h1, const float *__restrict__ params, int n,
                                   float *__restrict__ y) {
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (b >= n) return;
  const float *f2 = params + kP.f2;
  float acc = 0.0f;
  for (int j = lane; j < kHid; j += 32) acc += __bfloat162float(h1[(size_t)b * kHid + j]) * f2[j];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) y[b] = acc + params[kP.g2];
}

// Loss head (one block of 256 threads): loss = mean (y - c t)^2 with the
// net's target scale c (the product rounded to FP32 on its own), dy = 2 (y -
// c t) / n; grads of f2 and g2; dh1 = dy f2 [h1 > 0] (BF16, and transposed to
// [128][ldn]).
__global__ void head_backward_kernel(const float *__restrict__ y, const float *__restrict__ t, float tscale,
                                     const bf16 *__restrict__ h1, const float *__restrict__ params, int n, int ldn,
                                     float *__restrict__ grads, float *__restrict__ loss, bf16 *__restrict__ dh1,
                                     bf16 *__restrict__ dh1t) {
  __shared__ float red[256];
  __shared__ float s_dy[1024];
  const int tid = threadIdx.x;
  float l = 0.0f, gb = 0.0f;
  for (int b = tid; b < n; b += 256) {
    const float e = y[b] - __fmul_rn(t[b], tscale);
    l += e * e;
    const float d = 2.0f * e / (float)n;
    gb += d;
    if (b < 1024) s_dy[b] = d;
  }
  red[tid] = l;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0) *loss = red[0] / (float)n;
  __syncthreads();
  red[tid] = gb;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (tid < s) red[tid] += red[tid + s];
    __syncthreads();
  }
  if (tid == 0) grads[kP.g2] = red[0];
  __syncthreads();
  const float *f2 = params + kP.f2;
  for (int j = tid; j < kHid; j += 256) {
    float acc = 0.0f;
    for (int b = 0; b < n; ++b) acc += s_dy[b] * __bfloat162float(h1[(size_t)b * kHid + j]);
    grads[kP.f2 + j] = acc;
  }
  for (int e = tid; e < kHid * ldn; e += 256) {
    const int j = e / ldn, b = e % ldn;
    float d = 0.0f;
    if (b < n && __bfloat162float(h1[(size_t)b * kHid + j]) > 0.0f) d = s_dy[b] * f2[j];
    const bf16 v = __float2bfloat16_rn(d);
    dh1t[(size_t)j * ldn + b] = v;
    if (b < n) dh1[(size_t)b * kHid + j] = v;
  }
}

// out[c][r] = in[r][c] for r < rows (rows padded with zeros up to ldo), c < cols.
__global__ void transpose_kernel(const bf16 *__restrict__ in, int rows, int cols, int ldi, bf16 *__restrict__ out,
                                 int ldo) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ldi + c] : __float2bfloat16_rn(0.0f);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (c < cols && r < ldo) out[(size_t)c * ldo + r] = tile[threadIdx.x][k];
  }
}

// Column sums of a BF16 matrix [rows][cols] (bias gradients), one warp per
// column, fixed order.
__global__ void colsum_kernel(const bf16 *__restrict__ a, int64_t rows, int cols, float *__restrict__ out) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (c >= cols) return;
  float acc = 0.0f;
  for (int64_t r = lane; r < rows; r += 32) acc += __bfloat162float(a[r * cols + c]);
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) out[c] = acc;
}

// Split-K weight gradients: dW[co][k] = sum_z part[z][k][co], fixed z order.
// fc1's split-K partials (planes of n x 128 FP32) summed in split order, plus bias, ReLU, BF16.
__global__ void fc1_reduce_kernel(const float *__restrict__ part, int splits, int n, const float *__restrict__ bias,
                                  bf16 *__restrict__ h1) {
  const int64_t total = (int64_t)n * kHid;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    float acc = part[e];
    for (int z = 1; z < splits; ++z) acc += part[z * total + e];
    h1[e] = __float2bfloat16_rn(fmaxf(acc + bias[e % kHid], 0.0f));
  }
}

__global__ void wgrad_reduce_kernel(const float *__restrict__ part, int splits, int krows, int cout,
                                    float *__restrict__ dw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= krows * cout) return;
  const int k = e / cout, co = e % cout;
  float acc = 0.0f;
  for (int z = 0; z < splits; ++z) acc += part[(size_t)z * krows * cout + (size_t)k * cout + co];
  dw[(size_t)co * krows + k] = acc;
}

// Adam on the FP32 master parameters.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 operand copies of the weights: W_l [cout][27 cin] (forward B), WT_l
// [cin][27 cout] (input-gradient B), F1 [128][4104], F1T [4104][128].
__global__ void sync_weights_kernel(const float *__restrict__ p, bf16 *__restrict__ wb, bf16 *__restrict__ wtb,
                                    bf16 *__restrict__ f1b, bf16 *__restrict__ f1tb) {
  const int64_t total = kP.f1 + (int64_t)kHid * kFcIn;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < kP.f1) {
      // layer of this entry; every table access below uses a literal index
      const int l = e < kW1 ? 0 : (e < kW2 ? 1 : (e < kW3 ? 2 : 3));
      int cin, cout;
      int64_t wbase;
      switch (l) {
        case 0: cin = 8; cout = 16; wbase = kW0; break;
        case 1: cin = 16; cout = 32; wbase = kW1; break;
        case 2: cin = 32; cout = 64; wbase = kW2; break;
        default: cin = 64; cout = 64; wbase = kW3; break;
      }
      const int64_t o = e - wbase;
      const int kk = 27 * cin;
      if (o >= (int64_t)cout * kk) continue;  // bias entries
      const int co = (int)(o / kk), k = (int)(o % kk);
      const int tap = k / cin, ci = k % cin;
      const bf16 v = __float2bfloat16_rn(p[e]);
      wb[wbase + o] = v;
      wtb[wbase + (int64_t)ci * 27 * cout + tap * cout + co] = v;
    } else {
      const int64_t o = e - kP.f1;
      const int j = (int)(o / kFcIn), c = (int)(o % kFcIn);
      const bf16 v = __float2bfloat16_rn(p[e]);
      f1b[o] = v;
      f1tb[(int64_t)c * kHid + j] = v;
    }
  }
}

// Per-segment top-k (one CTA per segment of seg <= 8192 scores): bitonic
// sort in shared memory, descending score, ties to the lower index (so the
// order is deterministic); writes the kept global indices and, if asked,
// the kept poses.
__global__ void segment_topk_kernel(const float *__restrict__ scores, int seg, int keep, int pow2,
                                    int32_t *__restrict__ idx_out, const float *__restrict__ poses,
                                    float *__restrict__ poses_out) {
  extern __shared__ uint8_t sm[];
  float *key = (float *)sm;
  int32_t *id = (int32_t *)(key + pow2);
  const int64_t base = (int64_t)blockIdx.x * seg;
  for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
    const float v = i < seg ? scores[base + i] : -INFINITY;
    key[i] = v != v ? -INFINITY : v;  // NaN scores rank last
    id[i] = i;
  }
  __syncthreads();
  for (int k = 2; k <= pow2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < pow2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          // "before(a, b)": a ranks ahead of b
          const bool ab = key[i] > key[l] || (key[i] == key[l] && id[i] < id[l]);
          const bool desc = (i & k) == 0;
          if (desc ? !ab : ab) {
            const float tk = key[i];
            key[i] = key[l];
            key[l] = tk;
            const int32_t ti = id[i];
            id[i] = id[l];
            id[l] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < keep; r += blockDim.x) {
    const int64_t g = base + id[r];
    idx_out[(int64_t)blockIdx.x * keep + r] = (int32_t)g;
    if (poses && poses_out)
      for (int q = 0; q < 7; ++q) poses_out[((int64_t)blockIdx.x * keep + r) * 7 + q] = poses[g * 7 + q];
  }
}

// Per-segment argmax (one warp per segment): the largest value, ties to the
// lowest original index (idx maps position -> original index, or identity).
__global__ void segment_argmax_kernel(const float *__restrict__ vals, const int32_t *__restrict__ idx, int64_t n_seg,
                                      int seg, int32_t *__restrict__ best_idx, float *__restrict__ best_val) {
  const int64_t sgi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (sgi >= n_seg) return;
  float bv = -INFINITY;
  int32_t bi = INT32_MAX;
  for (int i = lane; i < seg; i += 32) {
    const int64_t p = sgi * seg + i;
    const float v = vals[p];
    const int32_t o = idx ? idx[p] : (int32_t)p;
    if (v > bv || (v == bv && o < bi)) {
      bv = v;
      bi = o;
    }
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const float ov = __shfl_xor_sync(0xffffffffu, bv, s);
    const int32_t oi = __shfl_xor_sync(0xffffffffu, bi, s);
    if (ov > bv || (ov == bv && oi < bi)) {
      bv = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    best_idx[sgi] = bi;
    if (best_val) best_val[sgi] = bv;
  }
}

// Test kernel of the bounded waits: the CTA holds all 512 TMEM columns of
// its SM and waits on an mbarrier that nothing ever completes, through the
// same bounded wait as the GEMM kernels; when the wait gives up it sets the
// error word, frees its tensor memory and returns.
__global__ void __launch_bounds__(128) tc_wait_probe_kernel(int *err) {
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const bool ok = __syncthreads_and(tc::mbar_wait(&bar, 0)) != 0;  // phase 0 never completes
  if (!ok && tid == 0) atomicExch(err, 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_base, 512);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

int *g_err[64] = {nullptr};

int dev_err_word(int **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return NBT_ECUDA;
  if (!g_err[dev]) {
    int *p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return NBT_ENOMEM;
    if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return NBT_ECUDA;
    g_err[dev] = p;
  }
  *out = g_err[dev];
  return NBT_OK;
}

template <int BN, class LA, class LB, class EP>
int launch_gemm(const LA &la, const LB &lb, const EP &ep, int M, int N, int K, int splits, cudaStream_t stream) {
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  // loaders that name a 16-byte source per chunk get the cp.async pipeline
  void (*kern)(LA, LB, EP, int, int, int, int *);
  size_t smem;
  if constexpr (LA::kAsync && LB::kAsync) {
    kern = tc::gemm_async_kernel<BN, LA, LB, EP>;
    smem = tc::gemm_async_smem_bytes(BN);
  } else {
    kern = tc::gemm_kernel<BN, LA, LB, EP>;
    smem = tc::gemm_smem_bytes(BN);
  }
  NBT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int kt_all = (K + tc::kBK - 1) / tc::kBK;
  splits = std::max(1, std::min(splits, kt_all));
  const int kt_split = (kt_all + splits - 1) / splits;
  splits = (kt_all + kt_split - 1) / kt_split;
  const dim3 grid((unsigned)((M + tc::kBM - 1) / tc::kBM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
  kern<<<grid, tc::kThreads, smem, stream>>>(la, lb, ep, M, K, kt_split, err);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

// BN for N columns (smallest supported tile >= N, at most 256 per tile).
template <class LA, class LB, class EP>
int gemm(const LA &la, const LB &lb, const EP &ep, int M, int N, int K, int splits, cudaStream_t s) {
  if (N <= 16) return launch_gemm<16>(la, lb, ep, M, N, K, splits, s);
  if (N <= 32) return launch_gemm<32>(la, lb, ep, M, N, K, splits, s);
  if (N <= 64) return launch_gemm<64>(la, lb, ep, M, N, K, splits, s);
  if (N <= 128) return launch_gemm<128>(la, lb, ep, M, N, K, splits, s);
  return launch_gemm<256>(la, lb, ep, M, N, K, splits, s);
}

int grid_1d(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, (int64_t)sm_count() * 32));
}

}  // namespace
}  // namespace nbt

using namespace nbt;

struct nbt_surrogate_s {
  int device = 0;
  int max_batch = 0, ldn = 0;  // ldn: batch padded to a multiple of 8
  float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  bf16 *wb = nullptr, *wtb = nullptr, *f1b = nullptr, *f1tb = nullptr;
  bf16 *act[kLayers] = {nullptr};   // outputs of conv layers 0..2 (layer 3 writes into x)
  bf16 *dact[kLayers] = {nullptr};  // gradients w.r.t. the outputs of conv layers 0..3
  bf16 *x = nullptr, *xt = nullptr, *h1 = nullptr, *dh1 = nullptr, *dh1t = nullptr;
  float *y = nullptr, *loss = nullptr, *part = nullptr;
  int64_t step = 0;
  float target_scale = 1.0f;  // training targets are multiplied by this in the loss
  // nbt_plan_pruned: crops of the next batch on a high-priority side stream while the caller's stream
  // runs the forward of the current one (fork / join through these events)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_crop[2] = {nullptr, nullptr}, ev_fwd[2] = {nullptr, nullptr};
};

namespace {

void free_net(nbt_surrogate n) {
  void *ptrs[] = {n->params, n->grads, n->adam_m, n->adam_v, n->wb, n->wtb, n->f1b, n->f1tb, n->x, n->xt, n->h1,
                  n->dh1, n->dh1t, n->y, n->loss, n->part};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int l = 0; l < kLayers; ++l) {
    if (n->act[l]) cudaFree(n->act[l]);
    if (n->dact[l]) cudaFree(n->dact[l]);
  }
  cudaEvent_t evs[] = {n->ev_fork, n->ev_crop[0], n->ev_crop[1], n->ev_fwd[0], n->ev_fwd[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (n->side) cudaStreamDestroy(n->side);
  (void)cudaGetLastError();
  delete n;
}

int check_net(nbt_surrogate n) {
  if (!n) return NBT_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NBT_ECUDA;
  return dev == n->device ? NBT_OK : NBT_EINVAL;
}

// Forward pass of n <= max_batch samples: crops [n, 32^3, 8], feats [n, 8].
// Layers 0 and 1 fused (inference): one persistent CTA per SM.
int launch_conv01(nbt_surrogate net, const uint8_t *crops, int n, cudaStream_t s) {
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  constexpr size_t smem = (size_t)fz::kSmem + 128;
  NBT_CUDA_TRY(cudaFuncSetAttribute(conv01_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(n, sm_count());
  conv01_kernel<<<(unsigned)grid, fz::kThreads + 32, smem, s>>>(crops, net->wb, net->params, n, net->act[1], err);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

// Layers 2 and 3 from shared-memory-staged inputs: one persistent CTA per SM.
template <int L>
int launch_conv23(nbt_surrogate net, const bf16 *in, bf16 *out, int n, cudaStream_t s) {
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  constexpr size_t smem = (size_t)c23::kSmem + 128;
  NBT_CUDA_TRY(cudaFuncSetAttribute(conv23_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min((n + 1) / 2, 2 * sm_count());
  conv23_kernel<L><<<(unsigned)grid, c23::kBuilders + 32, smem, s>>>(in, net->wb + (L == 2 ? kW2 : kW3),
                                                                     net->params + (L == 2 ? kB2 : kB3), n, out, err);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

// fused: layers 0 and 1 in one kernel (inference; training keeps the layer-0
// activation for the backward pass and runs them separately).
int forward_batch(nbt_surrogate net, const uint8_t *crops, const bf16 *feats, int n, float *pred, cudaStream_t s,
                  bool fused = false) {
  int first = 1;
  if (fused) {
    const int rc = launch_conv01(net, crops, n, s);
    if (rc != NBT_OK) return rc;
    first = 2;
  } else {
    const int64_t grid = std::min<int64_t>(n, (int64_t)sm_count() * 4);
    conv0_lookup_kernel<<<(unsigned)grid, 256, 0, s>>>(crops, net->wb + kP.w[0], net->params + kP.b[0], n,
                                                       net->act[0]);
    NBT_CUDA_TRY(cudaGetLastError());
  }
  const bf16 *in = net->act[first - 1];
  for (int l = first; l < kLayers; ++l) {
    if (l >= 2) {  // 4^3-output layers: inputs staged in shared memory, same sums as the generic GEMM
      const int rc = l == 2 ? launch_conv23<2>(net, in, net->act[2], n, s) : launch_conv23<3>(net, in, net->x, n, s);
      if (rc != NBT_OK) return rc;
      in = net->act[l];
      continue;
    }
    const LayerDims &L = kL[l];
    const int M = n * L.dout * L.dout * L.dout;
    const ConvFwdLoader la{in, M, L.din, L.stride, ilog2(L.dout), ilog2(L.cin / 8), L.cin};
    const MatLoader lb{net->wb + kP.w[l], L.cout, 27 * L.cin, 27 * L.cin};
    int rc;
    if (l + 1 < kLayers) {
      const EpiBiasRelu ep{net->act[l], net->params + kP.b[l], L.cout, L.cout};
      rc = gemm(la, lb, ep, M, L.cout, 27 * L.cin, 1, s);
      in = net->act[l];
    } else {
      const EpiConvToFlat ep{net->x, net->params + kP.b[l]};
      rc = gemm(la, lb, ep, M, L.cout, 27 * L.cin, 1, s);
    }
    if (rc != NBT_OK) return rc;
  }
  put_feats_kernel<<<(n * kFeat + 255) / 256, 256, 0, s>>>(feats, net->x, n);
  NBT_CUDA_TRY(cudaGetLastError());
  // fc1 (K = 4104: 65 stages of 64) split over K so that its ceil(n / 128) row tiles fill the SMs;
  // the partials are summed in split order with the bias and ReLU by fc1_reduce_kernel
  const MatLoader la{net->x, n, kFcIn, kFcIn};
  const MatLoader lb{net->f1b, kHid, kFcIn, kFcIn};
  const EpiF32 ep{net->part, kHid, kHid, (int64_t)n * kHid};
  int rc = gemm(la, lb, ep, n, kHid, kFcIn, kFc1Splits, s);
  if (rc != NBT_OK) return rc;
  fc1_reduce_kernel<<<grid_1d((int64_t)n * kHid), 256, 0, s>>>(net->part, fc1_splits(), n, net->params + kP.g1,
                                                              net->h1);
  NBT_CUDA_TRY(cudaGetLastError());
  fc2_forward_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(net->h1, net->params, n, pred ? pred : net->y);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int sync_weights(nbt_surrogate net, cudaStream_t s) {
  sync_weights_kernel<<<grid_1d(kP.f1 + (int64_t)kHid * kFcIn), 256, 0, s>>>(net->params, net->wb, net->wtb, net->f1b,
                                                                             net->f1tb);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

// Forward + backward of one batch; gradients into net->grads, loss into net->loss.
int backward_batch(nbt_surrogate net, const uint8_t *crops, const bf16 *feats, const float *targets, int n,
                   cudaStream_t s) {
  int rc = forward_batch(net, crops, feats, n, net->y, s);
  if (rc != NBT_OK) return rc;
  const int ldn = net->ldn;
  head_backward_kernel<<<1, 256, 0, s>>>(net->y, targets, net->target_scale, net->h1, net->params, n, ldn,
                                         net->grads, net->loss, net->dh1, net->dh1t);
  NBT_CUDA_TRY(cudaGetLastError());
  // fc1: dW1 = dh1^T X, db1 = colsum(dh1), dX = dh1 F1 (ReLU mask of the flattened conv output)
  {
    const dim3 tb(32, 8), tg((kFcIn + 31) / 32, (ldn + 31) / 32);
    transpose_kernel<<<tg, tb, 0, s>>>(net->x, n, kFcIn, kFcIn, net->xt, ldn);
    NBT_CUDA_TRY(cudaGetLastError());
    const MatLoader la{net->dh1t, kHid, n, ldn};
    const MatLoader lb{net->xt, kFcIn, n, ldn};
    const EpiF32 ep{net->grads + kP.f1, kFcIn, kFcIn, 0};
    rc = gemm(la, lb, ep, kHid, kFcIn, n, 1, s);
    if (rc != NBT_OK) return rc;
    colsum_kernel<<<(kHid * 32 + 255) / 256, 256, 0, s>>>(net->dh1, n, kHid, net->grads + kP.g1);
    NBT_CUDA_TRY(cudaGetLastError());
    const MatLoader la2{net->dh1, n, kHid, kHid};
    const MatLoader lb2{net->f1tb, kFlat, kHid, kHid};
    const EpiMaskRelu ep2{net->dact[kLayers - 1], net->x, kFlat, kFlat, kFcIn};
    rc = gemm(la2, lb2, ep2, n, kFlat, kHid, 1, s);
    if (rc != NBT_OK) return rc;
  }
  for (int l = kLayers - 1; l >= 0; --l) {
    const LayerDims &L = kL[l];
    const int Mout = n * L.dout * L.dout * L.dout;
    const bf16 *dy = net->dact[l];
    // bias gradient
    colsum_kernel<<<(L.cout * 32 + 255) / 256, 256, 0, s>>>(dy, Mout, L.cout, net->grads + kP.b[l]);
    NBT_CUDA_TRY(cudaGetLastError());
    if (l == 0) {
      // one-hot input: a table reduction instead of a GEMM
      const int64_t max_chunks = kSplitBytes / (27 * 3 * kC1 * 4);
      const int64_t chunk = std::max<int64_t>(kW0Sub, (Mout + max_chunks - 1) / max_chunks);
      const int chunks = (int)((Mout + chunk - 1) / chunk);
      conv0_wgrad_kernel<<<chunks, 256, 0, s>>>(crops, dy, Mout, chunk, net->part);
      NBT_CUDA_TRY(cudaGetLastError());
      conv0_wgrad_reduce_kernel<<<(kC1 * 27 * kC0 + 255) / 256, 256, 0, s>>>(net->part, chunks,
                                                                            net->grads + kP.w[0]);
      NBT_CUDA_TRY(cudaGetLastError());
      break;
    }
    const bf16 *in = net->act[l - 1];
    // weight gradient: split-K over output voxels, then a fixed-order reduction
    const int krows = 27 * L.cin;
    const int mtiles = (krows + tc::kBM - 1) / tc::kBM;
    const int kt_all = (Mout + tc::kBK - 1) / tc::kBK;
    int splits = std::max(1, std::min(kt_all, 4 * sm_count() / mtiles));
    splits = std::min<int>(splits, (int)(kSplitBytes / ((int64_t)krows * L.cout * 4)));
    const int kt_split = (kt_all + splits - 1) / splits;
    splits = (kt_all + kt_split - 1) / kt_split;
    const WgradColLoader la{in, Mout, L.din, L.stride, ilog2(L.dout), L.cin};
    const WgradDyLoader lb{dy, Mout, L.cout};
    const EpiF32 ep{net->part, L.cout, L.cout, (int64_t)krows * L.cout};
    rc = gemm(la, lb, ep, krows, L.cout, Mout, splits, s);
    if (rc != NBT_OK) return rc;
    wgrad_reduce_kernel<<<(krows * L.cout + 255) / 256, 256, 0, s>>>(net->part, splits, krows, L.cout,
                                                                     net->grads + kP.w[l]);
    NBT_CUDA_TRY(cudaGetLastError());
    // input gradient (not needed for the crop)
    if (l > 0) {
      const int Min = n * L.din * L.din * L.din;
      const ConvBwdDataLoader la2{dy, Min, L.din, L.dout, ilog2(L.stride), ilog2(L.din), ilog2(L.cout / 8), L.cout};
      const MatLoader lb2{net->wtb + kP.w[l], L.cin, 27 * L.cout, 27 * L.cout};
      const EpiMaskRelu ep2{net->dact[l - 1], net->act[l - 1], L.cin, L.cin, L.cin};
      rc = gemm(la2, lb2, ep2, Min, L.cin, 27 * L.cout, 1, s);
      if (rc != NBT_OK) return rc;
    }
  }
  return NBT_OK;
}

}  // namespace

extern "C" {

int nbt_tc_gemm(const void *a, const void *b, float *c, int32_t m, int32_t n, int32_t k, void *stream) {
  if (!a || !b || !c || m < 1 || n < 1 || n > 256 || k < 8 || (k % 8) != 0) return NBT_EINVAL;
  if (((uintptr_t)a & 15u) || ((uintptr_t)b & 15u)) return NBT_EINVAL;
  const MatLoader la{(const bf16 *)a, m, k, k};
  const MatLoader lb{(const bf16 *)b, n, k, k};
  const EpiF32 ep{c, n, n, 0};
  return gemm(la, lb, ep, m, n, k, 1, (cudaStream_t)stream);
}

int nbt_tc_error(int32_t *flag) {
  if (!flag) return NBT_EINVAL;
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  int v = 0;
  NBT_CUDA_TRY(cudaMemcpy(&v, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (v) NBT_CUDA_TRY(cudaMemset(err, 0, sizeof(int)));
  *flag = v;
  return NBT_OK;
}

int nbt_surrogate_param_count(int64_t *n) {
  if (!n) return NBT_EINVAL;
  *n = kP.total;
  return NBT_OK;
}

int nbt_surrogate_create(int32_t max_batch, nbt_surrogate *out) {
  if (!out || max_batch < 1 || max_batch > 4096) return NBT_EINVAL;
  *out = nullptr;
  nbt_surrogate n = new (std::nothrow) nbt_surrogate_s();
  if (!n) return NBT_ENOMEM;
  if (cudaGetDevice(&n->device) != cudaSuccess) {
    delete n;
    return NBT_ECUDA;
  }
  n->max_batch = max_batch;
  n->ldn = (max_batch + 7) / 8 * 8;
  const int64_t B = n->ldn;
  bool ok = true;
  auto alloc = [&](void **p, int64_t bytes) {
    if (ok && cudaMalloc(p, (size_t)bytes) != cudaSuccess) ok = false;
    if (ok && cudaMemset(*p, 0, (size_t)bytes) != cudaSuccess) ok = false;
  };
  alloc((void **)&n->params, kP.total * 4);
  alloc((void **)&n->grads, kP.total * 4);
  alloc((void **)&n->adam_m, kP.total * 4);
  alloc((void **)&n->adam_v, kP.total * 4);
  alloc((void **)&n->wb, kP.f1 * 2);
  alloc((void **)&n->wtb, kP.f1 * 2);
  alloc((void **)&n->f1b, (int64_t)kHid * kFcIn * 2);
  alloc((void **)&n->f1tb, (int64_t)kHid * kFcIn * 2);
  for (int l = 0; l < kLayers; ++l) {
    const int64_t vox = B * kL[l].dout * kL[l].dout * kL[l].dout * kL[l].cout;
    if (l + 1 < kLayers) alloc((void **)&n->act[l], vox * 2);
    alloc((void **)&n->dact[l], vox * 2);
  }
  alloc((void **)&n->x, B * kFcIn * 2);
  alloc((void **)&n->xt, B * kFcIn * 2);
  alloc((void **)&n->h1, B * kHid * 2);
  alloc((void **)&n->dh1, B * kHid * 2);
  alloc((void **)&n->dh1t, B * kHid * 2);
  alloc((void **)&n->y, B * 4);
  alloc((void **)&n->loss, 4);
  alloc((void **)&n->part, kSplitBytes);
  if (!ok) {
    free_net(n);
    return NBT_ENOMEM;
  }
  int lo = 0, hi = 0;
  bool sok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
             cudaStreamCreateWithPriority(&n->side, cudaStreamNonBlocking, hi) == cudaSuccess;
  cudaEvent_t *evs[] = {&n->ev_fork, &n->ev_crop[0], &n->ev_crop[1], &n->ev_fwd[0], &n->ev_fwd[1]};
  for (cudaEvent_t *e : evs) sok = sok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  if (!sok) {
    free_net(n);
    return NBT_ECUDA;
  }
  *out = n;
  return NBT_OK;
}

int nbt_surrogate_destroy(nbt_surrogate net) {
  if (!net) return NBT_OK;
  cudaDeviceSynchronize();
  free_net(net);
  return NBT_OK;
}

int nbt_surrogate_set_params(nbt_surrogate net, const float *host, int64_t n) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (!host || n != kP.total) return NBT_EINVAL;
  NBT_CUDA_TRY(cudaMemcpy(net->params, host, (size_t)n * 4, cudaMemcpyHostToDevice));
  NBT_CUDA_TRY(cudaMemset(net->adam_m, 0, (size_t)n * 4));
  NBT_CUDA_TRY(cudaMemset(net->adam_v, 0, (size_t)n * 4));
  net->step = 0;
  rc = sync_weights(net, nullptr);
  if (rc != NBT_OK) return rc;
  NBT_CUDA_TRY(cudaDeviceSynchronize());
  return NBT_OK;
}

int nbt_surrogate_get_params(nbt_surrogate net, float *host, int64_t n) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (!host || n != kP.total) return NBT_EINVAL;
  NBT_CUDA_TRY(cudaDeviceSynchronize());
  NBT_CUDA_TRY(cudaMemcpy(host, net->params, (size_t)n * 4, cudaMemcpyDeviceToHost));
  return NBT_OK;
}

int nbt_surrogate_crops(nbt_map map, const nbt_pose *poses, int64_t n, const nbt_camera *cam,
                        const nbt_ig_params *params, void *crops, void *feats, void *stream) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n < 0 || !cam || !params) return NBT_EINVAL;
  if (n == 0) return NBT_OK;
  if (!poses || !crops || !feats) return NBT_EINVAL;
  if ((uintptr_t)crops & 15u) return NBT_EINVAL;  // crops are written in 4-byte and read in 16-byte vectors
  if (!(cam->fov_h > 0.0f && cam->fov_h < 3.14159f) || !(cam->fov_v > 0.0f && cam->fov_v < 3.14159f) ||
      !(cam->max_range > 0.0f))
    return NBT_EINVAL;
  CropConst cc;
  const double dh = (double)cam->max_range * tan((double)cam->fov_h * 0.5);
  const double dv = (double)cam->max_range * tan((double)cam->fov_v * 0.5);
  cc.x0 = (float)(-dh + dh / kCrop);
  cc.xs = (float)(2.0 * dh / kCrop);
  cc.y0 = (float)(-dv + dv / kCrop);
  cc.ys = (float)(2.0 * dv / kCrop);
  cc.zc = cam->max_range;
  cc.inv_s = (float)(1.0 / (double)map->desc.voxel_size);
  cc.ox = map->desc.origin[0];
  cc.oy = map->desc.origin[1];
  cc.oz = map->desc.origin[2];
  cc.ext_x = (float)map->desc.nx * map->desc.voxel_size;  // one FP32 product (host, no contraction)
  cc.ext_y = (float)map->desc.ny * map->desc.voxel_size;
  cc.ext_z = (float)map->desc.nz * map->desc.voxel_size;
  cc.occ_thr = params->occ_threshold;
  cc.free_thr = params->free_threshold;
  DevMap m;
  m.payload = map->d_payload;  // raw states / probabilities (not derived gains)
  m.tab = map->d_tab;
  m.nx = map->desc.nx;
  m.ny = map->desc.ny;
  m.nz = map->desc.nz;
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = (int)std::min<int64_t>(n, (int64_t)sm_count() * 8);
  const bool lin = map->brick == 1;
  const float *pz = (const float *)poses;
  uint8_t *cr = (uint8_t *)crops;
  bf16 *ft = (bf16 *)feats;
  switch (map->desc.encoding) {
    case NBT_F32_PROB:
      if (lin)
        crop_kernel<PAYLOAD_GAIN_F32, true><<<grid, 256, 0, s>>>(m, cc, pz, n, cr, ft);
      else
        crop_kernel<PAYLOAD_GAIN_F32, false><<<grid, 256, 0, s>>>(m, cc, pz, n, cr, ft);
      break;
    case NBT_U2_STATE:
      if (lin)
        crop_kernel<PAYLOAD_U2, true><<<grid, 256, 0, s>>>(m, cc, pz, n, cr, ft);
      else
        crop_kernel<PAYLOAD_U2, false><<<grid, 256, 0, s>>>(m, cc, pz, n, cr, ft);
      break;
    default:
      if (lin)
        crop_kernel<PAYLOAD_U8, true><<<grid, 256, 0, s>>>(m, cc, pz, n, cr, ft);
      else
        crop_kernel<PAYLOAD_U8, false><<<grid, 256, 0, s>>>(m, cc, pz, n, cr, ft);
      break;
  }
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int nbt_surrogate_forward(nbt_surrogate net, const void *crops, const void *feats, int64_t n, float *pred,
                          void *stream) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (n < 0) return NBT_EINVAL;
  if (n == 0) return NBT_OK;
  if (!crops || !feats || !pred || ((uintptr_t)crops & 15u)) return NBT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t per = (int64_t)kCrop * kCrop * kCrop;
  for (int64_t b0 = 0; b0 < n; b0 += net->max_batch) {
    const int nb = (int)std::min<int64_t>(net->max_batch, n - b0);
    rc = forward_batch(net, (const uint8_t *)crops + b0 * per, (const bf16 *)feats + b0 * kFeat, nb, pred + b0, s,
                       true);
    if (rc != NBT_OK) return rc;
  }
  return NBT_OK;
}

int nbt_surrogate_backward(nbt_surrogate net, const void *crops, const void *feats, const float *targets, int32_t n,
                           float *grads_out, float *loss_out, void *stream) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (n < 1 || n > net->max_batch || n > 1024 || !crops || !feats || !targets || ((uintptr_t)crops & 15u))
    return NBT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  rc = backward_batch(net, (const uint8_t *)crops, (const bf16 *)feats, targets, n, s);
  if (rc != NBT_OK) return rc;
  if (grads_out) NBT_CUDA_TRY(cudaMemcpyAsync(grads_out, net->grads, kP.total * 4, cudaMemcpyDeviceToDevice, s));
  if (loss_out) NBT_CUDA_TRY(cudaMemcpyAsync(loss_out, net->loss, 4, cudaMemcpyDeviceToDevice, s));
  return NBT_OK;
}

int nbt_surrogate_train_step(nbt_surrogate net, const void *crops, const void *feats, const float *targets, int32_t n,
                             float lr, float *loss_out, void *stream) {
  int rc = nbt_surrogate_backward(net, crops, feats, targets, n, nullptr, loss_out, stream);
  if (rc != NBT_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - pow(0.9, (double)net->step)), c2 = (float)(1.0 - pow(0.999, (double)net->step));
  adam_kernel<<<grid_1d(kP.total), 256, 0, s>>>(net->params, net->grads, net->adam_m, net->adam_v, kP.total, lr, b1,
                                                b2, 1e-8f, c1, c2);
  NBT_CUDA_TRY(cudaGetLastError());
  return sync_weights(net, s);
}

int nbt_surrogate_set_target_scale(nbt_surrogate net, float scale) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (!std::isfinite(scale) || !(scale > 0.0f)) return NBT_EINVAL;
  net->target_scale = scale;
  return NBT_OK;
}

int nbt_surrogate_get_adam(nbt_surrogate net, float *m_host, float *v_host, int64_t n, int64_t *step) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (!m_host || !v_host || !step || n != kP.total) return NBT_EINVAL;
  NBT_CUDA_TRY(cudaDeviceSynchronize());
  NBT_CUDA_TRY(cudaMemcpy(m_host, net->adam_m, (size_t)n * 4, cudaMemcpyDeviceToHost));
  NBT_CUDA_TRY(cudaMemcpy(v_host, net->adam_v, (size_t)n * 4, cudaMemcpyDeviceToHost));
  *step = net->step;
  return NBT_OK;
}

int nbt_surrogate_set_adam(nbt_surrogate net, const float *m_host, const float *v_host, int64_t n, int64_t step) {
  int rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (!m_host || !v_host || n != kP.total || step < 0) return NBT_EINVAL;
  NBT_CUDA_TRY(cudaDeviceSynchronize());
  NBT_CUDA_TRY(cudaMemcpy(net->adam_m, m_host, (size_t)n * 4, cudaMemcpyHostToDevice));
  NBT_CUDA_TRY(cudaMemcpy(net->adam_v, v_host, (size_t)n * 4, cudaMemcpyHostToDevice));
  net->step = step;
  return NBT_OK;
}

int nbt_tc_set_wait_limit(uint64_t ns) {
  if (ns < 1000ull || ns > 60000000000ull) return NBT_EINVAL;
  NBT_CUDA_TRY(cudaMemcpyToSymbol(tc::c_wait_ns, &ns, sizeof(ns)));
  return NBT_OK;
}

int nbt_tc_wait_probe(void *stream) {
  int *err = nullptr;
  int rc = dev_err_word(&err);
  if (rc != NBT_OK) return rc;
  tc_wait_probe_kernel<<<(unsigned)sm_count(), 128, 0, (cudaStream_t)stream>>>(err);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

}  // extern "C"

extern "C" {

int nbt_segment_topk(const float *scores, int64_t n, int32_t seg, int32_t keep, int32_t *idx_out, const nbt_pose *poses,
                     nbt_pose *poses_out, void *stream) {
  if (!scores || !idx_out || seg < 1 || seg > 8192 || keep < 1 || keep > seg || n < 0 || n % seg) return NBT_EINVAL;
  if ((poses == nullptr) != (poses_out == nullptr)) return NBT_EINVAL;
  if (n == 0) return NBT_OK;
  int pow2 = 1;
  while (pow2 < seg) pow2 <<= 1;
  const size_t smem = (size_t)pow2 * 8;
  NBT_CUDA_TRY(cudaFuncSetAttribute(segment_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  segment_topk_kernel<<<(unsigned)(n / seg), 512, smem, (cudaStream_t)stream>>>(
      scores, seg, keep, pow2, idx_out, (const float *)poses, (float *)poses_out);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int nbt_segment_argmax(const float *values, const int32_t *idx, int64_t n, int32_t seg, int32_t *best_idx,
                       float *best_val, void *stream) {
  if (!values || !best_idx || seg < 1 || n < 0 || n % seg) return NBT_EINVAL;
  if (n == 0) return NBT_OK;
  const int64_t n_seg = n / seg;
  segment_argmax_kernel<<<(unsigned)((n_seg * 32 + 255) / 256), 256, 0, (cudaStream_t)stream>>>(values, idx, n_seg, seg,
                                                                                              best_idx, best_val);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Surrogate-pruned next-best-view selection in one call: crops and the
// network's score for every candidate, the keep best of each segment, the
// exact raycast (Section III IG) of those, and the best of them per segment.
// The exact IG judges the kept candidates, so pruning can miss the best view
// but never reports a wrong IG.  Scratch comes from the caller's workspace.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kCropBytes = (int64_t)kCrop * kCrop * kCrop;  // one uint8 class code per sample

int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }

struct PrunedLayout {
  int64_t crops, crops_stride, feats, feats_stride, scores, idx, kept, ig, ws, ws_bytes, total;
};

// Workspace regions (each 256-byte aligned): crops and features of one batch
// of max_batch candidates (two such buffers when there is more than one
// batch: the next batch's crops are formed while the current one's forward
// runs), all scores, the kept indices, kept poses and their exact IGs, and
// the raycast workspace of the kept views.
int pruned_layout(nbt_surrogate net, int64_t n, int32_t seg, int32_t keep, const nbt_camera *cam, PrunedLayout *L) {
  const int64_t chunk = std::min<int64_t>(n, net->max_batch);
  const int64_t bufs = n > chunk ? 2 : 1;
  const int64_t n_kept = n / seg * keep;
  int64_t ws_bytes = 0;
  const int rc = nbt_workspace_size(n_kept, cam, &ws_bytes);
  if (rc != NBT_OK) return rc;
  int64_t o = 0;
  L->crops = o;
  L->crops_stride = align256(chunk * kCropBytes);
  o += bufs * L->crops_stride;
  L->feats = o;
  L->feats_stride = align256(chunk * kFeat * 2);
  o += bufs * L->feats_stride;
  L->scores = o;
  o += align256(n * 4);
  L->idx = o;
  o += align256(n_kept * 4);
  L->kept = o;
  o += align256(n_kept * 28);
  L->ig = o;
  o += align256(n_kept * 4);
  L->ws = o;
  L->ws_bytes = ws_bytes;
  L->total = o + align256(ws_bytes);
  return NBT_OK;
}

bool pruned_shape_ok(int64_t n, int32_t seg, int32_t keep) {
  return n >= 0 && n <= INT32_MAX && seg >= 1 && seg <= 8192 && keep >= 1 && keep <= seg && n % seg == 0;
}

}  // namespace

extern "C" {

int nbt_pruned_workspace_size(nbt_surrogate net, int64_t n, int32_t seg, int32_t keep, const nbt_camera *cam,
                              int64_t *bytes) {
  if (!net || !bytes || !pruned_shape_ok(n, seg, keep) || !valid_camera(cam)) return NBT_EINVAL;
  PrunedLayout L;
  const int rc = pruned_layout(net, n, seg, keep, cam, &L);
  if (rc != NBT_OK) return rc;
  *bytes = L.total;
  return NBT_OK;
}

int nbt_plan_pruned(nbt_map map, nbt_surrogate net, const nbt_pose *poses, int64_t n, int32_t seg, int32_t keep,
                    const nbt_camera *cam, const nbt_ig_params *params, int32_t *best_out, float *best_ig_out,
                    int32_t *kept_out, void *workspace, int64_t workspace_bytes, void *stream) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  rc = check_net(net);
  if (rc != NBT_OK) return rc;
  if (!pruned_shape_ok(n, seg, keep) || !valid_camera(cam) || !valid_params(params)) return NBT_EINVAL;
  if (n == 0) return NBT_OK;
  if (!poses || !best_out) return NBT_EINVAL;
  PayloadKind kind;
  const void *payload = nullptr;
  rc = payload_kind(map, params, &kind, &payload);  // NBT_EUNSUPPORTED before anything is enqueued
  if (rc != NBT_OK) return rc;
  PrunedLayout L;
  rc = pruned_layout(net, n, seg, keep, cam, &L);
  if (rc != NBT_OK) return rc;
  if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255u)) return NBT_EWORKSPACE;
  char *w = (char *)workspace;
  float *scores = (float *)(w + L.scores);
  int32_t *idx = kept_out ? kept_out : (int32_t *)(w + L.idx);
  nbt_pose *kept = (nbt_pose *)(w + L.kept);
  float *ig = (float *)(w + L.ig);
  const int64_t n_kept = n / seg * keep;
  // Crops of batch b go into buffer b % 2 on the side stream (high priority: the latency-bound
  // gather fills issue slots the forward leaves idle), after the forward of batch b - 2 has released
  // that buffer; the caller's stream waits for them, runs the forward, and at the end has waited for
  // every side-stream launch (fork / join, so the call stays ordered on the caller's stream).
  cudaStream_t s = (cudaStream_t)stream;
  NBT_CUDA_TRY(cudaEventRecord(net->ev_fork, s));
  NBT_CUDA_TRY(cudaStreamWaitEvent(net->side, net->ev_fork, 0));
  int64_t b = 0;
  for (int64_t c0 = 0; c0 < n; c0 += net->max_batch, ++b) {
    const int64_t nc = std::min<int64_t>(net->max_batch, n - c0);
    const int buf = (int)(b & 1);
    uint8_t *crops = (uint8_t *)(w + L.crops + buf * L.crops_stride);
    void *feats = w + L.feats + buf * L.feats_stride;
    if (b >= 2) NBT_CUDA_TRY(cudaStreamWaitEvent(net->side, net->ev_fwd[buf], 0));
    rc = nbt_surrogate_crops(map, poses + c0, nc, cam, params, crops, feats, net->side);
    if (rc == NBT_OK) rc = cudaEventRecord(net->ev_crop[buf], net->side) == cudaSuccess ? NBT_OK : NBT_ECUDA;
    if (rc == NBT_OK) rc = cudaStreamWaitEvent(s, net->ev_crop[buf], 0) == cudaSuccess ? NBT_OK : NBT_ECUDA;
    if (rc != NBT_OK) {
      // join the side stream before returning, whatever was enqueued on it
      if (cudaEventRecord(net->ev_crop[buf], net->side) == cudaSuccess) (void)cudaStreamWaitEvent(s, net->ev_crop[buf], 0);
      (void)cudaGetLastError();
      return rc;
    }
    rc = nbt_surrogate_forward(net, crops, feats, nc, scores + c0, stream);
    if (rc != NBT_OK) return rc;
    NBT_CUDA_TRY(cudaEventRecord(net->ev_fwd[buf], s));
  }
  rc = nbt_segment_topk(scores, n, seg, keep, idx, poses, kept, stream);
  if (rc != NBT_OK) return rc;
  rc = nbt_views_ig(map, kept, n_kept, cam, params, ig, nullptr, w + L.ws, L.ws_bytes, stream);
  if (rc != NBT_OK) return rc;
  return nbt_segment_argmax(ig, idx, n_kept, keep, best_out, best_ig_out, stream);
}

}  // extern "C"
