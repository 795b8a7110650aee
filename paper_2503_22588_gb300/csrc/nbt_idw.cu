// IG between perspectives: the information-distribution (ID) buffer, the
// inverse-distance-weighted gain G(x) of Eq. 3, the orientation factor O(x)
// and the IG cost c_I (Section IV, "Orientation Factor O(x_k) and IG
// G(x_k)" and "Cost Function Extension").
//
// Layout: one device slab of n_b slots; a slot holds up to `cap`
// perspectives (a multiple of kBlock) as pairs, two float4 per pair:
//   {x_2k, x_2k+1, y_2k, y_2k+1}, {z_2k, z_2k+1, g_2k, g_2k+1}
// so one 128-bit shared-memory read feeds both lanes of a packed f32x2
// operation.  Slots are padded to a multiple of kBlock with start point
// (+inf, +inf, +inf) and gain 0: d^2 = +inf there, so the weight is 0 and the
// pad adds nothing to either sum.
//
// The query kernel is arithmetic-bound: per (query, perspective) pair it
// needs eight FP32 lane operations (four packed f32x2 instructions per two
// pairs) and one MUFU reciprocal (p = 2); both give the same ceiling of
// 16 pairs per clock per SM.  The perspectives are staged through shared
// memory and broadcast to the warp.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <new>

#include "nbt_internal.cuh"

using namespace nbt;

namespace {

constexpr int kMaxIds = 32;
constexpr int kBlock = 64;         // perspectives per FP32 lane-sum block (32 per f32x2 lane)
constexpr int kTile = 512;         // perspectives staged in shared memory per pass
constexpr int kIdwThreads = 128;
constexpr int kQ = 1;              // queries per thread

struct IdSet {
  const float4 *slots;
  int cap;                 // perspectives per slot (float4 per slot)
  int n;                   // IDs held
  int slot[kMaxIds];       // slot of ID m, m = 0 the oldest
  int views[kMaxIds];      // perspectives of ID m
  float weight[kMaxIds];   // 1 / (N_B - u) of ID m
};

struct CostConst {
  float poi[3];
  float tan_h, tan_v;
  float w_info, eps;
};

typedef unsigned long long u64;

__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void up2(u64 v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// Hardware reciprocal approximation (max error 1 ulp); a denormal or zero
// input gives +inf, +inf gives 0.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Weight d^-p from d^2: p = 2 is one reciprocal; otherwise 2^(-p/2 log2 d^2).
template <bool P2>
__device__ __forceinline__ float weight_of(float d2, float half_p) {
  if (P2) return rcp_approx(d2);
  return exp2f(-half_p * log2f(d2));
}

// Error-free addition into a (hi, lo) pair (Knuth's TwoSum).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b) {
  const float s = __fadd_rn(hi, b);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// FP32 d^2 of one perspective, in the order the packed loop uses per lane.
__device__ __forceinline__ float dist2(float qx, float qy, float qz, float px, float py, float pz) {
  const float dx = __fsub_rn(qx, px), dy = __fsub_rn(qy, py), dz = __fsub_rn(qz, pz);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}

// Rare path, taken when the FP32 denominator is not finite: the query
// coincides with start points (d^2 below the smallest normal float, where
// the reciprocal is +inf) -- then the mean gain of those points -- or the
// FP32 weights overflowed (very close points, large p) -- then the ID
// again with FP64 weights and sums.
template <bool P2>
__device__ float idw_slow(const float4 *slot, int views, float qx, float qy, float qz, float half_p) {
  float sum = 0.0f;
  int cnt = 0;
  double num = 0.0, den = 0.0;
  for (int j = 0; j < views; ++j) {
    const float4 a = slot[(j >> 1) * 2], b = slot[(j >> 1) * 2 + 1];
    const bool hi = j & 1;
    const float d2 = dist2(qx, qy, qz, hi ? a.y : a.x, hi ? a.w : a.z, hi ? b.y : b.x);
    const float g = hi ? b.w : b.z;
    if (d2 < 1.17549435e-38f) {
      sum = __fadd_rn(sum, g);
      ++cnt;
    } else {
      const double w = P2 ? 1.0 / (double)d2 : pow((double)d2, -(double)half_p);
      num += (double)g * w;
      den += w;
    }
  }
  return cnt ? __fdiv_rn(sum, (float)cnt) : (float)(num / den);
}

// Orientation factor O(x) of one camera pose (FP32; the inside decision in
// the fixed order documented in nbt.h).
__device__ __forceinline__ float orientation_factor(const float *pose, const CostConst &cc) {
  float r[9];
  quat_rot_f32(pose + 3, r);
  const float v0 = fsub(cc.poi[0], pose[0]), v1 = fsub(cc.poi[1], pose[1]), v2 = fsub(cc.poi[2], pose[2]);
  float c[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) c[k] = fadd(fadd(fmul(r[k], v0), fmul(r[3 + k], v1)), fmul(r[6 + k], v2));
  const bool inside = c[2] > 0.0f && fabsf(c[0]) <= fmul(c[2], cc.tan_h) && fabsf(c[1]) <= fmul(c[2], cc.tan_v);
  if (!inside) return 0.0f;
  const float len = __fsqrt_rn(fadd(fadd(fmul(v0, v0), fmul(v1, v1)), fmul(v2, v2)));
  return __fdiv_rn(c[2], len);
}

// One thread: kQ query poses.  For every ID, the perspectives stream
// through shared memory in tiles; per block of kBlock perspectives each
// query keeps packed FP32 lane sums of g w and w, then folds them into
// compensated totals.  COST adds O(x) and the c_I term.
template <bool P2, bool COST>
__global__ void __launch_bounds__(kIdwThreads)
    idw_kernel(IdSet ids, const float *__restrict__ poses, int64_t n, float half_p, CostConst cc,
               float *__restrict__ gain_out, float *__restrict__ orient_out, float *__restrict__ term_out) {
  __shared__ float4 tile[kTile];
  const int64_t q0 = ((int64_t)blockIdx.x * kIdwThreads + threadIdx.x) * kQ;
  float qx[kQ], qy[kQ], qz[kQ], gsum[kQ];
  u64 qx2[kQ], qy2[kQ], qz2[kQ];
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int64_t i = min(q0 + q, n - 1);
    qx[q] = __ldg(poses + i * 7 + 0);
    qy[q] = __ldg(poses + i * 7 + 1);
    qz[q] = __ldg(poses + i * 7 + 2);
    qx2[q] = pk2(qx[q], qx[q]);
    qy2[q] = pk2(qy[q], qy[q]);
    qz2[q] = pk2(qz[q], qz[q]);
    gsum[q] = 0.0f;
  }
  for (int m = 0; m < ids.n; ++m) {
    const int views = ids.views[m];
    if (views == 0) continue;  // an empty ID adds nothing
    const float4 *slot = ids.slots + (int64_t)ids.slot[m] * ids.cap;
    const int npad = (views + kBlock - 1) / kBlock * kBlock;
    float nh[kQ], nl[kQ], dh[kQ], dl[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) nh[q] = nl[q] = dh[q] = dl[q] = 0.0f;
    for (int t0 = 0; t0 < npad; t0 += kTile) {
      const int len = min(kTile, npad - t0);
      __syncthreads();
      for (int k = threadIdx.x; k < len; k += kIdwThreads) tile[k] = slot[t0 + k];
      __syncthreads();
      for (int b = 0; b < len; b += kBlock) {
        u64 an[kQ], ad[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) an[q] = ad[q] = 0ull;
#pragma unroll 8
        for (int k = 0; k < kBlock / 2; ++k) {
          const float4 A = tile[b + 2 * k], B = tile[b + 2 * k + 1];
          const u64 px = pk2(A.x, A.y), py = pk2(A.z, A.w), pz = pk2(B.x, B.y), pg = pk2(B.z, B.w);
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            const u64 dx = sub2(qx2[q], px), dy = sub2(qy2[q], py), dz = sub2(qz2[q], pz);
            const u64 d2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
            float a, c;
            up2(d2, a, c);
            const u64 w = pk2(weight_of<P2>(a, half_p), weight_of<P2>(c, half_p));
            an[q] = fma2(pg, w, an[q]);
            ad[q] = add2(ad[q], w);
          }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          float s0, s1;
          up2(an[q], s0, s1);
          two_sum_acc(nh[q], nl[q], __fadd_rn(s0, s1));
          up2(ad[q], s0, s1);
          two_sum_acc(dh[q], dl[q], __fadd_rn(s0, s1));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
      const float den = __fadd_rn(dh[q], dl[q]);
      float ratio;
      if (den < INFINITY) {
        ratio = __fdiv_rn(__fadd_rn(nh[q], nl[q]), den);
      } else {
        ratio = idw_slow<P2>(slot, views, qx[q], qy[q], qz[q], half_p);
      }
      gsum[q] = __fmaf_rn(ids.weight[m], ratio, gsum[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int64_t i = q0 + q;
    if (i >= n) break;
    if (gain_out) gain_out[i] = gsum[q];
    if (COST) {
      const float o = orientation_factor(poses + i * 7, cc);
      if (orient_out) orient_out[i] = o;
      term_out[i] = __fdiv_rn(cc.w_info, fadd(fmul(o, gsum[q]), cc.eps));
    }
  }
}

// One warp per trajectory: fixed-order FP64 sum of its states' cost terms.
__global__ void cost_reduce_kernel(const float *__restrict__ term, const int32_t *__restrict__ offsets,
                                   int32_t n_traj, int64_t n_poses, float *__restrict__ cost_out) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_traj) return;
  const int64_t b = min((int64_t)max(offsets[t], 0), n_poses);
  const int64_t e = min(max((int64_t)offsets[t + 1], b), n_poses);
  double acc = 0.0;
  for (int64_t p = b + lane; p < e; p += 32) acc += (double)term[p];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) cost_out[t] = (float)acc;
}

__global__ void id_push_kernel(const float *__restrict__ poses, const float *__restrict__ ig, int n_views, int n_pad,
                               float4 *__restrict__ slot) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_pad / 2; k += gridDim.x * blockDim.x) {
    float x[2], y[2], z[2], g[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * k + h;
      const bool in = j < n_views;
      x[h] = in ? poses[(int64_t)j * 7 + 0] : INFINITY;
      y[h] = in ? poses[(int64_t)j * 7 + 1] : INFINITY;
      z[h] = in ? poses[(int64_t)j * 7 + 2] : INFINITY;
      g[h] = in ? ig[j] : 0.0f;
    }
    slot[2 * k] = make_float4(x[0], x[1], y[0], y[1]);
    slot[2 * k + 1] = make_float4(z[0], z[1], g[0], g[1]);
  }
}

}  // namespace

struct nbt_id_buffer_s {
  int device = -1;
  int n_b = 0, max_views = 0, cap = 0;
  float4 *d_slots = nullptr;
  int head = 0;   // slot the next push writes
  int count = 0;  // IDs held
  int views[kMaxIds] = {};
  std::mutex mu;
};

namespace {

int check_buf(nbt_id_buffer buf) {
  if (!buf) return NBT_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NBT_ECUDA;
  return dev == buf->device ? NBT_OK : NBT_EINVAL;
}

// Snapshot of the buffer for one launch: IDs oldest first with their weights.
IdSet id_set(nbt_id_buffer buf) {
  std::lock_guard<std::mutex> lock(buf->mu);
  IdSet s{};
  s.slots = buf->d_slots;
  s.cap = buf->cap;
  s.n = buf->count;
  for (int m = 0; m < buf->count; ++m) {
    const int slot = ((buf->head - buf->count + m) % buf->n_b + buf->n_b) % buf->n_b;
    const int u = buf->n_b - buf->count + m;
    s.slot[m] = slot;
    s.views[m] = buf->views[slot];
    s.weight[m] = (float)(1.0 / (double)(buf->n_b - u));
  }
  return s;
}

bool valid_power(float p) { return std::isfinite(p) && p > 0.0f && p <= 8.0f; }

template <bool COST>
int launch_idw(nbt_id_buffer buf, const float *poses, int64_t n, float power, const CostConst &cc, float *gain_out,
               float *orient_out, float *term_out, cudaStream_t stream) {
  const IdSet ids = id_set(buf);
  const int64_t per_block = (int64_t)kIdwThreads * kQ;
  const int64_t grid = (n + per_block - 1) / per_block;
  if (grid > 0x7fffffff) return NBT_EINVAL;
  const float half_p = 0.5f * power;
  if (power == 2.0f)
    idw_kernel<true, COST><<<(unsigned)grid, kIdwThreads, 0, stream>>>(ids, poses, n, half_p, cc, gain_out,
                                                                       orient_out, term_out);
  else
    idw_kernel<false, COST><<<(unsigned)grid, kIdwThreads, 0, stream>>>(ids, poses, n, half_p, cc, gain_out,
                                                                        orient_out, term_out);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

}  // namespace

extern "C" {

int nbt_id_buffer_create(int32_t n_b, int32_t max_views, nbt_id_buffer *out) {
  if (!out) return NBT_EINVAL;
  *out = nullptr;
  if (n_b < 1 || n_b > kMaxIds || max_views < 1 || max_views > (1 << 20)) return NBT_EINVAL;
  nbt_id_buffer b = new (std::nothrow) nbt_id_buffer_s();
  if (!b) return NBT_ENOMEM;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return NBT_ECUDA;
  }
  b->n_b = n_b;
  b->max_views = max_views;
  b->cap = (max_views + kBlock - 1) / kBlock * kBlock;
  if (cudaMalloc((void **)&b->d_slots, (size_t)n_b * b->cap * sizeof(float4)) != cudaSuccess) {
    (void)cudaGetLastError();
    delete b;
    return NBT_ENOMEM;
  }
  *out = b;
  return NBT_OK;
}

int nbt_id_buffer_destroy(nbt_id_buffer buf) {
  if (!buf) return NBT_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != buf->device) cudaSetDevice(buf->device);
  cudaDeviceSynchronize();
  if (buf->d_slots) cudaFree(buf->d_slots);
  (void)cudaGetLastError();
  if (prev >= 0 && prev != buf->device) cudaSetDevice(prev);
  delete buf;
  return NBT_OK;
}

int nbt_id_buffer_push(nbt_id_buffer buf, const nbt_pose *poses, const float *ig, int32_t n_views, void *stream) {
  int rc = check_buf(buf);
  if (rc != NBT_OK) return rc;
  if (n_views < 0 || n_views > buf->max_views || (n_views > 0 && (!poses || !ig))) return NBT_EINVAL;
  std::lock_guard<std::mutex> lock(buf->mu);
  const int slot = buf->head;
  const int n_pad = (n_views + kBlock - 1) / kBlock * kBlock;
  if (n_pad > 0) {
    const int grid = std::min((n_pad / 2 + 255) / 256, 4096);
    id_push_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const float *)poses, ig, n_views, n_pad,
                                                           buf->d_slots + (int64_t)slot * buf->cap);
    NBT_CUDA_TRY(cudaGetLastError());
  }
  buf->views[slot] = n_views;
  buf->head = (slot + 1) % buf->n_b;
  buf->count = std::min(buf->count + 1, buf->n_b);
  return NBT_OK;
}

int nbt_id_buffer_clear(nbt_id_buffer buf) {
  if (!buf) return NBT_EINVAL;
  std::lock_guard<std::mutex> lock(buf->mu);
  buf->head = 0;
  buf->count = 0;
  return NBT_OK;
}

int nbt_id_buffer_count(nbt_id_buffer buf, int32_t *n_ids) {
  if (!buf || !n_ids) return NBT_EINVAL;
  std::lock_guard<std::mutex> lock(buf->mu);
  *n_ids = buf->count;
  return NBT_OK;
}

int nbt_idw_gain(nbt_id_buffer buf, const nbt_pose *poses, int64_t n, float power, float *gain_out, void *stream) {
  int rc = check_buf(buf);
  if (rc != NBT_OK) return rc;
  if (n < 0 || !valid_power(power) || (n > 0 && (!poses || !gain_out))) return NBT_EINVAL;
  if (n == 0) return NBT_OK;
  return launch_idw<false>(buf, (const float *)poses, n, power, CostConst{}, gain_out, nullptr, nullptr,
                           (cudaStream_t)stream);
}

int nbt_ig_cost(nbt_id_buffer buf, const nbt_pose *poses, int64_t n_poses, const int32_t *offsets, int32_t n_traj,
                const float *poi, float fov_h, float fov_v, const nbt_cost_params *params, float *gain_out,
                float *orient_out, float *term_out, float *cost_out, void *stream) {
  int rc = check_buf(buf);
  if (rc != NBT_OK) return rc;
  if (!params || !poi || n_poses < 0 || n_traj < 0 || !valid_power(params->power)) return NBT_EINVAL;
  if (!(params->w_info >= 0.0f) || !std::isfinite(params->w_info) || !(params->eps > 0.0f) ||
      !std::isfinite(params->eps))
    return NBT_EINVAL;
  if (!(fov_h > 0.0f && fov_h < 3.14159f) || !(fov_v > 0.0f && fov_v < 3.14159f)) return NBT_EINVAL;
  if (!std::isfinite(poi[0]) || !std::isfinite(poi[1]) || !std::isfinite(poi[2])) return NBT_EINVAL;
  if ((n_poses > 0 && (!poses || !term_out)) || (n_traj > 0 && (!offsets || !cost_out))) return NBT_EINVAL;
  CostConst cc;
  cc.poi[0] = poi[0];
  cc.poi[1] = poi[1];
  cc.poi[2] = poi[2];
  cc.tan_h = (float)std::tan((double)fov_h * 0.5);
  cc.tan_v = (float)std::tan((double)fov_v * 0.5);
  cc.w_info = params->w_info;
  cc.eps = params->eps;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_poses > 0) {
    rc = launch_idw<true>(buf, (const float *)poses, n_poses, params->power, cc, gain_out, orient_out, term_out, s);
    if (rc != NBT_OK) return rc;
  }
  if (n_traj > 0) {
    const int64_t threads = (int64_t)n_traj * 32;
    cost_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(term_out, offsets, n_traj, n_poses,
                                                                         cost_out);
    NBT_CUDA_TRY(cudaGetLastError());
  }
  return NBT_OK;
}

}  // extern "C"
