// Voxel-map update from a depth point cloud (Section III: every captured
// point cloud is voxel-filtered and inserted into the probabilistic map the
// IG is computed from), in the discrete form of occupancy-grid insertion:
//
//   1. points_kernel    each point's voxel; inside the map its bit is set in
//                       the hit bitmap (the voxel filter: one hit per voxel
//                       and scan); outside it joins the outside list;
//   2. enumerate_kernel the set bits of the hit bitmap become a list of
//                       distinct endpoint voxels (one ray each);
//   3. free_rays_kernel one ray per distinct endpoint, from the sensor to the
//                       endpoint voxel's centre, walked with the FP32
//                       reference walk of the IG path; every visited voxel's
//                       bit is set in the miss bitmap;
//   4. apply_kernel     one dense pass over the bitmaps: hit voxels take the
//                       occupied update, miss voxels that are not hits the
//                       free update; the pass clears both bitmaps for the
//                       next scan.
//
// Bitmaps are indexed by the linear voxel index (z ny + y) nx + x, which is
// also the payload index of the linear layout this update supports.  Set
// semantics make the result independent of the order atomics land in.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "nbt_internal.cuh"

using namespace nbt;

namespace {

constexpr float kMaxVoxelCoord = 4194304.0f;  // 2^22: beyond, index + 1/2 is not exact in FP32
constexpr int kPointRun = 8;                   // consecutive points one thread files
constexpr int kRayChunk = 4;                   // voxels a lane walks ahead of its bitmap reads
constexpr int kRayLanes = 8;                   // lanes that share one free-space ray

struct InsertConst {
  float ox, oy, oz;        // map origin (world)
  float sx, sy, sz;        // sensor (world)
  float vx, vy, vz;        // sensor (voxel units)
  float inv_s;
  float max_range2;        // <= 0: no range limit
  int nx, ny, nz;
};

__device__ __forceinline__ void set_bit(uint32_t *bits, uint32_t v) {
  uint32_t *w = bits + (v >> 5);
  const uint32_t m = 1u << (v & 31u);
  if (!(*(volatile uint32_t *)w & m)) atomicOr(w, m);
}

// 1. Endpoint voxel of every point.
__global__ void points_kernel(const float *__restrict__ pts, int64_t n, InsertConst c, uint32_t *__restrict__ hit,
                              int4 *__restrict__ outside, uint32_t *__restrict__ n_outside) {
  const int64_t n_runs = (n + kPointRun - 1) / kPointRun;
  for (int64_t run = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; run < n_runs;
       run += (int64_t)gridDim.x * blockDim.x)
  for (int64_t i = run * kPointRun, prev = -1, end = min(n, i + kPointRun); i < end; ++i) {
    const float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    if (!(isfinite(px) && isfinite(py) && isfinite(pz))) continue;
    if (c.max_range2 > 0.0f) {
      const float dx = fsub(px, c.sx), dy = fsub(py, c.sy), dz = fsub(pz, c.sz);
      const float r2 = fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
      if (!(r2 <= c.max_range2)) continue;
    }
    const float qx = fmul(fsub(px, c.ox), c.inv_s), qy = fmul(fsub(py, c.oy), c.inv_s),
                qz = fmul(fsub(pz, c.oz), c.inv_s);
    if (!(fabsf(qx) < kMaxVoxelCoord && fabsf(qy) < kMaxVoxelCoord && fabsf(qz) < kMaxVoxelCoord)) continue;
    const int x = (int)floorf(qx), y = (int)floorf(qy), z = (int)floorf(qz);
    if (x >= 0 && x < c.nx && y >= 0 && y < c.ny && z >= 0 && z < c.nz) {
      const int64_t v = ((int64_t)z * c.ny + y) * c.nx + x;
      if (v != prev) set_bit(hit, (uint32_t)v);   // neighbouring pixels usually share a voxel
      prev = v;
    } else {
      const uint32_t k = atomicAdd(n_outside, 1u);
      outside[k] = make_int4(x, y, z, 0);
    }
  }
}

// 2. Distinct in-map endpoints: the set bits of the hit bitmap.
__global__ void enumerate_kernel(const uint32_t *__restrict__ hit, int64_t n_words, uint32_t *__restrict__ list,
                                 uint32_t *__restrict__ n_list) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_words;
       w += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bits = hit[w];
    if (!bits) continue;
    uint32_t k = atomicAdd(n_list, (uint32_t)__popc(bits));
    while (bits) {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1u;
      list[k++] = (uint32_t)(w * 32 + b);
    }
  }
}

// 3. Free space: one ray per distinct endpoint (in-map list, then the
// outside list), sensor to the endpoint voxel's centre.  kRayLanes lanes walk
// one ray: lane l takes its share of the crossings (walk_lane_part), so a
// ray of a few hundred voxels costs each lane only its own part and many
// more walks are in flight than there are rays (a scan has ~75k rays, too
// few to hide the read latency one thread per ray).
__global__ void free_rays_kernel(const uint32_t *__restrict__ list, const uint32_t *__restrict__ n_list,
                                 const int4 *__restrict__ outside, const uint32_t *__restrict__ n_outside,
                                 InsertConst c, uint32_t *__restrict__ miss, unsigned long long *__restrict__ steps) {
  const int64_t n_in = *n_list, total = n_in + *n_outside;
  const float o[3] = {c.vx, c.vy, c.vz};
  const int lane = threadIdx.x & (kRayLanes - 1);
  const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kRayLanes;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) / kRayLanes;
  const int guard = c.nx + c.ny + c.nz + 3;
  unsigned long long steps_lane = 0ull;
  for (int64_t r = warp0; r < total; r += n_warps) {
    int x, y, z;
    if (r < n_in) {
      const uint32_t v = list[r];
      x = (int)(v % (uint32_t)c.nx);
      y = (int)((v / (uint32_t)c.nx) % (uint32_t)c.ny);
      z = (int)(v / ((uint32_t)c.nx * (uint32_t)c.ny));
    } else {
      const int4 e = outside[r - n_in];
      x = e.x;
      y = e.y;
      z = e.z;
    }
    const float d[3] = {fsub(fadd((float)x, 0.5f), o[0]), fsub(fadd((float)y, 0.5f), o[1]),
                        fsub(fadd((float)z, 0.5f), o[2])};
    Walk w;
    if (!walk_init(w, o, d, c.nx, c.ny, c.nz)) continue;
    walk_linear_steps(w, c.nx, c.ny);
    int lin = walk_linear_index(w, c.nx, c.ny);
    bool first, split_end;
    int A;
    if (!walk_lane_part(w, lin, lane, kRayLanes, c.nx, c.ny, c.nz, first, split_end, A)) continue;
    // The lane's voxels in groups of kRayChunk: walk ahead, read the group's
    // bitmap words together, then set the bits that are still clear (most
    // are set already: neighbouring rays cross the same voxels).
    bool pending = first, more = true;
    int g = 0;
    while (more) {
      uint32_t v[kRayChunk], word[kRayChunk];
      int n = 0;
#pragma unroll
      for (int k = 0; k < kRayChunk; ++k) {
        v[k] = (uint32_t)lin;
        if (more) {
          if (pending) {
            pending = false;
            n = k + 1;
          } else {
            float t;
            const int ax = walk_next_axis(w, t);
            if (g++ < guard && (t < w.tmax || (split_end && t == w.tmax && ax < A))) {
              walk_advance_lin(w, lin);   // takes exactly that crossing; its own end test is not needed
              v[k] = (uint32_t)lin;
              n = k + 1;
            } else {
              more = false;
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kRayChunk; ++k) word[k] = k < n ? __ldcg(miss + (v[k] >> 5)) : ~0u;
#pragma unroll
      for (int k = 0; k < kRayChunk; ++k) {
        const uint32_t m = 1u << (v[k] & 31u);
        if (k < n && !(word[k] & m)) atomicOr(miss + (v[k] >> 5), m);
      }
      steps_lane += (unsigned long long)n;
    }
  }
  // voxel steps walked, one atomic per warp
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) steps_lane += __shfl_xor_sync(0xffffffffu, steps_lane, s);
  if ((threadIdx.x & 31) == 0 && steps_lane) atomicAdd(steps, steps_lane);
}

// Bayes update of an occupancy probability by one observation of
// likelihood p, in ratio form with each operation rounded, then clamped.
__device__ __forceinline__ float occupancy_update(float P, float p, float q_p, float lo, float hi) {
  const float a = fmul(P, p);
  const float b = fmul(fsub(1.0f, P), q_p);
  const float r = __fdiv_rn(a, fadd(a, b));
  return r < lo ? lo : (r > hi ? hi : r);
}

struct UpdateConst {
  float p_hit, q_hit, p_miss, q_miss, lo, hi;   // q = 1 - p, rounded once
};

// 4. Apply the scan and clear the bitmaps.
template <int KIND>
__global__ void apply_kernel(uint32_t *__restrict__ hit, uint32_t *__restrict__ miss, int64_t n_words,
                             void *__restrict__ payload, int64_t n_elems, UpdateConst u) {
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n_words;
       w += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t h = hit[w], m0 = miss[w];
    if (!(h | m0)) continue;
    const uint32_t m = m0 & ~h;
    if (h) hit[w] = 0u;
    if (m0) miss[w] = 0u;
    if (KIND == PAYLOAD_GAIN_F32) {
      float *P = (float *)payload + w * 32;
      if ((w + 1) * 32 <= n_elems) {
        // whole 128-byte row: eight independent 16-byte loads, update, store
        float4 row[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) row[q] = ((const float4 *)P)[q];
        float *r = (float *)row;
#pragma unroll
        for (int b = 0; b < 32; ++b) {
          if (((h | m) >> b) & 1u) {
            const bool is_hit = (h >> b) & 1u;
            r[b] = occupancy_update(r[b], is_hit ? u.p_hit : u.p_miss, is_hit ? u.q_hit : u.q_miss, u.lo, u.hi);
          }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (((h | m) >> (4 * q)) & 15u) ((float4 *)P)[q] = row[q];
      } else {
        for (uint32_t bits = h | m; bits; bits &= bits - 1u) {
          const int b = __ffs(bits) - 1;
          const bool is_hit = (h >> b) & 1u;
          P[b] = occupancy_update(P[b], is_hit ? u.p_hit : u.p_miss, is_hit ? u.q_hit : u.q_miss, u.lo, u.hi);
        }
      }
    } else if (KIND == PAYLOAD_U8) {
      uint8_t *S = (uint8_t *)payload + w * 32;
      for (uint32_t bits = h | m; bits; bits &= bits - 1u) {
        const int b = __ffs(bits) - 1;
        S[b] = ((h >> b) & 1u) ? 2 : 1;
      }
    } else {
      // 2-bit states, four voxels per byte: the word's 32 voxels are bytes
      // 8w .. 8w + 7, which no other word touches.
      uint8_t *S = (uint8_t *)payload + w * 8;
      for (int q = 0; q < 8; ++q) {
        const uint32_t hq = (h >> (4 * q)) & 15u, mq = (m >> (4 * q)) & 15u;
        if (!(hq | mq)) continue;
        uint32_t byte = S[q];
        for (int k = 0; k < 4; ++k) {
          const uint32_t st = ((hq >> k) & 1u) ? 2u : (((mq >> k) & 1u) ? 1u : 4u);
          if (st < 4u) byte = (byte & ~(3u << (2 * k))) | (st << (2 * k));
        }
        S[q] = (uint8_t)byte;
      }
    }
  }
}

// Scan statistics: distinct in-map endpoints, rays cast, voxel steps walked.
__global__ void stats_kernel(const uint32_t *__restrict__ count, const unsigned long long *__restrict__ steps,
                             uint64_t *__restrict__ out) {
  if (threadIdx.x == 0) {
    out[0] = count[0];
    out[1] = (uint64_t)count[0] + count[1];
    out[2] = *steps;
  }
}

bool valid_insert(const nbt_insert_params *p) {
  auto open01 = [](float v) { return std::isfinite(v) && v > 0.0f && v < 1.0f; };
  return p && open01(p->prob_hit) && p->prob_hit > 0.5f && open01(p->prob_miss) && p->prob_miss < 0.5f &&
         open01(p->clamp_min) && open01(p->clamp_max) && p->clamp_min < p->clamp_max && std::isfinite(p->max_range);
}

}  // namespace

namespace nbt {

// Insert scratch owned by the map: bitmaps (zero between calls), endpoint
// lists and counters, grown to the largest point count seen.
int ensure_insert_scratch(nbt_map map, int64_t n_points) {
  const int64_t voxels = (int64_t)map->desc.nx * map->desc.ny * map->desc.nz;
  const int64_t words = (voxels + 31) / 32;
  if (!map->ins_hit) {
    if (cudaMalloc((void **)&map->ins_hit, (size_t)words * 4) != cudaSuccess ||
        cudaMalloc((void **)&map->ins_miss, (size_t)words * 4) != cudaSuccess ||
        cudaMalloc((void **)&map->ins_count, 16) != cudaSuccess) {
      (void)cudaGetLastError();
      return NBT_ENOMEM;
    }
    NBT_CUDA_TRY(cudaMemset(map->ins_hit, 0, (size_t)words * 4));
    NBT_CUDA_TRY(cudaMemset(map->ins_miss, 0, (size_t)words * 4));
  }
  if (map->ins_cap < n_points) {
    if (map->ins_list) cudaFree(map->ins_list);
    if (map->ins_outside) cudaFree(map->ins_outside);
    map->ins_list = nullptr;
    map->ins_outside = nullptr;
    map->ins_cap = 0;
    const int64_t list_n = std::min(n_points, voxels);
    if (cudaMalloc((void **)&map->ins_list, (size_t)list_n * 4) != cudaSuccess ||
        cudaMalloc((void **)&map->ins_outside, (size_t)n_points * 16) != cudaSuccess) {
      (void)cudaGetLastError();
      return NBT_ENOMEM;
    }
    map->ins_cap = n_points;
  }
  return NBT_OK;
}

}  // namespace nbt

extern "C" int nbt_map_insert_points(nbt_map map, const float *points, int64_t n, const float *sensor,
                                     const nbt_insert_params *params, uint64_t *stats_out, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n < 0 || n > 0x7fffffff || (n > 0 && !points) || !sensor || !valid_insert(params)) return NBT_EINVAL;
  if (map->brick != 1) return NBT_EUNSUPPORTED;
  InsertConst c;
  c.ox = map->desc.origin[0];
  c.oy = map->desc.origin[1];
  c.oz = map->desc.origin[2];
  c.sx = sensor[0];
  c.sy = sensor[1];
  c.sz = sensor[2];
  c.inv_s = (float)(1.0 / (double)map->desc.voxel_size);
  c.vx = (c.sx - c.ox) * c.inv_s;
  c.vy = (c.sy - c.oy) * c.inv_s;
  c.vz = (c.sz - c.oz) * c.inv_s;
  if (!(std::fabs(c.vx) < kMaxVoxelCoord && std::fabs(c.vy) < kMaxVoxelCoord && std::fabs(c.vz) < kMaxVoxelCoord))
    return NBT_EINVAL;
  c.max_range2 = params->max_range > 0.0f ? params->max_range * params->max_range : 0.0f;
  c.nx = map->desc.nx;
  c.ny = map->desc.ny;
  c.nz = map->desc.nz;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (n == 0) {
    if (stats_out) NBT_CUDA_TRY(cudaMemsetAsync(stats_out, 0, 24, stream));
    return NBT_OK;
  }
  std::lock_guard<std::mutex> lock(map->mu);
  rc = ensure_insert_scratch(map, n);
  if (rc != NBT_OK) return rc;
  const int64_t voxels = (int64_t)c.nx * c.ny * c.nz;
  const int64_t words = (voxels + 31) / 32;
  const int sms = sm_count();
  uint32_t *n_list = map->ins_count, *n_out = map->ins_count + 1;
  unsigned long long *steps = (unsigned long long *)(map->ins_count + 2);
  NBT_CUDA_TRY(cudaMemsetAsync(map->ins_count, 0, 16, stream));
  const int64_t n_runs = (n + kPointRun - 1) / kPointRun;
  const int64_t grid_pts = std::min<int64_t>((n_runs + 255) / 256, (int64_t)sms * 16);
  points_kernel<<<(unsigned)grid_pts, 256, 0, stream>>>(points, n, c, map->ins_hit, (int4 *)map->ins_outside, n_out);
  NBT_CUDA_TRY(cudaGetLastError());
  const int64_t grid_w = std::min<int64_t>((words + 255) / 256, (int64_t)sms * 16);
  enumerate_kernel<<<(unsigned)grid_w, 256, 0, stream>>>(map->ins_hit, words, map->ins_list, n_list);
  NBT_CUDA_TRY(cudaGetLastError());
  const int64_t grid_r = std::min<int64_t>((n * kRayLanes + 255) / 256, (int64_t)sms * 8);   // kRayLanes per ray
  free_rays_kernel<<<(unsigned)grid_r, 256, 0, stream>>>(map->ins_list, n_list, (const int4 *)map->ins_outside,
                                                          n_out, c, map->ins_miss, steps);
  NBT_CUDA_TRY(cudaGetLastError());
  UpdateConst u;
  u.p_hit = params->prob_hit;
  u.q_hit = 1.0f - params->prob_hit;
  u.p_miss = params->prob_miss;
  u.q_miss = 1.0f - params->prob_miss;
  u.lo = params->clamp_min;
  u.hi = params->clamp_max;
  const int kind = map->desc.encoding == NBT_F32_PROB ? PAYLOAD_GAIN_F32
                   : map->desc.encoding == NBT_U8_STATE ? PAYLOAD_U8 : PAYLOAD_U2;
  if (kind == PAYLOAD_GAIN_F32)
    apply_kernel<PAYLOAD_GAIN_F32><<<(unsigned)grid_w, 256, 0, stream>>>(map->ins_hit, map->ins_miss, words,
                                                                         map->d_payload, map->elems, u);
  else if (kind == PAYLOAD_U8)
    apply_kernel<PAYLOAD_U8><<<(unsigned)grid_w, 256, 0, stream>>>(map->ins_hit, map->ins_miss, words, map->d_payload,
                                                                   map->elems, u);
  else
    apply_kernel<PAYLOAD_U2><<<(unsigned)grid_w, 256, 0, stream>>>(map->ins_hit, map->ins_miss, words, map->d_payload,
                                                                   map->elems, u);
  NBT_CUDA_TRY(cudaGetLastError());
  if (stats_out) stats_kernel<<<1, 32, 0, stream>>>(map->ins_count, steps, stats_out);
  NBT_CUDA_TRY(cudaGetLastError());
  map->version += 1;  // derived gains are rebuilt before the next IG call
  return NBT_OK;
}
