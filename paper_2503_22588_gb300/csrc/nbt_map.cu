// nbt_map.cu -- voxel map handle: bricked device layout, upload, derived gains.
//
// The paper keeps its voxel map in an octree (UfoMap) on the host and moves
// map data to the GPU for every ID computation (Section V attributes the
// GPU's loss at few rays to that allocation and transfer).  Here the map
// lives on the device for its whole life: nbt_map_create allocates it once,
// nbt_map_upload lays a dense grid out on the device (linear x-fastest, the
// default, or B^3 Morton-ordered bricks) with one coalesced pass, and
// probability maps get a derived per-voxel signed gain table (|value| = g(v)
// of Eq. 2 / entropy / unknown indicator, sign = occupied) so the traversal
// reads one float per voxel step.

#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <unordered_map>
#include <vector>

#include "nbt_internal.cuh"

namespace nbt {

namespace {

constexpr int64_t kStageBytes = 64ll << 20;

int ceil_log2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Per-axis brick-index parts.  Morton: the bits of bx, by, bz are
// interleaved from the least significant end (x, y, z at each level),
// skipping an axis once it has no bits left.  Used when the padded Morton
// space is at most twice the brick count; otherwise bricks are linear.
void brick_parts(int nbx, int nby, int nbz, std::vector<int64_t> &px, std::vector<int64_t> &py,
                 std::vector<int64_t> &pz, int64_t *slots) {
  const int L[3] = {ceil_log2(nbx), ceil_log2(nby), ceil_log2(nbz)};
  const int64_t morton_slots = 1ll << (L[0] + L[1] + L[2]);
  const int64_t linear_slots = (int64_t)nbx * nby * nbz;
  px.assign(nbx, 0);
  py.assign(nby, 0);
  pz.assign(nbz, 0);
  if (morton_slots <= 2 * linear_slots) {
    int pos = 0;
    int64_t bitpos[3][32];
    const int maxl = std::max(L[0], std::max(L[1], L[2]));
    for (int k = 0; k < maxl; ++k)
      for (int a = 0; a < 3; ++a)
        if (k < L[a]) bitpos[a][k] = pos++;
    std::vector<int64_t> *parts[3] = {&px, &py, &pz};
    const int nb[3] = {nbx, nby, nbz};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < nb[a]; ++b) {
        int64_t v = 0;
        for (int k = 0; k < L[a]; ++k)
          if ((b >> k) & 1) v |= 1ll << bitpos[a][k];
        (*parts[a])[b] = v;
      }
    *slots = morton_slots;
  } else {
    for (int b = 0; b < nbx; ++b) px[b] = b;
    for (int b = 0; b < nby; ++b) py[b] = (int64_t)b * nbx;
    for (int b = 0; b < nbz; ++b) pz[b] = (int64_t)b * nbx * nby;
    *slots = linear_slots;
  }
}

__device__ __forceinline__ int32_t voxel_offset(const int32_t *tab, int nx, int ny, int x, int y, int z) {
  return tab[x] + tab[nx + y] + tab[nx + ny + z];
}

// Dense x-fastest slab (z in [z0, z0 + nzs)) -> bricked uint8 / float.
template <typename T>
__global__ void scatter_bricks_kernel(const T *__restrict__ src, T *__restrict__ dst, const int32_t *__restrict__ tab,
                                      int nx, int ny, int z0, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % nx);
    const int64_t r = k / nx;
    const int y = (int)(r % ny);
    const int z = z0 + (int)(r / ny);
    dst[voxel_offset(tab, nx, ny, x, y, z)] = src[k];
  }
}

// Dense uint8 states slab -> 2-bit packed bricks.  Each thread packs four
// x-consecutive voxels (x = 4g .. 4g+3), which are consecutive elements of
// one brick row because B >= 4 and 4 | B; voxels past nx pack as unknown.
__global__ void pack_u2_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst,
                               const int32_t *__restrict__ tab, int nx, int ny, int z0, int64_t n_groups) {
  const int gx = (nx + 3) / 4;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_groups;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(k % gx);
    const int64_t r = k / gx;
    const int y = (int)(r % ny);
    const int zl = (int)(r / ny);
    const int x0 = 4 * g;
    const uint8_t *row = src + ((int64_t)zl * ny + y) * nx;
    uint32_t byte = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int x = x0 + u;
      uint32_t s = x < nx ? row[x] : 0u;
      s = s > 2u ? 2u : s;
      byte |= s << (2 * u);
    }
    const int32_t off = voxel_offset(tab, nx, ny, x0, y, z0 + zl);
    dst[off >> 2] = (uint8_t)byte;
  }
}

// Dense uint8 states (voxels [v0, v0 + n) of the linear order) -> 2-bit
// elements of the linear layout: byte k holds voxels 4k .. 4k+3.  v0 is a
// multiple of 4, so every byte is written by exactly one thread.
__global__ void pack_u2_linear_kernel(const uint8_t *__restrict__ src, uint8_t *__restrict__ dst, int64_t v0,
                                      int64_t n) {
  const int64_t n_bytes = (n + 3) / 4;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_bytes; k += (int64_t)gridDim.x * blockDim.x) {
    uint32_t byte = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t v = 4 * k + u;
      uint32_t s = v < n ? src[v] : 0u;
      s = s > 2u ? 2u : s;
      byte |= s << (2 * u);
    }
    dst[v0 / 4 + k] = (uint8_t)byte;
  }
}

// Device layout -> dense x-fastest grid (the inverse of the upload): uint8
// states (2-bit maps unpacked) or float probabilities.
template <int ENC>
__global__ void gather_dense_kernel(const void *__restrict__ payload, const int32_t *__restrict__ tab, int nx, int ny,
                                    int64_t n, void *__restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(k % nx);
    const int64_t r = k / nx;
    const int y = (int)(r % ny);
    const int z = (int)(r / ny);
    const int32_t off = voxel_offset(tab, nx, ny, x, y, z);
    if (ENC == NBT_F32_PROB)
      ((float *)dst)[k] = ((const float *)payload)[off];
    else if (ENC == NBT_U8_STATE)
      ((uint8_t *)dst)[k] = ((const uint8_t *)payload)[off];
    else
      ((uint8_t *)dst)[k] = (uint8_t)((((const uint8_t *)payload)[off >> 2] >> ((off & 3) << 1)) & 3u);
  }
}

__device__ __forceinline__ float entropy_bits(float p) {
  if (!(p > 0.0f && p < 1.0f)) return 0.0f;
  const float q = 1.0f - p;
  return -p * log2f(p) - q * log2f(q);
}

// Bricked probabilities -> signed gains: |g| = g(v), sign bit = occupied.
__global__ void derive_gain_kernel(const float *__restrict__ p, float *__restrict__ g, int64_t n, int metric,
                                   float occ_thr, float free_thr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const float v = p[k];
    const bool occ = v > occ_thr;
    const bool fre = v < free_thr;
    float gain;
    if (metric == NBT_PAPER_EQ2) {
      gain = occ ? 1.0f - v : (fre ? v : 1.0f);            // Eq. 2
    } else if (metric == NBT_ENTROPY) {
      gain = entropy_bits(v);
    } else {
      gain = (!occ && !fre) ? 1.0f : 0.0f;
    }
    g[k] = occ ? -fabsf(gain) : fabsf(gain);
  }
}

// Brick summaries of a linear state map (one thread per kSkipB^3 brick):
// the class (0 unknown, 1 free, 2 occupied) of every voxel of the brick that
// lies inside the map; kSumUnknown / kSumFree if all equal, else kSumOther.
template <int ENC>
__global__ void brick_summary_kernel(const uint8_t *__restrict__ payload, int nx, int ny, int nz, int bsx, int bsy,
                                     int bsz, uint8_t *__restrict__ bsum) {
  const int64_t nb = (int64_t)bsx * bsy * bsz;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int x0 = (int)(b % bsx) * kSkipB;
    const int y0 = (int)((b / bsx) % bsy) * kSkipB;
    const int z0 = (int)(b / ((int64_t)bsx * bsy)) * kSkipB;
    const int x1 = min(x0 + kSkipB, nx), y1 = min(y0 + kSkipB, ny), z1 = min(z0 + kSkipB, nz);
    if ((nx & 7) == 0 && x1 - x0 == 8) {
      // whole 8-voxel rows (nx a multiple of 8): one aligned 16-bit (2-bit states) or 64-bit (bytes)
      // word per row, compared with the first voxel's class repeated
      const int64_t v0 = ((int64_t)z0 * ny + y0) * nx + x0;
      uint32_t first = ENC == NBT_U2_STATE ? payload[v0 >> 2] & 3u : payload[v0];
      bool uniform = first < 2u;
      const uint64_t pat = first ? (ENC == NBT_U2_STATE ? 0x5555ull : 0x0101010101010101ull) : 0ull;
      for (int z = z0; z < z1 && uniform; ++z)
        for (int y = y0; y < y1; ++y) {
          const int64_t v = ((int64_t)z * ny + y) * nx + x0;
          const uint64_t w = ENC == NBT_U2_STATE ? (uint64_t)*(const uint16_t *)(payload + (v >> 2))
                                                 : *(const uint64_t *)(payload + v);
          if (w != pat) {
            uniform = false;
            break;
          }
        }
      bsum[b] = (uint8_t)(uniform ? first : kSumOther);
      continue;
    }
    uint32_t first = 4u;
    bool uniform = true;
    for (int z = z0; z < z1 && uniform; ++z)
      for (int y = y0; y < y1 && uniform; ++y) {
        const int64_t row = ((int64_t)z * ny + y) * nx;
        for (int x = x0; x < x1; ++x) {
          const int64_t v = row + x;
          uint32_t st = ENC == NBT_U2_STATE ? (payload[v >> 2] >> ((v & 3) << 1)) & 3u : payload[v];
          st = st > 2u ? 2u : st;
          if (first == 4u) first = st;
          if (st != first || st == 2u) {
            uniform = false;
            break;
          }
        }
      }
    bsum[b] = (uint8_t)(uniform ? first : kSumOther);
  }
}

// Brick summaries of a linear FP32 map from its derived signed-gain table (one
// thread per kSkipB^3 brick): kSumUnknown where every gain inside the map is
// exactly +1 (an unknown voxel under all three metrics), kSumFree where every
// one is exactly +0, else kSumOther (an occupied voxel, or gains that vary).
__global__ void brick_summary_gain_kernel(const float *__restrict__ gain, int nx, int ny, int nz, int bsx, int bsy,
                                          int bsz, uint8_t *__restrict__ bsum) {
  const int64_t nb = (int64_t)bsx * bsy * bsz;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int x0 = (int)(b % bsx) * kSkipB;
    const int y0 = (int)((b / bsx) % bsy) * kSkipB;
    const int z0 = (int)(b / ((int64_t)bsx * bsy)) * kSkipB;
    const int x1 = min(x0 + kSkipB, nx), y1 = min(y0 + kSkipB, ny), z1 = min(z0 + kSkipB, nz);
    const uint32_t first = __float_as_uint(gain[((int64_t)z0 * ny + y0) * nx + x0]);
    bool uniform = first == 0x3f800000u || first == 0u;
    for (int z = z0; z < z1 && uniform; ++z)
      for (int y = y0; y < y1 && uniform; ++y) {
        const int64_t row = ((int64_t)z * ny + y) * nx;
        for (int x = x0; x < x1; ++x)
          if (__float_as_uint(gain[row + x]) != first) {
            uniform = false;
            break;
          }
      }
    bsum[b] = (uint8_t)(!uniform ? kSumOther : (first == 0u ? kSumFree : kSumUnknown));
  }
}

// Level l + 1 of the summary pyramid from level l (one thread per brick):
// uniform with class c exactly where every child inside the map is uniform
// with class c.
__global__ void brick_summary_up_kernel(const uint8_t *__restrict__ child, int cx, int cy, int cz,
                                        uint8_t *__restrict__ parent, int px, int py, int pz) {
  const int64_t nb = (int64_t)px * py * pz;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const int x0 = (int)(b % px) * 2, y0 = (int)((b / px) % py) * 2, z0 = (int)(b / ((int64_t)px * py)) * 2;
    uint32_t first = 4u;
    bool uniform = true;
    for (int z = z0; z < min(z0 + 2, cz); ++z)
      for (int y = y0; y < min(y0 + 2, cy); ++y)
        for (int x = x0; x < min(x0 + 2, cx); ++x) {
          const uint32_t c = child[((int64_t)z * cy + y) * cx + x];
          if (first == 4u) first = c;
          uniform = uniform && c == first && c != kSumOther;
        }
    parent[b] = (uint8_t)(uniform ? first : kSumOther);
  }
}

// Level-0 bytes rewritten as class | (L << 2): L = the highest level whose
// brick containing this 8^3 brick is uniform (with this brick's class).
// Reads only its own level-0 byte and levels >= 1, so it may run in place.
__global__ void brick_summary_levels_kernel(uint8_t *__restrict__ bsum, int bx, int by, int bz,
                                            const int3 *__restrict__ dims, const int64_t *__restrict__ offs) {
  const int64_t nb = (int64_t)bx * by * bz;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = bsum[b];
    if (c > kSumFree) continue;
    const int x = (int)(b % bx), y = (int)((b / bx) % by), z = (int)(b / ((int64_t)bx * by));
    uint32_t lvl = 0;
    for (int l = 1; l < kSkipLevels; ++l) {
      const int3 d = dims[l];
      const uint32_t p = bsum[offs[l] + ((int64_t)(z >> l) * d.y + (y >> l)) * d.x + (x >> l)];
      if (p != c) break;
      lvl = (uint32_t)l;
    }
    bsum[b] = (uint8_t)(c | (lvl << 2));
  }
}

int grid_for(int64_t n) {
  const int64_t blocks = (n + 255) / 256;
  return (int)std::min<int64_t>(std::max<int64_t>(blocks, 1), (int64_t)sm_count() * 16);
}

int elem_size(int encoding) { return encoding == NBT_F32_PROB ? 4 : 1; }

}  // namespace

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cached[dev] = n;
  }
  return cached[dev];
}

// Live maps: handle -> creation id.  Every handle-taking call checks that
// the handle names a live map before reading it, so a destroyed handle
// returns NBT_EINVAL instead of reading freed memory; a plan also checks the
// id, which a new map created at the same address does not share.
namespace {
std::mutex g_maps_mu;
std::unordered_map<const nbt_map_s *, uint64_t> g_maps;
uint64_t g_next_map_id = 1;

uint64_t register_map(nbt_map m) {
  std::lock_guard<std::mutex> lock(g_maps_mu);
  const uint64_t id = g_next_map_id++;
  g_maps[m] = id;
  return id;
}

bool unregister_map(nbt_map m) {
  std::lock_guard<std::mutex> lock(g_maps_mu);
  return g_maps.erase(m) == 1;
}
}  // namespace

bool map_alive(nbt_map map, uint64_t id) {
  std::lock_guard<std::mutex> lock(g_maps_mu);
  const auto it = g_maps.find(map);
  return it != g_maps.end() && (id == 0 || it->second == id);
}

int check_map(nbt_map map) {
  if (!map || !map_alive(map, 0)) return NBT_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NBT_ECUDA;
  return dev == map->device ? NBT_OK : NBT_EINVAL;
}

int prepare_gain(nbt_map map, const nbt_ig_params *prm, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(map->mu);
  if (map->gain_valid && map->gain_metric == prm->metric && map->gain_occ == prm->occ_threshold &&
      map->gain_free == prm->free_threshold && map->gain_version == map->version)
    return NBT_OK;
  derive_gain_kernel<<<grid_for(map->elems), 256, 0, stream>>>((const float *)map->d_payload, map->d_gain,
                                                               map->elems, prm->metric, prm->occ_threshold,
                                                               prm->free_threshold);
  NBT_CUDA_TRY(cudaGetLastError());
  map->gain_gen += 1;               // summaries built from older gains are stale
  map->gain_valid = true;
  map->gain_metric = prm->metric;
  map->gain_occ = prm->occ_threshold;
  map->gain_free = prm->free_threshold;
  map->gain_version = map->version;
  return NBT_OK;
}

namespace {

// The pyramid from the payload (state maps) or the derived gains (FP32 maps);
// the caller holds the map's lock.
int build_bsum(nbt_map map, cudaStream_t stream) {
  const nbt_map_desc &d = map->desc;
  const int64_t nb = (int64_t)map->bsx[0] * map->bsy[0] * map->bsz[0];
  const uint8_t *p = (const uint8_t *)map->d_payload;
  if (d.encoding == NBT_F32_PROB)
    brick_summary_gain_kernel<<<grid_for(nb), 256, 0, stream>>>(map->d_gain, d.nx, d.ny, d.nz, map->bsx[0],
                                                               map->bsy[0], map->bsz[0], map->d_bsum);
  else if (d.encoding == NBT_U2_STATE)
    brick_summary_kernel<NBT_U2_STATE><<<grid_for(nb), 256, 0, stream>>>(p, d.nx, d.ny, d.nz, map->bsx[0],
                                                                         map->bsy[0], map->bsz[0], map->d_bsum);
  else
    brick_summary_kernel<NBT_U8_STATE><<<grid_for(nb), 256, 0, stream>>>(p, d.nx, d.ny, d.nz, map->bsx[0],
                                                                         map->bsy[0], map->bsz[0], map->d_bsum);
  NBT_CUDA_TRY(cudaGetLastError());
  for (int l = 1; l < kSkipLevels; ++l) {
    const int64_t np = (int64_t)map->bsx[l] * map->bsy[l] * map->bsz[l];
    brick_summary_up_kernel<<<grid_for(np), 256, 0, stream>>>(map->d_bsum + map->boff[l - 1], map->bsx[l - 1],
                                                             map->bsy[l - 1], map->bsz[l - 1], map->d_bsum + map->boff[l],
                                                             map->bsx[l], map->bsy[l], map->bsz[l]);
    NBT_CUDA_TRY(cudaGetLastError());
  }
  brick_summary_levels_kernel<<<grid_for(nb), 256, 0, stream>>>(map->d_bsum, map->bsx[0], map->bsy[0], map->bsz[0],
                                                               map->d_bdims, map->d_boffs);
  NBT_CUDA_TRY(cudaGetLastError());
  map->bsum_valid = true;
  map->bsum_key = d.encoding == NBT_F32_PROB ? map->gain_gen : map->version;
  return NBT_OK;
}

}  // namespace

// Rebuild the summaries when the payload (state maps) or the derived gains
// (FP32 maps; prepare_gain runs first) changed since they were built.  Only
// the calls that run the skipping walk ask for them.
int prepare_bsum(nbt_map map, cudaStream_t stream) {
  std::lock_guard<std::mutex> lock(map->mu);
  if (!map->d_bsum) return NBT_OK;
  const uint64_t key = map->desc.encoding == NBT_F32_PROB ? map->gain_gen : map->version;
  if (map->bsum_valid && map->bsum_key == key) return NBT_OK;
  return build_bsum(map, stream);
}

int payload_kind(nbt_map map, const nbt_ig_params *prm, PayloadKind *kind, const void **payload) {
  switch (map->desc.encoding) {
    case NBT_U8_STATE:
      if (prm && prm->metric != NBT_COUNT_UNKNOWN) return NBT_EUNSUPPORTED;
      *kind = PAYLOAD_U8;
      *payload = map->d_payload;
      return NBT_OK;
    case NBT_U2_STATE:
      if (prm && prm->metric != NBT_COUNT_UNKNOWN) return NBT_EUNSUPPORTED;
      *kind = PAYLOAD_U2;
      *payload = map->d_payload;
      return NBT_OK;
    case NBT_F32_PROB:
      *kind = PAYLOAD_GAIN_F32;
      *payload = map->d_gain;
      return NBT_OK;
    default:
      return NBT_EINVAL;
  }
}

}  // namespace nbt

using namespace nbt;

extern "C" {

const char *nbt_status_string(int status) {
  switch (status) {
    case NBT_OK: return "NBT_OK";
    case NBT_EINVAL: return "NBT_EINVAL: invalid argument";
    case NBT_ENOMEM: return "NBT_ENOMEM: allocation failed";
    case NBT_ECUDA: return "NBT_ECUDA: CUDA runtime error";
    case NBT_ETIMEOUT: return "NBT_ETIMEOUT: bounded device wait gave up";
    case NBT_EUNSUPPORTED: return "NBT_EUNSUPPORTED: unsupported combination";
    case NBT_EWORKSPACE: return "NBT_EWORKSPACE: workspace missing or too small";
    case NBT_ESCRATCH: return "NBT_ESCRATCH: request exceeds the fixed scratch of nbt_views_ig_noalloc";
    default: return "unknown status";
  }
}

int nbt_get_version(int32_t *version) {
  if (!version) return NBT_EINVAL;
  *version = NBT_API_VERSION;
  return NBT_OK;
}

int nbt_map_create(const nbt_map_desc *desc, nbt_map *out) {
  if (!desc || !out) return NBT_EINVAL;
  *out = nullptr;
  const nbt_map_desc &d = *desc;
  if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > kMaxDim || d.ny > kMaxDim || d.nz > kMaxDim) return NBT_EINVAL;
  if ((int64_t)d.nx * d.ny * d.nz >= (1ll << 31)) return NBT_EINVAL;
  if (!(d.voxel_size > 0.0f) || !isfinite(d.voxel_size)) return NBT_EINVAL;
  if (!isfinite(d.origin[0]) || !isfinite(d.origin[1]) || !isfinite(d.origin[2])) return NBT_EINVAL;
  if (d.encoding != NBT_U8_STATE && d.encoding != NBT_F32_PROB && d.encoding != NBT_U2_STATE) return NBT_EINVAL;
  const int brick = d.brick == 0 ? 1 : d.brick;
  if (brick != 1 && brick != 4 && brick != 8) return NBT_EINVAL;

  nbt_map m = new (std::nothrow) nbt_map_s();
  if (!m) return NBT_ENOMEM;
  m->desc = d;
  m->desc.brick = brick;
  m->brick = brick;
  if (cudaGetDevice(&m->device) != cudaSuccess) {
    delete m;
    return NBT_ECUDA;
  }
  const int lb = brick == 8 ? 3 : (brick == 4 ? 2 : 0);
  m->nbx = (d.nx + brick - 1) / brick;
  m->nby = (d.ny + brick - 1) / brick;
  m->nbz = (d.nz + brick - 1) / brick;
  std::vector<int64_t> px, py, pz;
  int64_t slots = 0;
  const int64_t b3 = (int64_t)brick * brick * brick;
  if (brick == 1) {  // linear x-fastest layout: element index = (z * ny + y) * nx + x
    px.resize(m->nbx);
    py.resize(m->nby);
    pz.resize(m->nbz);
    for (int b = 0; b < m->nbx; ++b) px[b] = b;
    for (int b = 0; b < m->nby; ++b) py[b] = (int64_t)b * m->nbx;
    for (int b = 0; b < m->nbz; ++b) pz[b] = (int64_t)b * m->nbx * m->nby;
    slots = (int64_t)m->nbx * m->nby * m->nbz;
    m->elems = (slots + 3) / 4 * 4;  // whole bytes of 2-bit elements
  } else {
    brick_parts(m->nbx, m->nby, m->nbz, px, py, pz, &slots);
    m->elems = slots * b3;
  }
  if (m->elems >= (1ll << 31)) {
    delete m;
    return NBT_EINVAL;
  }
  std::vector<int32_t> tab((size_t)d.nx + d.ny + d.nz);
  const int mask = brick - 1;
  for (int x = 0; x < d.nx; ++x) tab[x] = (int32_t)(px[x >> lb] * b3 + (x & mask));
  for (int y = 0; y < d.ny; ++y) tab[d.nx + y] = (int32_t)(py[y >> lb] * b3 + (int64_t)(y & mask) * brick);
  for (int z = 0; z < d.nz; ++z)
    tab[d.nx + d.ny + z] = (int32_t)(pz[z >> lb] * b3 + (int64_t)(z & mask) * brick * brick);

  m->payload_bytes = d.encoding == NBT_F32_PROB ? m->elems * 4 : (d.encoding == NBT_U2_STATE ? m->elems / 4 : m->elems);
  m->payload_bytes = (m->payload_bytes + 15) / 16 * 16;  // whole 16-byte words: walks may read the word of the last element
  const int64_t dense_bytes = (int64_t)d.nx * d.ny * d.nz * elem_size(d.encoding);
  m->stage_bytes = std::min(dense_bytes, std::max<int64_t>(kStageBytes, (int64_t)d.nx * d.ny * elem_size(d.encoding)));
  int rc = NBT_OK;
  if (cudaMalloc(&m->d_payload, (size_t)m->payload_bytes) != cudaSuccess) rc = NBT_ENOMEM;
  if (rc == NBT_OK && d.encoding == NBT_F32_PROB &&
      cudaMalloc((void **)&m->d_gain, (size_t)m->elems * 4) != cudaSuccess)
    rc = NBT_ENOMEM;
  if (rc == NBT_OK && cudaMalloc((void **)&m->d_tab, tab.size() * sizeof(int32_t)) != cudaSuccess) rc = NBT_ENOMEM;
  if (rc == NBT_OK && cudaMalloc(&m->d_stage, (size_t)m->stage_bytes) != cudaSuccess) rc = NBT_ENOMEM;
  if (rc == NBT_OK && brick == 1) {
    int64_t total = 0;
    for (int l = 0; l < kSkipLevels; ++l) {
      const int e = kSkipB << l;
      m->bsx[l] = (d.nx + e - 1) / e;
      m->bsy[l] = (d.ny + e - 1) / e;
      m->bsz[l] = (d.nz + e - 1) / e;
      m->boff[l] = total;
      total += (int64_t)m->bsx[l] * m->bsy[l] * m->bsz[l];
    }
    if (cudaMalloc((void **)&m->d_bsum, (size_t)total) != cudaSuccess) rc = NBT_ENOMEM;
    // per-level brick counts and offsets for the level pass
    int3 dims[kSkipLevels];
    for (int l = 0; l < kSkipLevels; ++l) dims[l] = make_int3(m->bsx[l], m->bsy[l], m->bsz[l]);
    if (rc == NBT_OK && cudaMalloc((void **)&m->d_bdims, sizeof(dims)) != cudaSuccess) rc = NBT_ENOMEM;
    if (rc == NBT_OK && cudaMalloc((void **)&m->d_boffs, sizeof(m->boff)) != cudaSuccess) rc = NBT_ENOMEM;
    if (rc == NBT_OK && (cudaMemcpy(m->d_bdims, dims, sizeof(dims), cudaMemcpyHostToDevice) != cudaSuccess ||
                         cudaMemcpy(m->d_boffs, m->boff, sizeof(m->boff), cudaMemcpyHostToDevice) != cudaSuccess))
      rc = NBT_ECUDA;
  }
  if (rc == NBT_OK && cudaMemset(m->d_payload, 0, (size_t)m->payload_bytes) != cudaSuccess) rc = NBT_ECUDA;
  if (rc == NBT_OK && cudaMemcpy(m->d_tab, tab.data(), tab.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
                          cudaSuccess)
    rc = NBT_ECUDA;
  if (rc != NBT_OK) {
    (void)cudaGetLastError();
    free_map(m);
    return rc;
  }
  m->id = register_map(m);
  *out = m;
  return NBT_OK;
}

int nbt_map_destroy(nbt_map map) {
  if (!map) return NBT_OK;
  if (!unregister_map(map)) return NBT_EINVAL;  // not a live map (already destroyed)
  free_map(map);
  return NBT_OK;
}

}  // extern "C"

namespace nbt {

void free_map(nbt_map map) {
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != map->device) cudaSetDevice(map->device);
  cudaDeviceSynchronize();
  if (map->d_payload) cudaFree(map->d_payload);
  if (map->d_gain) cudaFree(map->d_gain);
  if (map->d_tab) cudaFree(map->d_tab);
  if (map->d_stage) cudaFree(map->d_stage);
  if (map->d_bsum) cudaFree(map->d_bsum);
  if (map->d_bdims) cudaFree(map->d_bdims);
  if (map->d_boffs) cudaFree(map->d_boffs);
  if (map->ins_hit) cudaFree(map->ins_hit);
  if (map->ins_miss) cudaFree(map->ins_miss);
  if (map->ins_count) cudaFree(map->ins_count);
  if (map->ins_list) cudaFree(map->ins_list);
  if (map->ins_outside) cudaFree(map->ins_outside);
  (void)cudaGetLastError();
  if (prev >= 0 && prev != map->device) cudaSetDevice(prev);
  delete map;
}

}  // namespace nbt

extern "C" {

int nbt_map_upload(nbt_map map, const void *src, int64_t bytes, int32_t src_on_device, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (!src) return NBT_EINVAL;
  const nbt_map_desc &d = map->desc;
  const int es = elem_size(d.encoding);
  const int64_t plane = (int64_t)d.nx * d.ny;
  if (bytes != plane * d.nz * es) return NBT_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  std::lock_guard<std::mutex> lock(map->mu);
  int slab = src_on_device ? d.nz : (int)std::max<int64_t>(1, map->stage_bytes / (plane * es));
  // linear 2-bit maps: slab starts must fall on whole bytes (4 voxels)
  if (d.encoding == NBT_U2_STATE && map->brick == 1 && slab < d.nz) slab = std::max(4, slab / 4 * 4);
  for (int z0 = 0; z0 < d.nz; z0 += slab) {
    const int nzs = std::min(slab, d.nz - z0);
    const char *s = (const char *)src + (int64_t)z0 * plane * es;
    if (!src_on_device) {
      NBT_CUDA_TRY(cudaMemcpyAsync(map->d_stage, s, (size_t)(nzs * plane * es), cudaMemcpyHostToDevice, stream));
      s = (const char *)map->d_stage;
    }
    const int64_t n = nzs * plane;
    if (d.encoding == NBT_U8_STATE) {
      scatter_bricks_kernel<uint8_t><<<grid_for(n), 256, 0, stream>>>((const uint8_t *)s, (uint8_t *)map->d_payload,
                                                                      map->d_tab, d.nx, d.ny, z0, n);
    } else if (d.encoding == NBT_F32_PROB) {
      scatter_bricks_kernel<float><<<grid_for(n), 256, 0, stream>>>((const float *)s, (float *)map->d_payload,
                                                                    map->d_tab, d.nx, d.ny, z0, n);
    } else if (map->brick == 1) {
      pack_u2_linear_kernel<<<grid_for((n + 3) / 4), 256, 0, stream>>>((const uint8_t *)s, (uint8_t *)map->d_payload,
                                                                      (int64_t)z0 * plane, n);
    } else {
      const int64_t groups = (int64_t)((d.nx + 3) / 4) * d.ny * nzs;
      pack_u2_kernel<<<grid_for(groups), 256, 0, stream>>>((const uint8_t *)s, (uint8_t *)map->d_payload, map->d_tab,
                                                           d.nx, d.ny, z0, groups);
    }
    NBT_CUDA_TRY(cudaGetLastError());
  }
  map->version += 1;
  map->gain_valid = false;
  return NBT_OK;
}

int nbt_map_download(nbt_map map, void *dst, int64_t bytes, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  const nbt_map_desc &d = map->desc;
  const int64_t n = (int64_t)d.nx * d.ny * d.nz;
  if (!dst || bytes != n * elem_size(d.encoding)) return NBT_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  if (d.encoding == NBT_F32_PROB)
    gather_dense_kernel<NBT_F32_PROB><<<grid_for(n), 256, 0, stream>>>(map->d_payload, map->d_tab, d.nx, d.ny, n, dst);
  else if (d.encoding == NBT_U8_STATE)
    gather_dense_kernel<NBT_U8_STATE><<<grid_for(n), 256, 0, stream>>>(map->d_payload, map->d_tab, d.nx, d.ny, n, dst);
  else
    gather_dense_kernel<NBT_U2_STATE><<<grid_for(n), 256, 0, stream>>>(map->d_payload, map->d_tab, d.nx, d.ny, n, dst);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int nbt_map_info(nbt_map map, nbt_map_desc *desc, int64_t *device_bytes) {
  if (!map || !map_alive(map, 0)) return NBT_EINVAL;
  if (desc) *desc = map->desc;
  if (device_bytes) {
    int64_t b = map->payload_bytes + (int64_t)(map->desc.nx + map->desc.ny + map->desc.nz) * 4 + map->stage_bytes;
    if (map->d_gain) b += map->elems * 4;
    if (map->d_bsum)
      b += map->boff[kSkipLevels - 1] +
           (int64_t)map->bsx[kSkipLevels - 1] * map->bsy[kSkipLevels - 1] * map->bsz[kSkipLevels - 1];
    *device_bytes = b;
  }
  return NBT_OK;
}

}  // extern "C"
