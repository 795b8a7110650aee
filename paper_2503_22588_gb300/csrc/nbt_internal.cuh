// nbt_internal.cuh -- internal types and device functions of the IG library.
//
// Layout of a map on the device
// -----------------------------
// The grid is stored in cubic bricks of B^3 voxels (B = 4 or 8), the voxels
// of a brick x-fastest, the bricks in Morton (Z) order of their brick
// coordinates (bit-interleaved x, y, z, with axes that run out of bits
// skipped).  Because the Morton bits of different axes and the in-brick bits
// of different axes never overlap, the element offset of voxel (x, y, z) is
//     tab[x] + tab[nx + y] + tab[nx + ny + z]
// with one per-axis table (int32, nx + ny + nz entries).  The kernels keep
// the three partial offsets in registers and refresh only the one of the
// axis a DDA step moves along, so any brick layout costs one table read per
// step.  Element = one byte (uint8 states), one float (gains), or 2 bits
// (packed states: byte offset >> 2, shift 2 * (offset & 3)).

#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/nbt.h"

namespace nbt {

// Internal encodings of the payload a kernel reads.
enum PayloadKind : int { PAYLOAD_U8 = 0, PAYLOAD_GAIN_F32 = 1, PAYLOAD_U2 = 2 };

constexpr int kMaxDim = 2048;
constexpr int kTileW = 32;          // ray tile: 32 x 8 pixels, 8 warps of 8 x 4 pixels
constexpr int kTileH = 8;
constexpr int kThreads = 256;
constexpr int kPartialBytes = 16;   // one per (pose, tile) item

struct Partial {                    // per-tile partial sums (16 bytes)
  float fsum;                       // FP32 gain sum (F32 payloads)
  uint32_t isum;                    // unknown-voxel count (state payloads)
  uint32_t steps;                   // visited voxels
  uint32_t pad;
};

}  // namespace nbt

struct nbt_map_s {
  nbt_map_desc desc;
  int device = 0;
  int brick = 8;
  int nbx = 0, nby = 0, nbz = 0;     // bricks per axis
  int64_t elems = 0;                 // padded element count of the bricked payload
  int64_t payload_bytes = 0;
  void *d_payload = nullptr;         // bricked u8 / u2 / f32 probabilities
  float *d_gain = nullptr;           // F32 maps: derived signed-gain cache (same layout)
  int32_t *d_tab = nullptr;          // offset tables: nx + ny + nz entries
  void *d_stage = nullptr;           // staging buffer for host uploads
  int64_t stage_bytes = 0;
  uint64_t version = 0;              // bumped by every upload
  // derived gain cache key
  bool gain_valid = false;
  int gain_metric = -1;
  float gain_occ = 0.0f, gain_free = 0.0f;
  uint64_t gain_version = 0;
  std::mutex mu;
};

namespace nbt {

// Map view passed to kernels by value.
struct DevMap {
  const void *payload;
  const int32_t *tab;
  int nx, ny, nz;
};

// Per-call camera constants (Section III endpoint grid), computed on the host.
struct CamConst {
  float x0, xstep, y0, ystep, zc;
  int spherical;
  int W, H;
  int tiles_x, tiles_per_pose;
  float inv_s;
  float ox, oy, oz;                  // map origin, world metres
};

// ---------------------------------------------------------------------------
// FP32 arithmetic with every operation rounded on its own: the __f*_rn
// intrinsics are never contracted into FMAs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }

// Segment (voxel units) of ray (i, j) for a pose: Section III endpoint grid.
__device__ __forceinline__ void ray_segment(const CamConst &cc, const float *pose, int i, int j, float o[3],
                                            float d[3]) {
  const float qw = pose[3], qx = pose[4], qy = pose[5], qz = pose[6];
  const float xx = fmul(qx, qx), yy = fmul(qy, qy), zz = fmul(qz, qz);
  const float xy = fmul(qx, qy), xz = fmul(qx, qz), yz = fmul(qy, qz);
  const float wx = fmul(qw, qx), wy = fmul(qw, qy), wz = fmul(qw, qz);
  float r[9];
  r[0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
  r[1] = fmul(2.0f, fsub(xy, wz));
  r[2] = fmul(2.0f, fadd(xz, wy));
  r[3] = fmul(2.0f, fadd(xy, wz));
  r[4] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
  r[5] = fmul(2.0f, fsub(yz, wx));
  r[6] = fmul(2.0f, fsub(xz, wy));
  r[7] = fmul(2.0f, fadd(yz, wx));
  r[8] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
  float cx = fadd(cc.x0, fmul((float)i, cc.xstep));
  float cy = fadd(cc.y0, fmul((float)j, cc.ystep));
  float cz = cc.zc;
  if (cc.spherical) {
    const float len = __fsqrt_rn(fadd(fadd(fmul(cx, cx), fmul(cy, cy)), fmul(cz, cz)));
    const float sc = __fdiv_rn(cc.zc, len);
    cx = fmul(cx, sc);
    cy = fmul(cy, sc);
    cz = fmul(cz, sc);
  }
  const float org[3] = {cc.ox, cc.oy, cc.oz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float wa = fadd(fadd(fmul(r[3 * a], cx), fmul(r[3 * a + 1], cy)), fmul(r[3 * a + 2], cz));
    o[a] = fmul(fsub(pose[a], org[a]), cc.inv_s);
    d[a] = fmul(wa, cc.inv_s);
  }
}

// ---------------------------------------------------------------------------
// The FP32 voxel walk (reference operation order documented in nbt.h).
// ---------------------------------------------------------------------------
struct Walk {
  int ix, iy, iz;
  int sx, sy, sz;
  float tx, ty, tz;
  float invx, invy, invz;
  float ox, oy, oz;
  float tmax;
};

__device__ __forceinline__ bool finite3(const float v[3]) {
  return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

// Clip the segment to the map box and find the first voxel.  Returns false
// if the segment visits no voxel.
__device__ __forceinline__ bool walk_init(Walk &w, const float o[3], const float d[3], int nx, int ny, int nz) {
  if (!finite3(o) || !finite3(d)) return false;
  const int dims[3] = {nx, ny, nz};
  float inv[3] = {0.0f, 0.0f, 0.0f};
  float tmin = 0.0f, tmax = 1.0f;
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float n = (float)dims[a];
    if (d[a] != 0.0f) {
      inv[a] = __fdiv_rn(1.0f, d[a]);
      const float t0 = fmul(fsub(0.0f, o[a]), inv[a]);
      const float t1 = fmul(fsub(n, o[a]), inv[a]);
      const float lo = inv[a] > 0.0f ? t0 : t1;
      const float hi = inv[a] > 0.0f ? t1 : t0;
      tmin = lo > tmin ? lo : tmin;
      tmax = hi < tmax ? hi : tmax;
    } else if (!(o[a] >= 0.0f && o[a] < n)) {
      ok = false;
    }
  }
  if (!ok || !(tmin < tmax)) return false;
  int idx[3], step[3];
  float tn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float p = fadd(o[a], fmul(tmin, d[a]));
    const float hi = (float)(dims[a] - 1);
    p = p < 0.0f ? 0.0f : p;
    p = p > hi ? hi : p;
    idx[a] = (int)floorf(p);
    step[a] = d[a] > 0.0f ? 1 : (d[a] < 0.0f ? -1 : 0);
    tn[a] = step[a] != 0 ? fmul(fsub((float)(idx[a] + (step[a] > 0)), o[a]), inv[a]) : __int_as_float(0x7f800000);
  }
  w.ix = idx[0]; w.iy = idx[1]; w.iz = idx[2];
  w.sx = step[0]; w.sy = step[1]; w.sz = step[2];
  w.tx = tn[0]; w.ty = tn[1]; w.tz = tn[2];
  w.invx = inv[0]; w.invy = inv[1]; w.invz = inv[2];
  w.ox = o[0]; w.oy = o[1]; w.oz = o[2];
  w.tmax = tmax;
  return true;
}

// One step of the walk; refreshes the partial offset of the moved axis from
// the offset table.  Returns false when the walk has ended (the current
// voxel was the last one).
__device__ __forceinline__ bool walk_step(Walk &w, int nx, int ny, int nz, const int32_t *tab, int &offx,
                                          int &offy, int &offz) {
  if (w.tx <= w.ty && w.tx <= w.tz) {
    if (!(w.tx < w.tmax)) return false;
    w.ix += w.sx;
    if ((unsigned)w.ix >= (unsigned)nx) return false;
    w.tx = fmul(fsub((float)(w.ix + (w.sx > 0)), w.ox), w.invx);
    offx = tab[w.ix];
  } else if (w.ty <= w.tz) {
    if (!(w.ty < w.tmax)) return false;
    w.iy += w.sy;
    if ((unsigned)w.iy >= (unsigned)ny) return false;
    w.ty = fmul(fsub((float)(w.iy + (w.sy > 0)), w.oy), w.invy);
    offy = tab[nx + w.iy];
  } else {
    if (!(w.tz < w.tmax)) return false;
    w.iz += w.sz;
    if ((unsigned)w.iz >= (unsigned)nz) return false;
    w.tz = fmul(fsub((float)(w.iz + (w.sz > 0)), w.oz), w.invz);
    offz = tab[nx + ny + w.iz];
  }
  return true;
}

// Host helpers (defined in nbt_map.cu).
int check_map(nbt_map map);
int prepare_gain(nbt_map map, const nbt_ig_params *params, cudaStream_t stream);
int payload_kind(nbt_map map, const nbt_ig_params *params, PayloadKind *kind, const void **payload);
int sm_count();

}  // namespace nbt

#define NBT_CUDA_TRY(expr)                 \
  do {                                     \
    cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) {               \
      (void)cudaGetLastError();            \
      return NBT_ECUDA;                    \
    }                                      \
  } while (0)
