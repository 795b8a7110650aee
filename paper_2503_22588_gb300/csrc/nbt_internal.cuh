// nbt_internal.cuh -- internal types and device functions of the IG library.
//
// Layout of a map on the device
// -----------------------------
// Two layouts.  Linear (brick = 1, the default): x-fastest, element index
// (z * ny + y) * nx + x; a DDA step adds a fixed per-axis stride.  Bricked
// (brick = 4 or 8): cubic bricks of B^3 voxels, x-fastest inside a brick,
// bricks in Morton (Z) order of their brick coordinates (bit-interleaved x, y,
// z, axes that run out of bits skipped).  Because the Morton bits of
// different axes and the in-brick bits of different axes never overlap, the
// element offset of voxel (x, y, z) is
//     tab[x] + tab[nx + y] + tab[nx + ny + z]
// with one per-axis table (int32, nx + ny + nz entries; built for both
// layouts).  The bricked kernel keeps the three partial offsets in registers
// and re-reads them from a shared-memory copy of the tables every step.
// Element = one byte (uint8 states), one float (gains), or 2 bits (packed
// states: byte offset >> 2, shift 2 * (offset & 3)).

#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/nbt.h"

namespace nbt {

// Internal encodings of the payload a kernel reads.
enum PayloadKind : int { PAYLOAD_U8 = 0, PAYLOAD_GAIN_F32 = 1, PAYLOAD_U2 = 2 };

constexpr int kMaxDim = 2048;
constexpr int kTileW = 32;          // ray tile: 32 x 8 pixels = 8 warp packets of 32 rays
constexpr int kTileH = 8;
constexpr int kThreads = 256;          // 8 warps, each working on its own tiles
constexpr int kPartialBytes = 16;   // one per (pose, tile) item

// Brick summaries (count walks on linear state maps): a pyramid of kSkipLevels
// levels; level l cuts the map into cubic bricks of edge 2^(kSkipLog + l)
// aligned to the origin, and a brick's byte says whether every voxel of it
// inside the map is unknown (kSumUnknown), every one is free (kSumFree), or
// neither (kSumOther: mixed, or holding an occupied voxel).  Level l + 1 is
// uniform exactly where its (up to) 8 children are uniform with one class.
// Once the pyramid is built, each level-0 byte is rewritten as class | (L <<
// 2), L the highest level whose brick around it is uniform, so that a walk
// finds the largest uniform brick around a voxel with one read (L < 64).
constexpr int kSkipLog = 3;
constexpr int kSkipB = 1 << kSkipLog;
#ifndef NBT_SKIP_LEVELS
#define NBT_SKIP_LEVELS 4
#endif
constexpr int kSkipLevels = NBT_SKIP_LEVELS;  // bricks of 8, 16, ..., 2^(2 + kSkipLevels) voxels
constexpr uint32_t kSumUnknown = 0, kSumFree = 1, kSumOther = 3;


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
  int packet_w = 8;                  // warp ray packet width (nbt_map_set_tuning)
  int skip = 1;                      // 1: count walks skip uniform bricks (nbt_map_set_tuning)
  int nbx = 0, nby = 0, nbz = 0;     // bricks per axis
  int64_t elems = 0;                 // padded element count of the bricked payload
  int64_t payload_bytes = 0;
  void *d_payload = nullptr;         // bricked u8 / u2 / f32 probabilities
  float *d_gain = nullptr;           // F32 maps: derived signed-gain cache (same layout)
  int32_t *d_tab = nullptr;          // offset tables: nx + ny + nz entries
  void *d_stage = nullptr;           // staging buffer for host uploads
  int64_t stage_bytes = 0;
  uint64_t id = 0;                   // unique per created map (live-map registry)
  uint64_t version = 0;              // bumped by every upload
  // derived gain cache key
  bool gain_valid = false;
  int gain_metric = -1;
  float gain_occ = 0.0f, gain_free = 0.0f;
  uint64_t gain_version = 0;
  uint64_t gain_gen = 0;             // bumped whenever the gains are derived anew
  // brick summaries of linear state maps (count walks skip uniform bricks):
  // one byte per kSkipB^3 brick, derived from the payload, rebuilt when stale
  uint8_t *d_bsum = nullptr;
  int bsx[nbt::kSkipLevels] = {0}, bsy[nbt::kSkipLevels] = {0}, bsz[nbt::kSkipLevels] = {0};  // bricks per axis, level
  int64_t boff[nbt::kSkipLevels] = {0};  // first byte of each level
  int3 *d_bdims = nullptr;           // device copies of the per-level brick counts and offsets
  int64_t *d_boffs = nullptr;
  bool bsum_valid = false;
  uint64_t bsum_key = 0;             // what the summaries were built from: the payload version (state
                                     // maps) or the gain generation (FP32 maps)
  // point-cloud insertion scratch (nbt_map_insert_points), allocated on first use
  uint32_t *ins_hit = nullptr;       // hit bitmap, one bit per voxel, zero between calls
  uint32_t *ins_miss = nullptr;      // miss bitmap, likewise
  uint32_t *ins_count = nullptr;     // [0] distinct in-map endpoints, [1] endpoints outside the map,
                                     // [2..3] voxel steps walked (uint64)
  uint32_t *ins_list = nullptr;      // distinct in-map endpoint voxels
  void *ins_outside = nullptr;       // int4 voxel coordinates of endpoints outside the map
  int64_t ins_cap = 0;               // points the lists hold
  std::mutex mu;
};

namespace nbt {

// Map view passed to kernels by value.
struct DevMap {
  const void *payload;
  const int32_t *tab;
  int nx, ny, nz;
  const uint8_t *bsum;               // brick summary pyramid (count walks), else null
  int bsx[kSkipLevels], bsy[kSkipLevels];  // bricks along x and y per level
  int boff[kSkipLevels];             // first byte of each level
};

// Per-call camera constants (Section III endpoint grid), computed on the host.
struct CamConst {
  float x0, xstep, y0, ystep, zc;
  int spherical;
  int W, H;
  int tiles_x, tiles_per_pose;
  int packet_w;                      // warp ray packet: packet_w x (32 / packet_w) pixels
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

// Camera-to-world rotation (row-major) of the unit quaternion q = (w, x, y, z),
// every operation rounded to FP32 in this fixed order.
__device__ __forceinline__ void quat_rot_f32(const float *q, float r[9]) {
  const float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
  const float xx = fmul(qx, qx), yy = fmul(qy, qy), zz = fmul(qz, qz);
  const float xy = fmul(qx, qy), xz = fmul(qx, qz), yz = fmul(qy, qz);
  const float wx = fmul(qw, qx), wy = fmul(qw, qy), wz = fmul(qw, qz);
  r[0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
  r[1] = fmul(2.0f, fsub(xy, wz));
  r[2] = fmul(2.0f, fadd(xz, wy));
  r[3] = fmul(2.0f, fadd(xy, wz));
  r[4] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
  r[5] = fmul(2.0f, fsub(yz, wx));
  r[6] = fmul(2.0f, fsub(xz, wy));
  r[7] = fmul(2.0f, fadd(yz, wx));
  r[8] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
}

// Segment (voxel units) of ray (i, j) for a pose whose rotation r =
// quat_rot_f32(pose + 3) is given: Section III endpoint grid.
__device__ __forceinline__ void ray_segment_rot(const CamConst &cc, const float *pose, const float *r, int i, int j,
                                                float o[3], float d[3]) {
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

__device__ __forceinline__ void ray_segment(const CamConst &cc, const float *pose, int i, int j, float o[3],
                                            float d[3]) {
  float r[9];
  quat_rot_f32(pose + 3, r);
  ray_segment_rot(cc, pose, r, i, j, o, d);
}

// ---------------------------------------------------------------------------
// The FP32 voxel walk (reference operation order documented in nbt.h).
//
// State per axis a: the parameter t_a of the next plane crossing, the
// coordinate b_a of that plane as an integer-valued float (b_a = i_a + [s_a >
// 0], exact below 2^24), the step s_a, o_a, 1/d_a, and the byte offset of
// voxel index i_a in the axis' offset table.  A step advances b_a by s_a
// (exact) and recomputes t_a = (b_a - o_a) * (1/d_a): the same two rounded
// operations as ((float)(i_a + [s_a > 0]) - o_a) * (1/d_a), so the sequence
// is bit-identical to the reference walk.  A step is branch-free (see
// walk_advance), so the lanes of a warp never diverge inside it.
//
// No index range check is needed per step: the plane that would take axis
// a out of the map has b_a = N_a (or 0), whose t is computed by exactly the
// expression of the clip value on that axis, which is >= t_max; the t_max
// test therefore always ends the walk first.
// ---------------------------------------------------------------------------
struct Walk {
  float tx, ty, tz;        // next crossing parameter (+inf: no crossing on that axis)
  float bx, by, bz;        // next crossing plane, integer-valued
  float sx, sy, sz;        // step: +1, -1 or 0
  float ox, oy, oz;        // segment start
  float vx, vy, vz;        // 1 / d
  int px, py, pz;          // byte offset of the current voxel's entry in each axis table
  int qx, qy, qz;          // byte step of those offsets: 4 * s
  float tmax;
};

__device__ __forceinline__ bool finite3(const float v[3]) {
  return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

__device__ __forceinline__ bool step_of(float s) { return s != 0.0f; }

__device__ __forceinline__ int tab_at(const int32_t *tab, int byte_off) {
  return *(const int32_t *)((const char *)tab + byte_off);
}

// Clip the segment to the map box and find the first voxel.  Table offsets
// are relative to each axis' table (x at 0, y at 4 nx, z at 4 (nx + ny)).
// Returns false if the segment visits no voxel.
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
      inv[a] = __frcp_rn(d[a]);  // correctly rounded 1 / d_a
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
  float b[3], t[3], s[3];
  int p[3], q[3];
  const int base[3] = {0, nx, nx + ny};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float pa = fadd(o[a], fmul(tmin, d[a]));
    const float hi = (float)(dims[a] - 1);
    pa = pa < 0.0f ? 0.0f : pa;
    pa = pa > hi ? hi : pa;
    const int idx = (int)floorf(pa);
    const int step = d[a] > 0.0f ? 1 : (d[a] < 0.0f ? -1 : 0);
    b[a] = (float)(idx + (step > 0));
    t[a] = step != 0 ? fmul(fsub(b[a], o[a]), inv[a]) : __int_as_float(0x7f800000);
    s[a] = (float)step;
    p[a] = 4 * (base[a] + idx);
    q[a] = 4 * step;
  }
  w.tx = t[0]; w.ty = t[1]; w.tz = t[2];
  w.bx = b[0]; w.by = b[1]; w.bz = b[2];
  w.sx = s[0]; w.sy = s[1]; w.sz = s[2];
  // An axis without a step (d_a = 0) must keep t_a = +inf when walk_advance
  // recomputes it: o_a = -inf and 1/d_a = 1 give (b_a - o_a) * 1 = +inf.
  const float ninf = -__int_as_float(0x7f800000);
  w.ox = step_of(s[0]) ? o[0] : ninf; w.oy = step_of(s[1]) ? o[1] : ninf; w.oz = step_of(s[2]) ? o[2] : ninf;
  w.vx = step_of(s[0]) ? inv[0] : 1.0f; w.vy = step_of(s[1]) ? inv[1] : 1.0f; w.vz = step_of(s[2]) ? inv[2] : 1.0f;
  w.px = p[0]; w.py = p[1]; w.pz = p[2];
  w.qx = q[0]; w.qy = q[1]; w.qz = q[2];
  w.tmax = tmax;
  return true;
}

// Voxel index of the current position on one axis.
__device__ __forceinline__ int walk_index(float b, float s) { return (int)b - (s > 0.0f ? 1 : 0); }

// One step of the walk: x if t_x <= t_y and t_x <= t_z, else y if t_y <=
// t_z, else z; false (and no change) when that crossing is not before t_max.
// Branch-free: the chosen axis' plane moves by its step (the others by 0,
// exact), all three crossing parameters are recomputed (unchanged planes
// give bit-identical values), and all three table entries are re-read.
__device__ __forceinline__ bool walk_advance(Walk &w, const int32_t *tab, int &offx, int &offy, int &offz) {
  const bool mx = (w.tx <= w.ty) & (w.tx <= w.tz);
  const bool my = !mx & (w.ty <= w.tz);
  const bool mz = !mx & !my;
  const float tsel = mx ? w.tx : (my ? w.ty : w.tz);
  if (!(tsel < w.tmax)) return false;
  w.bx = fadd(w.bx, mx ? w.sx : 0.0f);
  w.by = fadd(w.by, my ? w.sy : 0.0f);
  w.bz = fadd(w.bz, mz ? w.sz : 0.0f);
  w.tx = fmul(fsub(w.bx, w.ox), w.vx);
  w.ty = fmul(fsub(w.by, w.oy), w.vy);
  w.tz = fmul(fsub(w.bz, w.oz), w.vz);
  w.px += mx ? w.qx : 0;
  w.py += my ? w.qy : 0;
  w.pz += mz ? w.qz : 0;
  offx = tab_at(tab, w.px);
  offy = tab_at(tab, w.py);
  offz = tab_at(tab, w.pz);
  return true;
}

// Linear x-fastest layout: the element index moves by a fixed step per axis
// (+-1, +-nx, +-nx ny), so a step needs no table read.  Same walk, same
// reference operation order as walk_advance.
__device__ __forceinline__ void walk_linear_steps(Walk &w, int nx, int ny) {
  w.qx = w.sx > 0.0f ? 1 : (w.sx < 0.0f ? -1 : 0);
  w.qy = w.sy > 0.0f ? nx : (w.sy < 0.0f ? -nx : 0);
  w.qz = w.sz > 0.0f ? nx * ny : (w.sz < 0.0f ? -nx * ny : 0);
}

__device__ __forceinline__ int walk_linear_index(const Walk &w, int nx, int ny) {
  return (walk_index(w.bz, w.sz) * ny + walk_index(w.by, w.sy)) * nx + walk_index(w.bx, w.sx);
}

// One step of the walk on the linear layout, as predicated PTX: the axis
// predicates px / py / pz select the x / y / z crossing (same order and
// tie-break as walk_advance), and only the chosen axis' plane, crossing
// parameter and element index are updated, each operation rounded on its
// own.  The state advances on every call; the return value says whether the
// crossing was before t_max, i.e. whether the new voxel is part of the walk
// (callers stop at the first false and ignore the advanced state).  Because
// exactly one axis moves per call, the number of calls made while walking a
// ray equals the number of planes crossed, which ray_ig uses to count steps.
// Crossing parameters are never NaN (b - o has the sign of d and is nonzero,
// axes without a step hold +inf), so the three-input min equals the
// reference walk's selected parameter.
__device__ __forceinline__ bool walk_advance_lin(Walk &w, int &addr) {
  unsigned int end;
  asm("{\n\t"
      ".reg .pred px, py, pz, pe, pt;\n\t"
      ".reg .f32 ts, u;\n\t"
      "setp.le.f32 px, %0, %1;\n\t"          // x: t_x <= t_y and t_x <= t_z
      "setp.le.and.f32 px, %0, %2, px;\n\t"
      "setp.le.and.f32 py, %1, %2, !px;\n\t" // y: not x and t_y <= t_z
      "or.pred pt, px, py;\n\t"
      "not.pred pz, pt;\n\t"                  // z: neither
      "min.f32 ts, %0, %1, %2;\n\t"           // the chosen crossing
      "setp.geu.f32 pe, ts, %17;\n\t"         // not before t_max: the walk ends
      "selp.u32 %7, 1, 0, pe;\n\t"
      "@px add.rn.f32 %3, %3, %8;\n\t"        // b_x += s_x
      "@px sub.rn.f32 u, %3, %11;\n\t"        // t_x = (b_x - o_x) * (1 / d_x)
      "@px mul.rn.f32 %0, u, %14;\n\t"
      "@px add.s32 %6, %6, %18;\n\t"          // index += x stride
      "@py add.rn.f32 %4, %4, %9;\n\t"
      "@py sub.rn.f32 u, %4, %12;\n\t"
      "@py mul.rn.f32 %1, u, %15;\n\t"
      "@py add.s32 %6, %6, %19;\n\t"
      "@pz add.rn.f32 %5, %5, %10;\n\t"
      "@pz sub.rn.f32 u, %5, %13;\n\t"
      "@pz mul.rn.f32 %2, u, %16;\n\t"
      "@pz add.s32 %6, %6, %20;\n\t"
      "}"
      : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(addr), "=r"(end)
      : "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy), "f"(w.vz),
        "f"(w.tmax), "r"(w.qx), "r"(w.qy), "r"(w.qz));
  return end == 0u;
}

// ---------------------------------------------------------------------------
// One ray walked by a whole warp (linear layout), bit-identical to the
// sequential walk.  On axis a the k-th crossing ahead of the start has the
// parameter t_a(k) = ((b_a + k s_a) - o_a) * (1/d_a) -- the walk's own two
// rounded operations, non-decreasing in k -- and the walk takes crossings in
// (t, axis) order (ties: x, then y, then z) while t < t_max.  So the state
// after any prefix of that order is known from counts alone: with the split
// key (T, A) = the j-th crossing of axis A, axis a has taken the crossings
// with t_a(k) < T, or t_a(k) == T when a < A.  Lane l takes axis A's
// crossings [l L, (l + 1) L) and the other axes' crossings in between
// (L = the crossings of A before t_max divided among the ray's lanes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float walk_axis_t(float b, float s, float o, float v, int k) {
  return fmul(fsub(fadd(b, (float)k * s), o), v);
}

// Crossings k >= 0 of one axis that precede the key (T, A): the predicate
// "t_a(k) < T, or t_a(k) == T when tie_before" holds on a prefix of k, and
// at most `limit` crossings exist.  A real-arithmetic estimate is corrected
// by exact evaluations; a binary search takes over if it is more than a few
// crossings off.
__device__ __forceinline__ int walk_axis_count(float b, float s, float o, float v, float T, bool tie_before,
                                               int limit) {
  if (s == 0.0f) return 0;
  auto before = [&](int k) {
    const float t = walk_axis_t(b, s, o, v, k);
    return t < T || (tie_before && t == T);
  };
  const float est = fmaf(__fdividef(T, v), s, (o - b) * s);   // real k with t(k) = T
  int k = est > 0.0f ? (est < (float)limit ? (int)est : limit) : 0;
  for (int it = 0; it < 4; ++it) {
    const bool in_k = k < limit && before(k);
    const bool in_prev = k > 0 && before(k - 1);
    if (!in_k && (k == 0 || in_prev)) return k;   // first k outside the prefix
    k += in_k ? 1 : -1;
  }
  int lo = 0, hi = limit;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (before(mid))
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The walk's next crossing without taking it: axis (0 x, 1 y, 2 z) and t.
__device__ __forceinline__ int walk_next_axis(const Walk &w, float &t) {
  const bool mx = (w.tx <= w.ty) & (w.tx <= w.tz);
  const bool my = !mx & (w.ty <= w.tz);
  t = mx ? w.tx : (my ? w.ty : w.tz);
  return mx ? 0 : (my ? 1 : 2);
}

// Take crossing `axis` (linear layout): same operations as walk_advance_lin.
__device__ __forceinline__ void walk_take_lin(Walk &w, int axis, int &lin) {
  if (axis == 0) {
    w.bx = fadd(w.bx, w.sx);
    w.tx = fmul(fsub(w.bx, w.ox), w.vx);
    lin += w.qx;
  } else if (axis == 1) {
    w.by = fadd(w.by, w.sy);
    w.ty = fmul(fsub(w.by, w.oy), w.vy);
    lin += w.qy;
  } else {
    w.bz = fadd(w.bz, w.sz);
    w.tz = fmul(fsub(w.bz, w.oz), w.vz);
    lin += w.qz;
  }
}

// Set up part `lane` of n_parts of a ray whose walk w starts at linear index
// lin (walk_init + walk_linear_steps done).  On return w / lin hold the
// lane's start state and w.tmax its end; first is true for the lane that
// visits the start voxel itself; split_end tells whether the part ends at a
// split (then crossings tied with it on a lower axis still belong to it);
// axis_a is the split axis.  Returns false if the lane has nothing to walk.
__device__ __forceinline__ bool walk_lane_part(Walk &w, int &lin, int lane, int n_parts, int nx, int ny, int nz,
                                               bool &first, bool &split_end, int &axis_a) {
  const float ax = fabsf(w.vx), ay = fabsf(w.vy), az = fabsf(w.vz);   // smaller |1/d|: more crossings
  const bool sx = w.sx != 0.0f, sy = w.sy != 0.0f, sz = w.sz != 0.0f;
  int A = -1;
  float best = __int_as_float(0x7f800000);
  if (sx && ax < best) { A = 0; best = ax; }
  if (sy && ay < best) { A = 1; best = ay; }
  if (sz && az < best) { A = 2; best = az; }
  axis_a = A;
  first = lane == 0;
  split_end = false;
  if (A < 0) return lane == 0;   // no crossing at all: one voxel
  const float bA = A == 0 ? w.bx : (A == 1 ? w.by : w.bz), sA = A == 0 ? w.sx : (A == 1 ? w.sy : w.sz);
  const float oA = A == 0 ? w.ox : (A == 1 ? w.oy : w.oz), vA = A == 0 ? w.vx : (A == 1 ? w.vy : w.vz);
  const int dimA = A == 0 ? nx : (A == 1 ? ny : nz);
  const int nA = walk_axis_count(bA, sA, oA, vA, w.tmax, false, dimA + 1);   // crossings before t_max
  const int L = (nA + n_parts - 1) / n_parts;
  const int j0 = lane * L, j1 = j0 + L;
  if (lane > 0 && j0 >= nA) return false;
  if (j1 < nA) {
    w.tmax = walk_axis_t(bA, sA, oA, vA, j1);
    split_end = true;
  }
  if (lane == 0) return true;
  const float T = walk_axis_t(bA, sA, oA, vA, j0);
  const int cx = A == 0 ? j0 : walk_axis_count(w.bx, w.sx, w.ox, w.vx, T, 0 < A, nx + 1);
  const int cy = A == 1 ? j0 : walk_axis_count(w.by, w.sy, w.oy, w.vy, T, 1 < A, ny + 1);
  const int cz = A == 2 ? j0 : walk_axis_count(w.bz, w.sz, w.oz, w.vz, T, 2 < A, nz + 1);
  w.bx = fadd(w.bx, (float)cx * w.sx);
  w.by = fadd(w.by, (float)cy * w.sy);
  w.bz = fadd(w.bz, (float)cz * w.sz);
  w.tx = fmul(fsub(w.bx, w.ox), w.vx);
  w.ty = fmul(fsub(w.by, w.oy), w.vy);
  w.tz = fmul(fsub(w.bz, w.oz), w.vz);
  lin += cx * w.qx + cy * w.qy + cz * w.qz;
  return true;
}

// Host helpers (defined in nbt_map.cu).
bool valid_camera(const nbt_camera *c);     // ranges of nbt_camera (defined in nbt_raycast.cu)
bool valid_params(const nbt_ig_params *p);  // ranges of nbt_ig_params (defined in nbt_raycast.cu)
int check_map(nbt_map map);                 // NBT_EINVAL unless a live map on the current device
bool map_alive(nbt_map map, uint64_t id);   // live, and (id != 0) created with that id
void free_map(nbt_map map);                 // release a map's memory (no registry update)
int prepare_gain(nbt_map map, const nbt_ig_params *params, cudaStream_t stream);
int prepare_bsum(nbt_map map, cudaStream_t stream);  // (re)build stale brick summaries (after prepare_gain on FP32 maps)
int payload_kind(nbt_map map, const nbt_ig_params *params, PayloadKind *kind, const void **payload);
int sm_count();
int ensure_insert_scratch(nbt_map map, int64_t n_points);  // defined in nbt_insert.cu

}  // namespace nbt

#define NBT_CUDA_TRY(expr)                 \
  do {                                     \
    cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) {               \
      (void)cudaGetLastError();            \
      return NBT_ECUDA;                    \
    }                                      \
  } while (0)
