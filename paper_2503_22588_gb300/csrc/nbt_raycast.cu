// nbt_raycast.cu -- per-perspective and per-trajectory IG by voxel raycasting.
//
// Section III of the paper: for each perspective, rays from p_P to the
// endpoint grid on the far frustum plane; each ray sums g(v_i) over the
// voxels it crosses, up to and including the first occupied one (N_O); the
// ray IGs of a perspective are summed (or averaged, g_P).
//
// GPU mapping.  A work item is one (pose, 32 x 8 ray tile).  A CTA of 8
// warps takes items from a device work queue (one atomicAdd per item); each
// warp casts one 32-ray packet of the tile (packet_w x 32/packet_w pixels),
// one ray per lane, so the 256 rays a CTA walks at once start at the same
// camera and stay close, and their loads share L1 lines.  Each ray's walk is
// branch-free (see Walk), and the payload element of the next voxel is
// loaded before the current one is accumulated (the voxel sequence does not
// depend on the map, only the occlusion test does).  (Walks that skip
// uniform bricks on state maps let each warp take whole items instead, its
// 8 packets in turn.)  Per-ray sums go through a fixed warp-shuffle tree and
// a fixed 8-packet sum into one 16-byte partial per item; a second kernel
// adds the partials of each perspective
// (or trajectory) in a fixed order in FP64, so results do not depend on
// scheduling.

#include <math.h>

#include <cmath>

#include <algorithm>

#include <cuda.h>

#include "nbt_internal.cuh"

namespace nbt {

bool valid_camera(const nbt_camera *c) {
  if (!c) return false;
  if (c->width < 1 || c->height < 1 || c->width > 65535 || c->height > 65535) return false;
  const float pi = 3.14159265358979f;
  if (!(c->fov_h > 0.0f && c->fov_h < pi) || !(c->fov_v > 0.0f && c->fov_v < pi)) return false;
  if (!(c->max_range > 0.0f) || !isfinite(c->max_range)) return false;
  if (c->grid_mode != NBT_GRID_CORNERS && c->grid_mode != NBT_GRID_CENTERS) return false;
  if (c->range_mode != NBT_RANGE_PLANAR && c->range_mode != NBT_RANGE_SPHERICAL) return false;
  return true;
}

bool valid_params(const nbt_ig_params *p) {
  if (!p) return false;
  if (p->metric != NBT_COUNT_UNKNOWN && p->metric != NBT_PAPER_EQ2 && p->metric != NBT_ENTROPY) return false;
  if (p->reduce != NBT_REDUCE_SUM && p->reduce != NBT_REDUCE_MEAN) return false;
  if (!isfinite(p->occ_threshold) || !isfinite(p->free_threshold)) return false;
  return true;
}

namespace {

// Section III endpoint grid: d_h = d_Cam tan(FoV_h / 2), d_v likewise, in
// FP64 on the host; the grid start and spacing are each rounded once to FP32.
CamConst make_cam(nbt_map map, const nbt_camera *c) {
  CamConst cc;
  const double dh = (double)c->max_range * tan((double)c->fov_h * 0.5);
  const double dv = (double)c->max_range * tan((double)c->fov_v * 0.5);
  const int w = c->width, h = c->height;
  if (c->grid_mode == NBT_GRID_CORNERS) {
    cc.x0 = w > 1 ? (float)(-dh) : 0.0f;
    cc.xstep = w > 1 ? (float)(2.0 * dh / (double)(w - 1)) : 0.0f;
    cc.y0 = h > 1 ? (float)(-dv) : 0.0f;
    cc.ystep = h > 1 ? (float)(2.0 * dv / (double)(h - 1)) : 0.0f;
  } else {
    cc.x0 = (float)(-dh + dh / (double)w);
    cc.xstep = (float)(2.0 * dh / (double)w);
    cc.y0 = (float)(-dv + dv / (double)h);
    cc.ystep = (float)(2.0 * dv / (double)h);
  }
  cc.zc = c->max_range;
  cc.spherical = c->range_mode == NBT_RANGE_SPHERICAL;
  cc.W = w;
  cc.H = h;
  cc.tiles_x = (w + kTileW - 1) / kTileW;
  cc.tiles_per_pose = cc.tiles_x * ((h + kTileH - 1) / kTileH);
  cc.packet_w = map->packet_w;
  cc.inv_s = (float)(1.0 / (double)map->desc.voxel_size);
  cc.ox = map->desc.origin[0];
  cc.oy = map->desc.origin[1];
  cc.oz = map->desc.origin[2];
  return cc;
}

DevMap dev_map(nbt_map map, const void *payload) {
  DevMap m;
  m.payload = payload;
  m.tab = map->d_tab;
  m.nx = map->desc.nx;
  m.ny = map->desc.ny;
  m.nz = map->desc.nz;
  m.bsum = map->d_bsum;
  for (int l = 0; l < kSkipLevels; ++l) {
    m.bsx[l] = map->bsx[l];
    m.bsy[l] = map->bsy[l];
    m.boff[l] = (int)map->boff[l];
  }
  return m;
}

int64_t workspace_bytes_for(int64_t n_items) { return 256 + n_items * (int64_t)kPartialBytes; }

// Voxel payload read: gain magnitude, unknown indicator, occupied flag.
template <int KIND>
__device__ __forceinline__ void read_voxel(const void *payload, uint32_t off, float &g, uint32_t &unk, bool &occ) {
  if (KIND == PAYLOAD_GAIN_F32) {
    const float v = __ldg((const float *)payload + off);
    occ = (__float_as_uint(v) >> 31) != 0u;
    g = fabsf(v);
    unk = 0u;
  } else if (KIND == PAYLOAD_U8) {
    const uint32_t s = __ldg((const uint8_t *)payload + off);
    occ = s >= 2u;
    unk = s == 0u;
    g = 0.0f;
  } else {
    const uint32_t b = __ldg((const uint8_t *)payload + (off >> 2));
    const uint32_t s = (b >> ((off & 3u) << 1)) & 3u;
    occ = s >= 2u;
    unk = s == 0u;
    g = 0.0f;
  }
}

template <int KIND>
__device__ __forceinline__ uint32_t raw_load(const void *payload, uint32_t off) {
  if (KIND == PAYLOAD_GAIN_F32) return __float_as_uint(__ldg((const float *)payload + off));
  if (KIND == PAYLOAD_U8) return __ldg((const uint8_t *)payload + off);
  return __ldg((const uint8_t *)payload + (off >> 2));
}

// FP32-gain walk on the linear layout as one PTX loop (three voxels per
// pass, registers r0 / r1 / r2 rotating as current and prefetched voxel).  Per voxel:
// the walk_advance_lin step (same selection, same rounded operations; the
// axis is the first of x, y, z whose crossing equals the three-input min,
// which is walk_advance's tie-break since crossings are never NaN), the
// read of the next voxel unless the walk ends there (that read does not wait
// for the current voxel's value), then the current voxel's gain.  The walk
// stops when the chosen crossing is not before t_max or the current voxel is
// occupied (sign bit of its gain entry).
// Gains are added in visit order, one rounding each, as in ray_ig; the walk
// state advances once per visited voxel, so the plane travel counts them.
__constant__ int c_unit = 1;

template <bool HIT>
__device__ __forceinline__ void walk_gain_f32(Walk &w, int &lin, uint32_t raw, const float *payload,
                                              uint32_t addr_max, float &facc) {
#define NBT_WALK_PART                                                                            \
  "min.f32 ts, %0, %1, %2;\n\t"                                                                 \
  "setp.geu.f32 pm, ts, %18;\n\t"                                                               \
  "setp.eq.f32 px, %0, ts;\n\t"                                                                 \
  "setp.eq.and.f32 py, %1, ts, !px;\n\t"                                                        \
  "setp.neu.and.f32 pz, %1, ts, !px;\n\t"                                                       \
  "@px add.rn.f32 %3, %3, %9;\n\t"                                                              \
  "@px sub.rn.f32 u, %3, %12;\n\t"                                                              \
  "@px mul.rn.f32 %0, u, %15;\n\t"                                                              \
  "@px mad.lo.s32 %6, %19, %24, %6;\n\t"                                                        \
  "@py add.rn.f32 %4, %4, %10;\n\t"                                                             \
  "@py sub.rn.f32 u, %4, %13;\n\t"                                                              \
  "@py mul.rn.f32 %1, u, %16;\n\t"                                                              \
  "@py mad.lo.s32 %6, %20, %24, %6;\n\t"                                                        \
  "@pz add.rn.f32 %5, %5, %11;\n\t"                                                             \
  "@pz sub.rn.f32 u, %5, %14;\n\t"                                                              \
  "@pz mul.rn.f32 %2, u, %17;\n\t"                                                              \
  "@pz mad.lo.s32 %6, %21, %24, %6;\n\t"                                                        \
  "min.u32 lc, %6, %23;\n\t"
#define NBT_GAIN_BODY(CUR, NXT)                                                                  \
  NBT_WALK_PART                                                                                  \
  "mad.wide.u32 a, lc, 4, %22;\n\t"                                                             \
  "@!pm ld.global.nc.b32 " NXT ", [a];\n\t"                                                     \
  "abs.f32 g, " CUR ";\n\t"
#define NBT_GAIN_HIT(CUR)                                                                        \
  "setp.lt.or.s32 pe, " CUR ", 0, pm;\n\t"                                                      \
  "add.rn.f32 %7, %7, g;\n\t"
#define NBT_GAIN_MISS(CUR)                                                                       \
  "setp.lt.s32 po, " CUR ", 0;\n\t"                                                             \
  "or.pred pe, pm, po;\n\t"                                                                     \
  "@!po add.rn.f32 %7, %7, g;\n\t"
// Three voxels per pass (registers r0 -> r1 -> r2 -> r0): measured 2.4 %
// faster than two and 1.5 % faster than four on the 256^3 probability map.
#define NBT_GAIN_LOOP(END)                                                                       \
  "LOOP:\n\t" NBT_GAIN_BODY("r0", "r1") END("r0") "@pe bra DONE;\n\t"                          \
  NBT_GAIN_BODY("r1", "r2") END("r1") "@pe bra DONE;\n\t"                                       \
  NBT_GAIN_BODY("r2", "r0") END("r2") "@!pe bra LOOP;\n\t"                                      \
  "DONE:\n\t"
  // The index steps are multiply-adds by a unit read from constant memory
  // (opaque to the compiler), so they run on the FMA pipe next to the
  // float work instead of adding to the compare/select ALU pipe.
  const int unit = c_unit;
  if (HIT) {
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, pe;\n\t"
        ".reg .f32 ts, u, g;\n\t"
        ".reg .b32 r0, r1, r2, lc;\n\t"
        ".reg .b64 a;\n\t"
        "mov.b32 r0, %8;\n\t" NBT_GAIN_LOOP(NBT_GAIN_HIT) "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+f"(facc)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(w.tmax), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, po, pe;\n\t"
        ".reg .f32 ts, u, g;\n\t"
        ".reg .b32 r0, r1, r2, lc;\n\t"
        ".reg .b64 a;\n\t"
        "mov.b32 r0, %8;\n\t" NBT_GAIN_LOOP(NBT_GAIN_MISS) "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+f"(facc)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(w.tmax), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit)
        : "memory");
  }
#undef NBT_GAIN_LOOP
#undef NBT_GAIN_HIT
#undef NBT_GAIN_MISS
#undef NBT_GAIN_BODY
}

// Count IG on 1-byte and 2-bit state maps (linear layout): the same PTX walk
// as walk_gain_f32 (same selection, operations, clamp and three-voxel pass);
// per voxel the unknown count grows by one for state 0 and the walk stops
// after an occupied voxel (state >= 2).  2-bit states: four voxels per byte,
// voxel v in bits 2 (v & 3) of byte v / 4; the byte is replicated into all
// four byte lanes of a word (multiply by 0x01010101) so that a funnel shift
// by 2 v (taken mod 32) brings bits 2 (v & 3) of one copy to bit 0.  The
// +1 of the count and the 2 v are multiply-adds by opaque units, like the
// index steps.
template <int KIND>
__device__ __forceinline__ void walk_count(Walk &w, int &lin, uint32_t raw, uint32_t addr, const uint8_t *payload,
                                           uint32_t addr_max, uint32_t &iacc) {
  const int unit = c_unit, two = unit + unit;
  if constexpr (KIND == PAYLOAD_U8) {
#define NBT_U8_BODY(CUR, NXT)                                                                    \
  NBT_WALK_PART                                                                                  \
  "mad.wide.u32 a, lc, %24, %22;\n\t"                                                           \
  "@!pm ld.global.nc.u8 " NXT ", [a];\n\t"                                                      \
  "setp.eq.u32 pu, " CUR ", 0;\n\t"                                                             \
  "@pu mad.lo.s32 %7, %24, %24, %7;\n\t"                                                        \
  "setp.gt.or.u32 pe, " CUR ", 1, pm;\n\t"
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, pu, pe;\n\t"
        ".reg .f32 ts, u;\n\t"
        ".reg .b32 r0, r1, r2, lc;\n\t"
        ".reg .b64 a;\n\t"
        "mov.b32 r0, %8;\n\t"
        "LOOP:\n\t" NBT_U8_BODY("r0", "r1") "@pe bra DONE;\n\t"
        NBT_U8_BODY("r1", "r2") "@pe bra DONE;\n\t"
        NBT_U8_BODY("r2", "r0") "@!pe bra LOOP;\n\t"
        "DONE:\n\t"
        "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+r"(iacc)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(w.tmax), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit)
        : "memory");
#undef NBT_U8_BODY
  } else {
#define NBT_U2_BODY(CUR, SC, NXT, SN)                                                            \
  NBT_WALK_PART                                                                                  \
  "shr.u32 wb, lc, 2;\n\t"                                                                       \
  "mad.wide.u32 a, wb, %24, %22;\n\t"                                                           \
  "@!pm ld.global.nc.u8 " NXT ", [a];\n\t"                                                      \
  "mad.lo.s32 " SN ", lc, %25, 0;\n\t"                                                          \
  "mul.lo.u32 st, " CUR ", 16843009;\n\t"                                                       \
  "shf.r.wrap.b32 st, st, st, " SC ";\n\t"                                                      \
  "and.b32 st, st, 3;\n\t"                                                                      \
  "setp.eq.u32 pu, st, 0;\n\t"                                                                  \
  "@pu mad.lo.s32 %7, %24, %24, %7;\n\t"                                                        \
  "setp.gt.or.u32 pe, st, 1, pm;\n\t"
    const uint32_t s_first = addr * 2u;
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, pu, pe;\n\t"
        ".reg .f32 ts, u;\n\t"
        ".reg .b32 r0, r1, r2, s0, s1, s2, lc, wb, st;\n\t"
        ".reg .b64 a;\n\t"
        "mov.b32 r0, %8;\n\t"
        "mov.b32 s0, %26;\n\t"
        "LOOP:\n\t" NBT_U2_BODY("r0", "s0", "r1", "s1") "@pe bra DONE;\n\t"
        NBT_U2_BODY("r1", "s1", "r2", "s2") "@pe bra DONE;\n\t"
        NBT_U2_BODY("r2", "s2", "r0", "s0") "@!pe bra LOOP;\n\t"
        "DONE:\n\t"
        "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+r"(iacc)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(w.tmax), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit),
          "r"(two), "r"(s_first)
        : "memory");
#undef NBT_U2_BODY
  }
}
#undef NBT_WALK_PART

// ---------------------------------------------------------------------------
// Count walks that skip uniform bricks (linear 1-byte and 2-bit state maps).
//
// The walk takes plane crossings in (t, axis) order, and on each axis the
// crossing parameters t_a(k) = ((b_a + k s_a) - o_a) (1/d_a), each operation
// rounded, do not decrease with k.  So the state after every crossing that
// comes before a key (T, A) is known from per-axis counts alone: axis a has
// taken the crossings with t_a(k) < T, or t_a(k) == T when a < A (the x-y-z
// tie-break).  Inside a brick whose voxels are all unknown or all free (brick
// summary), nothing depends on the voxels' values, so the walk through it is
// replaced by those counts: with (T, A) the first crossing of the brick's
// boundary (or t_max if the walk ends inside), the brick contributes
// 1 + sum_a c_a visited voxels (each crossing enters one new voxel), all
// unknown or none, and the walk continues from the state after them -- the
// same voxels, the same counts and the same final state as stepping voxel
// by voxel.  A warp takes such a macro step only when all its active lanes
// sit in uniform bricks; otherwise every lane walks voxel by voxel (the PTX
// loop of walk_count, with the brick exit as an extra limit) up to the exit
// of its current brick, so the lanes stay converged.
// ---------------------------------------------------------------------------

// One axis of a jump to the key: its crossings k before the key, t(k) < T,
// or t(k) == T when tie, with t(k) = ((b + k s) - o) (1/d), the walk's own
// rounded operations (the answer lies in [0, kin], kin = the axis' planes
// inside the brick); the exit axis takes all kin of them and then the exit
// plane itself.  The plane b and its crossing t move past the crossings
// taken, as kin single steps would move them.  A real-arithmetic estimate
// from the current crossing t and |d| is checked by two exact evaluations --
// one of them the new crossing itself -- (the predicate is monotone in k)
// and corrected step by step when they fail, so the result never depends on
// the estimate.  Returns the crossings before the key (kin on the exit axis).
__device__ __forceinline__ int skip_axis_jump(float &b, float s, float o, float v, float ad, float &t, float T,
                                              int kin, bool exit, bool tie) {
  auto before = [&](float tk) { return tk < T || (tie && tk == T); };
  int c = kin;
  if (!exit) {
    const float e = ceilf((T - t) * ad);
    c = e > 0.0f ? (e < (float)kin ? (int)e : kin) : 0;
  }
  float bn = fadd(b, (float)(c + (int)exit) * s);
  float tn = fmul(fsub(bn, o), v);
  if (!exit) {
    const float tp = fmul(fsub(fsub(bn, s), o), v);   // t(c - 1): b + (c - 1) s is exact
    if (!((c == 0 || before(tp)) && (c == kin || !before(tn)))) {
      auto tk = [&](int k) { return fmul(fsub(fadd(b, (float)k * s), o), v); };
      while (c > 0 && !before(tk(c - 1))) --c;
      while (c < kin && before(tk(c))) ++c;
      bn = fadd(b, (float)c * s);
      tn = fmul(fsub(bn, o), v);
    }
  }
  b = bn;
  t = tn;
  return c;
}

// The walk_count loop from the current voxel (payload entry raw, already
// loaded: the state byte on 1-byte maps, the 32-bit word holding its 2-bit
// state on 2-bit maps) for at most `passes` passes of three voxels, up to the
// first occupied voxel or the first crossing not before tlim.  The walk state
// ends one crossing past the last visited voxel (so the plane travel is the
// number visited); sacc = the sum of the visited voxels' states (every
// visited voxel but the last is unknown, 0, or free, 1, so the caller gets
// the unknown count from it, the visited count and the last state with one
// add per voxel instead of a test and a conditional add); last = state of the
// last visited voxel, ts_out = the crossing the loop stopped on (before tlim
// if it stopped on the pass count).  2-bit maps are read a 32-bit word (16
// voxels) at a time: the state of element e is bits 2 (e mod 16) of word
// e / 16, one funnel shift away.
template <int KIND>
__device__ __forceinline__ void walk_count_run(Walk &w, int &lin, uint32_t raw, uint32_t addr, const uint8_t *payload,
                                               uint32_t addr_max, float tlim, int passes, uint32_t &sacc,
                                               uint32_t &last, float &ts_out) {
#define NBT_RUN_PART                                                                             \
  "min.f32 ts, %0, %1, %2;\n\t"                                                                 \
  "setp.geu.f32 pm, ts, %20;\n\t"                                                               \
  "setp.eq.f32 px, %0, ts;\n\t"                                                                 \
  "setp.eq.and.f32 py, %1, ts, !px;\n\t"                                                        \
  "setp.neu.and.f32 pz, %1, ts, !px;\n\t"                                                       \
  "@px add.rn.f32 %3, %3, %11;\n\t"                                                             \
  "@px sub.rn.f32 u, %3, %14;\n\t"                                                              \
  "@px mul.rn.f32 %0, u, %17;\n\t"                                                              \
  "@px mad.lo.s32 %6, %21, %26, %6;\n\t"                                                        \
  "@py add.rn.f32 %4, %4, %12;\n\t"                                                             \
  "@py sub.rn.f32 u, %4, %15;\n\t"                                                              \
  "@py mul.rn.f32 %1, u, %18;\n\t"                                                              \
  "@py mad.lo.s32 %6, %22, %26, %6;\n\t"                                                        \
  "@pz add.rn.f32 %5, %5, %13;\n\t"                                                             \
  "@pz sub.rn.f32 u, %5, %16;\n\t"                                                              \
  "@pz mul.rn.f32 %2, u, %19;\n\t"                                                              \
  "@pz mad.lo.s32 %6, %23, %26, %6;\n\t"                                                        \
  "min.u32 lc, %6, %25;\n\t"
  const int unit = c_unit, two = unit + unit;
  if constexpr (KIND == PAYLOAD_U8) {
#define NBT_U8_RUN(CUR, NXT)                                                                     \
  NBT_RUN_PART                                                                                   \
  "mad.wide.u32 a, lc, %26, %24;\n\t"                                                           \
  "@!pm ld.global.nc.u8 " NXT ", [a];\n\t"                                                      \
  "add.u32 %7, %7, " CUR ";\n\t"                                                                \
  "setp.gt.or.u32 pe, " CUR ", 1, pm;\n\t"
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, pe, pc;\n\t"
        ".reg .f32 ts, u;\n\t"
        ".reg .b32 r0, r1, r2, lc, cnt;\n\t"
        ".reg .b64 a;\n\t"
        "mov.b32 r0, %10;\n\t"
        "mov.b32 cnt, %27;\n\t"
        "LOOP:\n\t" NBT_U8_RUN("r0", "r1") "@pe bra D0;\n\t"
        NBT_U8_RUN("r1", "r2") "@pe bra D1;\n\t"
        NBT_U8_RUN("r2", "r0")
        "sub.s32 cnt, cnt, 1;\n\t"
        "setp.ne.and.s32 pc, cnt, 0, !pe;\n\t"
        "@pc bra LOOP;\n\t"
        "mov.b32 %8, r2;\n\t"
        "bra DONE;\n\t"
        "D0:\n\t"
        "mov.b32 %8, r0;\n\t"
        "bra DONE;\n\t"
        "D1:\n\t"
        "mov.b32 %8, r1;\n\t"
        "DONE:\n\t"
        "mov.f32 %9, ts;\n\t"
        "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+r"(sacc),
          "=r"(last), "=f"(ts_out)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(tlim), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit),
          "r"(passes)
        : "memory");
#undef NBT_U8_RUN
  } else {
#define NBT_U2_RUN(CUR, SC, NXT, SN)                                                             \
  NBT_RUN_PART                                                                                   \
  "shr.u32 wb, lc, 4;\n\t"                                                                       \
  "mad.wide.u32 a, wb, 4, %24;\n\t"                                                             \
  "@!pm ld.global.nc.b32 " NXT ", [a];\n\t"                                                     \
  "mad.lo.s32 " SN ", lc, %27, 0;\n\t"                                                          \
  "shf.r.wrap.b32 st, " CUR ", " CUR ", " SC ";\n\t"                                            \
  "and.b32 st, st, 3;\n\t"                                                                      \
  "add.u32 %7, %7, st;\n\t"                                                                     \
  "setp.gt.or.u32 pe, st, 1, pm;\n\t"
    const uint32_t s_first = addr * 2u;
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, pe, pc;\n\t"
        ".reg .f32 ts, u;\n\t"
        ".reg .b32 r0, r1, r2, s0, s1, s2, lc, wb, st, cnt;\n\t"
        ".reg .b64 a;\n\t"
        "mov.b32 r0, %10;\n\t"
        "mov.b32 s0, %28;\n\t"
        "mov.b32 cnt, %29;\n\t"
        "LOOP:\n\t" NBT_U2_RUN("r0", "s0", "r1", "s1") "@pe bra DONE;\n\t"
        NBT_U2_RUN("r1", "s1", "r2", "s2") "@pe bra DONE;\n\t"
        NBT_U2_RUN("r2", "s2", "r0", "s0")
        "sub.s32 cnt, cnt, 1;\n\t"
        "setp.ne.and.s32 pc, cnt, 0, !pe;\n\t"
        "@pc bra LOOP;\n\t"
        "DONE:\n\t"
        "mov.b32 %8, st;\n\t"
        "mov.f32 %9, ts;\n\t"
        "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+r"(sacc),
          "=r"(last), "=f"(ts_out)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(tlim), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit),
          "r"(two), "r"(s_first), "r"(passes)
        : "memory");
#undef NBT_U2_RUN
  }
#undef NBT_RUN_PART
}

// The walk_gain_f32 loop (FP32 signed gains) from the current voxel, for at
// most `passes` passes of three voxels, up to the first occupied voxel or the
// first crossing not before tlim; outputs as walk_count_run (last = the raw
// gain entry of the last visited voxel: negative when occupied).
template <bool HIT>
__device__ __forceinline__ void walk_gain_run(Walk &w, int &lin, uint32_t raw, const float *payload,
                                              uint32_t addr_max, float tlim, int passes, float &facc, uint32_t &last,
                                              float &ts_out) {
#define NBT_GRUN_PART                                                                            \
  "min.f32 ts, %0, %1, %2;\n\t"                                                                 \
  "setp.geu.f32 pm, ts, %20;\n\t"                                                               \
  "setp.eq.f32 px, %0, ts;\n\t"                                                                 \
  "setp.eq.and.f32 py, %1, ts, !px;\n\t"                                                        \
  "setp.neu.and.f32 pz, %1, ts, !px;\n\t"                                                       \
  "@px add.rn.f32 %3, %3, %11;\n\t"                                                             \
  "@px sub.rn.f32 u, %3, %14;\n\t"                                                              \
  "@px mul.rn.f32 %0, u, %17;\n\t"                                                              \
  "@px mad.lo.s32 %6, %21, %26, %6;\n\t"                                                        \
  "@py add.rn.f32 %4, %4, %12;\n\t"                                                             \
  "@py sub.rn.f32 u, %4, %15;\n\t"                                                              \
  "@py mul.rn.f32 %1, u, %18;\n\t"                                                              \
  "@py mad.lo.s32 %6, %22, %26, %6;\n\t"                                                        \
  "@pz add.rn.f32 %5, %5, %13;\n\t"                                                             \
  "@pz sub.rn.f32 u, %5, %16;\n\t"                                                              \
  "@pz mul.rn.f32 %2, u, %19;\n\t"                                                              \
  "@pz mad.lo.s32 %6, %23, %26, %6;\n\t"                                                        \
  "min.u32 lc, %6, %25;\n\t"                                                                    \
  "mad.wide.u32 a, lc, 4, %24;\n\t"
#define NBT_GRUN_HIT(CUR, NXT)                                                                   \
  NBT_GRUN_PART                                                                                  \
  "@!pm ld.global.nc.b32 " NXT ", [a];\n\t"                                                     \
  "abs.f32 g, " CUR ";\n\t"                                                                     \
  "setp.lt.or.s32 pe, " CUR ", 0, pm;\n\t"                                                      \
  "add.rn.f32 %7, %7, g;\n\t"
#define NBT_GRUN_MISS(CUR, NXT)                                                                  \
  NBT_GRUN_PART                                                                                  \
  "@!pm ld.global.nc.b32 " NXT ", [a];\n\t"                                                     \
  "abs.f32 g, " CUR ";\n\t"                                                                     \
  "setp.lt.s32 po, " CUR ", 0;\n\t"                                                             \
  "or.pred pe, pm, po;\n\t"                                                                     \
  "@!po add.rn.f32 %7, %7, g;\n\t"
#define NBT_GRUN_LOOP(BODY)                                                                      \
  "mov.b32 r0, %10;\n\t"                                                                        \
  "mov.b32 cnt, %27;\n\t"                                                                       \
  "LOOP:\n\t" BODY("r0", "r1") "@pe bra D0;\n\t" BODY("r1", "r2") "@pe bra D1;\n\t"             \
  BODY("r2", "r0")                                                                               \
  "sub.s32 cnt, cnt, 1;\n\t"                                                                    \
  "setp.ne.and.s32 pc, cnt, 0, !pe;\n\t"                                                        \
  "@pc bra LOOP;\n\t"                                                                           \
  "mov.b32 %8, r2;\n\t"                                                                         \
  "bra DONE;\n\t"                                                                               \
  "D0:\n\t"                                                                                     \
  "mov.b32 %8, r0;\n\t"                                                                         \
  "bra DONE;\n\t"                                                                               \
  "D1:\n\t"                                                                                     \
  "mov.b32 %8, r1;\n\t"                                                                         \
  "DONE:\n\t"                                                                                   \
  "mov.f32 %9, ts;\n\t"
  const int unit = c_unit;
  if (HIT) {
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, pe, pc;\n\t"
        ".reg .f32 ts, u, g;\n\t"
        ".reg .b32 r0, r1, r2, lc, cnt;\n\t"
        ".reg .b64 a;\n\t" NBT_GRUN_LOOP(NBT_GRUN_HIT) "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+f"(facc),
          "=r"(last), "=f"(ts_out)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(tlim), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit),
          "r"(passes)
        : "memory");
  } else {
    asm volatile(
        "{\n\t"
        ".reg .pred px, py, pz, pm, po, pe, pc;\n\t"
        ".reg .f32 ts, u, g;\n\t"
        ".reg .b32 r0, r1, r2, lc, cnt;\n\t"
        ".reg .b64 a;\n\t" NBT_GRUN_LOOP(NBT_GRUN_MISS) "}"
        : "+f"(w.tx), "+f"(w.ty), "+f"(w.tz), "+f"(w.bx), "+f"(w.by), "+f"(w.bz), "+r"(lin), "+f"(facc),
          "=r"(last), "=f"(ts_out)
        : "r"(raw), "f"(w.sx), "f"(w.sy), "f"(w.sz), "f"(w.ox), "f"(w.oy), "f"(w.oz), "f"(w.vx), "f"(w.vy),
          "f"(w.vz), "f"(tlim), "r"(w.qx), "r"(w.qy), "r"(w.qz), "l"(payload), "r"(addr_max), "r"(unit),
          "r"(passes)
        : "memory");
  }
#undef NBT_GRUN_LOOP
#undef NBT_GRUN_MISS
#undef NBT_GRUN_HIT
#undef NBT_GRUN_PART
}

#ifndef NBT_RUN_PASSES
#define NBT_RUN_PASSES 8
#endif
#ifndef NBT_SKIP_LOOKUP_LEVELS
#define NBT_SKIP_LOOKUP_LEVELS kSkipLevels
#endif
constexpr int kRunPasses = NBT_RUN_PASSES;               // voxel-by-voxel stretch between two votes (passes of 3)
constexpr int kLookupLevels = NBT_SKIP_LOOKUP_LEVELS;    // pyramid levels a lane consults (bricks 8 .. 2^(2+L))

// IG and visited voxels of one ray on a linear map, skipping uniform bricks
// (see above): unknown counts on state maps (KIND U8 / U2, into iacc), or FP32
// gains (KIND GAIN_F32, into facc: a uniform brick's voxels all have gain
// exactly 1 or 0, so the brick adds its visited count or nothing).  Each lane looks up the largest uniform brick of
// the summary pyramid (8 to 64 voxels) around its current voxel; when every
// active lane of the warp has one, each replaces the walk through it by the
// per-axis counts up to the brick's exit.  Called by all 32 lanes of a warp
// together (valid = the lane has a ray); per-ray results equal ray_ig's.
template <int KIND, bool HIT>
__device__ __forceinline__ void ray_skip(const DevMap &m, uint32_t addr_max, const float o[3], const float d[3],
                                         bool valid, float &facc, uint32_t &iacc, uint32_t &steps) {
  Walk w;
  bool done = !valid || !walk_init(w, o, d, m.nx, m.ny, m.nz);
  int lin = 0;
  float adx = 0.0f, ady = 0.0f, adz = 0.0f;
  int upx = 0, upy = 0, upz = 0;            // [s_a > 0]: the current voxel is b_a - up_a
  if (!done) {
    walk_linear_steps(w, m.nx, m.ny);
    lin = walk_linear_index(w, m.nx, m.ny);
    adx = fabsf(d[0]);
    ady = fabsf(d[1]);
    adz = fabsf(d[2]);
    upx = w.sx > 0.0f;
    upy = w.sy > 0.0f;
    upz = w.sz > 0.0f;
  }
  const uint8_t *payload = (const uint8_t *)m.payload;
  while (__any_sync(0xffffffffu, !done)) {
    int ix = 0, iy = 0, iz = 0, lvl = -1;
    uint32_t cls = kSumOther;
    if (!done) {
      ix = (int)w.bx - upx;
      iy = (int)w.by - upy;
      iz = (int)w.bz - upz;
      // the largest uniform brick around the voxel: its level-0 byte holds class | (level << 2)
      const uint32_t v = __ldg(m.bsum + ((int64_t)(iz >> kSkipLog) * m.bsy[0] + (iy >> kSkipLog)) * m.bsx[0] +
                               (ix >> kSkipLog));
      cls = v & 3u;
      if (cls <= kSumFree) lvl = min((int)(v >> 2), kLookupLevels - 1);
    }
    const bool macro = __all_sync(0xffffffffu, done || lvl >= 0);
    if (done) continue;
    if (macro) {
      // exit planes of the uniform brick and their crossings
      const int sh = kSkipLog + lvl;
      const float ex = (float)(((ix >> sh) + upx) << sh), ey = (float)(((iy >> sh) + upy) << sh),
                  ez = (float)(((iz >> sh) + upz) << sh);
      const float tex = fmul(fsub(ex, w.ox), w.vx);    // +inf on an axis without a step
      const float tey = fmul(fsub(ey, w.oy), w.vy);
      const float tez = fmul(fsub(ez, w.oz), w.vz);
      const float T = fminf(tex, fminf(tey, tez));
      const bool end = !(T < w.tmax);                   // the walk ends inside this brick
      const float key = end ? w.tmax : T;
      const int A = end ? 3 : (tex == T ? 0 : (tey == T ? 1 : 2));  // exit axis (x-y-z tie-break)
      // crossings of each axis inside the brick; the exit axis takes exactly those
      const int kx = w.sx != 0.0f ? (int)fabsf(ex - w.bx) : 0;
      const int ky = w.sy != 0.0f ? (int)fabsf(ey - w.by) : 0;
      const int kz = w.sz != 0.0f ? (int)fabsf(ez - w.bz) : 0;
      const int cx = skip_axis_jump(w.bx, w.sx, w.ox, w.vx, adx, w.tx, key, kx, A == 0, 0 < A && !end);
      const int cy = skip_axis_jump(w.by, w.sy, w.oy, w.vy, ady, w.ty, key, ky, A == 1, 1 < A && !end);
      const int cz = skip_axis_jump(w.bz, w.sz, w.oz, w.vz, adz, w.tz, key, kz, A == 2, 2 < A && !end);
      const uint32_t nvis = 1u + (uint32_t)(cx + cy + cz);
      steps += nvis;
      if (cls == kSumUnknown) {
        if constexpr (KIND == PAYLOAD_GAIN_F32)
          facc = fadd(facc, (float)nvis);       // nvis voxels of gain exactly 1
        else
          iacc += nvis;
      }
      // the walk state now sits past those crossings and, unless the walk ends, the exit crossing (T, A)
      const int mx = cx + (A == 0), my = cy + (A == 1), mz = cz + (A == 2);
      lin += mx * w.qx + my * w.qy + mz * w.qz;
      done = end;
    } else {
      // every lane walks the same number of voxels (kRunPasses passes of three) before the next
      // vote, so the lanes stay in step
      const float bx0 = w.bx, by0 = w.by, bz0 = w.bz;
      const uint32_t addr = min((uint32_t)lin, addr_max);
      // the first voxel's payload entry (2-bit maps: the 32-bit word holding it)
      const uint32_t raw = KIND == PAYLOAD_U2 ? __ldg((const uint32_t *)payload + (addr >> 4))
                                             : raw_load<KIND>(payload, addr);
      uint32_t last = 0u;
      float ts = 0.0f;
      bool occ;
      uint32_t sacc = 0u;
      if constexpr (KIND == PAYLOAD_GAIN_F32) {
        walk_gain_run<HIT>(w, lin, raw, (const float *)m.payload, addr_max, w.tmax, kRunPasses, facc, last, ts);
        occ = (int32_t)last < 0;                     // sign bit: occupied
      } else {
        walk_count_run<KIND>(w, lin, raw, addr, payload, addr_max, w.tmax, kRunPasses, sacc, last, ts);
        occ = last >= 2u;
      }
      const uint32_t nvis = (uint32_t)(fabsf(w.bx - bx0) + fabsf(w.by - by0) + fabsf(w.bz - bz0));
      steps += nvis;
      // every visited voxel but the last has state 0 (unknown) or 1 (free)
      if constexpr (KIND != PAYLOAD_GAIN_F32) iacc += nvis - 1u - (sacc - last) + (last == 0u ? 1u : 0u);
      done = occ || !(ts < w.tmax);                  // occluded, or the walk's end reached
    }
  }
}

// IG of one ray: walk, read, accumulate, stop after the first occupied voxel.
// HIT: the occupied voxel adds its gain (the Section III sum runs to N_O).
// LINEAR: linear layout with stride steps; else bricked with table reads.
// Every payload read uses min(index, addr_max), a safety net that keeps
// reads inside the payload (the walk itself never leaves the map).
template <int KIND, bool HIT, bool LINEAR>
__device__ __forceinline__ void ray_ig(const void *payload, const int32_t *tab, uint32_t addr_max, int nx, int ny,
                                       int nz, const float o[3], const float d[3], float &facc, uint32_t &iacc,
                                       uint32_t &steps) {
  Walk w;
  if (!walk_init(w, o, d, nx, ny, nz)) return;
  int offx = 0, offy = 0, offz = 0, lin = 0;
  if (LINEAR) {
    walk_linear_steps(w, nx, ny);
    lin = walk_linear_index(w, nx, ny);
  } else {
    offx = tab_at(tab, w.px);
    offy = tab_at(tab, w.py);
    offz = tab_at(tab, w.pz);
  }
  uint32_t addr = min(LINEAR ? (uint32_t)lin : (uint32_t)(offx + offy + offz), addr_max);
  uint32_t raw = raw_load<KIND>(payload, addr);
  const float bx0 = w.bx, by0 = w.by, bz0 = w.bz;
  if constexpr (LINEAR) {
    if constexpr (KIND == PAYLOAD_GAIN_F32)
      walk_gain_f32<HIT>(w, lin, raw, (const float *)payload, addr_max, facc);
    else
      walk_count<KIND>(w, lin, raw, addr, (const uint8_t *)payload, addr_max, iacc);
    // one walk step per visited voxel, each moving one plane by one: the
    // visited count is the plane travel (exact integer-valued floats)
    steps += (uint32_t)(fabsf(w.bx - bx0) + fabsf(w.by - by0) + fabsf(w.bz - bz0));
  } else {
    // Bricked layouts: three voxels per iteration for FP32 gains (fewer
    // register moves and back-edges); the 1-byte and 2-bit payloads measured
    // no gain from it.
#pragma unroll(KIND == PAYLOAD_GAIN_F32 ? 3 : 1)
    for (;;) {
      const bool more = walk_advance(w, tab, offx, offy, offz);
      steps += 1u;
      const uint32_t naddr = min((uint32_t)(offx + offy + offz), addr_max);
      const uint32_t nraw = more ? raw_load<KIND>(payload, naddr) : 0u;
      bool occ;
      if (KIND == PAYLOAD_GAIN_F32) {
        occ = (int32_t)raw < 0;
        const float g = fabsf(__uint_as_float(raw));
        if (HIT || !occ) facc += g;
      } else {
        uint32_t st = raw;
        if (KIND == PAYLOAD_U2) st = (st >> ((addr & 3u) << 1)) & 3u;
        occ = st >= 2u;
        iacc += st == 0u ? 1u : 0u;  // an occupied voxel is never unknown
      }
      if (occ || !more) break;
      raw = nraw;
      addr = naddr;
    }
  }
}

// Latency-bound variant of ray_ig (linear layout): the walk runs K voxels
// ahead of the reads -- it records K addresses, issues the K loads back to
// back, then consumes them in order -- so a ray waits for memory once per K
// steps instead of once per step.  Same visit order and the same sums as
// ray_ig; up to K - 1 voxels past the occluding one are walked and read but
// not used.  Used when there are too few rays to hide the per-step latency.
template <int KIND, bool HIT, int K>
__device__ __forceinline__ void ray_ig_chunked(const void *payload, uint32_t addr_max, int nx, int ny, int nz,
                                               const float o[3], const float d[3], float &facc, uint32_t &iacc,
                                               uint32_t &steps) {
  Walk w;
  if (!walk_init(w, o, d, nx, ny, nz)) return;
  walk_linear_steps(w, nx, ny);
  int lin = walk_linear_index(w, nx, ny);
  bool alive = true;  // the walk has a current voxel not yet recorded
  for (;;) {
    uint32_t a[K], r[K];
    int n = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      a[k] = min((uint32_t)lin, addr_max);
      if (alive) {
        n = k + 1;
        alive = walk_advance_lin(w, lin);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) r[k] = k < n ? raw_load<KIND>(payload, a[k]) : 0u;
    bool stop = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (k < n && !stop) {
        steps += 1u;
        bool occ;
        if (KIND == PAYLOAD_GAIN_F32) {
          occ = (int32_t)r[k] < 0;
          const float g = fabsf(__uint_as_float(r[k]));
          if (HIT || !occ) facc += g;
        } else {
          uint32_t st = r[k];
          if (KIND == PAYLOAD_U2) st = (st >> ((a[k] & 3u) << 1)) & 3u;
          occ = st >= 2u;
          iacc += st == 0u ? 1u : 0u;
        }
        stop = occ;
      }
    }
    if (stop || !alive) break;
  }
}

// Items = (pose, 32 x 8 ray tile).  A CTA takes one item at a time; warp w
// casts packet w of the tile; the 8 packet sums are added in warp order
// into partials[item].  CHUNK > 0 (linear layout only) walks CHUNK voxels
// ahead of the reads (ray_ig_chunked).  SKIP (linear state maps, count
// metric, or FP32 gains) skips uniform bricks (ray_skip).
#ifndef NBT_SKIP_MIN_BLOCKS
#define NBT_SKIP_MIN_BLOCKS 5
#endif
template <int KIND, bool HIT, bool LINEAR, int CHUNK, bool SKIP = false>
__global__ void __launch_bounds__(kThreads, SKIP ? NBT_SKIP_MIN_BLOCKS : (CHUNK ? 4 : (LINEAR ? 6 : 5)))
    ig_tiles_kernel(DevMap m, CamConst cc, const float *__restrict__ poses, int64_t n_items, uint32_t addr_max,
                    unsigned long long *queue, Partial *partials) {
  extern __shared__ int32_t stab[];
  __shared__ float s_pose[8], s_rot[9];
  __shared__ float s_f[kThreads / 32];
  __shared__ uint32_t s_i[kThreads / 32], s_s[kThreads / 32];
  __shared__ long long s_item;
  __shared__ int s_x0, s_y0;
  if (!LINEAR) {
    const int ntab = m.nx + m.ny + m.nz;
    for (int k = threadIdx.x; k < ntab; k += blockDim.x) stab[k] = m.tab[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pw = cc.packet_w, ph = 32 / pw, across = 32 / pw;
  const int di = (warp % across) * pw + lane % pw;  // pixel of this lane within the tile
  const int dj = (warp / across) * ph + lane / pw;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(queue, 1ull);
      s_item = it;
      if (it < n_items) {
        // the item's pose, its rotation and the tile's first pixel, once per CTA
        const long long pose = it / cc.tiles_per_pose;
        const int tile = (int)(it - pose * cc.tiles_per_pose);
        float q[7], r[9];
#pragma unroll
        for (int k = 0; k < 7; ++k) s_pose[k] = q[k] = __ldg(poses + pose * 7 + k);
        quat_rot_f32(q + 3, r);
#pragma unroll
        for (int k = 0; k < 9; ++k) s_rot[k] = r[k];
        s_x0 = (tile % cc.tiles_x) * kTileW;
        s_y0 = (tile / cc.tiles_x) * kTileH;
      }
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= n_items) break;
    const int i = s_x0 + di;
    const int j = s_y0 + dj;
    float facc = 0.0f;
    uint32_t iacc = 0u, steps = 0u;
    const bool inside = i < cc.W && j < cc.H;
    if constexpr (SKIP) {
      float o[3] = {0.0f, 0.0f, 0.0f}, d[3] = {0.0f, 0.0f, 0.0f};
      if (inside) ray_segment_rot(cc, s_pose, s_rot, i, j, o, d);
      ray_skip<KIND, HIT>(m, addr_max, o, d, inside, facc, iacc, steps);   // all lanes together
    } else if (inside) {
      float o[3], d[3];
      ray_segment_rot(cc, s_pose, s_rot, i, j, o, d);
      if constexpr (CHUNK > 0)
        ray_ig_chunked<KIND, HIT, CHUNK>(m.payload, addr_max, m.nx, m.ny, m.nz, o, d, facc, iacc, steps);
      else
        ray_ig<KIND, HIT, LINEAR>(m.payload, stab, addr_max, m.nx, m.ny, m.nz, o, d, facc, iacc, steps);
    }
    // FP32-gain walks leave the count at 0 and count walks the gain: reduce
    // only what the payload kind produces
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      if (KIND == PAYLOAD_GAIN_F32)
        facc += __shfl_xor_sync(0xffffffffu, facc, s);
      else
        iacc += __shfl_xor_sync(0xffffffffu, iacc, s);
      steps += __shfl_xor_sync(0xffffffffu, steps, s);
    }
    if (lane == 0) {
      s_f[warp] = facc;
      s_i[warp] = iacc;
      s_s[warp] = steps;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Partial p;
      p.fsum = 0.0f;
      p.isum = 0u;
      p.steps = 0u;
      p.pad = 0u;
      for (int k = 0; k < kThreads / 32; ++k) {
        p.fsum += s_f[k];
        p.isum += s_i[k];
        p.steps += s_s[k];
      }
      partials[item] = p;
    }
  }
}

// Uniform-brick skipping walks on state maps (linear layout, many rays):
// each warp takes whole items from the device queue and casts the item's 8
// packets one after another, so no warp waits at a CTA barrier for a slower
// one (the walks of one packet take very different times once uniform
// bricks are skipped).  Lane 0 forms the item's rotation into the warp's
// shared slot.
// The per-item sum is the same fixed shuffle tree per packet and the same
// packet order as ig_tiles_kernel's 8-warp sum, so partials are
// bit-identical to it.
template <int KIND, bool HIT>
__global__ void __launch_bounds__(kThreads, NBT_SKIP_MIN_BLOCKS)
    ig_warp_tiles_kernel(DevMap m, CamConst cc, const float *__restrict__ poses, int64_t n_items, uint32_t addr_max,
                         unsigned long long *queue, Partial *partials) {
  constexpr int kPk = kThreads / 32;   // packets per item
  // per warp: the item's pose, rotation and first pixel; the packets' sums (kept out of registers)
  __shared__ float s_pose[kThreads / 32][8], s_rot[kThreads / 32][9];
  __shared__ int s_xy[kThreads / 32][2];
  __shared__ long long s_item[kThreads / 32];
  __shared__ float s_f[kThreads / 32][kPk];
  __shared__ uint32_t s_i[kThreads / 32][kPk], s_s[kThreads / 32][kPk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pw = cc.packet_w, ph = 32 / pw, across = 32 / pw;
  float *sp = s_pose[warp], *sr = s_rot[warp];
  for (;;) {
    long long item = 0;
    if (lane == 0) {
      item = (long long)atomicAdd(queue, 1ull);
      s_item[warp] = item;
      if (item < n_items) {
        const long long pose = item / cc.tiles_per_pose;
        const int tile = (int)(item - pose * cc.tiles_per_pose);
        float q[7], r[9];
#pragma unroll
        for (int k = 0; k < 7; ++k) sp[k] = q[k] = __ldg(poses + pose * 7 + k);
        quat_rot_f32(q + 3, r);
#pragma unroll
        for (int k = 0; k < 9; ++k) sr[k] = r[k];
        s_xy[warp][0] = (tile % cc.tiles_x) * kTileW;
        s_xy[warp][1] = (tile / cc.tiles_x) * kTileH;
      }
    }
    if (__shfl_sync(0xffffffffu, item, 0) >= n_items) break;
    __syncwarp();
    for (int pk = 0; pk < kPk; ++pk) {
      const int i = s_xy[warp][0] + (pk % across) * pw + lane % pw;
      const int j = s_xy[warp][1] + (pk / across) * ph + lane / pw;
      float facc = 0.0f;
      uint32_t iacc = 0u, steps = 0u;
      const bool inside = i < cc.W && j < cc.H;
      float o[3] = {0.0f, 0.0f, 0.0f}, d[3] = {0.0f, 0.0f, 0.0f};
      if (inside) ray_segment_rot(cc, sp, sr, i, j, o, d);
      ray_skip<KIND, HIT>(m, addr_max, o, d, inside, facc, iacc, steps);   // all lanes together
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        if (KIND == PAYLOAD_GAIN_F32)
          facc += __shfl_xor_sync(0xffffffffu, facc, s);
        else
          iacc += __shfl_xor_sync(0xffffffffu, iacc, s);
        steps += __shfl_xor_sync(0xffffffffu, steps, s);
      }
      if (lane == 0) {
        s_f[warp][pk] = facc;
        s_i[warp][pk] = iacc;
        s_s[warp][pk] = steps;
      }
    }
    __syncwarp();   // every lane is done with the slot before lane 0 refills it
    if (lane == 0) {
      Partial p;
      p.fsum = 0.0f;
      p.isum = 0u;
      p.steps = 0u;
      p.pad = 0u;
      for (int k = 0; k < kPk; ++k) {
        p.fsum += s_f[warp][k];
        p.isum += s_i[warp][k];
        p.steps += s_s[warp][k];
      }
      partials[s_item[warp]] = p;
    }
  }
}

// Few rays (the paper's operating point: a few thousand rays per call):
// LANES lanes walk each ray (walk_lane_part), each its share of the
// crossings, kSplitChunk voxels ahead of its reads.  A lane stops at its
// first occupied voxel; the ray's IG is the sum of its lanes up to and
// including the first lane that found one (the lanes are in walk order).
// Items as ig_tiles_kernel: (pose, 32 x 8 tile), one partial per item; the
// tile's rays are taken 32 at a time.
constexpr int kSplitChunk = 4;

template <int KIND, bool HIT, int LANES>
__device__ __forceinline__ void lane_ray_ig(const void *payload, uint32_t addr_max, int nx, int ny, int nz,
                                            const float o[3], const float d[3], int part, float &facc,
                                            uint32_t &iacc, uint32_t &steps, bool &occ_found) {
  Walk w;
  if (!walk_init(w, o, d, nx, ny, nz)) return;
  walk_linear_steps(w, nx, ny);
  int lin = walk_linear_index(w, nx, ny);
  bool first, split_end;
  int A;
  if (!walk_lane_part(w, lin, part, LANES, nx, ny, nz, first, split_end, A)) return;
  const int guard = nx + ny + nz + 3;
  bool pending = first, more = true;
  int g = 0;
  while (more) {
    uint32_t a[kSplitChunk], r[kSplitChunk];
    int n = 0;
#pragma unroll
    for (int k = 0; k < kSplitChunk; ++k) {
      a[k] = min((uint32_t)lin, addr_max);
      if (more) {
        if (pending) {
          pending = false;
          n = k + 1;
        } else {
          float t;
          const int ax = walk_next_axis(w, t);
          if (g++ < guard && (t < w.tmax || (split_end && t == w.tmax && ax < A))) {
            walk_advance_lin(w, lin);   // takes exactly that crossing
            a[k] = min((uint32_t)lin, addr_max);
            n = k + 1;
          } else {
            more = false;
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kSplitChunk; ++k) r[k] = k < n ? raw_load<KIND>(payload, a[k]) : 0u;
#pragma unroll
    for (int k = 0; k < kSplitChunk; ++k) {
      if (k < n && !occ_found) {
        steps += 1u;
        bool occ;
        if (KIND == PAYLOAD_GAIN_F32) {
          occ = (int32_t)r[k] < 0;
          const float gk = fabsf(__uint_as_float(r[k]));
          if (HIT || !occ) facc += gk;
        } else {
          uint32_t st = r[k];
          if (KIND == PAYLOAD_U2) st = (st >> ((a[k] & 3u) << 1)) & 3u;
          occ = st >= 2u;
          iacc += st == 0u ? 1u : 0u;
        }
        occ_found = occ;
      }
    }
    if (occ_found) return;
  }
}

template <int KIND, bool HIT, int LANES>
__global__ void __launch_bounds__(kThreads)
    ig_split_kernel(DevMap m, CamConst cc, const float *__restrict__ poses, int64_t n_items, uint32_t addr_max,
                    unsigned long long *queue, Partial *partials) {
  __shared__ float s_pose[8];
  __shared__ float s_f[kThreads / 32];
  __shared__ uint32_t s_i[kThreads / 32], s_s[kThreads / 32];
  __shared__ long long s_item;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int part = threadIdx.x % LANES;   // position of this lane in its ray's group
  const int slot = threadIdx.x / LANES;   // ray of the pass
  const unsigned group = (LANES == 32 ? 0xffffffffu : ((1u << LANES) - 1u)) << (lane & ~(LANES - 1));
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(queue, 1ull);
      s_item = it;
      if (it < n_items) {
        const long long pose = it / cc.tiles_per_pose;
#pragma unroll
        for (int k = 0; k < 7; ++k) s_pose[k] = __ldg(poses + pose * 7 + k);
      }
    }
    __syncthreads();
    const long long item = s_item;
    if (item >= n_items) break;
    const long long pose = item / cc.tiles_per_pose;
    const int tile = (int)(item - pose * cc.tiles_per_pose);
    const int x0 = (tile % cc.tiles_x) * kTileW, y0 = (tile / cc.tiles_x) * kTileH;
    const int tw = min(kTileW, cc.W - x0), th = min(kTileH, cc.H - y0);
    const int n_rays = tw * th;
    float facc = 0.0f;
    uint32_t iacc = 0u, steps = 0u;
    for (int r0 = 0; r0 < n_rays; r0 += kThreads / LANES) {
      const int r = r0 + slot;
      float f = 0.0f;
      uint32_t ic = 0u, st = 0u;
      bool occ = false;
      if (r < n_rays) {
        float o[3], d[3];
        ray_segment(cc, s_pose, x0 + r % tw, y0 + r / tw, o, d);
        lane_ray_ig<KIND, HIT, LANES>(m.payload, addr_max, m.nx, m.ny, m.nz, o, d, part, f, ic, st, occ);
      }
      // lanes past the first one that met an occupied voxel contribute nothing
      const unsigned hit = __ballot_sync(0xffffffffu, occ) & group;
      if (hit && lane > __ffs(hit) - 1) {
        f = 0.0f;
        ic = 0u;
        st = 0u;
      }
      facc += f;
      iacc += ic;
      steps += st;
    }
    // FP32-gain walks leave the count at 0 and count walks the gain: reduce
    // only what the payload kind produces
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      if (KIND == PAYLOAD_GAIN_F32)
        facc += __shfl_xor_sync(0xffffffffu, facc, s);
      else
        iacc += __shfl_xor_sync(0xffffffffu, iacc, s);
      steps += __shfl_xor_sync(0xffffffffu, steps, s);
    }
    if (lane == 0) {
      s_f[warp] = facc;
      s_i[warp] = iacc;
      s_s[warp] = steps;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Partial p;
      p.fsum = 0.0f;
      p.isum = 0u;
      p.steps = 0u;
      p.pad = 0u;
      for (int k = 0; k < kThreads / 32; ++k) {
        p.fsum += s_f[k];
        p.isum += s_i[k];
        p.steps += s_s[k];
      }
      partials[item] = p;
    }
  }
}

// One warp per perspective: fixed-order FP64 sum of its tiles' partials.
__global__ void views_reduce_kernel(const Partial *__restrict__ partials, int64_t n_views, int tiles, int mean,
                                    double n_rays, float *__restrict__ ig_out, uint64_t *__restrict__ steps_out) {
  const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (v >= n_views) return;
  double f = 0.0;
  unsigned long long a = 0ull, b = 0ull;
  for (int t = lane; t < tiles; t += 32) {
    const Partial p = partials[v * tiles + t];
    f += (double)p.fsum;
    a += p.isum;
    b += p.steps;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    f += __shfl_xor_sync(0xffffffffu, f, s);
    a += __shfl_xor_sync(0xffffffffu, a, s);
    b += __shfl_xor_sync(0xffffffffu, b, s);
  }
  if (lane == 0) {
    double total = f + (double)a;
    if (mean) total /= n_rays;
    ig_out[v] = (float)total;
    if (steps_out) steps_out[v] = b;
  }
}

// One warp per trajectory: lanes take whole poses, each pose's IG in FP64
// (sum or mean over its tiles), then a fixed shuffle tree over lanes.
// Offsets are clamped to [0, n_poses] so malformed CSR input cannot read
// outside the partials; it only yields wrong sums.
__global__ void traj_reduce_kernel(const Partial *__restrict__ partials, const int32_t *__restrict__ offsets,
                                   int32_t n_traj, int32_t n_poses, int tiles, int mean, double n_rays,
                                   float *__restrict__ traj_out, float *__restrict__ pose_out) {
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= n_traj) return;
  const int32_t b = min(max(offsets[t], 0), n_poses);
  const int32_t e = min(max(offsets[t + 1], b), n_poses);
  double acc = 0.0;
  for (int32_t p = b + lane; p < e; p += 32) {
    double f = 0.0;
    unsigned long long a = 0ull;
    for (int k = 0; k < tiles; ++k) {
      const Partial q = partials[(int64_t)p * tiles + k];
      f += (double)q.fsum;
      a += q.isum;
    }
    double pig = f + (double)a;
    if (mean) pig /= n_rays;
    if (pose_out) pose_out[p] = (float)pig;
    acc += pig;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
  if (lane == 0) traj_out[t] = (float)acc;
}

__global__ void view_segments_kernel(CamConst cc, const float *__restrict__ poses, int64_t n_rays,
                                     float *__restrict__ o_out, float *__restrict__ d_out) {
  const int64_t n_per = (int64_t)cc.W * cc.H;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rays; r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = r / n_per;
    const int k = (int)(r - v * n_per);
    float pz[7];
    for (int q = 0; q < 7; ++q) pz[q] = poses[v * 7 + q];
    float o[3], d[3];
    ray_segment(cc, pz, k % cc.W, k / cc.W, o, d);
    for (int a = 0; a < 3; ++a) {
      o_out[r * 3 + a] = o[a];
      d_out[r * 3 + a] = d[a];
    }
  }
}

// Test kernel: the voxel sequence of each segment, walked by the same step
// function as the IG kernel for the map's layout.
template <int KIND, bool LINEAR>
__global__ void trace_kernel(DevMap m, const float *__restrict__ o, const float *__restrict__ d, int n_rays,
                             int use_occ, uint32_t addr_max, int32_t *__restrict__ idx_out, int cap,
                             int32_t *__restrict__ n_out) {
  extern __shared__ int32_t stab[];
  const int ntab = m.nx + m.ny + m.nz;
  if (!LINEAR)
    for (int k = threadIdx.x; k < ntab; k += blockDim.x) stab[k] = m.tab[k];
  __syncthreads();
  const int limit = ntab + 2;  // a walk visits at most nx + ny + nz - 2 voxels
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rays; r += gridDim.x * blockDim.x) {
    const float oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
    const float dd[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
    Walk w;
    int count = 0;
    if (walk_init(w, oo, dd, m.nx, m.ny, m.nz)) {
      int offx = 0, offy = 0, offz = 0, lin = 0;
      if (LINEAR) {
        walk_linear_steps(w, m.nx, m.ny);
        lin = walk_linear_index(w, m.nx, m.ny);
      } else {
        offx = tab_at(stab, w.px);
        offy = tab_at(stab, w.py);
        offz = tab_at(stab, w.pz);
      }
      while (count < limit) {
        const int ix = walk_index(w.bx, w.sx), iy = walk_index(w.by, w.sy), iz = walk_index(w.bz, w.sz);
        if (count < cap) idx_out[(int64_t)r * cap + count] = (iz * m.ny + iy) * m.nx + ix;
        ++count;
        if (use_occ) {
          float g;
          uint32_t unk;
          bool occ;
          const uint32_t a = min(LINEAR ? (uint32_t)lin : (uint32_t)(offx + offy + offz), addr_max);
          read_voxel<KIND>(m.payload, a, g, unk, occ);
          if (occ) break;
        }
        const bool more = LINEAR ? walk_advance_lin(w, lin) : walk_advance(w, stab, offx, offy, offz);
        if (!more) break;
      }
    }
    n_out[r] = count;
  }
}

size_t tile_smem(nbt_map map) { return (size_t)(map->desc.nx + map->desc.ny + map->desc.nz) * sizeof(int32_t); }

uint32_t addr_max_of(nbt_map map) { return (uint32_t)(map->elems - 1); }

// Resident CTAs per SM of one tile-kernel instantiation: queried once per
// device for the linear layout (no dynamic shared memory), per call for
// bricked layouts (their table size varies).
template <int KIND, bool HIT, bool LINEAR, int CHUNK, bool SKIP = false>
int tiles_per_sm(nbt_map map, size_t smem, int *per_sm) {
  static int cached[64] = {0};
  const int dev = map->device;
  if (LINEAR && dev >= 0 && dev < 64 && cached[dev] > 0) {
    *per_sm = cached[dev];
    return NBT_OK;
  }
  int n = 0;
  NBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, ig_tiles_kernel<KIND, HIT, LINEAR, CHUNK, SKIP>,
                                                             kThreads, smem));
  *per_sm = std::max(n, 1);
  if (LINEAR && dev >= 0 && dev < 64) cached[dev] = *per_sm;
  return NBT_OK;
}

template <int KIND, bool HIT, bool LINEAR, int CHUNK, bool SKIP = false>
int launch_tiles_t(nbt_map map, const void *payload, const CamConst &cc, const float *poses, int64_t n_items,
                   void *workspace, cudaStream_t stream) {
  const size_t smem = LINEAR ? 0 : tile_smem(map);
  int per_sm = 1;
  int rc = tiles_per_sm<KIND, HIT, LINEAR, CHUNK, SKIP>(map, smem, &per_sm);
  if (rc != NBT_OK) return rc;
  const int64_t grid = std::min<int64_t>(n_items, (int64_t)sm_count() * per_sm);
  unsigned long long *queue = (unsigned long long *)workspace;
  Partial *partials = (Partial *)((char *)workspace + 256);
  NBT_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream));
  ig_tiles_kernel<KIND, HIT, LINEAR, CHUNK, SKIP><<<(unsigned)grid, kThreads, smem, stream>>>(
      dev_map(map, payload), cc, poses, n_items, addr_max_of(map), queue, partials);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

template <int KIND, bool HIT>
int launch_warp_tiles(nbt_map map, const void *payload, const CamConst &cc, const float *poses, int64_t n_items,
                      void *workspace, cudaStream_t stream) {
  static int cached[64] = {0};
  const int dev = map->device;
  int per_sm = dev >= 0 && dev < 64 ? cached[dev] : 0;
  if (per_sm <= 0) {
    NBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ig_warp_tiles_kernel<KIND, HIT>, kThreads, 0));
    per_sm = std::max(per_sm, 1);
    if (dev >= 0 && dev < 64) cached[dev] = per_sm;
  }
  const int64_t warps = (int64_t)sm_count() * per_sm * (kThreads / 32);
  const int64_t grid = (std::min<int64_t>(n_items, warps) + kThreads / 32 - 1) / (kThreads / 32);
  unsigned long long *queue = (unsigned long long *)workspace;
  Partial *partials = (Partial *)((char *)workspace + 256);
  NBT_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream));
  ig_warp_tiles_kernel<KIND, HIT><<<(unsigned)grid, kThreads, 0, stream>>>(dev_map(map, payload), cc, poses, n_items,
                                                                          addr_max_of(map), queue, partials);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

// Voxels the latency-bound variant walks ahead of its reads.
constexpr int kChunk = 8;

// Calls with at most this many rays (linear layout) take the split-ray
// kernel: 16 lanes per ray up to kSplit16Rays, 8 up to kSplit8Rays (measured
// on the paper-mode sweep; beyond, more rays than lanes hide the latency).
constexpr int64_t kSplit16Rays = 4096;
constexpr int64_t kSplit8Rays = 32768;

template <int KIND, bool HIT, int LANES>
int launch_split(nbt_map map, const void *payload, const CamConst &cc, const float *poses, int64_t n_items,
                 void *workspace, cudaStream_t stream) {
  static int cached[64] = {0};
  const int dev = map->device;
  int per_sm = dev >= 0 && dev < 64 ? cached[dev] : 0;
  if (per_sm <= 0) {
    NBT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ig_split_kernel<KIND, HIT, LANES>, kThreads,
                                                               0));
    per_sm = std::max(per_sm, 1);
    if (dev >= 0 && dev < 64) cached[dev] = per_sm;
  }
  const int64_t grid = std::min<int64_t>(n_items, (int64_t)sm_count() * per_sm);
  unsigned long long *queue = (unsigned long long *)workspace;
  Partial *partials = (Partial *)((char *)workspace + 256);
  NBT_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), stream));
  ig_split_kernel<KIND, HIT, LANES><<<(unsigned)grid, kThreads, 0, stream>>>(
      dev_map(map, payload), cc, poses, n_items, addr_max_of(map), queue, partials);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

// Linear layout, by the number of rays in the call: a few thousand take the
// split-ray kernel (several lanes per ray); up to two per thread slot of the
// throughput kernel's resident CTAs, the walk-ahead kernel (neither can hide
// the per-step read latency otherwise); more take the rolling one-voxel
// prefetch, which issues the fewest instructions per step.  The split
// kernel adds each ray's gains lane part by lane part, so its FP32 sums may
// differ from the other kernels' in the last bits (counts and steps equal).
template <int KIND, bool HIT>
int launch_tiles_linear(nbt_map map, const void *payload, const CamConst &cc, const float *poses, int64_t n_items,
                        void *workspace, cudaStream_t stream) {
  int per_sm = 1;
  int rc = tiles_per_sm<KIND, HIT, true, 0>(map, 0, &per_sm);
  if (rc != NBT_OK) return rc;
  const int64_t n_rays = n_items / cc.tiles_per_pose * cc.W * cc.H;
  if (n_rays <= kSplit16Rays) return launch_split<KIND, HIT, 16>(map, payload, cc, poses, n_items, workspace, stream);
  if (n_rays <= kSplit8Rays) return launch_split<KIND, HIT, 8>(map, payload, cc, poses, n_items, workspace, stream);
  if (n_rays <= 2 * (int64_t)sm_count() * per_sm * kThreads)
    return launch_tiles_t<KIND, HIT, true, kChunk>(map, payload, cc, poses, n_items, workspace, stream);
  if (map->skip && map->d_bsum) {
    // skip uniform bricks (summaries built here, only for the calls that use them); on state maps the
    // occupied voxel adds nothing, so HIT is moot there
    rc = prepare_bsum(map, stream);
    if (rc != NBT_OK) return rc;
    constexpr bool H = KIND == PAYLOAD_GAIN_F32 ? HIT : true;
    // state maps: warps take whole items (no CTA barrier between packets, measured +3 % on the
    // tabletop trajectories); FP32 gains keep the 8-warp CTA items, which measured 3 % faster there
    if constexpr (KIND == PAYLOAD_GAIN_F32)
      return launch_tiles_t<KIND, H, true, 0, true>(map, payload, cc, poses, n_items, workspace, stream);
    else
      return launch_warp_tiles<KIND, H>(map, payload, cc, poses, n_items, workspace, stream);
  }
  return launch_tiles_t<KIND, HIT, true, 0>(map, payload, cc, poses, n_items, workspace, stream);
}

template <int KIND>
int launch_tiles(nbt_map map, const void *payload, const CamConst &cc, const float *poses, int64_t n_items,
                 int include_hit, void *workspace, cudaStream_t stream) {
  const bool lin = map->brick == 1;
  if (include_hit)
    return lin ? launch_tiles_linear<KIND, true>(map, payload, cc, poses, n_items, workspace, stream)
               : launch_tiles_t<KIND, true, false, 0>(map, payload, cc, poses, n_items, workspace, stream);
  return lin ? launch_tiles_linear<KIND, false>(map, payload, cc, poses, n_items, workspace, stream)
             : launch_tiles_t<KIND, false, false, 0>(map, payload, cc, poses, n_items, workspace, stream);
}

template <int KIND>
void launch_trace(nbt_map map, const DevMap &m, unsigned grid, cudaStream_t stream, const float *o, const float *d,
                  int n_rays, int use_occ, int32_t *idx_out, int cap, int32_t *n_out) {
  const size_t smem = tile_smem(map);
  const uint32_t amax = addr_max_of(map);
  if (map->brick == 1)
    trace_kernel<KIND, true><<<grid, 128, 0, stream>>>(m, o, d, n_rays, use_occ, amax, idx_out, cap, n_out);
  else
    trace_kernel<KIND, false><<<grid, 128, smem, stream>>>(m, o, d, n_rays, use_occ, amax, idx_out, cap, n_out);
}

int run_tiles(nbt_map map, const nbt_pose *poses, int64_t n_poses, const nbt_camera *cam,
              const nbt_ig_params *params, void *workspace, int64_t workspace_bytes, cudaStream_t stream,
              CamConst *cc_out) {
  PayloadKind kind;
  const void *payload = nullptr;
  int rc = payload_kind(map, params, &kind, &payload);
  if (rc != NBT_OK) return rc;
  const CamConst cc = make_cam(map, cam);
  *cc_out = cc;
  const int64_t n_items = n_poses * cc.tiles_per_pose;
  if (!workspace || workspace_bytes < workspace_bytes_for(n_items) || ((uintptr_t)workspace & 15u))
    return NBT_EWORKSPACE;
  if (kind == PAYLOAD_GAIN_F32) {
    rc = prepare_gain(map, params, stream);
    if (rc != NBT_OK) return rc;
  }
  const float *pp = (const float *)poses;
  switch (kind) {
    case PAYLOAD_U8:
      return launch_tiles<PAYLOAD_U8>(map, payload, cc, pp, n_items, params->include_hit, workspace, stream);
    case PAYLOAD_U2:
      return launch_tiles<PAYLOAD_U2>(map, payload, cc, pp, n_items, params->include_hit, workspace, stream);
    default:
      return launch_tiles<PAYLOAD_GAIN_F32>(map, payload, cc, pp, n_items, params->include_hit, workspace, stream);
  }
}

}  // namespace
}  // namespace nbt

using namespace nbt;

extern "C" {

int nbt_camera_from_grid_scale(float fov_h, float fov_v, float max_range, float voxel_size, float grid_scale,
                               nbt_camera *cam) {
  if (!cam) return NBT_EINVAL;
  const float args[5] = {fov_h, fov_v, max_range, voxel_size, grid_scale};
  for (float a : args)
    if (!std::isfinite(a) || !(a > 0.0f)) return NBT_EINVAL;
  if (!(fov_h < 3.14159265f) || !(fov_v < 3.14159265f)) return NBT_EINVAL;
  const double step = (double)grid_scale * (double)voxel_size;
  int32_t side[2];
  const float fovs[2] = {fov_h, fov_v};
  for (int a = 0; a < 2; ++a) {
    const double half = (double)max_range * std::tan((double)fovs[a] * 0.5);
    const double n = std::floor((2.0 * half) / step) + 1.0;
    if (!(n <= 65535.0)) return NBT_EINVAL;
    side[a] = std::max(2, (int32_t)n);
  }
  cam->width = side[0];
  cam->height = side[1];
  cam->fov_h = fov_h;
  cam->fov_v = fov_v;
  cam->max_range = max_range;
  cam->grid_mode = NBT_GRID_CORNERS;
  cam->range_mode = NBT_RANGE_PLANAR;
  return NBT_OK;
}

int nbt_workspace_size(int64_t n_poses, const nbt_camera *cam, int64_t *bytes) {
  // n_poses <= INT32_MAX keeps n_poses * tiles * 16 below 2^59 (tiles < 2^24)
  if (!bytes || n_poses < 0 || n_poses > INT32_MAX || !valid_camera(cam)) return NBT_EINVAL;
  const int64_t tiles = (int64_t)((cam->width + kTileW - 1) / kTileW) * ((cam->height + kTileH - 1) / kTileH);
  *bytes = workspace_bytes_for(n_poses * tiles);
  return NBT_OK;
}

int nbt_views_ig(nbt_map map, const nbt_pose *poses, int64_t n_views, const nbt_camera *cam,
                 const nbt_ig_params *params, float *ig_out, uint64_t *steps_out, void *workspace,
                 int64_t workspace_bytes, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n_views < 0 || n_views > INT32_MAX || !valid_camera(cam) || !valid_params(params)) return NBT_EINVAL;
  if (n_views == 0) return NBT_OK;
  if (!poses || !ig_out) return NBT_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  CamConst cc;
  rc = run_tiles(map, poses, n_views, cam, params, workspace, workspace_bytes, stream, &cc);
  if (rc != NBT_OK) return rc;
  const Partial *partials = (const Partial *)((const char *)workspace + 256);
  const int64_t threads = n_views * 32;
  views_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(
      partials, n_views, cc.tiles_per_pose, params->reduce == NBT_REDUCE_MEAN, (double)cc.W * cc.H, ig_out, steps_out);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int nbt_traj_ig(nbt_map map, const nbt_pose *poses, int64_t n_poses, const int32_t *offsets, int32_t n_traj,
                const nbt_camera *cam, const nbt_ig_params *params, float *traj_ig_out, float *pose_ig_out,
                void *workspace, int64_t workspace_bytes, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n_poses < 0 || n_traj < 0 || !valid_camera(cam) || !valid_params(params)) return NBT_EINVAL;
  if (n_traj == 0) return n_poses == 0 ? NBT_OK : NBT_EINVAL;
  if (!offsets || !traj_ig_out || (n_poses > 0 && !poses)) return NBT_EINVAL;
  if (n_poses > INT32_MAX) return NBT_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  CamConst cc = make_cam(map, cam);
  if (n_poses > 0) {
    rc = run_tiles(map, poses, n_poses, cam, params, workspace, workspace_bytes, stream, &cc);
    if (rc != NBT_OK) return rc;
  } else if (!workspace || workspace_bytes < workspace_bytes_for(0)) {
    return NBT_EWORKSPACE;
  }
  const Partial *partials = (const Partial *)((const char *)workspace + 256);
  const int64_t threads = (int64_t)n_traj * 32;
  traj_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(
      partials, offsets, n_traj, (int32_t)n_poses, cc.tiles_per_pose, params->reduce == NBT_REDUCE_MEAN,
      (double)cc.W * cc.H, traj_ig_out, pose_ig_out);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int nbt_trace_segments(nbt_map map, const float *o, const float *d, int32_t n_rays, const nbt_ig_params *params,
                       int32_t *idx_out, int32_t cap, int32_t *n_out, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n_rays < 0 || cap < 0 || (params && !valid_params(params))) return NBT_EINVAL;
  if (n_rays == 0) return NBT_OK;
  if (!o || !d || !n_out || (cap > 0 && !idx_out)) return NBT_EINVAL;
  cudaStream_t stream = (cudaStream_t)stream_;
  PayloadKind kind = PAYLOAD_U8;
  const void *payload = map->d_payload;
  if (params) {
    rc = payload_kind(map, params, &kind, &payload);
    if (rc != NBT_OK) return rc;
    if (kind == PAYLOAD_GAIN_F32) {
      rc = prepare_gain(map, params, stream);
      if (rc != NBT_OK) return rc;
    }
  }
  const DevMap m = dev_map(map, payload);
  const unsigned grid = (unsigned)std::min<int64_t>((n_rays + 127) / 128, (int64_t)sm_count() * 8);
  const int use_occ = params != nullptr;
  switch (kind) {
    case PAYLOAD_U8: launch_trace<PAYLOAD_U8>(map, m, grid, stream, o, d, n_rays, use_occ, idx_out, cap, n_out); break;
    case PAYLOAD_U2: launch_trace<PAYLOAD_U2>(map, m, grid, stream, o, d, n_rays, use_occ, idx_out, cap, n_out); break;
    default: launch_trace<PAYLOAD_GAIN_F32>(map, m, grid, stream, o, d, n_rays, use_occ, idx_out, cap, n_out); break;
  }
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

int nbt_view_segments(nbt_map map, const nbt_pose *poses, int64_t n_views, const nbt_camera *cam, float *o_out,
                      float *d_out, void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n_views < 0 || n_views > INT32_MAX || !valid_camera(cam)) return NBT_EINVAL;
  if (n_views == 0) return NBT_OK;
  if (!poses || !o_out || !d_out) return NBT_EINVAL;
  const CamConst cc = make_cam(map, cam);
  const int64_t n_rays = n_views * cam->width * (int64_t)cam->height;
  const unsigned grid = (unsigned)std::min<int64_t>((n_rays + 255) / 256, (int64_t)sm_count() * 32);
  view_segments_kernel<<<grid, 256, 0, (cudaStream_t)stream_>>>(cc, (const float *)poses, n_rays, o_out, d_out);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// nbt_views_ig_noalloc: the per-perspective IG path with its scratch (work
// queue counter + per-tile partials) in a fixed device array instead of a
// caller workspace, for callers that may not allocate device memory (see
// include/nbt.h).  The array is file-scope, so every device that loads the
// library holds it until the process exits.  Host code only ever uses the
// device address looked up below; the array's name is a host-side stand-in.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char nbt_noalloc_scratch[NBT_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};
unsigned long long g_noalloc_ctx[kNoallocMaxDevices] = {0};

// Unique id of the calling thread's current CUDA context (0 if it cannot be
// read).  The driver calls are looked up through the runtime, so the library
// does not link the driver library itself.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      get_current = (GetCurrent)a;
      get_id = (GetId)b;
    }
    (void)cudaGetLastError();
    looked_up = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on `device` (the current device).
// Looked up once per device and context: if the device's context was torn
// down and created again (cudaDeviceReset), the module is loaded anew and
// the array may have moved, so a new context id triggers a new lookup.
int noalloc_scratch(int device, void **ptr) {
  if (device < 0 || device >= kNoallocMaxDevices) return NBT_EINVAL;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_noalloc_ptr[device] || ctx == 0 || ctx != g_noalloc_ctx[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, nbt_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();
      return NBT_ECUDA;
    }
    g_noalloc_ptr[device] = p;
    g_noalloc_ctx[device] = ctx;
  }
  *ptr = g_noalloc_ptr[device];
  return NBT_OK;
}

}  // namespace

extern "C" int nbt_views_ig_noalloc(nbt_map map, const nbt_pose *poses, int64_t n_views, const nbt_camera *cam,
                                    const nbt_ig_params *params, float *ig_out, uint64_t *steps_out,
                                    void *stream_) {
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (n_views < 0 || !valid_camera(cam) || !valid_params(params)) return NBT_EINVAL;
  if (n_views == 0) return NBT_OK;
  if (!poses || !ig_out) return NBT_EINVAL;
  // bound n_views before any product: at most this many views fit the array
  const int64_t tiles = (int64_t)((cam->width + kTileW - 1) / kTileW) * ((cam->height + kTileH - 1) / kTileH);
  if (n_views > ((int64_t)NBT_NOALLOC_SCRATCH_BYTES - 256) / ((int64_t)kPartialBytes * tiles)) return NBT_ESCRATCH;
  int64_t need = 0;
  rc = nbt_workspace_size(n_views, cam, &need);
  if (rc != NBT_OK) return rc;
  if (need > (int64_t)NBT_NOALLOC_SCRATCH_BYTES) return NBT_ESCRATCH;
  void *scratch = nullptr;
  rc = noalloc_scratch(map->device, &scratch);
  if (rc != NBT_OK) return rc;
  cudaStream_t stream = (cudaStream_t)stream_;
  // run_tiles zeroes the queue counter on the stream before the tile
  // kernel; the tile kernel writes every partial the reduce kernel reads.
  CamConst cc;
  rc = run_tiles(map, poses, n_views, cam, params, scratch, (int64_t)NBT_NOALLOC_SCRATCH_BYTES, stream, &cc);
  if (rc != NBT_OK) return rc;
  const Partial *partials = (const Partial *)((const char *)scratch + 256);
  const int64_t threads = n_views * 32;
  views_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(
      partials, n_views, cc.tiles_per_pose, params->reduce == NBT_REDUCE_MEAN, (double)cc.W * cc.H, ig_out, steps_out);
  NBT_CUDA_TRY(cudaGetLastError());
  return NBT_OK;
}

extern "C" int nbt_map_set_tuning(nbt_map map, const nbt_tuning *tuning) {
  if (!map || !tuning || !map_alive(map, 0)) return NBT_EINVAL;
  const int pw = tuning->packet_w == 0 ? 8 : tuning->packet_w;
  if (pw != 4 && pw != 8 && pw != 16 && pw != 32) return NBT_EINVAL;
  if (tuning->skip != 0 && tuning->skip != 1) return NBT_EINVAL;
  std::lock_guard<std::mutex> lock(map->mu);
  map->packet_w = pw;
  map->skip = tuning->skip;
  return NBT_OK;
}

extern "C" int nbt_map_get_tuning(nbt_map map, nbt_tuning *tuning) {
  if (!map || !tuning || !map_alive(map, 0)) return NBT_EINVAL;
  tuning->packet_w = map->packet_w;
  tuning->brick = map->brick;
  tuning->skip = map->skip;
  return NBT_OK;
}
