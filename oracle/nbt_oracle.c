/*
 * nbt_oracle.c -- CPU oracle for information-gain (IG) raycasting.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  This is the plain, slow reference
 * the CUDA library is checked against.  Only the test suite, the smoke check
 * and the benchmark's CPU baseline load it; the library never does, and the
 * two share no code.
 *
 * What it computes (paper, Section III "Online Local Information
 * Distribution"):
 *   - "Endpoint Calculation": per perspective, N_E = W x H endpoints on the
 *     far frustum plane at distance d_Cam, on a grid spanning
 *     [-d_h, d_h] x [-d_v, d_v] with d_h = d_Cam tan(FoV_h / 2) and
 *     d_v = d_Cam tan(FoV_v / 2), the four border rays included;
 *   - "IG Calculation": the voxels each ray from p_P to p_E passes through,
 *     in order; the ray IG g_R = sum_{i=0}^{N_O} g(v_i) with g from Eq. 2
 *     (or the unknown-voxel count / binary-entropy variants), where N_O
 *     stops at the first occupied voxel or at the endpoint;
 *   - per-perspective sums and the mean g_P = (1 / N_E) sum_k g_R,k.
 *
 * Three walks enumerate the voxels of a segment o + t d, t in [0, 1]
 * (voxel units, voxel (x, y, z) = [x, x+1) x [y, y+1) x [z, z+1)):
 *   orc_walk_brute : every voxel of the map is slab-tested in FP64; the voxels
 *                    whose interior the segment crosses with positive length,
 *                    sorted by entry parameter.  The definition; tiny maps.
 *   orc_walk_f64   : Amanatides-Woo stepping in FP64.
 *   orc_walk_f32   : Amanatides-Woo stepping in FP32 in one fixed operation
 *                    order, every operation rounded on its own (this file is
 *                    built with -ffp-contract=off).  The reference traversal.
 * IG is accumulated in FP64 along whichever walk is chosen.
 *
 * Readings where the paper is silent (each is a choice both sides follow):
 *   - rays are clipped to the map box; voxels outside contribute nothing;
 *   - the voxel holding the clipped start point is visited; a further voxel
 *     is visited iff the segment enters it before its end (entry t < t_max);
 *   - the first occupied voxel is visited and, with include_hit = 1, adds
 *     its gain (the sum in Eq. 2's ray IG runs to i = N_O inclusive);
 *   - probability maps: occupied iff p > occ_threshold, free iff
 *     p < free_threshold, unknown otherwise (both compared in FP32);
 *   - entropy uses log base 2, so p = 0.5 (unknown) gains 1 as in Eq. 2.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U8_STATE 0
#define ORC_F32_PROB 1

#define ORC_COUNT_UNKNOWN 0
#define ORC_PAPER_EQ2 1
#define ORC_ENTROPY 2

#define ORC_REDUCE_SUM 0
#define ORC_REDUCE_MEAN 1

#define ORC_GRID_CORNERS 0
#define ORC_GRID_CENTERS 1

#define ORC_RANGE_PLANAR 0
#define ORC_RANGE_SPHERICAL 1

#define ORC_WALK_F32 0
#define ORC_WALK_F64 1
#define ORC_WALK_BRUTE 2

typedef struct {
  int32_t nx, ny, nz;
  int32_t encoding;        /* ORC_U8_STATE or ORC_F32_PROB */
  float voxel_size;        /* metres */
  float origin[3];         /* world position of the map's min corner */
  const void *data;        /* dense grid, x fastest: idx = (z*ny + y)*nx + x */
} orc_map;

typedef struct {
  int32_t width, height;   /* W x H rays per perspective, N_E = W * H */
  float fov_h, fov_v;      /* full opening angles, radians */
  float max_range;         /* d_Cam, metres */
  int32_t grid_mode;       /* ORC_GRID_CORNERS (paper) or ORC_GRID_CENTERS */
  int32_t range_mode;      /* ORC_RANGE_PLANAR (paper) or ORC_RANGE_SPHERICAL */
} orc_camera;

typedef struct {
  int32_t metric;          /* ORC_COUNT_UNKNOWN, ORC_PAPER_EQ2, ORC_ENTROPY */
  float occ_threshold;     /* probability maps: occupied iff p > this */
  float free_threshold;    /* probability maps: free iff p < this */
  int32_t include_hit;     /* 1: the first occupied voxel adds its gain */
  int32_t reduce;          /* ORC_REDUCE_SUM or ORC_REDUCE_MEAN */
} orc_params;

/* Far-plane grid in the camera frame, rounded once to FP32. */
typedef struct {
  float x0, xstep, y0, ystep, zc;
  int32_t spherical;
} orc_cam_consts;

/* ------------------------------------------------------------------------ */
/* Endpoint calculation (Section III).                                       */
/* ------------------------------------------------------------------------ */

/* d_h = d_Cam tan(FoV_h / 2), d_v = d_Cam tan(FoV_v / 2), evaluated in FP64.
 * Corner mode: x_i = -d_h + i * 2 d_h / (W - 1) (the border rays are rays
 * 0 and W - 1); centre mode: x_i = -d_h + (i + 1/2) * 2 d_h / W.  The start
 * and the spacing are each rounded once to FP32; x_i itself is formed in
 * FP32 by orc_view_ray_f32. */
void orc_camera_consts(const orc_camera *cam, orc_cam_consts *cc) {
  double dh = (double)cam->max_range * tan((double)cam->fov_h * 0.5);
  double dv = (double)cam->max_range * tan((double)cam->fov_v * 0.5);
  int w = cam->width, h = cam->height;
  if (cam->grid_mode == ORC_GRID_CORNERS) {
    cc->x0 = w > 1 ? (float)(-dh) : 0.0f;
    cc->xstep = w > 1 ? (float)(2.0 * dh / (double)(w - 1)) : 0.0f;
    cc->y0 = h > 1 ? (float)(-dv) : 0.0f;
    cc->ystep = h > 1 ? (float)(2.0 * dv / (double)(h - 1)) : 0.0f;
  } else {
    cc->x0 = (float)(-dh + dh / (double)w);
    cc->xstep = (float)(2.0 * dh / (double)w);
    cc->y0 = (float)(-dv + dv / (double)h);
    cc->ystep = (float)(2.0 * dv / (double)h);
  }
  cc->zc = cam->max_range;
  cc->spherical = cam->range_mode == ORC_RANGE_SPHERICAL;
}

/* Camera-to-world rotation of the unit quaternion (w, x, y, z), in FP32. */
static void quat_to_rot_f32(const float *q, float r[9]) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  float xx = x * x, yy = y * y, zz = z * z;
  float xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  r[0] = 1.0f - 2.0f * (yy + zz);
  r[1] = 2.0f * (xy - wz);
  r[2] = 2.0f * (xz + wy);
  r[3] = 2.0f * (xy + wz);
  r[4] = 1.0f - 2.0f * (xx + zz);
  r[5] = 2.0f * (yz - wx);
  r[6] = 2.0f * (xz - wy);
  r[7] = 2.0f * (yz + wx);
  r[8] = 1.0f - 2.0f * (xx + yy);
}

/* Ray (i, j) of one perspective as a segment in voxel units: start o (the
 * camera position p_P) and displacement d (to the endpoint p_E), in FP32.
 * pose = {px, py, pz, qw, qx, qy, qz}. */
void orc_view_ray_f32(const orc_map *m, const orc_cam_consts *cc, const float *pose, int32_t i,
                      int32_t j, float o[3], float d[3]) {
  float r[9];
  quat_to_rot_f32(pose + 3, r);
  float inv_s = (float)(1.0 / (double)m->voxel_size);
  float cx = cc->x0 + (float)i * cc->xstep;
  float cy = cc->y0 + (float)j * cc->ystep;
  float cz = cc->zc;
  if (cc->spherical) {
    float len = sqrtf((cx * cx + cy * cy) + cz * cz);
    float sc = cc->zc / len;
    cx = cx * sc;
    cy = cy * sc;
    cz = cz * sc;
  }
  for (int a = 0; a < 3; ++a) {
    float wa = (r[3 * a + 0] * cx + r[3 * a + 1] * cy) + r[3 * a + 2] * cz;
    o[a] = (pose[a] - m->origin[a]) * inv_s;
    d[a] = wa * inv_s;
  }
}

/* ------------------------------------------------------------------------ */
/* Walks.  A visitor receives each voxel in order and returns 1 to stop.     */
/* ------------------------------------------------------------------------ */

typedef int (*orc_visit_fn)(void *ctx, int32_t x, int32_t y, int32_t z);

static int all_finite3(const float *v) {
  return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}

/* FP32 reference traversal.  Fixed operation order:
 *   inv_a = 1 / d_a;  clip: t0 = (0 - o_a) inv_a, t1 = (N_a - o_a) inv_a,
 *   t_min = max(0, near), t_max = min(1, far);  empty unless t_min < t_max;
 *   start: p_a = o_a + t_min d_a, i_a = floor(clamp(p_a, 0, N_a - 1));
 *   next crossing on axis a: t_a = ((float)(i_a + [s_a > 0]) - o_a) inv_a,
 *   recomputed from the integer index after every step on that axis;
 *   advance x if t_x <= t_y and t_x <= t_z, else y if t_y <= t_z, else z;
 *   stop when the chosen t is not < t_max, or the index leaves the map. */
int64_t orc_walk_f32(const int32_t dims[3], const float o[3], const float d[3], orc_visit_fn fn,
                     void *ctx) {
  if (!all_finite3(o) || !all_finite3(d)) return 0;
  float inv[3] = {0.0f, 0.0f, 0.0f};
  float tmin = 0.0f, tmax = 1.0f;
  for (int a = 0; a < 3; ++a) {
    float n = (float)dims[a];
    if (d[a] != 0.0f) {
      inv[a] = 1.0f / d[a];
      float t0 = (0.0f - o[a]) * inv[a];
      float t1 = (n - o[a]) * inv[a];
      float lo = inv[a] > 0.0f ? t0 : t1;
      float hi = inv[a] > 0.0f ? t1 : t0;
      tmin = lo > tmin ? lo : tmin;
      tmax = hi < tmax ? hi : tmax;
    } else if (!(o[a] >= 0.0f && o[a] < n)) {
      return 0;
    }
  }
  if (!(tmin < tmax)) return 0;
  int32_t idx[3], step[3];
  float tn[3];
  for (int a = 0; a < 3; ++a) {
    float p = o[a] + tmin * d[a];
    float hi = (float)(dims[a] - 1);
    p = p < 0.0f ? 0.0f : p;
    p = p > hi ? hi : p;
    idx[a] = (int32_t)floorf(p);
    step[a] = d[a] > 0.0f ? 1 : (d[a] < 0.0f ? -1 : 0);
    tn[a] = step[a] != 0 ? ((float)(idx[a] + (step[a] > 0)) - o[a]) * inv[a] : INFINITY;
  }
  int64_t count = 0;
  for (;;) {
    ++count;
    if (fn && fn(ctx, idx[0], idx[1], idx[2])) break;
    int a = (tn[0] <= tn[1] && tn[0] <= tn[2]) ? 0 : (tn[1] <= tn[2] ? 1 : 2);
    if (!(tn[a] < tmax)) break;
    idx[a] += step[a];
    if (idx[a] < 0 || idx[a] >= dims[a]) break;
    tn[a] = ((float)(idx[a] + (step[a] > 0)) - o[a]) * inv[a];
  }
  return count;
}

/* The same stepping in FP64, crossings as (boundary - o) / d. */
int64_t orc_walk_f64(const int32_t dims[3], const float of[3], const float df[3], orc_visit_fn fn,
                     void *ctx) {
  if (!all_finite3(of) || !all_finite3(df)) return 0;
  double o[3] = {of[0], of[1], of[2]}, d[3] = {df[0], df[1], df[2]};
  double tmin = 0.0, tmax = 1.0;
  for (int a = 0; a < 3; ++a) {
    double n = (double)dims[a];
    if (d[a] != 0.0) {
      double t0 = (0.0 - o[a]) / d[a];
      double t1 = (n - o[a]) / d[a];
      double lo = d[a] > 0.0 ? t0 : t1;
      double hi = d[a] > 0.0 ? t1 : t0;
      if (lo > tmin) tmin = lo;
      if (hi < tmax) tmax = hi;
    } else if (!(o[a] >= 0.0 && o[a] < n)) {
      return 0;
    }
  }
  if (!(tmin < tmax)) return 0;
  int32_t idx[3], step[3];
  double tn[3];
  for (int a = 0; a < 3; ++a) {
    double p = o[a] + tmin * d[a];
    double hi = (double)(dims[a] - 1);
    if (p < 0.0) p = 0.0;
    if (p > hi) p = hi;
    idx[a] = (int32_t)floor(p);
    step[a] = d[a] > 0.0 ? 1 : (d[a] < 0.0 ? -1 : 0);
    tn[a] = step[a] != 0 ? ((double)(idx[a] + (step[a] > 0)) - o[a]) / d[a] : INFINITY;
  }
  int64_t count = 0;
  for (;;) {
    ++count;
    if (fn && fn(ctx, idx[0], idx[1], idx[2])) break;
    int a = (tn[0] <= tn[1] && tn[0] <= tn[2]) ? 0 : (tn[1] <= tn[2] ? 1 : 2);
    if (!(tn[a] < tmax)) break;
    idx[a] += step[a];
    if (idx[a] < 0 || idx[a] >= dims[a]) break;
    tn[a] = ((double)(idx[a] + (step[a] > 0)) - o[a]) / d[a];
  }
  return count;
}

typedef struct {
  double tin;
  int32_t x, y, z;
} brute_hit;

static int cmp_hit(const void *a, const void *b) {
  double ta = ((const brute_hit *)a)->tin, tb = ((const brute_hit *)b)->tin;
  return ta < tb ? -1 : (ta > tb ? 1 : 0);
}

/* The definition: slab-test every voxel; keep those whose open interior the
 * segment crosses over a positive parameter length; order by entry t. */
int64_t orc_walk_brute(const int32_t dims[3], const float of[3], const float df[3], orc_visit_fn fn,
                       void *ctx) {
  if (!all_finite3(of) || !all_finite3(df)) return 0;
  double o[3] = {of[0], of[1], of[2]}, d[3] = {df[0], df[1], df[2]};
  int64_t cap = (int64_t)dims[0] + dims[1] + dims[2] + 3, n = 0;
  brute_hit *hits = (brute_hit *)malloc((size_t)cap * sizeof(brute_hit));
  if (!hits) return -1;
  for (int32_t z = 0; z < dims[2]; ++z)
    for (int32_t y = 0; y < dims[1]; ++y)
      for (int32_t x = 0; x < dims[0]; ++x) {
        int32_t c[3] = {x, y, z};
        double tin = 0.0, tout = 1.0;
        int inside = 1;
        for (int a = 0; a < 3 && inside; ++a) {
          if (d[a] != 0.0) {
            double t0 = ((double)c[a] - o[a]) / d[a];
            double t1 = ((double)c[a] + 1.0 - o[a]) / d[a];
            double lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
            if (lo > tin) tin = lo;
            if (hi < tout) tout = hi;
          } else if (!(o[a] > (double)c[a] && o[a] < (double)c[a] + 1.0)) {
            inside = 0;
          }
        }
        if (inside && tin < tout) {
          if (n < cap) {
            hits[n].tin = tin;
            hits[n].x = x;
            hits[n].y = y;
            hits[n].z = z;
          }
          ++n;
        }
      }
  int64_t m = n < cap ? n : cap;
  qsort(hits, (size_t)m, sizeof(brute_hit), cmp_hit);
  int64_t count = 0;
  for (int64_t k = 0; k < m; ++k) {
    ++count;
    if (fn && fn(ctx, hits[k].x, hits[k].y, hits[k].z)) break;
  }
  free(hits);
  return count;
}

typedef int64_t (*orc_walk_fn)(const int32_t *, const float *, const float *, orc_visit_fn, void *);

static orc_walk_fn walk_of(int mode) {
  return mode == ORC_WALK_F64 ? orc_walk_f64 : (mode == ORC_WALK_BRUTE ? orc_walk_brute : orc_walk_f32);
}

/* Smallest gap, in segment parameter t, between two events of the walk that
 * an exact and a rounded walk might order differently: plane crossings of
 * two different axes (the ray passes near a voxel edge or corner), or a
 * plane crossing and the clip parameters t_min / t_max (the ray enters near
 * an edge, or ends near a plane).  FP64; +inf when there is no such pair. */
double orc_min_tie_gap(const int32_t dims[3], const float of[3], const float df[3]) {
  double o[3] = {of[0], of[1], of[2]}, d[3] = {df[0], df[1], df[2]};
  double tmin = 0.0, tmax = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (d[a] != 0.0) {
      double t0 = (0.0 - o[a]) / d[a], t1 = ((double)dims[a] - o[a]) / d[a];
      double lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
      if (lo > tmin) tmin = lo;
      if (hi < tmax) tmax = hi;
    }
  }
  if (!(tmin < tmax)) return INFINITY;
  int64_t cap = (int64_t)dims[0] + dims[1] + dims[2] + 8, n = 0;
  brute_hit *c = (brute_hit *)malloc((size_t)cap * sizeof(brute_hit));
  if (!c) return -1.0;
  for (int a = 0; a < 3; ++a) {
    if (d[a] == 0.0) continue;
    double pa = o[a] + tmin * d[a], pb = o[a] + tmax * d[a];
    double lo = pa < pb ? pa : pb, hi = pa < pb ? pb : pa;
    for (double b = ceil(lo - 1e-6); b <= floor(hi + 1e-6) && n < cap - 2; b += 1.0) {
      c[n].tin = (b - o[a]) / d[a];
      c[n].x = a; /* event label: the axis */
      ++n;
    }
  }
  c[n].tin = tmin;
  c[n].x = 3;
  ++n;
  c[n].tin = tmax;
  c[n].x = 4;
  ++n;
  qsort(c, (size_t)n, sizeof(brute_hit), cmp_hit);
  double best = INFINITY;
  for (int64_t k = 1; k < n; ++k) {
    if (c[k].x == c[k - 1].x) continue;
    double g = c[k].tin - c[k - 1].tin;
    /* a clip event coincides exactly with the face crossing that defines it */
    if (g == 0.0 && (c[k].x >= 3 || c[k - 1].x >= 3)) continue;
    if (g < best) best = g;
  }
  free(c);
  return best;
}

/* ------------------------------------------------------------------------ */
/* Gain (Eq. 2 and variants).                                                */
/* ------------------------------------------------------------------------ */

/* Binary entropy in bits; H(0) = H(1) = 0. */
double orc_entropy(double p) {
  if (!(p > 0.0 && p < 1.0)) return 0.0;
  return -p * log2(p) - (1.0 - p) * log2(1.0 - p);
}

/* Gain g(v) of one voxel and whether it is occupied (ends the ray).
 * Eq. 2: occupied -> 1 - P(v); free -> P(v); unknown -> 1. */
void orc_voxel_gain(const orc_map *m, int64_t idx, const orc_params *prm, double *g, int *occupied) {
  if (m->encoding == ORC_U8_STATE) {
    uint8_t s = ((const uint8_t *)m->data)[idx];
    *occupied = s >= 2;
    *g = s == 0 ? 1.0 : 0.0; /* state maps carry no P(v): count unknown voxels */
    return;
  }
  float p = ((const float *)m->data)[idx];
  int occ = p > prm->occ_threshold;
  int fre = p < prm->free_threshold;
  *occupied = occ;
  switch (prm->metric) {
    case ORC_PAPER_EQ2:
      *g = occ ? 1.0 - (double)p : (fre ? (double)p : 1.0);
      break;
    case ORC_ENTROPY:
      *g = orc_entropy((double)p);
      break;
    default:
      *g = (!occ && !fre) ? 1.0 : 0.0;
      break;
  }
}

typedef struct {
  const orc_map *m;
  const orc_params *prm;
  double ig;
  int64_t steps;
} ray_acc;

static int visit_gain(void *ctx, int32_t x, int32_t y, int32_t z) {
  ray_acc *acc = (ray_acc *)ctx;
  int64_t idx = ((int64_t)z * acc->m->ny + y) * acc->m->nx + x;
  double g;
  int occ;
  orc_voxel_gain(acc->m, idx, acc->prm, &g, &occ);
  acc->steps += 1;
  if (occ) {
    if (acc->prm->include_hit) acc->ig += g;
    return 1;
  }
  acc->ig += g;
  return 0;
}

/* Ray IG g_R and voxel steps (visited voxels, the occluding one included). */
void orc_ray_ig(const orc_map *m, const float o[3], const float d[3], const orc_params *prm, int walk,
                double *ig, int64_t *steps) {
  int32_t dims[3] = {m->nx, m->ny, m->nz};
  ray_acc acc = {m, prm, 0.0, 0};
  walk_of(walk)(dims, o, d, visit_gain, &acc);
  *ig = acc.ig;
  *steps = acc.steps;
}

/* Per-ray IG and steps for explicit segments o[n][3], d[n][3]. */
void orc_segments_ig(const orc_map *m, const float *o, const float *d, int64_t n, const orc_params *prm,
                     int walk, double *ig, int64_t *steps) {
  for (int64_t k = 0; k < n; ++k) orc_ray_ig(m, o + 3 * k, d + 3 * k, prm, walk, ig + k, steps + k);
}

typedef struct {
  int64_t *out;
  int64_t cap, n;
  int32_t nx, ny;
} trace_ctx;

static int visit_trace(void *ctx, int32_t x, int32_t y, int32_t z) {
  trace_ctx *t = (trace_ctx *)ctx;
  if (t->n < t->cap) t->out[t->n] = ((int64_t)z * t->ny + y) * t->nx + x;
  t->n += 1;
  return 0;
}

/* The whole voxel sequence of a segment (no occlusion), linear indices. */
int64_t orc_trace(const int32_t dims[3], const float o[3], const float d[3], int walk, int64_t *out,
                  int64_t cap) {
  trace_ctx t = {out, cap, 0, dims[0], dims[1]};
  walk_of(walk)(dims, o, d, visit_trace, &t);
  return t.n;
}

typedef struct {
  trace_ctx t;
  ray_acc acc;
} trace_occ_ctx;

static int visit_trace_occ(void *ctx, int32_t x, int32_t y, int32_t z) {
  trace_occ_ctx *c = (trace_occ_ctx *)ctx;
  visit_trace(&c->t, x, y, z);
  return visit_gain(&c->acc, x, y, z);
}

/* The voxel sequence of a segment up to and including the first occupied
 * voxel (what the IG sum visits). */
int64_t orc_trace_occluded(const orc_map *m, const float o[3], const float d[3], const orc_params *prm,
                           int walk, int64_t *out, int64_t cap) {
  int32_t dims[3] = {m->nx, m->ny, m->nz};
  trace_occ_ctx c = {{out, cap, 0, m->nx, m->ny}, {m, prm, 0.0, 0}};
  walk_of(walk)(dims, o, d, visit_trace_occ, &c);
  return c.t.n;
}

/* All rays of one perspective, ray k = j * W + i: o[k][3], d[k][3]. */
void orc_view_rays(const orc_map *m, const orc_camera *cam, const float *pose, float *o, float *d) {
  orc_cam_consts cc;
  orc_camera_consts(cam, &cc);
  for (int32_t j = 0; j < cam->height; ++j)
    for (int32_t i = 0; i < cam->width; ++i) {
      int64_t k = (int64_t)j * cam->width + i;
      orc_view_ray_f32(m, &cc, pose, i, j, o + 3 * k, d + 3 * k);
    }
}

/* Perspective IG: the sum over the N_E rays, or the mean g_P (Section III). */
static void view_ig(const orc_map *m, const orc_camera *cam, const orc_cam_consts *cc, const float *pose,
                    const orc_params *prm, int walk, double *ig, int64_t *steps) {
  double sum = 0.0;
  int64_t st = 0;
  for (int32_t j = 0; j < cam->height; ++j)
    for (int32_t i = 0; i < cam->width; ++i) {
      float o[3], d[3];
      double g;
      int64_t s;
      orc_view_ray_f32(m, cc, pose, i, j, o, d);
      orc_ray_ig(m, o, d, prm, walk, &g, &s);
      sum += g;
      st += s;
    }
  int64_t ne = (int64_t)cam->width * cam->height;
  *ig = (prm->reduce == ORC_REDUCE_MEAN && ne > 0) ? sum / (double)ne : sum;
  *steps = st;
}

typedef struct {
  const orc_map *m;
  const orc_camera *cam;
  const float *poses;
  const orc_params *prm;
  int walk;
  int64_t begin, end;
  double *ig;
  int64_t *steps;
} view_job;

static void *view_worker(void *arg) {
  view_job *jb = (view_job *)arg;
  orc_cam_consts cc;
  orc_camera_consts(jb->cam, &cc);
  for (int64_t v = jb->begin; v < jb->end; ++v)
    view_ig(jb->m, jb->cam, &cc, jb->poses + 7 * v, jb->prm, jb->walk, jb->ig + v, jb->steps + v);
  return NULL;
}

/* IG of n_views perspectives, split over n_threads host threads by
 * contiguous view ranges.  Returns 0, or -1 if a thread could not start. */
int orc_views_ig(const orc_map *m, const float *poses, int64_t n_views, const orc_camera *cam,
                 const orc_params *prm, int walk, int n_threads, double *ig, int64_t *steps) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > n_views) n_threads = n_views > 0 ? (int)n_views : 1;
  view_job *jobs = (view_job *)calloc((size_t)n_threads, sizeof(view_job));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return -1;
  }
  int rc = 0;
  for (int t = 0; t < n_threads; ++t) {
    jobs[t] = (view_job){m, cam, poses, prm, walk, n_views * t / n_threads, n_views * (t + 1) / n_threads,
                         ig, steps};
  }
  int started = 0;
  for (int t = 1; t < n_threads; ++t) {
    if (pthread_create(&th[t], NULL, view_worker, &jobs[t]) != 0) {
      rc = -1;
      break;
    }
    started = t;
  }
  view_worker(&jobs[0]);
  for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
  if (rc != 0) /* finish the ranges of threads that did not start */
    for (int t = started + 1; t < n_threads; ++t) view_worker(&jobs[t]);
  free(jobs);
  free(th);
  return 0;
}

/* Trajectory IG: the sum of the perspective IGs of poses
 * offsets[t] .. offsets[t+1]-1, for each trajectory t. */
int orc_traj_ig(const orc_map *m, const float *poses, const int32_t *offsets, int32_t n_traj,
                const orc_camera *cam, const orc_params *prm, int walk, int n_threads, double *traj_ig,
                int64_t *traj_steps) {
  int64_t n_poses = n_traj > 0 ? offsets[n_traj] : 0;
  double *pig = (double *)malloc((size_t)(n_poses > 0 ? n_poses : 1) * sizeof(double));
  int64_t *pst = (int64_t *)malloc((size_t)(n_poses > 0 ? n_poses : 1) * sizeof(int64_t));
  if (!pig || !pst) {
    free(pig);
    free(pst);
    return -1;
  }
  int rc = orc_views_ig(m, poses, n_poses, cam, prm, walk, n_threads, pig, pst);
  for (int32_t t = 0; t < n_traj; ++t) {
    double s = 0.0;
    int64_t st = 0;
    for (int32_t k = offsets[t]; k < offsets[t + 1]; ++k) {
      s += pig[k];
      st += pst[k];
    }
    traj_ig[t] = s;
    traj_steps[t] = st;
  }
  free(pig);
  free(pst);
  return rc;
}
