/*
 * nbt.h -- C ABI of the GB300 information-gain (IG) raycasting library.
 *
 * The library computes the Online Local Information Distribution of the
 * paper's Section III: for each camera perspective around a point of
 * interest, N_E rays are cast from the perspective p_P to endpoints p_E on
 * the far frustum plane ("Endpoint Calculation"), each ray sums the per-voxel
 * gains g(v_i) of Eq. 2 over the voxels it crosses up to and including the
 * first occupied voxel ("IG Calculation", N_O), and the ray IGs are reduced
 * to one value per perspective (the sum, or the mean g_P of Section III).
 * Trajectory IG adds the perspective IGs of each pose sequence.
 *
 * Conventions (all entry points):
 *   - Every function returns an int status: NBT_OK (0) or a negative NBT_E*
 *     code; nbt_status_string() names it.  No C++ exception crosses the ABI.
 *   - Arguments are validated on the host before anything is enqueued; a
 *     call that returns an error has enqueued no work.
 *   - "device" pointers are CUDA global-memory pointers on the device the
 *     map was created on, which must be the current device of the calling
 *     thread.  The caller owns every pointer it passes; the library keeps
 *     none beyond the call, except what a handle owns (maps, ID buffers,
 *     surrogates) and the buffers a trajectory plan captures.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous: results are valid once the stream has
 *     reached the call.  Calls do not synchronise, except where a
 *     function's comment says so: uploads from pageable host memory (CUDA
 *     copies pageable memory synchronously), destroying a map, ID buffer or
 *     surrogate (so no enqueued call still reads it), creating a
 *     trajectory plan, reading the tensor-core error word and copying
 *     surrogate parameters to or from the host.
 *   - A map handle may be used from several host threads; calls that read
 *     it may overlap on different streams, but an upload must not overlap
 *     with calls that read the same map.
 *
 * Geometry: voxel (x, y, z) covers [origin + x*s, origin + (x+1)*s) on x and
 * likewise on y and z (s = voxel size).  Dense host/device grids are
 * x-fastest: linear index (z * ny + y) * nx + x.  A pose is the camera
 * position (world metres) and the unit quaternion (w, x, y, z) of the
 * camera-to-world rotation; camera +z is the optical axis, +x right, +y down.
 *
 * Traversal: every ray is walked in FP32 by the reference operation order
 * documented in nbt_trace_segments (bit-exact with the project's CPU
 * reference walk); gains are accumulated in FP32 per ray, per-perspective
 * sums in FP64, and returned as float.
 */
#ifndef NBT_H
#define NBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NBT_API_VERSION 1

/* Status codes. */
#define NBT_OK 0
#define NBT_EINVAL (-1)          /* an argument is invalid (NULL, size, range, mismatch) */
#define NBT_ENOMEM (-2)          /* device or host allocation failed */
#define NBT_ECUDA (-3)           /* a CUDA runtime call or kernel launch failed */
#define NBT_ETIMEOUT (-4)        /* a bounded device-side wait gave up */
#define NBT_EUNSUPPORTED (-5)    /* valid but unsupported combination (e.g. Eq. 2 on a state map) */
#define NBT_EWORKSPACE (-6)      /* workspace missing or smaller than nbt_workspace_size() */
#define NBT_ESCRATCH (-7)        /* request larger than the fixed scratch of nbt_views_ig_noalloc */

/* Map encodings (voxel payload stored on the device). */
#define NBT_U8_STATE 0           /* uint8 state per voxel: 0 unknown, 1 free, >= 2 occupied */
#define NBT_F32_PROB 1           /* float occupancy probability P(v) per voxel */
#define NBT_U2_STATE 2           /* states packed 4 per byte (2 bits; 3 reads as occupied) */

/* IG metrics (per-voxel gain g(v), Section III). */
#define NBT_COUNT_UNKNOWN 0      /* g = 1 if unknown, else 0 */
#define NBT_PAPER_EQ2 1          /* Eq. 2: 1 - P occupied, P free, 1 unknown (F32 maps only) */
#define NBT_ENTROPY 2            /* g = H(P) in bits (F32 maps only) */

#define NBT_REDUCE_SUM 0         /* per-perspective IG = sum over the N_E rays */
#define NBT_REDUCE_MEAN 1        /* per-perspective IG = g_P = sum / N_E (Section III) */

#define NBT_GRID_CORNERS 0       /* endpoint grid includes the four border rays (paper) */
#define NBT_GRID_CENTERS 1       /* endpoint grid at pixel centres */

#define NBT_RANGE_PLANAR 0       /* endpoints on the far plane at d_Cam (paper) */
#define NBT_RANGE_SPHERICAL 1    /* every ray has length d_Cam */

typedef struct nbt_map_s *nbt_map; /* opaque; owns the device copy of the map */

/* Map description.  Each of nx, ny, nz in [1, 2048]; nx*ny*nz < 2^31.
 * brick: the device layout -- 1 (linear x-fastest, the default; 0 selects
 * it too) or 4 / 8 (cubic bricks of that edge in Morton order; see
 * nbt_map_create). */
typedef struct {
  int32_t nx, ny, nz;
  float voxel_size;              /* s_Vox, metres, > 0 */
  float origin[3];               /* world position of the map's min corner */
  int32_t encoding;              /* NBT_U8_STATE | NBT_F32_PROB | NBT_U2_STATE */
  int32_t brick;                 /* 0 or 1 (linear), 4 or 8 (Morton bricks) */
} nbt_map_desc;

/* Camera pose: 28 bytes, arrays of poses are tightly packed. */
typedef struct {
  float pos[3];                  /* p_P, world metres */
  float quat[4];                 /* camera-to-world rotation, (w, x, y, z), unit */
} nbt_pose;

/* Camera: W x H rays per perspective (N_E = W * H), opening angles FoV_h,
 * FoV_v and range d_Cam (Section III "Endpoint Calculation": half extents
 * d_h = d_Cam tan(FoV_h / 2), d_v = d_Cam tan(FoV_v / 2)). */
typedef struct {
  int32_t width, height;         /* each in [1, 65535] */
  float fov_h, fov_v;            /* full angles, radians, in (0, pi) */
  float max_range;               /* d_Cam, metres, > 0 */
  int32_t grid_mode;             /* NBT_GRID_CORNERS | NBT_GRID_CENTERS */
  int32_t range_mode;            /* NBT_RANGE_PLANAR | NBT_RANGE_SPHERICAL */
} nbt_camera;

/* IG parameters. */
typedef struct {
  int32_t metric;                /* NBT_COUNT_UNKNOWN | NBT_PAPER_EQ2 | NBT_ENTROPY */
  float occ_threshold;           /* F32 maps: occupied iff P > occ_threshold (e.g. 0.7) */
  float free_threshold;          /* F32 maps: free iff P < free_threshold (e.g. 0.3) */
  int32_t include_hit;           /* 1: the first occupied voxel adds its gain (sum to N_O) */
  int32_t reduce;                /* NBT_REDUCE_SUM | NBT_REDUCE_MEAN */
} nbt_ig_params;

/* Name of a status code (static string, never NULL). */
const char *nbt_status_string(int status);

/* Library ABI version (NBT_API_VERSION) into *version. */
int nbt_get_version(int32_t *version);

/* Create a map on the current device and allocate its device storage
 * (zero-filled: all voxels unknown / P = 0).  Layout: linear x-fastest
 * (brick 1; a voxel step adds a fixed stride -- the fastest layout on GB300
 * because the whole map stays L2-resident), or B^3 bricks (B = 4 or 8) in
 * Morton (Z) order of their brick coordinates, addressed through per-axis
 * offset tables (a voxel's offset is the sum of three table entries).
 * Ownership of the handle passes to the caller, who releases it with
 * nbt_map_destroy.  Errors: NBT_EINVAL (desc out of range), NBT_ENOMEM,
 * NBT_ECUDA. */
int nbt_map_create(const nbt_map_desc *desc, nbt_map *out);

/* Release a map and its device memory (synchronises the device first so no
 * enqueued call still reads it).  NULL is accepted and ignored; a handle that
 * names no live map (already destroyed) returns NBT_EINVAL.  Every other
 * call that takes a map handle also returns NBT_EINVAL for such a handle. */
int nbt_map_destroy(nbt_map map);

/* Upload a dense x-fastest grid (the paper's voxel map, Section III) into
 * the map's bricked device layout.  src holds nx*ny*nz elements: uint8
 * states for NBT_U8_STATE and NBT_U2_STATE maps, float probabilities for
 * NBT_F32_PROB maps; bytes must equal that size.  src_on_device: 1 if src is
 * a device pointer, 0 for host memory (copied in slabs through a staging
 * buffer the map owns).  Asynchronous on `stream`; invalidates derived gain
 * tables.  Host src: pageable memory has been read when the call returns;
 * page-locked memory is read when the stream reaches the copy, so it must
 * stay valid until then.  The staging buffer is shared by the map's uploads:
 * issue uploads of one map on one stream.  Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_map_upload(nbt_map map, const void *src, int64_t bytes, int32_t src_on_device, void *stream);

/* Description and device bytes held by the map (either output may be NULL). */
int nbt_map_info(nbt_map map, nbt_map_desc *desc, int64_t *device_bytes);

/* Copy the map back out as the dense x-fastest grid nbt_map_upload takes:
 * uint8 states (2-bit maps unpacked to 0..3) or float probabilities, into
 * the device buffer dst of exactly nx*ny*nz elements (bytes must match).
 * Asynchronous on stream.  Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_map_download(nbt_map map, void *dst, int64_t bytes, void *stream);

/* Occupancy update from one depth scan (Section III: every captured point
 * cloud is voxel-filtered and inserted into the probabilistic voxel map),
 * in the discrete form of occupancy-grid insertion:
 *   - voxel filter: each point stands for the voxel that contains it; every
 *     distinct such voxel inside the map is observed occupied once ("hit");
 *   - free space: a ray from the sensor to the centre of each distinct
 *     endpoint voxel (inside the map or not), walked with the FP32 reference
 *     walk of nbt_trace_segments and clipped to the map, observes every voxel
 *     it visits free ("miss"), at most once per scan; a voxel that is also a
 *     hit in the scan takes only the hit;
 *   - NBT_F32_PROB maps: P <- P p / (P p + (1 - P)(1 - p)) with p = prob_hit
 *     or prob_miss, each operation rounded in FP32 in this order, then
 *     clamped to [clamp_min, clamp_max]; state maps: hit -> 2 (occupied),
 *     miss -> 1 (free).
 * Points that are not finite, farther than max_range from the sensor (if
 * max_range > 0) or 2^22 voxels or more from the map origin on an axis are
 * ignored.  points: device float[n][3], world metres; sensor: host float[3]
 * (within 2^22 voxels of the origin); stats_out: NULL or device uint64[3],
 * written with the number of distinct endpoint voxels inside the map (hits),
 * the number of rays cast and the number of voxel steps they walked.  Only the linear layout (brick 1) is
 * supported (NBT_EUNSUPPORTED otherwise).  The map allocates its insertion
 * scratch on the first call and when n exceeds every earlier n (two voxel
 * bitmaps and endpoint lists; cudaMalloc synchronises); inserts into one map
 * must be ordered on one stream.  Derived gains of an FP32 map are rebuilt
 * before its next IG call.  Errors: NBT_EINVAL, NBT_EUNSUPPORTED,
 * NBT_ENOMEM, NBT_ECUDA. */
typedef struct {
  float prob_hit;                /* p_hit in (0.5, 1), e.g. 0.7 */
  float prob_miss;               /* p_miss in (0, 0.5), e.g. 0.4 */
  float clamp_min, clamp_max;    /* 0 < clamp_min < clamp_max < 1, e.g. 0.1192, 0.971 */
  float max_range;               /* metres; <= 0: no range limit */
} nbt_insert_params;

int nbt_map_insert_points(nbt_map map, const float *points, int64_t n, const float *sensor,
                          const nbt_insert_params *params, uint64_t *stats_out, void *stream);

/* The paper's endpoint grid for grid factor s_G (Section III "Endpoint
 * Calculation": corner rays on the far plane at d_Cam, grid spacing
 * s_G * s_Vox): fills *cam with fov_h, fov_v, max_range, corner grid mode,
 * planar range and
 *   width  = max(2, floor((2 d_h) / (s_G s_Vox)) + 1),  d_h = d_Cam tan(fov_h / 2),
 *   height = max(2, floor((2 d_v) / (s_G s_Vox)) + 1),  d_v = d_Cam tan(fov_v / 2),
 * evaluated in FP64 from the float arguments: the densest grid whose
 * spacing is not finer than s_G s_Vox.  Host only.  Errors: NBT_EINVAL
 * (an argument not finite and positive, a FoV not below pi, a side above
 * 65535). */
int nbt_camera_from_grid_scale(float fov_h, float fov_v, float max_range, float voxel_size, float grid_scale,
                               nbt_camera *cam);

/* Device workspace, in bytes, that nbt_views_ig / nbt_traj_ig need for
 * n_poses perspectives of camera `cam` (per-tile partial sums).  The caller
 * allocates it (any device allocator) and passes it to those calls; it may
 * be reused by calls that do not overlap on the device.  Errors: NBT_EINVAL
 * (n_poses outside [0, INT32_MAX], an invalid camera). */
int nbt_workspace_size(int64_t n_poses, const nbt_camera *cam, int64_t *bytes);

/* Per-perspective IG (Section III "IG Calculation"): for each of n_views
 * poses (device array), cast the W x H rays, sum g(v_i) along each ray to
 * the first occupied voxel, and reduce over rays (params->reduce).
 *   ig_out:    device float[n_views], written.
 *   steps_out: device uint64[n_views] or NULL: voxels visited per view
 *              (the occluding voxel included).
 *   workspace: device buffer of >= nbt_workspace_size(n_views, cam) bytes,
 *              16-byte aligned.
 * n_views in [0, INT32_MAX]; n_views == 0 is valid and enqueues nothing.
 * Errors: NBT_EINVAL, NBT_EUNSUPPORTED (Eq. 2 / entropy on a state map),
 * NBT_EWORKSPACE, NBT_ECUDA. */
int nbt_views_ig(nbt_map map, const nbt_pose *poses, int64_t n_views, const nbt_camera *cam,
                 const nbt_ig_params *params, float *ig_out, uint64_t *steps_out, void *workspace,
                 int64_t workspace_bytes, void *stream);

/* Trajectory IG: per trajectory t, the sum of the perspective IGs of poses
 * offsets[t] .. offsets[t+1]-1 (device int32 CSR offsets, n_traj + 1
 * entries, non-decreasing, offsets[0] == 0, offsets[n_traj] == n_poses).
 * Poses of all trajectories go through one persistent launch that takes
 * (pose, ray tile) items from a device work queue.
 *   traj_ig_out: device float[n_traj]; pose_ig_out: device float[n_poses]
 *   or NULL; workspace as for nbt_views_ig with n_poses perspectives.
 * Errors as for nbt_views_ig; NBT_EINVAL also if n_poses does not match. */
int nbt_traj_ig(nbt_map map, const nbt_pose *poses, int64_t n_poses, const int32_t *offsets, int32_t n_traj,
                const nbt_camera *cam, const nbt_ig_params *params, float *traj_ig_out, float *pose_ig_out,
                void *workspace, int64_t workspace_bytes, void *stream);

/* Test entry point: the voxels visited by n_rays explicit segments.
 * o, d: device float[n_rays][3], segment start and displacement in voxel
 * units (point o + t d, t in [0, 1], relative to the map's min corner).
 * The walk (Section III "IG Calculation": all voxels from p_P to p_E) runs
 * in FP32 in this fixed operation order, each operation rounded on its own:
 *   inv_a = 1 / d_a; clip t0 = (0 - o_a) inv_a, t1 = (N_a - o_a) inv_a,
 *   t_min = max(0, near), t_max = min(1, far), no voxel unless t_min < t_max;
 *   start p_a = o_a + t_min d_a, i_a = floor(clamp(p_a, 0, N_a - 1));
 *   next crossing t_a = ((float)(i_a + [d_a > 0]) - o_a) inv_a, recomputed
 *   from the index after each step; step x if t_x <= t_y and t_x <= t_z,
 *   else y if t_y <= t_z, else z; stop when that t is not < t_max or the
 *   index leaves the map.
 * params: NULL walks the whole segment; otherwise the walk also stops after
 * the first occupied voxel as the IG sum does.
 *   idx_out: device int32[n_rays][cap], linear voxel indices in visit order
 *            (entries past the count are left untouched);
 *   n_out:   device int32[n_rays], the number of visited voxels (may
 *            exceed cap; only cap are stored). */
int nbt_trace_segments(nbt_map map, const float *o, const float *d, int32_t n_rays, const nbt_ig_params *params,
                       int32_t *idx_out, int32_t cap, int32_t *n_out, void *stream);

/* Test entry point: the ray segments (voxel units, as nbt_trace_segments
 * takes them) that the IG kernels generate for every ray of n_views poses,
 * ray k = j * W + i of view v at row v * W * H + k.  Endpoint grid (Section
 * III): d_h, d_v in FP64 on the host; x_i = x_0 + i * x_step in FP32 with
 * x_0 = -d_h, x_step = 2 d_h / (W - 1) (corners) or x_0 = -d_h + d_h / W,
 * x_step = 2 d_h / W (centres), both rounded once to FP32; likewise y_j;
 * camera-frame direction (x_i, y_j, d_Cam), scaled to length d_Cam in the
 * spherical range mode; world direction R c with R from the quaternion;
 * o = (p_P - origin) / s and d = (R c) / s, with 1/s rounded once to FP32.
 *   o_out, d_out: device float[n_views * W * H][3]. */
int nbt_view_segments(nbt_map map, const nbt_pose *poses, int64_t n_views, const nbt_camera *cam, float *o_out,
                      float *d_out, void *stream);

/* CUDA-graph executor for repeated trajectory IG (the Section IV planner
 * re-scores candidate trajectories every cycle with unchanged shapes).
 * nbt_plan_create_traj captures one nbt_traj_ig call with exactly these
 * arguments (work-queue reset, the persistent tile kernel, the per-
 * trajectory reduction) into a CUDA graph; nbt_plan_launch replays it on
 * `stream`.  The graph keeps the pointers: the map and every buffer passed
 * here must stay alive until nbt_plan_destroy, and the caller may change the
 * contents of poses, offsets and the map between launches (not n_poses,
 * n_traj, the camera or the params).  A probability map's derived gains
 * are refreshed outside the graph when the map was re-uploaded.  Creating
 * a plan synchronises an internal stream; launching does not synchronise.
 * Errors: as nbt_traj_ig, plus NBT_ECUDA if capture fails; nbt_plan_launch
 * returns NBT_EINVAL (and launches nothing) once the plan's map has been
 * destroyed, even if a new map now lives at the same address. */
typedef struct nbt_plan_s *nbt_plan;
int nbt_plan_create_traj(nbt_map map, const nbt_pose *poses, int64_t n_poses, const int32_t *offsets, int32_t n_traj,
                         const nbt_camera *cam, const nbt_ig_params *params, float *traj_ig_out, float *pose_ig_out,
                         void *workspace, int64_t workspace_bytes, nbt_plan *out);
int nbt_plan_launch(nbt_plan plan, void *stream);
int nbt_plan_destroy(nbt_plan plan);

/* Launch tuning of the IG kernels for one map (chosen by the autotuner in
 * the Python package).  packet_w: width of a warp's ray packet in pixels,
 * 4, 8, 16 or 32 (height 32 / packet_w; 0 = default 8).  brick: read-only
 * in nbt_map_get_tuning (the brick edge is fixed at nbt_map_create).
 * skip: 1 (the default) lets walks on linear maps replace the voxel-by-voxel
 * walk through a uniform brick -- the largest cube of 8, 16, 32 or 64
 * voxels aligned to the map origin around the current voxel whose voxels
 * are all unknown or all free (state maps), or whose derived gains are all
 * exactly 1 or all exactly 0 (probability maps) -- by per-axis crossing
 * counts (used by calls with enough rays to fill the GPU); 0 always walks
 * voxel by voxel.  Only speed changes: every setting visits the same voxels
 * and returns the same unknown counts; FP32 gain sums may differ in their
 * rounding order (a brick's unit gains are added at once). */
typedef struct {
  int32_t packet_w;
  int32_t brick;
  int32_t skip;
} nbt_tuning;

/* Set / read a map's kernel tuning.  Errors: NBT_EINVAL. */
int nbt_map_set_tuning(nbt_map map, const nbt_tuning *tuning);
int nbt_map_get_tuning(nbt_map map, nbt_tuning *tuning);

/* Tensor-core GEMM behind the learned IG surrogate (the paper has no
 * learned component; the surrogate prunes candidate perspectives before the
 * exact Section III raycast re-scores them).  Test entry point:
 * c[m][n] = sum_k a[m][k] * b[n][k] with BF16 a (m x k) and b (n x k),
 * row-major, 16-byte aligned, k % 8 == 0, 1 <= n <= 256; FP32 c (m x n,
 * row-major), accumulated in FP32 by tcgen05 MMAs.  Device pointers.
 * Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_tc_gemm(const void *a, const void *b, float *c, int32_t m, int32_t n, int32_t k, void *stream);

/* The tensor-core kernels' device error word on the current device: 1 if a
 * bounded device-side wait gave up since the last read (then the results
 * of that launch are invalid).  Synchronises; reading clears the word. */
int nbt_tc_error(int32_t *flag);

/* Bound, in nanoseconds of the GPU's global timer, on every device-side
 * mbarrier wait of the tensor-core kernels on the current device (default
 * 2 s).  A wait that reaches it gives up: the kernel sets the error word
 * (nbt_tc_error), waits (bounded again) for its own tensor-core operations
 * in flight, frees its tensor memory and returns, so the context stays
 * usable.  ns in [1e3, 6e10].  Synchronous (a copy to device constant
 * memory); do not change it while tensor-core kernels run.  Errors:
 * NBT_EINVAL, NBT_ECUDA. */
int nbt_tc_set_wait_limit(uint64_t ns);

/* Test entry point of that failure path (no counterpart in the paper): on
 * every SM, a CTA takes all 512 tensor-memory columns and waits on an
 * mbarrier that nothing completes; when the bounded wait gives up it sets
 * the error word, frees the columns and returns.  The launch therefore ends
 * after about the wait limit (shorten it first with nbt_tc_set_wait_limit)
 * and leaves the error word set.  Asynchronous on stream.  Errors:
 * NBT_ECUDA. */
int nbt_tc_wait_probe(void *stream);

/* The learned IG surrogate (no counterpart in the paper; it prunes
 * candidate perspectives before the exact Section III raycast re-scores
 * them).  Input per perspective: a view-aligned crop -- 32 x 32 x 32
 * samples on the rays through the pixel centres of a 32 x 32 image of the
 * field of view, at depth fractions (k + 1/2) / 32 of d_Cam, each the class
 * of the voxel holding it as a uint8 code (0 outside the map, 1 unknown,
 * 2 free, 3 occupied), [n][32 (depth k)][32 (row j)][32 (column i)], the
 * array 16-byte aligned (every call that takes crops returns NBT_EINVAL
 * otherwise) -- and 8
 * BF16 pose features ((position - origin) / map extent, the quaternion, 1).
 * The network sees code c as the one-hot vector with a 1 in channel c - 1 of
 * 8 (all zero for code 0).  Output: the predicted mean ray IG (the training target
 * the caller chooses, e.g. g_P with a target scale of 0.01, see
 * nbt_surrogate_set_target_scale).  Network: 3^3 convolutions 8->16,
 * 16->32, 32->64 (stride 2) and 64->64 (stride 1), ReLU; 4096 + 8 -> 128
 * (ReLU) -> 1; BF16 weights and activations, FP32 accumulation on tcgen05
 * tensor cores, FP32 master weights, MSE loss, Adam. */
typedef struct nbt_surrogate_s *nbt_surrogate;

/* Number of FP32 parameters (the layout of set/get_params: per conv layer
 * W [C_out][27 C_in] (tap (dz*3+dy)*3+dx, then C_in) and b [C_out]; then
 * F1 [128][4104], g1 [128], f2 [128], g2 [1]). */
int nbt_surrogate_param_count(int64_t *n);

/* Create a network on the current device with activation buffers for up
 * to max_batch (1 .. 4096) samples per pass; parameters start at zero.
 * Also creates the side stream and events nbt_plan_pruned uses.
 * Errors: NBT_EINVAL, NBT_ENOMEM, NBT_ECUDA. */
int nbt_surrogate_create(int32_t max_batch, nbt_surrogate *out);
int nbt_surrogate_destroy(nbt_surrogate net);

/* Copy all parameters from / to host memory (n must equal the count);
 * set_params also resets the Adam state.  Synchronous. */
int nbt_surrogate_set_params(nbt_surrogate net, const float *host, int64_t n);
int nbt_surrogate_get_params(nbt_surrogate net, float *host, int64_t n);

/* Crops and pose features of n poses (device arrays as described above).
 * params supplies the occupancy thresholds of probability maps.
 * Asynchronous on stream. */
int nbt_surrogate_crops(nbt_map map, const nbt_pose *poses, int64_t n, const nbt_camera *cam,
                        const nbt_ig_params *params, void *crops, void *feats, void *stream);

/* Predictions (device float[n]) for n crops, in passes of max_batch. */
int nbt_surrogate_forward(nbt_surrogate net, const void *crops, const void *feats, int64_t n, float *pred,
                          void *stream);

/* Loss (mean squared error against targets) and its gradient w.r.t. every
 * parameter for one batch (n <= max_batch, n <= 1024), without updating.
 * grads_out: device float[count] or NULL; loss_out: device float or NULL. */
int nbt_surrogate_backward(nbt_surrogate net, const void *crops, const void *feats, const float *targets, int32_t n,
                           float *grads_out, float *loss_out, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on one batch. */
int nbt_surrogate_train_step(nbt_surrogate net, const void *crops, const void *feats, const float *targets, int32_t n,
                             float lr, float *loss_out, void *stream);

/* Scale c > 0 (finite) applied to the targets of nbt_surrogate_backward and
 * nbt_surrogate_train_step: the loss is mean (pred - c t)^2, with c t
 * rounded to FP32.  Default 1.  Lets the caller pass Section III's mean ray
 * IG g_P as the target while the network predicts g_P c (e.g. c = 0.01, so
 * that outputs are of order 1).  Host-side setting.  Errors: NBT_EINVAL. */
int nbt_surrogate_set_target_scale(nbt_surrogate net, float scale);

/* Checkpoint / resume of training: the Adam moments m and v (FP32 host
 * arrays in the parameter layout, n = the parameter count) and the number of
 * Adam steps taken.  Together with nbt_surrogate_get_params / set_params
 * (set_params first: it resets the Adam state) and the target scale they
 * are the whole training state, so training resumed from them continues
 * bit for bit.  Synchronous.  Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_surrogate_get_adam(nbt_surrogate net, float *m_host, float *v_host, int64_t n, int64_t *step);
int nbt_surrogate_set_adam(nbt_surrogate net, const float *m_host, const float *v_host, int64_t n, int64_t step);

/* Surrogate-pruned planning helpers.  Candidates come in segments of seg
 * perspectives (e.g. the views around one PoI); n % seg == 0.
 * nbt_segment_topk: for each segment, the global indices of its keep
 * highest scores (descending; ties to the lower index; NaN last), device
 * int32[n / seg][keep]; with poses / poses_out (both or neither) also the
 * kept poses, device nbt_pose[n / seg][keep].  seg <= 8192.
 * nbt_segment_argmax: for each segment the largest value and the index
 * that holds it (idx[position] if idx is given, else the position; ties
 * to the lowest index), device int32 / float[n / seg] (best_val nullable). */
int nbt_segment_topk(const float *scores, int64_t n, int32_t seg, int32_t keep, int32_t *idx_out, const nbt_pose *poses,
                     nbt_pose *poses_out, void *stream);
int nbt_segment_argmax(const float *values, const int32_t *idx, int64_t n, int32_t seg, int32_t *best_idx,
                       float *best_val, void *stream);

/* IG between perspectives (Section IV, paragraphs "Orientation Factor
 * O(x_k) and IG G(x_k)" with Eq. 3, and "Cost Function Extension").  An information distribution (ID) is one
 * set of N_P perspectives: start points p_P,j (metres, world frame) and
 * IGs g_P,j (e.g. the mean ray IG nbt_views_ig returns).  The buffer keeps
 * the N_B most recent IDs; a camera position x between perspectives gets
 *   G(x) = sum_{u=0}^{N_B-1} 1 / (N_B - u) * IDW_u(x),
 *   IDW_u(x) = sum_j g_P,j d_j^-p / sum_j d_j^-p,  d_j = |x - p_P,j|,
 * for the IDs u of the buffer, u = 0 the oldest.  With n < N_B IDs stored
 * the n IDs take u = N_B - n .. N_B - 1 (the newest always weighs 1).  A
 * position that coincides with start points (FP32 d_j^2 == 0) takes, for
 * that ID, the mean gain of those points; an empty ID adds nothing.
 * Arithmetic: FP32 per pair (rcp.approx for p = 2, else exp2f / log2f),
 * sums of 32 terms per lane folded into compensated FP32 totals, one IEEE
 * division per ID; an ID whose FP32 sums overflow (points very close to
 * the query, large p) is recomputed with FP64 weights and sums.  Positions
 * must be finite; distinct positions closer than about 1e-19 m (FP32 d^2
 * below the smallest normal float) read as coincident. */
typedef struct nbt_id_buffer_s *nbt_id_buffer;

/* Create an empty buffer of n_b (1 .. 32) IDs of up to max_views
 * (1 .. 1 << 20) perspectives each on the current device.
 * Errors: NBT_EINVAL, NBT_ENOMEM, NBT_ECUDA. */
int nbt_id_buffer_create(int32_t n_b, int32_t max_views, nbt_id_buffer *out);
int nbt_id_buffer_destroy(nbt_id_buffer buf);

/* Append one ID: n_views (0 .. max_views) perspectives, poses as device
 * nbt_pose[n_views] (the start point is the position; the rotation is not
 * used) and ig as device float[n_views].  When the buffer already holds n_b
 * IDs the oldest is dropped.  Asynchronous on stream: a query enqueued
 * later on the same stream sees the new ID; the bookkeeping (which slot is
 * oldest, how many perspectives each holds) is host-side and updated at
 * once.  Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_id_buffer_push(nbt_id_buffer buf, const nbt_pose *poses, const float *ig, int32_t n_views, void *stream);

/* Forget every ID (host-side; nothing is enqueued). */
int nbt_id_buffer_clear(nbt_id_buffer buf);

/* Number of IDs held (0 .. n_b). */
int nbt_id_buffer_count(nbt_id_buffer buf, int32_t *n_ids);

/* G(x) for n query poses (device nbt_pose[n]; positions used) with
 * distance power p = power (0 < power <= 8), written to device
 * float[n].  n == 0 enqueues nothing.  Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_idw_gain(nbt_id_buffer buf, const nbt_pose *poses, int64_t n, float power, float *gain_out, void *stream);

/* Parameters of the IG cost: distance power p, weight w_I >= 0 and the
 * epsilon of c_I (the paper uses 1e-7). */
typedef struct {
  float power;
  float w_info;
  float eps;
} nbt_cost_params;

/* IG cost of n_traj candidate trajectories (the states x_0 .. x_K of
 * trajectory t are the camera poses offsets[t] .. offsets[t+1]-1 of poses,
 * device int32 CSR offsets, n_traj + 1 entries, clamped to [0, n_poses]):
 *   O(x) = cos of the angle between the optical axis (camera +z) and the
 *          direction to poi, 0 when the PoI lies outside the field of view
 *          (camera-frame direction c: inside iff c_z > 0,
 *          |c_x| <= c_z tan(fov_h / 2), |c_y| <= c_z tan(fov_v / 2); the
 *          decision in FP32: c_k = (R_0k v_0 + R_1k v_1) + R_2k v_2, v =
 *          poi - position, R from the quaternion, each operation rounded,
 *          the tangents evaluated in FP64 on the host and rounded once);
 *   G(x) as nbt_idw_gain;
 *   term(x) = w_I / (O(x) G(x) + eps);  cost_out[t] = sum_k term(x_k)
 *   (per-trajectory sums in FP64, fixed order).
 * poi: host float[3].  gain_out, orient_out: device float[n_poses] or NULL;
 * term_out: device float[n_poses] (required); cost_out: device
 * float[n_traj].  Errors: NBT_EINVAL, NBT_ECUDA. */
int nbt_ig_cost(nbt_id_buffer buf, const nbt_pose *poses, int64_t n_poses, const int32_t *offsets, int32_t n_traj,
                const float *poi, float fov_h, float fov_v, const nbt_cost_params *params, float *gain_out,
                float *orient_out, float *term_out, float *cost_out, void *stream);

/* Surrogate-pruned next-best-view selection in one call.  n candidate
 * perspectives (device poses) in segments of seg (e.g. the candidates
 * around one PoI; n % seg == 0, 1 <= keep <= seg <= 8192, n <= INT32_MAX):
 *   1. crops and network scores of every candidate (nbt_surrogate_crops and
 *      nbt_surrogate_forward, in batches of the net's max_batch);
 *   2. per segment, the keep highest scores (nbt_segment_topk);
 *   3. the exact IG of those keep candidates (nbt_views_ig: Section III,
 *      Eq. 2 / the unknown count along the rays to N_O, reduced per params);
 *   4. per segment, the kept candidate of highest exact IG
 *      (nbt_segment_argmax; ties to the lowest candidate index).
 * Exact raycasting judges the kept candidates, so pruning may miss the
 * best view but never reports a wrong IG; keep = seg gives exactly the
 * choice of raycasting every candidate.  The surrogate is not part of the
 * paper.
 *   best_out:    device int32[n / seg], global candidate index per segment;
 *   best_ig_out: device float[n / seg] or NULL, its exact IG;
 *   kept_out:    device int32[n / seg][keep] or NULL, the kept indices
 *                (descending score);
 *   workspace:   device buffer of >= nbt_pruned_workspace_size bytes,
 *                256-byte aligned, owned by the caller.
 * Allocates nothing; asynchronous on stream.  n == 0 enqueues nothing.
 * With more than one batch, the crops of the next batch run on the
 * network's own high-priority side stream while stream runs the current
 * batch's forward (event fork / join: the call is ordered on stream as a
 * whole).  A network
 * serves one call at a time (its buffers, side stream and events are its
 * own).
 * Errors: NBT_EINVAL, NBT_EUNSUPPORTED, NBT_EWORKSPACE, NBT_ECUDA. */
int nbt_pruned_workspace_size(nbt_surrogate net, int64_t n, int32_t seg, int32_t keep, const nbt_camera *cam,
                              int64_t *bytes);
int nbt_plan_pruned(nbt_map map, nbt_surrogate net, const nbt_pose *poses, int64_t n, int32_t seg, int32_t keep,
                    const nbt_camera *cam, const nbt_ig_params *params, int32_t *best_out, float *best_ig_out,
                    int32_t *kept_out, void *workspace, int64_t workspace_bytes, void *stream);

/* Size of the fixed device scratch array behind nbt_views_ig_noalloc. */
#define NBT_NOALLOC_SCRATCH_BYTES (4 << 20)

/* nbt_views_ig without any device allocation, for callers that cannot
 * allocate.  The paper has no counterpart; this is a deployment variant.
 *
 * Who needs it: code that must never call cudaMalloc -- a real-time
 * planning loop (the planner of the paper runs at 10 Hz) where a
 * cudaMalloc can synchronise the device and stall for milliseconds, a
 * host process whose device memory is already reserved by another
 * allocator or capped by a budget, or a plugin that is not allowed to
 * allocate inside its callbacks.  Such a caller cannot create the
 * workspace nbt_views_ig takes, so this entry point uses a file-scope
 * __device__ array of NBT_NOALLOC_SCRATCH_BYTES instead.  That array exists
 * on every device that loads the library and stays there until the
 * process exits.
 *
 * Arguments and results are those of nbt_views_ig, without the workspace
 * (the map, the poses and the outputs are still the caller's).  The request
 * must fit the array: n_views * ceil(W / 32) * ceil(H / 8) tiles, 16 bytes
 * each, plus a 256-byte header, at most NBT_NOALLOC_SCRATCH_BYTES (262,128
 * tiles, e.g. 3,495 views of 160 x 120 rays); larger requests (n_views is
 * bounded before any size is multiplied out) return NBT_ESCRATCH before
 * anything is enqueued -- split them into several calls.
 *
 * The first call on a device looks up the array's device address there
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  The address is kept per device and CUDA
 * context: after the device's context was destroyed and created again
 * (cudaDeviceReset), the next call looks it up anew, so that first call on
 * the new context too should come before any stream capture.  Every call on a device shares the one array
 * and clears the part that must start at zero itself; calls whose work
 * overlaps on the GPU (different streams, no ordering between them) race
 * on the array and give wrong results, so order them on one stream or with
 * events.  Errors as for nbt_views_ig, plus NBT_ESCRATCH. */
int nbt_views_ig_noalloc(nbt_map map, const nbt_pose *poses, int64_t n_views, const nbt_camera *cam,
                         const nbt_ig_params *params, float *ig_out, uint64_t *steps_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* NBT_H */
