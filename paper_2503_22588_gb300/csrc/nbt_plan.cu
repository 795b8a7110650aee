// nbt_plan.cu -- CUDA-graph executor for repeated trajectory IG.
//
// A moving-horizon planner (paper, Section IV) re-scores candidate
// trajectories every planning cycle (10 Hz in Section V) with the same
// shapes: same number of poses and trajectories, same camera.  A plan
// captures one nbt_traj_ig call (work-queue reset, the persistent tile
// kernel and the per-trajectory reduction) into a CUDA graph once; every
// planning cycle then costs one graph launch.  The graph reads the pose and
// offset buffers at launch time, so the caller refills them in place between
// launches; it also reads the map, so a re-uploaded map is picked up as well
// (a probability map's derived gains are refreshed before the graph runs).

#include <new>

#include "nbt_internal.cuh"

struct nbt_plan_s {
  nbt_map map = nullptr;
  uint64_t map_id = 0;  // the map's creation id: a destroyed map is detected at launch
  nbt_ig_params params;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

using namespace nbt;

extern "C" {

int nbt_plan_create_traj(nbt_map map, const nbt_pose *poses, int64_t n_poses, const int32_t *offsets, int32_t n_traj,
                         const nbt_camera *cam, const nbt_ig_params *params, float *traj_ig_out, float *pose_ig_out,
                         void *workspace, int64_t workspace_bytes, nbt_plan *out) {
  if (!out) return NBT_EINVAL;
  *out = nullptr;
  int rc = check_map(map);
  if (rc != NBT_OK) return rc;
  if (!params || !cam) return NBT_EINVAL;
  cudaStream_t s = nullptr;
  NBT_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  // derived gains are produced outside the graph (the graph must not re-derive them every cycle)
  PayloadKind kind;
  const void *payload = nullptr;
  rc = payload_kind(map, params, &kind, &payload);
  if (rc == NBT_OK && kind == PAYLOAD_GAIN_F32) rc = prepare_gain(map, params, s);
  if (rc == NBT_OK && map->skip) rc = prepare_bsum(map, s);  // built outside the graph, refreshed per launch
  if (rc == NBT_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = NBT_ECUDA;
  nbt_plan p = nullptr;
  if (rc == NBT_OK) {
    p = new (std::nothrow) nbt_plan_s();
    if (!p) rc = NBT_ENOMEM;
  }
  if (rc == NBT_OK) {
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      rc = NBT_ECUDA;
    } else {
      rc = nbt_traj_ig(map, poses, n_poses, offsets, n_traj, cam, params, traj_ig_out, pose_ig_out, workspace,
                       workspace_bytes, s);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(s, &g);
      if (rc == NBT_OK && (e != cudaSuccess || !g)) rc = NBT_ECUDA;
      if (rc == NBT_OK) {
        p->graph = g;
        if (cudaGraphInstantiate(&p->exec, g, 0) != cudaSuccess) rc = NBT_ECUDA;
      } else if (g) {
        cudaGraphDestroy(g);
      }
    }
  }
  (void)cudaGetLastError();
  cudaStreamDestroy(s);
  if (rc != NBT_OK) {
    if (p) {
      if (p->exec) cudaGraphExecDestroy(p->exec);
      if (p->graph) cudaGraphDestroy(p->graph);
      delete p;
    }
    return rc;
  }
  p->map = map;
  p->map_id = map->id;
  p->params = *params;
  *out = p;
  return NBT_OK;
}

int nbt_plan_launch(nbt_plan plan, void *stream) {
  if (!plan || !plan->exec) return NBT_EINVAL;
  if (!map_alive(plan->map, plan->map_id)) return NBT_EINVAL;  // the plan's map was destroyed
  int rc = check_map(plan->map);
  if (rc != NBT_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  PayloadKind kind;
  const void *payload = nullptr;
  rc = payload_kind(plan->map, &plan->params, &kind, &payload);
  if (rc != NBT_OK) return rc;
  // derived data (gains, brick summaries) are refreshed outside the graph: no-ops unless the map changed
  if (kind == PAYLOAD_GAIN_F32) rc = prepare_gain(plan->map, &plan->params, s);
  if (rc == NBT_OK && plan->map->skip) rc = prepare_bsum(plan->map, s);
  if (rc != NBT_OK) return rc;
  NBT_CUDA_TRY(cudaGraphLaunch(plan->exec, s));
  return NBT_OK;
}

int nbt_plan_destroy(nbt_plan plan) {
  if (!plan) return NBT_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  (void)cudaGetLastError();
  delete plan;
  return NBT_OK;
}

}  // extern "C"
