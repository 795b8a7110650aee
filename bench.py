"""Benchmark of the IG raycasting hot path on one or more GPUs.

Default workload ``room512-pruned`` (the headline: exact vs surrogate-pruned
next-best-view selection, same best view): per step one seeded 512^3 2-bit
room of 2000 primitives (40 % unknown) with 8 PoIs x 4096 candidate views of
320 x 240 rays.  The pruned arm uploads the map and runs nbt_plan_pruned
(surrogate scores of every candidate, the top 5 % per PoI raycast exactly,
the best of them); the exact arm raycasts every candidate (paper Section
III IG: unknown voxels along each ray up to the first occupied one).  The
surrogate is trained inside the run, before timing.  Other workloads
(``--workload``): prob256, exact64, traj256, room512, surrogate, idw_cost,
fig3, insert -- each step one pass of its path over one batch of input.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
       [--impl reference]
With N > 1 launch under torch.distributed.run: every rank processes its own
batch (replicas; no data-path collective), timings are reduced with a max.
"""

from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IG views/sec & voxel-steps/s at 1 GB300 (exact vs surrogate-pruned, same best view)"
L2_FLUSH_BYTES = 256 << 20
BYTES_PER_STEP = {"f32": 4.0, "u8": 1.0, "u2": 0.25}
SKIP_WALK_MIN_RAYS = 2 * 152 * 6 * 256   # rays per call above which linear maps take the skipping walk
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SOURCES = ["paper_2503_22588_gb300/csrc/nbt_raycast.cu", "paper_2503_22588_gb300/csrc/nbt_internal.cuh"]


def describe(w) -> str:
    return {
        "prob256": "prob256: 256^3 FP32 tabletop (200 primitives), 1024 views on a 0.3-0.8 m Fibonacci shell, "
                   "160x120 rays, entropy IG until p>0.7",
        "exact64": "exact64: 64^3 uint8 states (20 boxes/spheres, half unknown), 64 views on a 0.5 m sphere, "
                   "64x48 rays, unknown-voxel count",
        "room512": "room512: 512^3 2-bit states (2000 primitives, 40% unknown), 8 PoIs x 4096 views, "
                   "320x240 rays, unknown-voxel count",
        "traj256": "traj256: 256^3 uint8 tabletop, 512 trajectories of 5-40 poses around 4 PoIs, 128x96 rays, "
                   "trajectory IG = sum of per-pose unknown counts, one CUDA-graph replay per step",
        "idw_cost": "idw_cost: c_I of 16384 candidate trajectories x 31 states (3 s horizon, 0.1 s steps) against "
                    "N_B=10 buffered IDs of N_P=500 perspectives (Eq. 3, p=2, orientation factor, eps=1e-7)",
    }.get(w.name, w.name)


def kernel_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def load_peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The reference walk's lane operations per visited voxel (its FP32 operation order): the axis choice
# (3 comparisons), the chosen crossing (1 min) and its end test (1), the plane step (1 add), the
# crossing recomputed from the plane (1 sub + 1 mul), the element index step (1 add), the address
# and the payload read (2), the gain test and sum (2) and the occlusion test (1).  Unpacking 2-bit
# states is not counted.
WALK_OPS_PER_STEP = 14
ISSUE_LANES_PER_CLK_PER_SM = 128     # 4 schedulers x one 32-lane warp instruction per clock


def walk_alu_roofline(steps: float, ms: float, kernel: str) -> dict:
    """The walk against the instruction-issue bound that binds it: the reference walk's lane operations
    per voxel step x the launch's voxel steps, over the launch time, against the SMs' issue rate
    (uniform bricks resolved without stepping count their voxels' operations as done, as the gather
    roofline counts their bytes)."""
    peak = ISSUE_LANES_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9      # G lane-ops/s
    achieved = WALK_OPS_PER_STEP * steps / (ms * 1e-3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Glane-op/s", "frac": achieved / peak,
            "kernel": kernel,
            "algorithmic": f"{WALK_OPS_PER_STEP} lane ops per voxel step of the reference walk x {steps:.0f} steps",
            "peak_kind": f"derived: {ISSUE_LANES_PER_CLK_PER_SM} lane ops/clk/SM (4 schedulers x 32 lanes) x "
                         f"{SM_COUNT} SMs x {SM_MAX_MHZ:.0f} MHz"}


def ncu_traffic(workload: str):
    """DRAM bytes per launch (per forward of the batch, for the surrogate) from the committed ncu summary, if current."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    t = json.load(open(TRAFFIC_FILE)).get(workload)
    if not t or t.get("kernel_hash") != kernel_hash(t.get("sources", KERNEL_SOURCES)):
        return None
    return t.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"nbt_clocks_rank{index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [s for s in sm if s >= 0.5 * top] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest per-rank value over all ranks (the slowest rank sets the job's time)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, total_ms: float) -> float:
    """Whole-job units per second: every rank processes units_per_rank in at most total_ms."""
    return world * units_per_rank / (total_ms * 1e-3)


def build_workload(name: str, rank: int):
    from workload import configs
    if name == "idw_cost":
        return configs.idw_cost(seed=rank)
    return configs.WORKLOADS[name](seed=rank)


def cpu_baseline(w, budget_s: float = 12.0) -> dict:
    """The oracle as it stands (FP32 reference walk, FP64 sums) on a bounded sample of the workload."""
    import oracle
    threads = os.cpu_count() or 1
    m = oracle.Map(w.grid, w.voxel_size, w.origin)
    cam = oracle.camera_of(w.camera)
    prm = oracle.params(w.metric)
    n_cal = min(threads, w.n_poses)
    t0 = time.perf_counter()
    oracle.views_ig(m, w.poses[:n_cal], cam, prm, "f32", threads)
    t_cal = time.perf_counter() - t0
    n = int(min(w.n_poses, max(n_cal, n_cal * budget_s / max(t_cal, 1e-3))))
    n = max(threads, (n // threads) * threads) if n >= threads else n
    t0 = time.perf_counter()
    _, st = oracle.views_ig(m, w.poses[:n], cam, prm, "f32", threads)
    dt = time.perf_counter() - t0
    # one thread as well: the paper's CPU version was sequential
    n1 = int(max(1, min(w.n_poses, 0.5 * budget_s / max(t_cal / n_cal * threads, 1e-6))))
    t0 = time.perf_counter()
    _, st1 = oracle.views_ig(m, w.poses[:n1], cam, prm, "f32", 1)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": "views/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n} of {w.n_poses} views of the same workload ({int(st.sum())} voxel steps)",
            "voxel_steps_per_s": float(st.sum()) / dt,
            "single_thread": {"value": n1 / dt1, "unit": "views/s", "cores": 1,
                              "sample": f"first {n1} views ({int(st1.sum())} voxel steps)",
                              "voxel_steps_per_s": float(st1.sum()) / dt1}}


def traj_cpu_baseline(w, budget_s: float = 12.0) -> dict:
    """The oracle on a bounded sample of trajectories (all their poses)."""
    import oracle
    threads = os.cpu_count() or 1
    m = oracle.Map(w.grid, w.voxel_size, w.origin)
    cam = oracle.camera_of(w.camera)
    prm = oracle.params(w.metric)
    t0 = time.perf_counter()
    oracle.views_ig(m, w.poses[:threads], cam, prm, "f32", threads)
    per_pose = (time.perf_counter() - t0) / threads
    n_traj, n_poses = 0, 0
    while n_traj < len(w.offsets) - 1 and (n_poses + 1) * per_pose < budget_s:
        n_traj += 1
        n_poses = int(w.offsets[n_traj])
    t0 = time.perf_counter()
    _, st = oracle.traj_ig(m, w.poses[:n_poses], w.offsets[:n_traj + 1], cam, prm, "f32", threads)
    dt = time.perf_counter() - t0
    return {"value": n_poses / dt, "unit": "views/s", "cores": threads, "kind": "oracle",
            "sample": f"first {n_traj} of {len(w.offsets) - 1} trajectories ({n_poses} poses, {int(st.sum())} "
                      f"voxel steps)", "voxel_steps_per_s": float(st.sum()) / dt}


COST_METRIC = "IG cost states/s (Eq. 3 interpolation + orientation factor + c_I per candidate trajectory)"
MUFU_PER_CLK_PER_SM = 16     # reciprocal / log2 / exp2 results per SM per clock
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def cost_cpu_sample(w, n_traj: int):
    """Run the oracle's c_I on the first n_traj trajectories; returns (seconds, states)."""
    from oracle import idw as I
    ids = [(pz[:, :3].astype(np.float64), g.astype(np.float64)) for pz, g in w.ids]
    n = int(w.offsets[n_traj])
    t0 = time.perf_counter()
    I.ig_cost(w.poses[:n], w.offsets[:n_traj + 1], w.poi.astype(np.float64), w.fov_h, w.fov_v, ids, w.n_b, w.power,
              w.w_info, w.eps)
    return time.perf_counter() - t0, n


def cost_cpu_baseline(w, budget_s: float = 12.0) -> dict:
    """The oracle as it stands (FP64 numpy, one host thread) on a bounded sample of trajectories."""
    dt1, _ = cost_cpu_sample(w, 1)
    n_traj = int(max(1, min(len(w.offsets) - 1, budget_s / max(dt1, 1e-4))))
    dt, n = cost_cpu_sample(w, n_traj)
    return {"value": n / dt, "unit": "states/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n_traj} of {len(w.offsets) - 1} trajectories ({n} states)"}


def run_reference_cost(args) -> None:
    w = build_workload("idw_cost", 0)
    dt1, _ = cost_cpu_sample(w, 1)
    per_step_s = min(8.0, 120.0 / max(1, args.steps + args.warmup))
    n_traj = int(max(1, min(len(w.offsets) - 1, per_step_s / max(dt1, 1e-4))))
    for _ in range(args.warmup):
        cost_cpu_sample(w, n_traj)
    times = [cost_cpu_sample(w, n_traj) for _ in range(args.steps)]
    total = sum(t for t, _ in times)
    n = times[0][1]
    value = n * args.steps / total
    line = {"impl": "reference", "metric": COST_METRIC, "value": value, "unit": "states/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(w), "states_per_step": n, "parallelism": "one host thread"},
            "cpu_baseline": {"value": value, "unit": "states/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {n_traj} trajectories ({n} states) per step"},
            "e2e": {"value": value, "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_step_budget(args) -> float:
    """Seconds of oracle work per step, so that warmup + steps end within about two minutes."""
    return min(8.0, 120.0 / max(1, args.steps + args.warmup))


def timed_reference(args, fn) -> float:
    """args.warmup untimed calls of fn, then the total seconds of args.steps timed calls."""
    for _ in range(args.warmup):
        fn()
    total = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        fn()
        total += time.perf_counter() - t0
    return total


def reference_line(args, metric: str, value: float, unit: str, higher_is_better: bool, total_s: float,
                   config: dict, cores: int, sample: str) -> dict:
    return {"impl": "reference", "metric": metric, "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / max(1, args.steps),
            "higher_is_better": higher_is_better, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config,
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference_insert(args, budget_s: float | None = None) -> dict:
    """The oracle's map update (one host thread) on the first scans of the insert workload."""
    from oracle import insert as I
    from workload import configs
    scans, n, vs = configs.insert_scans(seed=0)
    budget_s = reference_step_budget(args) if budget_s is None else budget_s
    grid0 = np.full((n, n, n), 0.5, np.float32)
    t0 = time.perf_counter()
    I.insert(grid0, scans[0][1], scans[0][0][:3], vs)
    k = int(max(1, min(len(scans), budget_s / max(time.perf_counter() - t0, 1e-3))))

    def step():
        g = grid0
        for pose, p in scans[:k]:
            g = I.insert(g, p, pose[:3], vs)

    total = timed_reference(args, step)
    pts = sum(len(p) for _, p in scans[:k])
    value = pts * args.steps / total
    return reference_line(args, INSERT_METRIC, value, "points/s", True, total,
                          {"workload": f"insert: 640x576 depth scans into a {n}^3 FP32 map",
                           "points_per_step": pts, "parallelism": "one host thread"},
                          1, f"the first {k} of {len(scans)} scans ({pts} points) per step, from a fresh map")


def run_reference_fig3(args) -> dict:
    """The oracle on the paper's chosen ID (s_G 100, N_P 500): ms per ID, lower is better."""
    import oracle
    from oracle.endpoints import grid_size as orc_grid
    from workload import configs
    grid, _, poses = configs.fig3_scene(seed=0)
    fov_h, fov_v = math.radians(60.0), math.radians(45.0)
    m = oracle.Map(grid, configs.VOXEL, (0.0, 0.0, 0.0))
    prm = oracle.params("eq2", reduce="mean")
    ow, oh = orc_grid(fov_h, fov_v, 1.0, configs.VOXEL, 100)
    cam = oracle.camera(ow, oh, fov_h, fov_v, 1.0)
    threads = os.cpu_count() or 1
    total = timed_reference(args, lambda: oracle.views_ig(m, poses[:500], cam, prm, "f32", threads))
    value = 1e3 * total / max(1, args.steps)
    return reference_line(args, FIG3_METRIC, value, "ms", False, total,
                          {"workload": "fig3: 256^3 FP32 tabletop, N_P 500 perspectives by Eq. 1 (r_S = 1 m), "
                                       f"s_G 100 ({ow}x{oh} rays), d_Cam 1 m, Eq. 2 mean IG",
                           "parallelism": "host threads"},
                          threads, "the whole ID (500 perspectives) per step")


def run_reference_surrogate(args, budget_s: float | None = None) -> dict:
    """The oracle's crop (FP32 sample arithmetic) and FP64 forward on candidate views of the tabletop."""
    from oracle import surrogate as S
    from workload import configs, poses as wp
    w = configs.traj256(seed=0)
    cc = S.crop_consts(math.radians(60.0), math.radians(45.0), 1.0)
    params = {k: np.asarray(v, np.float64) for k, v in S.init_params(0).items()}
    pz = np.concatenate([wp.shell_views(p, 4096, 0.3, 0.8, k) for k, p in enumerate(w.pois)])
    budget_s = reference_step_budget(args) if budget_s is None else budget_s

    def views(k):
        cr, ft = zip(*(S.frustum_crop(w.grid, w.voxel_size, w.origin, pz[i], cc) for i in range(k)))
        S.forward(params, np.stack(cr).astype(np.float64), np.stack(ft), bf16_activations=True)

    t0 = time.perf_counter()
    views(1)
    k = int(max(1, min(len(pz), budget_s / max(time.perf_counter() - t0, 1e-3))))
    total = timed_reference(args, lambda: views(k))
    value = k * args.steps / total
    return reference_line(args, SURROGATE_METRIC, value, "views/s", True, total,
                          {"workload": "surrogate: 32^3 view-aligned crops + forward, candidate views of the "
                                       "256^3 uint8 tabletop", "views_per_step": k,
                           "parallelism": "one host thread; numpy matrix products may use every core (BLAS)"},
                          os.cpu_count() or 1, f"crop + forward of the first {k} of {len(pz)} candidates per step")


REFERENCE_ARMS = {"insert": run_reference_insert, "fig3": run_reference_fig3, "surrogate": run_reference_surrogate}


def reference_views_workload(name: str) -> str:
    """Workload whose views the oracle scores; the pruned selection's reference is the exact
    scoring of the same room512 candidates."""
    return "room512" if name == "room512-pruned" else name


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "idw_cost":
        run_reference_cost(args)
        return
    if args.workload in REFERENCE_ARMS:
        print(json.dumps(REFERENCE_ARMS[args.workload](args)), flush=True)
        return
    import oracle
    w = build_workload(reference_views_workload(args.workload), 0)
    threads = os.cpu_count() or 1
    m = oracle.Map(w.grid, w.voxel_size, w.origin)
    cam = oracle.camera_of(w.camera)
    prm = oracle.params(w.metric)
    # a bounded sample per step so that warmup + steps end within a few minutes
    t0 = time.perf_counter()
    oracle.views_ig(m, w.poses[:threads], cam, prm, "f32", threads)
    per_view = (time.perf_counter() - t0) / threads
    per_step_s = min(8.0, 120.0 / max(1, args.steps + args.warmup))
    n = int(max(threads, min(w.n_poses, per_step_s / max(per_view, 1e-6))))
    for _ in range(args.warmup):
        oracle.views_ig(m, w.poses[:n], cam, prm, "f32", threads)
    times, steps = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, st = oracle.views_ig(m, w.poses[:n], cam, prm, "f32", threads)
        times.append(time.perf_counter() - t0)
        steps += int(st.sum())
    total = sum(times)
    value = n * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "views/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": (pruned_describe() + " (reference: the oracle's exact scoring of the candidates)"
                                    if args.workload == "room512-pruned" else describe(w)),
                       "views_per_step": n, "parallelism": "host threads"},
            "voxel_steps_per_s": steps / total,
            "cpu_baseline": {"value": value, "unit": "views/s", "cores": threads, "kind": "oracle",
                             "sample": f"first {n} of {w.n_poses} views per step"},
            "e2e": {"value": value, "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


WORKLOAD_CHOICES = ["prob256", "exact64", "room512", "traj256", "room512-pruned", "idw_cost", "fig3", "insert",
                    "surrogate"]

# (steps, warm-up steps) when not given: each workload's timed work ends within a minute or so
DEFAULT_STEPS = {"prob256": (1000, 20), "exact64": (1000, 20), "traj256": (200, 5), "room512": (20, 3),
                 "room512-pruned": (25, 3), "idw_cost": (200, 5), "fig3": (20, 3), "insert": (200, 5),
                 "surrogate": (100, 5)}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: per workload)")
    ap.add_argument("--warmup", type=int, default=None, help="untimed warm-up steps (default: per workload)")
    ap.add_argument("--workload", default="room512-pruned", choices=WORKLOAD_CHOICES)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip", type=int, default=None, choices=[0, 1],
                    help="state-map count walks: skip uniform 8^3 bricks (1) or not (0); default: the library's")
    ap.add_argument("--views", type=int, default=None,
                    help="view workloads: only the first N views (a reduced launch, for profiling)")
    ap.add_argument("--train-epochs", type=int, default=30,
                    help="room512-pruned: surrogate training epochs before timing (0: untrained, for profiling)")
    ap.add_argument("--scenes", type=int, default=PRUNED_MIN_SCENES,
                    help="room512-pruned: scenes scored for the same-best-view rate (at least the timed steps)")
    args = ap.parse_args(argv)
    steps, warmup = DEFAULT_STEPS[args.workload]
    args.steps = steps if args.steps is None else args.steps
    args.warmup = max(3, warmup if args.warmup is None else args.warmup)  # at least three untimed steps
    return args


def main() -> None:
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import paper_2503_22588_gb300 as nbt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    nbt.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    def finish():
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()

    runners = {"idw_cost": run_cost, "fig3": run_fig3, "insert": run_insert, "surrogate": run_surrogate}
    if args.workload == "room512-pruned":
        run_pruned(args, nbt, torch, dev, world, rank, local, dist)
        return finish()
    if args.workload in runners:
        runners[args.workload](args, nbt, torch, dev, stream, world, rank, local, dist)
        return finish()
    w = build_workload(args.workload, rank)
    if w.offsets is not None:
        run_traj(args, w, nbt, torch, dev, stream, world, rank, local, dist)
        return finish()
    if args.views is not None:   # a reduced launch of the same workload (profiling)
        w.poses = np.ascontiguousarray(w.poses[:args.views])
    cam = nbt.camera(w.camera.width, w.camera.height, w.camera.fov_h, w.camera.fov_v, w.camera.max_range)
    prm = nbt.ig_params(w.metric)
    grid_dev = torch.from_numpy(np.ascontiguousarray(w.grid)).to(dev)
    poses_dev = torch.from_numpy(w.poses).to(dev)
    m = nbt.Map(w.n, w.n, w.n, w.voxel_size, w.origin, w.encoding)
    if args.skip is not None:
        m.set_tuning(8, skip=bool(args.skip))
    # the library takes the uniform-brick skipping walk on linear maps above this many rays per call
    skip_walk = args.skip != 0 and w.n_poses * w.camera.width * w.camera.height > SKIP_WALK_MIN_RAYS
    ws = nbt.workspace(w.n_poses, cam, dev)
    ig = torch.empty(w.n_poses, dtype=torch.float32, device=dev)
    steps = torch.empty(w.n_poses, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        m.upload(grid_dev, stream)
        nbt.views_ig(m, poses_dev, cam, prm, ig, steps, ws, stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        step()
    barrier()
    n_steps_voxel = int(steps.sum().item())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)  # evict the map from L2 between timed steps (not timed)
        a, b, c = ev[k]
        a.record(stream)
        m.upload(grid_dev, stream)
        b.record(stream)
        nbt.views_ig(m, poses_dev, cam, prm, ig, steps, ws, stream)
        c.record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    ig_ms = [b.elapsed_time(c) for a, b, c in ev]
    upload_ms = float(np.mean([a.elapsed_time(b) for a, b, c in ev]))
    total_ms = float(sum(step_ms))
    ig_mean_ms = float(np.mean(ig_ms))
    total_ms = max_over_ranks(total_ms, dist, dev)

    # end to end through the public API with host buffers: pinned host grid and
    # poses in, per-perspective IG out, copies inside the timed region
    grid_host = torch.from_numpy(np.ascontiguousarray(w.grid)).pin_memory()
    poses_host = torch.from_numpy(w.poses).pin_memory()
    ig_host = torch.empty(w.n_poses, dtype=torch.float32).pin_memory()
    poses_e2e = torch.empty_like(poses_dev)

    def e2e_step():
        m.upload(grid_host.numpy(), stream)
        poses_e2e.copy_(poses_host, non_blocking=True)
        nbt.views_ig(m, poses_e2e, cam, prm, ig, None, ws, stream, want_steps=False)
        ig_host.copy_(ig, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, _, c = ev[k]
        a.record(stream)
        e2e_step()
        c.record(stream)
        c.synchronize()
        e_ms.append(a.elapsed_time(c))
    e2e_total = float(sum(e_ms))
    e2e_total = max_over_ranks(e2e_total, dist, dev)

    peak, peak_kind = load_peaks()
    bps = BYTES_PER_STEP[w.encoding]
    achieved = n_steps_voxel * bps / (ig_mean_ms * 1e-3) / 1e9
    traffic = ncu_traffic(args.workload)
    line = {
        "metric": METRIC,
        "value": job_throughput(w.n_poses * args.steps, world, total_ms),
        "unit": "views/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": describe(w) + (f" (reduced: first {w.n_poses} views)" if args.views else ""),
                   "views_per_gpu": w.n_poses, "rays_per_view": w.rays_per_pose,
                   "map": f"{w.n}^3 {w.encoding}", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "step": "map upload+gain derivation + views_ig (tile kernel + reduce)"},
        "voxel_steps_per_s": world * n_steps_voxel * args.steps / (total_ms * 1e-3),
        "voxel_steps_per_step": n_steps_voxel,
        "views_ig_ms": ig_mean_ms,
        "upload_ms": upload_ms,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "the tile kernel the call selects (ig_tiles_kernel or ig_warp_tiles_kernel) + views_reduce",
                     "algorithmic": f"{bps} B per voxel step x {n_steps_voxel} steps",
                     "peak_kind": f"{peak_kind} (hbm_gbs)"},
        "roofline_alu": walk_alu_roofline(n_steps_voxel, ig_mean_ms, "the tile kernel the call selects + views_reduce"),
        "e2e": {"value": job_throughput(w.n_poses * args.steps, world, e2e_total), "unit": "views/s",
                "h2d_bytes_per_step": int(grid_host.numel() * grid_host.element_size()
                                          + poses_host.numel() * 4),
                "d2h_bytes_per_step": int(ig_host.numel() * 4)},
        # per step: upload (scatter / pack), gain derivation (probability maps only), the brick summaries
        # of the new map when the call takes the skipping walk (5), tile kernel, reduce
        "gpu_launches": ((4 if w.encoding == "f32" else 3) + (5 if skip_walk else 0)) * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_traj(args, w, nbt, torch, dev, stream, world, rank, local, dist) -> None:
    """Trajectory workload: autotuned map + one CUDA-graph replay of nbt_traj_ig per step."""
    cam = nbt.camera(w.camera.width, w.camera.height, w.camera.fov_h, w.camera.fov_v, w.camera.max_range)
    prm = nbt.ig_params(w.metric)
    grid_dev = torch.from_numpy(np.ascontiguousarray(w.grid)).to(dev)
    poses_dev = torch.from_numpy(w.poses).to(dev)
    off_dev = torch.from_numpy(w.offsets).to(dev)
    m, tuned, _ = nbt.autotune(grid_dev, w.voxel_size, w.origin, w.encoding, poses_dev, cam, prm, offsets=off_dev,
                               skips=(0, 1), reps=2)
    _, st = nbt.views_ig(m, poses_dev, cam, prm)
    n_steps_voxel = int(st.sum().item())
    plan = nbt.TrajPlan(m, poses_dev, off_dev, cam, prm)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        m.upload(grid_dev, stream)
        plan.launch(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b, c = ev[k]
        a.record(stream)
        m.upload(grid_dev, stream)
        b.record(stream)
        plan.launch(stream)
        c.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = float(sum(a.elapsed_time(c) for a, b, c in ev))
    ig_ms = float(np.mean([b.elapsed_time(c) for a, b, c in ev]))
    total_ms = max_over_ranks(total_ms, dist, dev)
    # end to end: host grid, poses and offsets in, trajectory IG out
    grid_host = torch.from_numpy(np.ascontiguousarray(w.grid)).pin_memory()
    poses_host = torch.from_numpy(w.poses).pin_memory()
    off_host = torch.from_numpy(w.offsets).pin_memory()
    out_host = torch.empty(len(w.offsets) - 1, dtype=torch.float32).pin_memory()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, _, c = ev[k]
        a.record(stream)
        m.upload(grid_host.numpy(), stream)
        poses_dev.copy_(poses_host, non_blocking=True)
        off_dev.copy_(off_host, non_blocking=True)
        out_host.copy_(plan.launch(stream), non_blocking=True)
        c.record(stream)
        c.synchronize()
        e_ms.append(a.elapsed_time(c))
    e2e_total = float(sum(e_ms))
    e2e_total = max_over_ranks(e2e_total, dist, dev)
    peak, peak_kind = load_peaks()
    bps = BYTES_PER_STEP[w.encoding]
    line = {
        "metric": METRIC, "value": job_throughput(w.n_poses * args.steps, world, total_ms), "unit": "views/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": describe(w), "poses_per_gpu": w.n_poses, "trajectories": len(w.offsets) - 1,
                   "rays_per_pose": w.rays_per_pose, "map": f"{w.n}^3 {w.encoding}", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write)", "tuned": tuned,
                   "step": "map upload + CUDA-graph replay of nbt_traj_ig"},
        "voxel_steps_per_s": world * n_steps_voxel * args.steps / (total_ms * 1e-3),
        "voxel_steps_per_step": n_steps_voxel, "traj_ig_ms": ig_ms,
        "roofline": {"bound": "hbm", "achieved": n_steps_voxel * bps / (ig_ms * 1e-3) / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": n_steps_voxel * bps / (ig_ms * 1e-3) / 1e9 / peak,
                     "traffic": ncu_traffic(args.workload), "kernel": "the tile kernel the plan selects (ig_tiles_kernel or ig_warp_tiles_kernel) + traj_reduce",
                     "algorithmic": f"{bps} B per voxel step x {n_steps_voxel} steps",
                     "peak_kind": f"{peak_kind} (hbm_gbs)"},
        "roofline_alu": walk_alu_roofline(n_steps_voxel, ig_ms, "the tile kernel the plan selects + traj_reduce"),
        "e2e": {"value": job_throughput(w.n_poses * args.steps, world, e2e_total), "unit": "views/s",
                "h2d_bytes_per_step": int(grid_host.numel() + poses_host.numel() * 4 + off_host.numel() * 4),
                "d2h_bytes_per_step": int(out_host.numel() * 4)},
        # per step: upload, the brick summaries of the new map when the plan takes the skipping walk (5),
        # and the graph's tile kernel and reduce
        "gpu_launches": (3 + (5 if tuned.get("skip") else 0)) * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = traj_cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    plan.close()
    m.close()


def run_cost(args, nbt, torch, dev, stream, world, rank, local, dist) -> None:
    """IG cost of candidate trajectories: per step, push the newest ID, then nbt_ig_cost over all candidates."""
    w = build_workload("idw_cost", rank)
    buf = nbt.IdBuffer(w.n_b, max(len(g) for _, g in w.ids))
    id_dev = [(torch.from_numpy(pz).to(dev), torch.from_numpy(g).to(dev)) for pz, g in w.ids]
    for pz, g in id_dev:
        buf.push(pz, g, stream)
    poses_dev = torch.from_numpy(w.poses).to(dev)
    off_dev = torch.from_numpy(w.offsets).to(dev)
    n_states, n_traj = w.poses.shape[0], len(w.offsets) - 1
    pairs = n_states * sum(len(g) for _, g in w.ids)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(k, poses, off, mid=None):
        pz, g = id_dev[k % len(id_dev)]
        buf.push(pz, g, stream)
        if mid is not None:
            mid.record(stream)
        return nbt.ig_cost(buf, poses, off, w.poi, w.fov_h, w.fov_v, w.w_info, w.power, w.eps, stream=stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for k in range(max(args.warmup, 3)):
        step(k, poses_dev, off_dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, b, c = ev[k]
        a.record(stream)
        step(k, poses_dev, off_dev, b)
        c.record(stream)
    barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    cost_ms = float(np.mean([b.elapsed_time(c) for a, b, c in ev]))
    total_ms = float(sum(step_ms))
    total_ms = max_over_ranks(total_ms, dist, dev)
    # end to end: pinned host poses and offsets in, per-trajectory cost out
    poses_host = torch.from_numpy(w.poses).pin_memory()
    off_host = torch.from_numpy(w.offsets).pin_memory()
    cost_host = torch.empty(n_traj, dtype=torch.float32).pin_memory()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, _, c = ev[k]
        a.record(stream)
        poses_dev.copy_(poses_host, non_blocking=True)
        off_dev.copy_(off_host, non_blocking=True)
        cost_host.copy_(step(k, poses_dev, off_dev), non_blocking=True)
        c.record(stream)
        c.synchronize()
        e_ms.append(a.elapsed_time(c))
    e2e_total = float(sum(e_ms))
    e2e_total = max_over_ranks(e2e_total, dist, dev)
    peak = MUFU_PER_CLK_PER_SM * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9   # Gpair/s at one MUFU op per pair
    achieved = pairs / (cost_ms * 1e-3) / 1e9
    line = {
        "metric": COST_METRIC, "value": job_throughput(n_states * args.steps, world, total_ms), "unit": "states/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": describe(w), "states_per_gpu": n_states, "trajectories": n_traj,
                   "ids": len(w.ids), "perspectives_per_id": len(w.ids[0][1]), "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "step": "nbt_id_buffer_push (newest ID) + nbt_ig_cost (IDW/orientation/term kernel + reduce)"},
        "pairs_per_step": pairs, "ig_cost_ms": cost_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s", "frac": achieved / peak,
                     "traffic": ncu_traffic("idw_cost"), "kernel": "idw_kernel (+cost_reduce)",
                     "algorithmic": f"1 MUFU reciprocal and 8 FP32 lane ops per (state, perspective) pair x {pairs} "
                                    "pairs",
                     "peak_kind": f"derived: {MUFU_PER_CLK_PER_SM} MUFU/clk/SM (= 128 FP32 lanes / 8) x {SM_COUNT} "
                                  f"SMs x {SM_MAX_MHZ} MHz"},
        "e2e": {"value": job_throughput(n_states * args.steps, world, e2e_total), "unit": "states/s",
                "h2d_bytes_per_step": int(poses_host.numel() * 4 + off_host.numel() * 4),
                "d2h_bytes_per_step": int(cost_host.numel() * 4)},
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cost_cpu_baseline(w)
    if rank == 0:
        print(json.dumps(line), flush=True)
    buf.close()


FIG3_METRIC = ("ID computation ms over grid factor s_G x perspectives N_P (Fig. 3 sweep; Eq. 1 perspectives, s_G "
               "endpoint grid, Eq. 2 mean IG)")


def run_fig3(args, nbt, torch, dev, stream, world, rank, local, dist) -> None:
    """The paper's Fig. 3 sweep on the GPU and the CPU oracle: one ID per (s_G, N_P) cell.

    Per cell: kernel-only time of nbt_views_ig with device-resident poses
    (device time only: the call is enqueued behind a short GPU spin before
    the start event fires), end-to-end time through the public API (poses
    from pinned host memory, IGs back to the host, copies and host launch
    overhead inside the timed region), and the CPU oracle on the same
    perspectives.  value = the end-to-end ms of the paper's chosen
    setting (s_G = 100, N_P = 500).
    """
    import oracle
    from oracle.endpoints import grid_size as orc_grid
    from workload import configs
    grid, poi, poses = configs.fig3_scene(seed=rank)
    n = grid.shape[0]
    m = nbt.Map(n, n, n, configs.VOXEL, (0.0, 0.0, 0.0), "f32")
    m.upload(torch.from_numpy(grid).to(dev), stream)
    prm = nbt.ig_params("eq2", reduce="mean")
    fov_h, fov_v = math.radians(60.0), math.radians(45.0)
    orc_map = oracle.Map(grid, configs.VOXEL, (0.0, 0.0, 0.0))
    orc_prm = oracle.params("eq2", reduce="mean")
    threads = os.cpu_count() or 1
    reps = max(args.steps, 3)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    cells, best_roof, launches = [], None, 0
    for sg in configs.FIG3_GRID_SCALES:
        cam = nbt.camera_from_grid_scale(fov_h, fov_v, 1.0, configs.VOXEL, sg)
        for n_p in configs.FIG3_VIEW_COUNTS:
            pz_host = torch.from_numpy(np.ascontiguousarray(poses[:n_p])).pin_memory()
            pz = pz_host.to(dev)
            ws = nbt.workspace(n_p, cam, dev)
            ig = torch.empty(n_p, dtype=torch.float32, device=dev)
            st = torch.empty(n_p, dtype=torch.int64, device=dev)
            ig_host = torch.empty(n_p, dtype=torch.float32).pin_memory()
            for _ in range(max(args.warmup, 3)):
                nbt.views_ig(m, pz, cam, prm, ig, st, ws, stream)
            torch.cuda.synchronize(dev)
            k_ms, e_ms, h_us = [], [], []
            for r in range(reps):
                flush.fill_(r & 0xFF)
                a, c = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                # kernel-only: the GPU spins ~0.1 ms first, so the call is enqueued before the start event fires
                torch.cuda._sleep(200000)
                a.record(stream)
                t_host = time.perf_counter()
                nbt.views_ig(m, pz, cam, prm, ig, st, ws, stream)
                h_us.append(1e6 * (time.perf_counter() - t_host))
                c.record(stream)
                c.synchronize()
                k_ms.append(a.elapsed_time(c))
                flush.fill_(r & 0xFF)
                a.record(stream)
                pz.copy_(pz_host, non_blocking=True)
                nbt.views_ig(m, pz, cam, prm, ig, None, ws, stream, want_steps=False)
                ig_host.copy_(ig, non_blocking=True)
                c.record(stream)
                c.synchronize()
                e_ms.append(a.elapsed_time(c))
            launches += 4 * reps
            steps = int(st.sum().item())
            ow, oh = orc_grid(fov_h, fov_v, 1.0, configs.VOXEL, sg)
            t0 = time.perf_counter()
            oracle.views_ig(orc_map, poses[:n_p], oracle.camera(ow, oh, fov_h, fov_v, 1.0), orc_prm, "f32", threads)
            cpu_ms = 1e3 * (time.perf_counter() - t0)
            cell = {"s_g": sg, "n_p": n_p, "n_e": cam.width * cam.height, "gpu_kernel_ms": float(np.mean(k_ms)),
                    "gpu_e2e_ms": float(np.mean(e_ms)), "host_enqueue_us": float(np.median(h_us)),
                    "cpu_oracle_ms": cpu_ms, "voxel_steps": steps}
            cells.append(cell)
            if best_roof is None or steps > best_roof[0]:
                best_roof = (steps, cell["gpu_kernel_ms"], sg, n_p)
    clk = clocks.stop()
    chosen = next(c for c in cells if c["s_g"] == 100 and c["n_p"] == 500)
    peak, peak_kind = load_peaks()
    steps, k_ms, sg, n_p = best_roof
    achieved = steps * BYTES_PER_STEP["f32"] / (k_ms * 1e-3) / 1e9
    line = {
        "metric": FIG3_METRIC, "value": chosen["gpu_e2e_ms"], "unit": "ms", "n_gpus": world, "steps": reps,
        "warmup": args.warmup, "ms_per_step": chosen["gpu_e2e_ms"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "fig3: 256^3 FP32 tabletop, PoI at the centre, N_P perspectives by Eq. 1 (r_S = 1 m), "
                               "FoV 60x45, d_Cam 1 m, s_Vox 1 cm, Eq. 2 mean IG; value = s_G 100, N_P 500 "
                               "end to end", "parallelism": f"replicas x{world}",
                   "l2": "flushed before every timed call (256 MiB write)"},
        "sweep": cells,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": f"ig_tiles_kernel (+views_reduce) at s_G {sg}, N_P {n_p}",
                     "algorithmic": f"4.0 B per voxel step x {steps} steps", "peak_kind": f"{peak_kind} (hbm_gbs)"},
        "e2e": {"value": chosen["gpu_e2e_ms"], "unit": "ms", "h2d_bytes_per_step": 500 * 28,
                "d2h_bytes_per_step": 500 * 4},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": {"value": chosen["cpu_oracle_ms"], "unit": "ms", "cores": threads, "kind": "oracle",
                         "sample": "the same ID (s_G 100, N_P 500), all perspectives"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()


INSERT_METRIC = "map update points/s (depth scans inserted into the probabilistic voxel map)"


def insert_cpu_baseline(scans, n, vs, budget_s: float = 12.0) -> dict:
    """The oracle's insertion (FP32 update, FP32 walk in C, one host thread) on a bounded number of scans."""
    from oracle import insert as I
    grid = np.full((n, n, n), 0.5, np.float32)
    t0 = time.perf_counter()
    done, pts = 0, 0
    while done < len(scans) and (done == 0 or time.perf_counter() - t0 < budget_s):
        pose, p = scans[done]
        grid = I.insert(grid, p, pose[:3], vs)
        done += 1
        pts += len(p)
    dt = time.perf_counter() - t0
    return {"value": pts / dt, "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {done} of {len(scans)} scans ({pts} points) into the same 256^3 map"}


def run_insert(args, nbt, torch, dev, stream, world, rank, local, dist) -> None:
    """Map update: one 640 x 576 depth scan inserted per step (scans used in rotation)."""
    from workload import configs
    scans, n, vs = configs.insert_scans(seed=rank)
    grid = torch.full((n, n, n), 0.5, dtype=torch.float32, device=dev)
    m = nbt.Map.from_grid(grid, vs, (0.0, 0.0, 0.0), "f32")
    pts_dev = [torch.from_numpy(p).to(dev) for _, p in scans]
    sensors = [tuple(float(v) for v in pose[:3]) for pose, _ in scans]
    stats = torch.zeros(3, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for k in range(max(args.warmup, 3)):
        m.insert_points(pts_dev[k % len(scans)], sensors[k % len(scans)], stats=stats, stream=stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    st_hist = torch.zeros((args.steps, 3), dtype=torch.int64, device=dev)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, c = ev[k]
        a.record(stream)
        m.insert_points(pts_dev[k % len(scans)], sensors[k % len(scans)], stats=st_hist[k], stream=stream)
        c.record(stream)
    barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(c) for a, c in ev]
    total_ms = float(sum(ms))
    total_ms = max_over_ranks(total_ms, dist, dev)
    sh = st_hist.cpu().numpy()
    points = sum(len(scans[k % len(scans)][1]) for k in range(args.steps))
    # end to end: points from pinned host memory, the scan statistics back to the host
    host_pts = [torch.from_numpy(p).pin_memory() for _, p in scans]
    stats_host = torch.zeros(3, dtype=torch.int64).pin_memory()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, c = ev[k]
        a.record(stream)
        buf = pts_dev[k % len(scans)]
        buf.copy_(host_pts[k % len(scans)], non_blocking=True)
        m.insert_points(buf, sensors[k % len(scans)], stats=stats, stream=stream)
        stats_host.copy_(stats, non_blocking=True)
        c.record(stream)
        c.synchronize()
        e_ms.append(a.elapsed_time(c))
    e2e_total = float(sum(e_ms))
    e2e_total = max_over_ranks(e2e_total, dist, dev)
    peak, peak_kind = load_peaks()
    mean_s = total_ms * 1e-3 / args.steps
    steps_walked = float(sh[:, 2].mean())
    algo_bytes = points / args.steps * 12.0 + steps_walked * 4.0 + 2 * (n ** 3 / 8) * 2
    achieved = algo_bytes / mean_s / 1e9
    line = {
        "metric": INSERT_METRIC, "value": job_throughput(points, world, total_ms), "unit": "points/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "insert: 640x576 depth scans (Azure Kinect NFOV geometry, 75x65 deg, 3.86 m, 2 mm "
                               "noise) of an analytic tabletop into a 256^3 FP32 probability map of 1 cm voxels; "
                               f"{len(scans)} scans in rotation, one per step", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write)",
                   "step": "nbt_map_insert_points (points, distinct endpoints, free rays, update pass)"},
        "rays_per_step": float(sh[:, 1].mean()), "hits_per_step": float(sh[:, 0].mean()),
        "voxel_steps_per_step": steps_walked, "voxel_steps_per_s": steps_walked / mean_s,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "nbt_map_insert_points (free_rays_kernel dominant)",
                     "algorithmic": "12 B per point + 4 B (miss-bitmap word) per voxel step + 2 bitmaps read and "
                                    "cleared per scan", "peak_kind": f"{peak_kind} (hbm_gbs)"},
        "e2e": {"value": job_throughput(points, world, e2e_total), "unit": "points/s",
                "h2d_bytes_per_step": int(np.mean([p.numel() * 4 for p in host_pts])), "d2h_bytes_per_step": 24},
        # per scan: points, enumerate, free rays, apply, stats
        "gpu_launches": 5 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = insert_cpu_baseline(scans, n, vs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()


SURROGATE_METRIC = "surrogate inference views/s (frustum crops + 3D-CNN forward on tcgen05), 16,384 candidates per step"


def surrogate_flops_per_view() -> int:
    """Multiply-adds x 2 of one forward pass: the four 3^3 convolutions, fc1 and fc2."""
    from paper_2503_22588_gb300.surrogate import CROP, FC_IN, HIDDEN, LAYERS
    flops, size = 0, CROP
    for cin, cout, stride in LAYERS:
        size = (size - 1) // stride + 1
        flops += 2 * size ** 3 * cout * 27 * cin
    return flops + 2 * FC_IN * HIDDEN + 2 * HIDDEN


def surrogate_cpu_baseline(crops, feats, params, budget_s: float = 10.0) -> dict:
    """The oracle's FP64 forward (numpy, BF16-rounded as on the GPU) on a bounded number of the same crops
    (class codes, expanded to the one-hot input the oracle takes)."""
    from oracle import surrogate as S
    q = {k: np.asarray(v, np.float64) for k, v in params.items()}
    n, t0 = 0, time.perf_counter()
    while n < len(crops) and (n == 0 or time.perf_counter() - t0 < budget_s):
        S.forward(q, S.codes_to_onehot(crops[n:n + 8]), feats[n:n + 8], bf16_activations=True)
        n += len(crops[n:n + 8])
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "views/s", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"forward of the first {n} crops of the same step (crops given); numpy matrix products "
                      f"may use every core through BLAS"}


def run_surrogate(args, nbt, torch, dev, stream, world, rank, local, dist) -> None:
    """Surrogate inference: crops and predictions for 16,384 candidate views per step."""
    import math
    from paper_2503_22588_gb300 import surrogate as gs
    from workload import configs, poses as wp
    w = configs.traj256(seed=rank)
    m = nbt.Map.from_grid(torch.from_numpy(np.ascontiguousarray(w.grid)).to(dev), w.voxel_size, w.origin, "u8")
    cam = nbt.camera(128, 96, math.radians(60), math.radians(45), 1.0)
    prm = nbt.ig_params("count")
    pz_np = np.concatenate([wp.shell_views(p, 4096, 0.3, 0.8, 100 * rank + k) for k, p in enumerate(w.pois)])
    pz = torch.from_numpy(pz_np).to(dev)
    n, batch = len(pz_np), 4096
    net = gs.Surrogate(max_batch=batch, params=gs.he_init(rank))
    scores = torch.empty(n, dtype=torch.float32, device=dev)
    cr = torch.empty((batch, gs.CROP, gs.CROP, gs.CROP), dtype=torch.uint8, device=dev)
    ft = torch.empty((batch, gs.FEATS), dtype=torch.bfloat16, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(poses_dev, fwd_events=None):
        for b0 in range(0, n, batch):
            c_b, f_b = gs.crops(m, poses_dev[b0:b0 + batch], cam, prm, stream, out=(cr, ft))
            if fwd_events is not None:
                fwd_events[b0 // batch][0].record(stream)
            net.forward(c_b, f_b, scores[b0:b0 + batch], stream)
            if fwd_events is not None:
                fwd_events[b0 // batch][1].record(stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 3)):
        step(pz)
    n_b = (n + batch - 1) // batch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    fev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_b)]
           for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, c = ev[k]
        a.record(stream)
        step(pz, fev[k])
        c.record(stream)
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(float(sum(a.elapsed_time(c) for a, c in ev)), dist, dev)
    fwd_ms = float(np.mean([sum(x.elapsed_time(y) for x, y in f) for f in fev]))
    # end to end: candidate poses from pinned host memory, scores back to the host
    pz_host = torch.from_numpy(pz_np).pin_memory()
    sc_host = torch.empty(n, dtype=torch.float32).pin_memory()
    e_ms = []
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        a, c = ev[k]
        a.record(stream)
        pz.copy_(pz_host, non_blocking=True)
        step(pz)
        sc_host.copy_(scores, non_blocking=True)
        c.record(stream)
        c.synchronize()
        e_ms.append(a.elapsed_time(c))
    e2e_total = max_over_ranks(float(sum(e_ms)), dist, dev)
    fl = surrogate_method_flops_per_view()       # the method's own FLOPs (layer 0 as its one-hot GEMM)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = fl * n / (fwd_ms * 1e-3) / 1e12
    line = {
        "metric": SURROGATE_METRIC, "value": job_throughput(n * args.steps, world, total_ms), "unit": "views/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "surrogate: 16,384 candidate views (4 PoIs x 4096 on a 0.3-0.8 m shell) of the 256^3 "
                               "uint8 tabletop; 32^3 class-code crops (one-hot over 8 channels), convs 8-16-32-64-64, "
                               "MLP 4104-128-1, batches of 4096; random-init weights", "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write)", "step": "nbt_surrogate_crops + forward"},
        "forward_ms_per_step": fwd_ms, "flops_per_view": fl,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": "surrogate forward (implicit-GEMM convolutions + MLP on tcgen05)",
                     "algorithmic": f"{fl} FLOP per view (layer 0 as its K = 112 one-hot GEMM) x {n} views",
                     "peak_kind": "measured (bf16_tflops, burst)"},
        "e2e": {"value": job_throughput(n * args.steps, world, e2e_total), "unit": "views/s",
                "h2d_bytes_per_step": int(pz_host.numel() * 4), "d2h_bytes_per_step": int(sc_host.numel() * 4)},
        # per batch: crops, fused layers 0-1, layer 2, layer 3, features, fc1 GEMM, fc2
        "gpu_launches": 8 * n_b * args.steps,   # per batch: crops, conv01, conv23 x 2, features, fc1, fc1 reduce, fc2
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = surrogate_cpu_baseline(cr[:64].cpu().numpy(), ft.float().cpu().numpy()[:64],
                                                      net.get_params())
    if rank == 0:
        print(json.dumps(line), flush=True)
    net.close()
    m.close()


PRUNED_MIN_SCENES = 100  # agreement is scored on at least this many scenes (8 PoIs each: >= 800 cases)
PRUNED_SEG, PRUNED_KEEP = 4096, 205


def pruned_describe() -> str:
    return ("room512-pruned: 512^3 2-bit room (2000 primitives, 40% unknown), 8 PoIs x 4096 candidate views of "
            "320x240 rays per scene, unknown-voxel count; best view per PoI by exact raycasting of all "
            "candidates vs of the surrogate's top 5 % (205 per PoI)")


def wilson_interval(k: int, n: int, z: float = 1.959964) -> tuple[float, float]:
    """95 % Wilson score interval of a binomial rate k / n."""
    if n == 0:
        return 0.0, 1.0
    p = k / n
    den = 1.0 + z * z / n
    mid = (p + z * z / (2 * n)) / den
    half = z * math.sqrt(p * (1.0 - p) / n + z * z / (4.0 * n * n)) / den
    # at k = 0 (k = n) the lower (upper) bound is exactly 0 (1); keep rounding from moving it
    return (0.0 if k == 0 else max(0.0, mid - half)), (1.0 if k == n else min(1.0, mid + half))


def surrogate_method_flops_per_view() -> int:
    """FLOPs of one inference forward as the kernels run it: layer 0 is a tensor-core GEMM over the
    one-hot crop with K = 112 (28 taps x 4 class slots; 27 real taps) instead of a dense 8-channel
    convolution (K = 216); layers 1-3 are implicit-GEMM convolutions (K = 27 C_in); fc1 and fc2."""
    from paper_2503_22588_gb300.surrogate import CROP, FC_IN, HIDDEN, LAYERS
    flops, size = 0, CROP
    for i, (cin, cout, stride) in enumerate(LAYERS):
        size = (size - 1) // stride + 1
        k = 112 if i == 0 else 27 * cin
        flops += 2 * size ** 3 * cout * k
    return flops + 2 * FC_IN * HIDDEN + 2 * HIDDEN


def room_scenes(seeds, workers: int):
    """The room512 workloads of ``seeds``, generated on host cores (spawned worker processes)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from workload import configs
    if workers <= 1:
        return [configs.room512(seed=s) for s in seeds]
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(configs.room512, seeds))


TRAIN_ROOMS, TRAIN_PRIMS, TRAIN_EPOCHS = 24, 250, 30


def train_room_surrogate(nbt, torch, dev, cam, prm, epochs: int = TRAIN_EPOCHS, log=None):
    """The surrogate trained inside the run on exact labels (mean ray IG) of 24 seeded 256^3 rooms with
    room512's primitive density (250 primitives in 256^3, 2000 in 512^3) and 40 % unknown."""
    from paper_2503_22588_gb300 import planning as P, surrogate as gs
    from workload import poses as wp, scenes
    maps, poses, targets = [], [], []
    for sidx in range(TRAIN_ROOMS):
        g = scenes.room_states(256, TRAIN_PRIMS, 0.4, seed=1000 + sidx)
        m = nbt.Map.from_grid(torch.from_numpy(g).to(dev), 0.01, (0, 0, 0), "u8")
        rng = np.random.default_rng(2000 + sidx)
        pois = rng.uniform(0.6, 2.56 - 0.6, size=(8, 3))
        pz = np.concatenate([wp.shell_views(p, 1024, 0.3, 0.8, 3000 + sidx * 10 + k) for k, p in enumerate(pois)])
        pt = torch.from_numpy(pz).to(dev)
        maps.append(m)
        poses.append(pt)
        targets.append(P.label_views(m, pt, cam, prm))
    net = gs.Surrogate(max_batch=4096, params=gs.he_init(0), target_scale=P.TARGET_SCALE)
    t0 = time.perf_counter()
    losses = P.train(net, maps, poses, targets, cam, prm, epochs=epochs, lr=1e-3, batch=256, log=log)
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    for m in maps:
        m.close()
    return net, {"seconds": train_s, "final_loss": losses[-1] if losses else None,
                 "samples": TRAIN_ROOMS * 8 * 1024, "epochs": epochs,
                 "scenes": f"{TRAIN_ROOMS} seeded 256^3 rooms, {TRAIN_PRIMS} primitives, 40 % unknown",
                 "target": "mean ray IG x 0.01 (scale applied in the loss kernel)"}


def pruned_cpu_baseline(w, budget_s: float = 12.0, single_s: float = 6.0) -> dict:
    """The oracle's exact scoring (FP32 reference walk, FP64 sums) of a bounded sample of the same room512
    candidates, on every host core and on one thread (the paper's CPU version was sequential)."""
    import oracle
    threads = os.cpu_count() or 1
    m = oracle.Map(w.grid, w.voxel_size, w.origin)
    cam = oracle.camera_of(w.camera)
    prm = oracle.params(w.metric)
    t0 = time.perf_counter()
    oracle.views_ig(m, w.poses[:threads], cam, prm, "f32", threads)
    per = (time.perf_counter() - t0) / threads
    n = int(max(threads, min(w.n_poses, budget_s / max(per, 1e-6))))
    t0 = time.perf_counter()
    oracle.views_ig(m, w.poses[:n], cam, prm, "f32", threads)
    dt = time.perf_counter() - t0
    n1 = int(max(1, min(w.n_poses, single_s / max(per * threads, 1e-6))))
    t0 = time.perf_counter()
    oracle.views_ig(m, w.poses[:n1], cam, prm, "f32", 1)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": "views/s", "cores": threads, "kind": "oracle",
            "sample": f"exact scoring of the first {n} of the {w.n_poses} candidate views of room512 scene 0",
            "single_thread": {"value": n1 / dt1, "unit": "views/s", "cores": 1,
                              "sample": f"the first {n1} candidate views of the same scene"}}


def run_pruned(args, nbt, torch, dev, world, rank, local, dist) -> None:
    """room512 next-best-view selection, exact vs surrogate-pruned (the headline metric).

    The surrogate is trained first, inside this run, on exact labels of seeded 256^3 rooms.  Then each
    timed step takes one room512 scene (8 PoIs x 4096 candidate views of 320 x 240 rays): the pruned
    arm uploads the map and runs nbt_plan_pruned (crops and network scores of every candidate, the top
    5 % per PoI raycast exactly, the best of them); the exact arm uploads the map and raycasts every
    candidate.  Both are timed with CUDA events on the launching stream, the L2 flushed before each.
    The same-best-view rate is scored on at least 100 scenes (>= 800 PoI cases); scenes beyond the
    timed steps are evaluated untimed.
    """
    import math
    from paper_2503_22588_gb300 import planning as P, surrogate as gs

    cam = nbt.camera(320, 240, math.radians(60), math.radians(45), 1.0)
    prm = nbt.ig_params("count")
    seg, keep = PRUNED_SEG, PRUNED_KEEP
    stream = torch.cuda.current_stream(dev)
    n_eval = max(args.scenes, args.steps)
    seeds = [1000 * rank + k for k in range(n_eval)]
    t0 = time.perf_counter()
    scenes_w = room_scenes(seeds, min(8, os.cpu_count() or 1))
    gen_s = time.perf_counter() - t0
    net, train_info = train_room_surrogate(nbt, torch, dev, cam, prm, args.train_epochs)
    n_views = scenes_w[0].n_poses
    nseg = n_views // seg
    grids = [torch.from_numpy(np.ascontiguousarray(w.grid)).to(dev) for w in scenes_w]
    poses = [torch.from_numpy(w.poses).to(dev) for w in scenes_w]
    m = nbt.Map(512, 512, 512, 0.01, (0.0, 0.0, 0.0), "u2")
    if args.skip is not None:
        m.set_tuning(8, skip=bool(args.skip))
    ws_exact = nbt.workspace(n_views, cam, dev)
    ws_pruned = P.pruned_workspace(net, n_views, seg, keep, cam, dev)
    ig_all = torch.empty(n_views, dtype=torch.float32, device=dev)
    steps_all = torch.empty(n_views, dtype=torch.int64, device=dev)
    best_p = torch.empty(nseg, dtype=torch.int32, device=dev)
    val_p = torch.empty(nseg, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def pruned_step(k):
        m.upload(grids[k], stream)
        P.pruned_best(net, m, poses[k], seg, keep, cam, prm, ws_pruned, stream, (best_p, val_p), want_kept=False)

    def exact_step(k, ev=None):
        m.upload(grids[k], stream)
        if ev is not None:
            ev[0].record(stream)
        nbt.views_ig(m, poses[k], cam, prm, ig_all, steps_all, ws_exact, stream)
        if ev is not None:
            ev[1].record(stream)
        return P.segment_argmax(ig_all, seg, stream=stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):                 # untimed passes of both arms
        pruned_step(0)
        exact_step(0)
    barrier()
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ev_p = [(E(), E()) for _ in range(args.steps)]
    ev_x = [(E(), E()) for _ in range(args.steps)]
    ev_k = [(E(), E()) for _ in range(args.steps)]
    same = optimal = cases = 0
    vox_steps = 0
    exact_best, exact_ig = [], []
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                    # evict the map from L2 (untimed)
        ev_p[k][0].record(stream)
        pruned_step(k)
        ev_p[k][1].record(stream)
        flush.fill_((k + 1) & 0xFF)
        ev_x[k][0].record(stream)
        bx, vx = exact_step(k, ev_k[k])
        ev_x[k][1].record(stream)
        torch.cuda.synchronize(dev)
        same += int((bx == best_p).sum().item())
        optimal += int((vx == val_p).sum().item())
        cases += nseg
        vox_steps += int(steps_all.sum().item())
        exact_best.append(bx.clone())
        exact_ig.append(ig_all.clone())
    barrier()
    clk = clocks.stop()
    pr_ms = [a.elapsed_time(b) for a, b in ev_p]
    ex_ms = [a.elapsed_time(b) for a, b in ev_x]
    kern_ms = [a.elapsed_time(b) for a, b in ev_k]
    pr_total = max_over_ranks(float(sum(pr_ms)), dist, dev)
    ex_total = max_over_ranks(float(sum(ex_ms)), dist, dev)

    # agreement on the scenes beyond the timed steps (untimed), same calls
    for k in range(args.steps, n_eval):
        pruned_step(k)
        bx, vx = exact_step(k)
        torch.cuda.synchronize(dev)
        same += int((bx == best_p).sum().item())
        optimal += int((vx == val_p).sum().item())
        cases += nseg
        exact_best.append(bx.clone())
        exact_ig.append(ig_all.clone())

    # pruning baselines at the same exact budget (205 raycast views per PoI), same scenes: random
    # candidates, the untrained network, and Eq. 3's interpolation (a random half of the budget
    # raycast and pushed as one ID, G(x) at the other candidates, the top of G(x) raycast)
    base = {"random": 0, "untrained_network": 0, "idw_eq3": 0}
    net0 = gs.Surrogate(max_batch=4096, params=gs.he_init(0))
    ws0 = P.pruned_workspace(net0, n_views, seg, keep, cam, dev)
    k1 = keep // 2
    k2 = keep - k1
    idbuf = nbt.IdBuffer(n_b=1, max_views=k1)
    g_all = torch.empty(n_views, dtype=torch.float32, device=dev)
    for k in range(n_eval):
        m.upload(grids[k], stream)
        bx, ig_k, pt = exact_best[k], exact_ig[k], poses[k]
        rs = torch.from_numpy(np.random.default_rng(4000 + seeds[k]).random(n_views, dtype=np.float32)).to(dev)
        idx_r, _ = P.segment_topk(rs, seg, keep)
        b_r, _ = P.segment_argmax(ig_k[idx_r.reshape(-1).long()].contiguous(), keep, idx_r.reshape(-1).contiguous())
        base["random"] += int((bx == b_r).sum().item())
        b_u, _, _ = P.pruned_best(net0, m, pt, seg, keep, cam, prm, ws0, want_kept=False)
        base["untrained_network"] += int((bx == b_u).sum().item())
        idx_1, kept_1 = P.segment_topk(rs, seg, k1, pt)
        ig_1 = ig_k[idx_1.reshape(-1).long()].contiguous()
        for s_ in range(nseg):
            idbuf.push(kept_1[s_ * k1:(s_ + 1) * k1], ig_1[s_ * k1:(s_ + 1) * k1])
            nbt.idw_gain(idbuf, pt[s_ * seg:(s_ + 1) * seg], 2.0, g_all[s_ * seg:(s_ + 1) * seg])
        g_all.index_fill_(0, idx_1.reshape(-1).long(), float("-inf"))  # already raycast
        idx_2, _ = P.segment_topk(g_all, seg, k2)
        idxs = torch.cat([idx_1, idx_2], 1).reshape(-1).contiguous()
        b_i, _ = P.segment_argmax(ig_k[idxs.long()].contiguous(), keep, idxs)
        base["idw_eq3"] += int((bx == b_i).sum().item())
    torch.cuda.synchronize(dev)
    idbuf.close()
    net0.close()

    # surrogate forward alone (crops excluded), for its tensor-core roofline: the timed scenes' candidates
    cr = torch.empty((net.max_batch, gs.CROP, gs.CROP, gs.CROP), dtype=torch.uint8, device=dev)
    ft = torch.empty((net.max_batch, gs.FEATS), dtype=torch.bfloat16, device=dev)
    sc = torch.empty(n_views, dtype=torch.float32, device=dev)
    fwd_ms = []
    for k in range(min(args.steps, 4)):
        m.upload(grids[k], stream)
        t_k = 0.0
        for c0 in range(0, n_views, net.max_batch):
            c_b, f_b = gs.crops(m, poses[k][c0:c0 + net.max_batch], cam, prm, stream, out=(cr, ft))
            a, b = E(), E()
            a.record(stream)
            net.forward(c_b, f_b, sc[c0:c0 + net.max_batch], stream)
            b.record(stream)
            b.synchronize()
            t_k += a.elapsed_time(b)
        fwd_ms.append(t_k)

    # end to end through the public API: the dense grid and the candidate poses from pinned host memory,
    # the best views and their IGs back to the host, every step
    grid_h = torch.empty(grids[0].shape, dtype=torch.uint8).pin_memory()
    poses_h = torch.empty(poses[0].shape, dtype=torch.float32).pin_memory()
    best_h = torch.empty(nseg, dtype=torch.int32).pin_memory()
    val_h = torch.empty(nseg, dtype=torch.float32).pin_memory()
    pz_dev = torch.empty_like(poses[0])
    e2e_ms = []
    for k in range(args.steps):
        grid_h.numpy()[...] = scenes_w[k].grid            # staging into pinned memory (untimed)
        poses_h.numpy()[...] = scenes_w[k].poses
        flush.fill_(k & 0xFF)
        a, b = E(), E()
        a.record(stream)
        m.upload(grid_h.numpy(), stream)
        pz_dev.copy_(poses_h, non_blocking=True)
        P.pruned_best(net, m, pz_dev, seg, keep, cam, prm, ws_pruned, stream, (best_p, val_p), want_kept=False)
        best_h.copy_(best_p, non_blocking=True)
        val_h.copy_(val_p, non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = max_over_ranks(float(sum(e2e_ms)), dist, dev)

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm, hbm_kind = load_peaks()
    bf16 = float(peaks.get("bf16_tflops", 1900.0))
    bf16_kind = "measured (bf16_tflops, burst)" if "bf16_tflops" in peaks else "fallback (1.9 PFLOP/s burst)"
    kern_mean = float(np.mean(kern_ms))
    steps_per_launch = vox_steps / args.steps
    achieved = steps_per_launch * BYTES_PER_STEP["u2"] / (kern_mean * 1e-3) / 1e9
    fl = surrogate_method_flops_per_view()
    fwd_mean = float(np.mean(fwd_ms))
    s_achieved = fl * n_views / (fwd_mean * 1e-3) / 1e12
    lo, hi = wilson_interval(same, cases)
    n_chunks = (n_views + net.max_batch - 1) // net.max_batch
    line = {
        "metric": METRIC, "value": job_throughput(n_views * args.steps, world, pr_total), "unit": "views/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": pr_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 surrogate + u2 exact",
        "data": "synthetic",
        "config": {"workload": pruned_describe(), "views_per_step": n_views, "rays_per_view": 320 * 240,
                   "map": "512^3 u2", "scenes": f"seeds {seeds[0]}..{seeds[-1]} (timed: first {args.steps})",
                   "train": f"{TRAIN_ROOMS} seeded 256^3 rooms ({TRAIN_PRIMS} primitives) x 8 PoIs x 1024 views, "
                            f"exact labels, {args.train_epochs} epochs (before timing)",
                   "parallelism": f"replicas x{world}", "l2": "flushed before every timed arm (256 MiB write)",
                   "step": "pruned: map upload + nbt_plan_pruned (crops, forward, top-k, exact re-score, argmax); "
                           "exact: map upload + nbt_views_ig of all candidates + argmax"},
        "exact_views_per_s": job_throughput(n_views * args.steps, world, ex_total),
        "pruned_views_per_s": job_throughput(n_views * args.steps, world, pr_total),
        "speedup": ex_total / pr_total,
        "voxel_steps_per_s": world * vox_steps / (float(sum(kern_ms)) * 1e-3),
        "voxel_steps_per_exact_step": steps_per_launch,
        "exact_views_ig_ms": kern_mean,
        "same_best_view": {"agree": same, "cases": cases, "rate": same / max(1, cases), "wilson95": [lo, hi],
                           "target": 0.95, "scenes": n_eval,
                           "optimal_ig": {"agree": optimal, "rate": optimal / max(1, cases),
                                          "what": "pruned choice's exact IG equals the exact maximum"}},
        "pruning_baselines": {
            "exact_views_per_poi": keep,
            **{k: {"agree": v, "cases": cases, "rate": v / max(1, cases)} for k, v in base.items()},
            "idw_eq3_scheme": f"{k1} random candidates per PoI raycast, G(x) of Eq. 3 (p = 2, one ID) at the "
                              f"others, its top {k2} raycast; best of the {keep}"},
        "train": train_info,
        "scene_generation_s": gen_s,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": ncu_traffic("room512"), "kernel": "ig_warp_tiles_kernel<u2> (exact arm, + views_reduce)",
                     "algorithmic": f"0.25 B per voxel step x {steps_per_launch:.0f} steps per launch",
                     "peak_kind": f"{hbm_kind} (hbm_gbs)"},
        "roofline_alu": walk_alu_roofline(steps_per_launch, kern_mean, "ig_warp_tiles_kernel<u2> (exact arm, + views_reduce)"),
        "roofline_surrogate": {"bound": "tensor", "achieved": s_achieved, "peak": bf16, "unit": "TFLOP/s",
                               "frac": s_achieved / bf16, "traffic": ncu_traffic("surrogate_forward"),
                               "kernel": "surrogate forward (fused layers 0-1, layers 2-3, fc1, fc2)",
                               "algorithmic": f"{fl} FLOP per view (layer 0 as its K = 112 one-hot GEMM) x {n_views}",
                               "forward_ms_per_step": fwd_mean, "peak_kind": bf16_kind},
        "e2e": {"value": job_throughput(n_views * args.steps, world, e2e_total), "unit": "views/s",
                "h2d_bytes_per_step": int(grid_h.numel() + poses_h.numel() * 4),
                "d2h_bytes_per_step": int(best_h.numel() * 4 + val_h.numel() * 4)},
        # per timed step, pruned arm: upload (1) + brick summaries of the new map (5) + per batch of 4096
        # (crops, fused layers 0-1, layer 2, layer 3, features, fc1, fc1 reduce, fc2) + top-k + tile
        # kernel + reduce + argmax; exact arm: upload (1) + brick summaries (5) + tile kernel + reduce +
        # argmax
        "gpu_launches": ((1 + 5 + 8 * n_chunks + 4) + (1 + 5 + 3)) * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = pruned_cpu_baseline(scenes_w[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    net.close()
    m.close()


if __name__ == "__main__":
    main()
