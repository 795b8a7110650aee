"""Host-side logic of bench.py that the reported numbers depend on (no GPU)."""

import argparse
import json

import pytest

import bench


def test_stored_traffic_only_for_the_sources_it_was_measured_on(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("// kernel v1\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    good = bench.kernel_hash(["kernel.cu"])
    table = {"w": {"kernel_hash": good, "bytes_per_launch": 1234, "sources": ["kernel.cu"]}}
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(table))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic("w") == 1234
    assert bench.ncu_traffic("other") is None
    src.write_text("// kernel v2\n")            # the kernel changed after the capture: no traffic claim
    assert bench.ncu_traffic("w") is None


def test_peak_falls_back_when_no_measured_peaks(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.5}))
    assert bench.load_peaks() == (6000.5, "measured")


def test_surrogate_flops_by_hand():
    # 32^3 crop, 3^3 convolutions 8->16 /2, 16->32 /2, 32->64 /2, 64->64 /1, fc 4104->128->1
    by_hand = (2 * 16 ** 3 * 16 * 27 * 8 + 2 * 8 ** 3 * 32 * 27 * 16 + 2 * 4 ** 3 * 64 * 27 * 32
               + 2 * 4 ** 3 * 64 * 27 * 64 + 2 * 4104 * 128 + 2 * 128)
    assert by_hand == 64_751_872
    assert bench.surrogate_flops_per_view() == by_hand


@pytest.mark.parametrize("name", ["prob256", "exact64", "room512", "traj256"])
def test_workload_descriptions_name_the_workload(name):
    class W:
        pass
    w = W()
    w.name = name
    assert bench.describe(w).startswith(name)


def test_every_workload_has_a_reference_arm():
    from workload import configs
    for name in bench.WORKLOAD_CHOICES:
        if name == "idw_cost" or name in bench.REFERENCE_ARMS:
            continue
        assert bench.reference_views_workload(name) in configs.WORKLOADS, name


@pytest.mark.parametrize("arm", ["insert", "fig3", "surrogate"])
def test_reference_arm_lines(arm):
    """The oracle arms of the non-view workloads print the native line's metric, unit and direction."""
    args = argparse.Namespace(steps=1, warmup=0, gpus=1, workload=arm)
    fn = bench.REFERENCE_ARMS[arm]
    line = fn(args) if arm == "fig3" else fn(args, budget_s=0.01)
    metric, unit, hib = {"insert": (bench.INSERT_METRIC, "points/s", True),
                         "fig3": (bench.FIG3_METRIC, "ms", False),
                         "surrogate": (bench.SURROGATE_METRIC, "views/s", True)}[arm]
    assert line["impl"] == "reference" and line["metric"] == metric and line["unit"] == unit
    assert line["higher_is_better"] is hib and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    json.dumps(line)


def test_step_defaults_per_workload_and_explicit_flags_win():
    a = bench.parse_args([])
    assert (a.workload, a.steps, a.warmup, a.gpus, a.impl) == ("room512-pruned", 25, 3, 1, "native")
    assert set(bench.DEFAULT_STEPS) == set(bench.WORKLOAD_CHOICES)
    assert all(w >= 3 for _, w in bench.DEFAULT_STEPS.values())
    b = bench.parse_args(["--workload", "room512"])
    assert (b.steps, b.warmup) == (20, 3)
    c = bench.parse_args(["--workload", "room512", "--steps", "7", "--warmup", "4"])
    assert (c.steps, c.warmup) == (7, 4)
    assert bench.parse_args(["--warmup", "1"]).warmup == 3        # never fewer than three warm-up steps


def test_wilson_interval_against_closed_cases():
    """The 95 % Wilson score interval: 39/40 gives a lower bound near 0.87 (far below a 95 % target),
    190/200 about 0.91, and k = n has an upper bound of exactly 1; the interval contains k / n."""
    lo, hi = bench.wilson_interval(39, 40)
    assert abs(lo - 0.8709) < 2e-3 and hi < 1.0
    lo, hi = bench.wilson_interval(190, 200)
    assert abs(lo - 0.9103) < 2e-3 and lo < 0.95 < hi
    lo, hi = bench.wilson_interval(200, 200)
    assert hi == 1.0 and abs(lo - 0.9812) < 2e-3
    for k, n in ((0, 10), (3, 7), (10, 10)):
        lo, hi = bench.wilson_interval(k, n)
        assert lo <= k / n <= hi


def test_surrogate_flop_counts():
    """Dense-equivalent forward: 2 x (16^3 16 216 + 8^3 32 432 + 4^3 64 864 + 4^3 64 1728) + fc; the method's
    own count replaces layer 0's K = 216 by the K = 112 one-hot GEMM the kernels run."""
    dense = 2 * (16 ** 3 * 16 * 216 + 8 ** 3 * 32 * 432 + 4 ** 3 * 64 * 864 + 4 ** 3 * 64 * 1728) + 2 * 4104 * 128 + 256
    assert bench.surrogate_flops_per_view() == dense
    assert dense - bench.surrogate_method_flops_per_view() == 2 * 16 ** 3 * 16 * (216 - 112)


def test_walk_alu_roofline_by_hand():
    # 2e9 voxel steps in 10 ms at 14 lane ops per step, against 128 lanes x 152 SMs x 2070 MHz
    r = bench.walk_alu_roofline(2e9, 10.0, "k")
    assert r["bound"] == "alu" and r["unit"] == "Glane-op/s"
    assert r["peak"] == pytest.approx(128 * 152 * 2070e6 / 1e9)
    assert r["achieved"] == pytest.approx(14 * 2e9 / 10e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
