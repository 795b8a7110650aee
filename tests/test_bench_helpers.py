"""Host-side logic of bench.py that the reported numbers depend on (no GPU)."""

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
