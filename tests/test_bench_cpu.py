"""CPU: bench.py's host helpers - the DRAM-traffic lookup keyed by the kernel
source it was captured on, the clock-sample summary that decides whether a
timed run is kept, the HBM peak lookup and the oracle's z-slab sample of the
sphere workload, and the reference arm on ranks other than 0."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_traffic_is_reported_only_for_the_source_it_was_captured_on(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    entry = {"source": "k.cu", "source_sha256_16": bench.source_hash(str(src)),
             "dram_bytes_per_launch": 123.0}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"stage2": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("stage2") == 123.0
    assert bench.traffic_for("stage1") is None          # no capture of that kernel
    src.write_text("kernel v2\n")
    assert bench.traffic_for("stage2") is None          # the source changed since


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        t = json.load(f)
    kernels = [k for k in t if not k.startswith("_")]
    assert {"stage1", "stage2", "batch_stage1", "batch_stage2"} <= set(kernels)
    for k in kernels:
        e = t[k]
        assert os.path.exists(os.path.join(ROOT, e["source"])), k
        assert len(e["source_sha256_16"]) == 16 and e["dram_bytes_per_launch"] > 0


class _Finished:
    """Stands in for the nvidia-smi sampler process once it has exited."""

    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _sampler_with(rows, tmp_path):
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = _Finished()
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s.f = open(s.path)
    return s


def test_clock_summary_takes_the_median_clock_and_the_active_reasons(tmp_path):
    rows = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1100.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "not a sample"]
    r = _sampler_with(rows, tmp_path).stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] == 3
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clock_summary_reports_a_thermal_slowdown(tmp_path):
    rows = ["0, 1500, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active",
            "0, 1600, 2070, 1300.0, 0x40, Active, Active, Not Active, Not Active"]
    r = _sampler_with(rows, tmp_path).stop()
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert r["sm_mhz"] == 1550.0


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.proc = None
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_hbm_peak_is_the_measured_one_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6787.6}))
    assert bench.measured_peaks() == (6787.6, "measured")


def test_oracle_slab_keeps_the_sphere_markers_whose_support_fits():
    c = bench.C.heated_sphere(n=64)
    for nz in (8, 16, 40, 64, 200):
        gs, X, Tw = bench.oracle_slab(c, nz)
        want = max(8, min(nz, c.grid.n[2]))
        assert gs.n == (c.grid.n[0], c.grid.n[1], want) and gs.h == c.grid.h
        assert gs.lo[2] == -0.5 * want * gs.h and gs.lo[:2] == c.grid.lo[:2]
        cz = np.floor((X[:, 2] - gs.lo[2]) / gs.h)
        assert len(X) == len(Tw) and len(X) > 0
        assert cz.min() >= 2 and cz.max() <= want - 3
        # every marker of the full set whose owner plane fits is kept
        cz_all = np.floor((c.X[:, 2] - gs.lo[2]) / gs.h)
        assert len(X) == int(((cz_all >= 2) & (cz_all <= want - 3)).sum())
    gs, X, _ = bench.oracle_slab(c, c.grid.n[2])
    assert len(X) == len(c.X)          # the whole grid keeps every marker


def test_reference_arm_runs_on_rank_0_only(capsys):
    """Under torchrun the oracle arm is timed and printed by rank 0 alone;
    every other rank exits 0 without work or output."""
    import argparse
    args = argparse.Namespace(gpus=2, steps=1, warmup=1, n=256, workload="sphere",
                              impl="reference", cpu_seconds=1.0, no_cpu_baseline=True, every=50)
    for run in (bench.run_reference, bench.run_reference_batched):
        assert run(args, 1, 2) == 0
    assert capsys.readouterr().out == ""
