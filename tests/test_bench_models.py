"""Host-side pieces of bench.py: the algorithmic byte models of the roofline
and the reading of the committed ncu traffic summaries (no GPU needed)."""
import glob
import os

import numpy as np
import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sweep_bytes_per_row_and_wall():
    # MIXED (4-byte values): 8 bytes per slot (index + coefficient) and 20 per
    # fluid row (RHS, omega/D, count, p read, p written); 8 per wall entry and
    # 16 per wall row (count, 1/S, H, p_w)
    counts = np.full(10, 29)
    fluid, walls = bench.sweep_bytes(counts, 3, np.array([12, 12, 12]), 4)
    assert fluid == 10 * (8 * 29 + 20)
    assert walls == 3 * 12 * 8 + 3 * 16
    # FP64: 12 bytes per slot (4-byte index from the list, 8-byte coefficient)
    fluid, walls = bench.sweep_bytes(counts, 0, np.zeros(0), 8)
    assert fluid == 10 * (12 * 29 + 36) and walls == 0


def test_filter_bytes():
    # per particle 32 bytes, per skin entry 4 read, per kept entry 4 written
    assert bench.kernel_bytes("filter", True, 3, 7, 10, 50, 60, 90) == 10 * 32 + 4 * 90 + 4 * 60
    assert bench.kernel_bytes("no_such_site", True, 3, 1, 1, 1, 1, 1) is None


@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(ROOT, "profiles", "*_traffic.md"))))
def test_traffic_summaries_are_read_only_for_the_kernel_they_measured(path):
    name = os.path.basename(path)[:-len("_traffic.md")]
    site, workload = name.rsplit("_", 1)
    assert site in bench.SITES
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    ratio = float(vals["dram_bytes_per_algorithmic_byte"])
    assert ratio > 0
    current = bench.kernel_source_sha(site)
    got = bench.measured_traffic(workload, site, 1.0e9)
    if vals["kernel_source_sha1"] == current:
        assert got == pytest.approx(ratio * 1.0e9)
    else:
        assert got is None        # the kernel changed since the counters were taken
    assert bench.measured_traffic(workload, site, 0.0) is None


def test_launch_options_follow_the_tune_flag(tmp_path, monkeypatch):
    import argparse
    import workloads
    from paper_1908_01762_gb300 import autotune, sisph
    monkeypatch.setattr(autotune, "device_name", lambda: "GPU sm_103 x152")
    cases = [workloads.taylor_green(50)]
    path = str(tmp_path / "cache.json")
    args = argparse.Namespace(tune="off", tune_cache=path, tune_steps=5)
    assert bench.launch_options(args, cases, sisph.MIXED) == ({}, {"source": "library defaults"})
    args.tune = "cache"
    opts, note = bench.launch_options(args, cases, sisph.MIXED)
    assert opts == {} and note["source"].startswith("library defaults")
    autotune.tune(cases, sisph.MIXED, path=path, device="GPU sm_103 x152", sms=152,
                  timer=lambda o: 1.0 if o["block"] == 128 and o["skin"] == 0.1 else 2.0)
    opts, note = bench.launch_options(args, cases, sisph.MIXED)
    assert opts == {"block": 128, "skin": 0.1, "ppe_sync": 0}
    assert note == {"source": "autotune cache", **opts}
    # the shipped cache is what the benchmark reads by default
    assert os.path.dirname(autotune.DEFAULT_CACHE) == os.path.join(ROOT, "paper_1908_01762_gb300")


def test_cpu_sample_keeps_the_workloads_resolution():
    # the oracle is timed on a bounded sample of the same dam break: the same
    # dx and physics, tank and column scaled by 1/4 per axis (about 1/64 of
    # the particles); the batch on its first case
    import workloads
    big = workloads.dam_break_3d(dx=0.00524)
    sample, what = bench.cpu_sample("c4l", [big])
    assert sample["params"]["h"] == big["params"]["h"]
    assert sample["params"]["rho0"] == big["params"]["rho0"] and sample["dim"] == 3
    nf_big = int(np.sum(big["kind"] == 0))
    nf = int(np.sum(sample["kind"] == 0))
    assert 0.7 / 64 < nf / nf_big < 1.3 / 64
    assert "1/4" in what
    cases = workloads.batch_ensemble(64)
    sample, what = bench.cpu_sample("c5", cases)
    assert sample is cases[0]


def test_step_bytes_sums_the_modelled_sites():
    sites = {"ppe_sweeps": {"launches_per_step": 1.0}, "filter": {"launches_per_step": 2.0},
             "sync": {"launches_per_step": 2.0}}
    fb = bench.kernel_bytes("filter", True, 3, 7, 10, 50, 60, 90)
    assert bench.step_bytes(sites, 1000.0, True, 3, 7, 10, 50, 60, 90) == 1000.0 + 2 * fb
