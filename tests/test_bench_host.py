"""Host-side figures of bench.py (no GPU): the utilisation figures derived
from a region trace and the shared-memory line."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_trace_utilisation_on_a_hand_made_trace():
    # two CTAs, 30 ns of span; regions busy 10 + 10 + 20 = 40 ns
    tr = np.array([[100, 110], [105, 115], [110, 130]], dtype=np.uint64)
    u = bench.trace_utilisation(tr, ctas=2)
    assert u["regions"] == 3
    assert u["cta_busy_fraction"] == pytest.approx(40 / (2 * 30))
    assert u["mean_regions_in_flight"] == pytest.approx(40 / 30)
    assert u["mean_region_us"] == pytest.approx(40 / 3 / 1e3)


def test_smem_line_uses_the_sampled_clock():
    r = bench.smem_roofline(1_000_000, 1.0, {"sm_mhz": 1000.0})
    assert r["peak"] == pytest.approx(152 * 128 * 1e9 / 1e9)
    assert r["achieved"] == pytest.approx(96 * 1e6 / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    m = bench.smem_roofline(1_000_000, 1.0, {"sm_mhz": 1000.0}, measured_gbs=30000.0)
    assert m["peak"] == 30000.0 and m["peak_kind"].startswith("measured")


def test_alu_line_counts_the_site_update_flops():
    r = bench.alu_roofline(2_000_000, 2.0, 50.0)
    assert r["achieved"] == pytest.approx(41 * 2e6 / 2e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 50.0) and r["bound"] == "alu"


@pytest.mark.parametrize("shape", ["split", "lattice"])
def test_traffic_record_is_used_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch, shape):
    """roofline.traffic comes from the committed ncu record of the kernel
    (region or lattice) only while every source that shapes that kernel's
    memory traffic is byte-identical to the one the record was taken on and
    the region base is the record's; it is the record's bytes per site-update
    times the launch's site-updates."""
    import hashlib
    import json

    for i, rel in enumerate(bench.KERNEL_SOURCES[shape]):
        p = tmp_path / rel
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_text(f"source {i}\n")
    h = hashlib.sha256()
    for rel in bench.KERNEL_SOURCES[shape]:
        h.update((tmp_path / rel).read_bytes())
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / bench.TRAFFIC_RECORD[shape]).write_text(json.dumps({
        "kernel_sources_sha256_16": h.hexdigest()[:16], "region_base": 16, "site_updates": 4,
        "dram_bytes_read_per_launch": 7, "dram_bytes_write_per_launch": 5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic(16, 4, shape) == 12
    assert bench.ncu_traffic(16, 40, shape) == 120
    assert bench.ncu_traffic(32, 4, shape) is None
    other = "lattice" if shape == "split" else "split"
    assert bench.ncu_traffic(16, 4, other) is None  # the other kernel's record is absent here
    (tmp_path / bench.KERNEL_SOURCES[shape][0]).write_text("changed\n")
    assert bench.ncu_traffic(16, 4, shape) is None


def test_lattice_layers_match_the_library():
    """The bench counts a lattice call's regions with the layer rule of
    lattice.h: three layers cut by the call's first level plus one per s
    levels."""
    assert bench.lattice_layers(16, 128) == 35 and bench.lattice_layers(16, 64) == 19
    assert bench.lattice_layers(8, 1) == 4 and bench.lattice_layers(24, 50) == 12


def test_pass_schedule_continues_and_restarts():
    """Bench steps continue the run and start over (a restore) only when the
    next step would pass the run's last level."""
    assert bench.pass_schedule(5, 64, 2048) == [0, 64, 128, 192, 256]
    s = bench.pass_schedule(40, 64, 2048)
    assert s[31] == 1984 and s[32] == 0 and s[33] == 64
    assert bench.pass_schedule(3, 256, 256) == [0, 0, 0]


def test_clock_parsing_reports_median_and_reasons():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1900, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2000, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.parse_clocks(lines)
    assert c == {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}


@pytest.mark.parametrize("shape,kernel", [("split", "region_kernel"), ("lattice", "lattice_kernel")])
def test_committed_traffic_record_names_its_capture(shape, kernel):
    import json

    rec = json.load(open(os.path.join(ROOT, "profiles", bench.TRAFFIC_RECORD[shape])))
    assert rec["kernel"] == kernel and "ncu" in rec["command"] and "--clock-control none" in rec["command"]
    assert f"regex:{kernel}" in rec["command"]
    assert rec["region_base"] in (8, 16, 32) and rec["site_updates"] > 0
    assert rec["dram_bytes_read_per_launch"] > 0 and rec["dram_bytes_write_per_launch"] > 0


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints
    one JSON line with the fields the driver reads, on the same metric and
    workload as the GPU arm."""
    import json
    import subprocess

    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "site-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == bench.workload_name(bench.BIG)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
