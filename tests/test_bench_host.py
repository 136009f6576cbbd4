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
