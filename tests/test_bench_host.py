"""Host-side pieces of bench.py's measurement: the algorithmic pair count behind
the roofline, the space-time roofline's arithmetic, and the rule that reports
the row kernel's DRAM traffic only while the captured sources are unchanged."""
import math
import os
import shutil

import numpy as np

import bench
from paper_2103_03348_b300 import synth


def brute_band_pairs(t, r, params):
    """Causal pairs (t_m < t_n) whose time gap is within the excitation's FP32
    underflow band, cut = (128 + max r log2 e) / (omega log2 e), by direct count."""
    log2e = 1.4426950408889634
    cut = (128.0 + float(np.max(r)) * log2e) / (params[4] * log2e)
    n = len(t)
    count = 0
    for i in range(n):
        for j in range(n):
            if t[j] < t[i] and t[i] - t[j] <= cut:
                count += 1
    return count


def test_band_pairs_match_a_direct_count():
    rng = np.random.default_rng(3)
    for omega, t_max in ((0.1, 200.0), (5.0, 60.0), (40.0, 20.0)):
        t = np.sort(np.round(rng.uniform(0.0, t_max, 400), 1))  # rounding makes ties
        r = rng.normal(0.0, 0.7, t.size)
        params = (0.5, 1.0, 1.0, 0.5, omega, 1.0)
        w = synth.Workload("t", np.zeros_like(t), np.zeros_like(t), t, r, params, np.ones(t.size, bool))
        assert bench.band_pairs(w) == brute_band_pairs(t, r, params)


def test_st_roofline_arithmetic():
    pairs = {"row_background_pairs": 1000, "row_excitation_pairs": 300, "column_pairs": 200}
    peak = 1.0e6  # slots per second
    out = bench.st_roofline(pairs, [2.0, 2.0], [1.0], peak)
    row_slots = 14 * 1000 + 7 * 300
    assert out["algorithmic_slots_per_launch"] == row_slots
    assert math.isclose(out["frac"], row_slots / 2.0e-3 / peak)
    assert math.isclose(out["col_frac"], 7 * 200 / 1.0e-3 / peak)
    assert out["row_background_pairs"] == 1000


def test_profile_traffic_follows_the_captured_sources(tmp_path, monkeypatch):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    csrc = root / "paper_2103_03348_b300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "row32_large_N100000.txt"), root / "profiles")
    for f in os.listdir(os.path.join(bench.ROOT, "paper_2103_03348_b300", "csrc")):
        if f.endswith((".cu", ".cuh")):
            shutil.copy(os.path.join(bench.ROOT, "paper_2103_03348_b300", "csrc", f), csrc)
    monkeypatch.setattr(bench, "ROOT", str(root))
    traffic = bench.profile_traffic()
    assert traffic is not None and traffic > 0
    with open(csrc / "row32_pair.cuh", "a") as fh:  # a change to any source the capture lists
        fh.write("\n// changed\n")
    assert bench.profile_traffic() is None
