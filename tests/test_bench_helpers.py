"""Host-side logic of bench.py (CPU): rank sharding of an ensemble, the
algorithmic work counts behind the roofline fraction, and the bounded
sample of the oracle baseline."""
import os
import sys

import numpy as np
import pytest

from paper_1712_07739_gb300 import synth

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_rank_configs_partition_the_ensemble():
    for world in (1, 2, 3, 8):
        parts = [bench.rank_configs(64, world, r) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1


def test_cubic_alignment_detection():
    assert bench.is_cubic_aligned(synth.cubic_voigt())
    assert bench.is_cubic_aligned(synth.isotropic_voigt(1.0, 0.3))
    assert not bench.is_cubic_aligned(synth.rotated_voigt(synth.cubic_voigt(), synth.rotation()))


def test_near_work_counts():
    work = {"near_pairs": 1000, "points": 10}
    wl = dict(bench.WORKLOADS["c3"])
    p = wl["p"]
    l2p = 10 * (12 * p ** 3 + 30 * p)
    flops, kernel = bench.near_flops(wl, work)
    assert kernel == "k_near_sym"
    # one unit-circle evaluation per unordered pair, one contraction per direction
    q = wl["circle_q"]
    assert flops == 1000 * ((193 * q + 77) / 2 + 229) + l2p
    one_sided = bench.near_pair_flops("mixed", "circle", q, True)
    assert 1000 * one_sided + l2p > flops
    general = dict(wl, C=lambda: synth.rotated_voigt(synth.cubic_voigt(), synth.rotation()))
    assert bench.near_flops(general, work)[0] > flops
    fp64, k64 = bench.near_flops(dict(wl, precision="fp64"), work)
    assert k64 == "k_near_sym64" and fp64 == flops  # the FP64 pass's symmetric kernel does the same work
    fiso, kfiso = bench.near_flops(dict(bench.WORKLOADS["c3_iso"], precision="fp64"), work)
    assert kfiso == "k_leaf_eval_f64" and fiso == 1000 * 341 + l2p
    iso, kiso = bench.near_flops(bench.WORKLOADS["c3_iso"], work)
    assert kiso == "k_near_mixed" and iso == 1000 * 202 + l2p


def test_oracle_sample_is_bounded_and_scaled():
    wl = bench.WORKLOADS["c1"]
    nodes, segs, b = wl["gen"](0)
    rate, used, desc, dt = bench.oracle_sample_rate(wl, nodes, segs, b, budget_s=1.0)
    assert rate > 0 and used >= 1 and dt < 30.0
    assert "source points" in desc and "segments/s" in desc
    assert np.isfinite(rate)


def test_roofline_traffic_belongs_to_its_capture():
    """The near field's DRAM traffic is reported only for a launch a capture
    describes: the uniform tree (250k capture, scaled by points) or the 1M
    headline on the adaptive tree (its own capture); anything else is null."""
    peaks = {"fp64_tflops": 1.0, "fp32_tflops": 80.0, "source": "test"}
    work = {"near_pairs": 3_627_757_324, "m2l_pairs": 18_013_294, "points": 4_000_000}
    head = dict(bench.WORKLOADS["c3"])
    assert head["refine_points"] == 128
    r = bench.roofline_of(head, work, 75.0, 170.0, 1, peaks, ranks={"r1": 832, "r2": 960})
    assert r["bound"] == "alu" and r["traffic"] == bench.NEAR_SYM_ADAPTIVE_1M_DRAM_BYTES
    uni = dict(bench.WORKLOADS["c3u"])
    r = bench.roofline_of(uni, work, 64.0, 190.0, 1, peaks, ranks={"r1": 832, "r2": 960})
    assert r["traffic"] == pytest.approx(bench.NEAR_SYM_DRAM_BYTES_PER_POINT * 4_000_000)
    other = dict(head, refine_points=64)
    r = bench.roofline_of(other, work, 75.0, 170.0, 1, peaks, ranks={"r1": 832, "r2": 960})
    assert r["traffic"] is None
