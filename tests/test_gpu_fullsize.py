"""Parity at the full 1M-segment size, in the launch configuration bench.py
times (mixed precision, p = 6, 7-level octree, cubic unit-circle rule with
Q = 20), on nodes the oracle can compute one by one: the direct Mura sum of
Eq. "stress3" against all 4M source points (oracle Q = 32, ~2e-10 in h).
"""
import os
import sys

import numpy as np
import pytest

import oracle
from paper_1712_07739_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_workload(name):
    sys.path.insert(0, ROOT)
    import bench

    return bench.WORKLOADS[name]


@pytest.fixture(scope="module")
def c3_case():
    wl = _bench_workload("c3")
    nodes, segs, b = wl["gen"](0)
    rng = np.random.default_rng(2024)
    ids = rng.choice(len(nodes), 4, replace=False)
    mat = oracle.Material.aniso(wl["C"](), Q=32)
    Fo, used = oracle.sampled_node_forces(mat, nodes, segs, b, ids)
    return nodes, segs, b, wl, ids, Fo, used


def _forces(nodes, segs, b, wl, **over):
    import paper_1712_07739_gb300 as gb

    kw = dict(p=wl["p"], levels=wl["levels"], precision=wl["precision"], h_mode=wl["h_mode"], circle_q=wl["circle_q"])
    kw.update(over)
    f = gb.FMM(**kw).set_material(wl["C"]())
    f.build(torch.tensor(nodes, device="cuda"), torch.tensor(segs, device="cuda"), torch.tensor(b, device="cuda"))
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    return F


@pytest.mark.parametrize("label,over", [("bench configuration", {}),
                                        ("BF16 split on all offsets, Q=32", {"m2l_split": 2, "circle_q": 32}),
                                        ("FP16 scaled operands", {"m2l_split": 4}),
                                        ("p=7, FP16 scaled operands", {"p": 7, "m2l_split": 4})])
def test_full_size_sampled_nodes_match_direct_sum(c3_case, label, over):
    nodes, segs, b, wl, ids, Fo, used = c3_case
    F = _forces(nodes, segs, b, wl, **over)
    assert np.isfinite(F).all()
    err = np.linalg.norm(F[ids] - Fo) / np.linalg.norm(Fo)
    print(f"1M segments, {label}: {len(ids)} sampled nodes vs direct sum ({used} threads): rel L2 {err:.3e}")
    assert err < 1e-3


def test_full_size_repeatable_and_linear_in_b():
    """Properties that hold at any size: a second pass gives bit-identical
    forces (fixed summation orders everywhere; each node receives exactly two
    end forces), and scaling every Burgers vector by 2 scales the forces by
    4 (the stress is linear in b, the force linear in stress and b)."""
    import paper_1712_07739_gb300 as gb

    wl = _bench_workload("c3")
    nodes, segs, b = wl["gen"](0)
    f = gb.FMM(p=wl["p"], levels=wl["levels"], precision=wl["precision"], h_mode=wl["h_mode"],
               circle_q=wl["circle_q"]).set_material(wl["C"]())
    dn, ds = torch.tensor(nodes, device="cuda"), torch.tensor(segs, device="cuda")
    f.build(dn, ds, torch.tensor(b, device="cuda"))
    F1 = f.nodal_forces().cpu().numpy()
    F2 = f.nodal_forces().cpu().numpy()
    assert np.array_equal(F1, F2)
    f.build(dn, ds, torch.tensor(2.0 * b, device="cuda"))
    F4 = f.nodal_forces().cpu().numpy()
    assert np.linalg.norm(F4 - 4.0 * F1) <= 1e-6 * np.linalg.norm(F1)
