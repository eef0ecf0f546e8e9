"""Parity at the full 1M-segment size, in the launch configuration bench.py
times (mixed precision, p = 7 on Chebyshev nodes, 7-level octree, cubic
unit-circle rule with Q = 16, SVD-compressed tensor-core M2L), and in the
dense-M2L configuration on equispaced nodes (FP16 Legendre moments with
residual passes on the low-order moments), on nodes the oracle computed one
by one: the direct Mura
sum of Eq. "stress3" against all 4M source points (oracle Q = 32, ~2e-10 in
h), stored in tests/golden/c3_sampled_forces.json by
tests/golden/make_c3_sampled_forces.py.  The 1e-4 bar of the method's
accuracy target applies to the bench configuration.  On a quarter-size
network the same configuration and the FP64 pass are held against stored
direct-sum forces too.
"""
import json
import os
import sys

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden", "c3_sampled_forces.json")


def _bench_workload(name):
    sys.path.insert(0, ROOT)
    import bench

    return bench.WORKLOADS[name]


@pytest.fixture(scope="module")
def c3_case():
    wl = _bench_workload("c3")
    nodes, segs, b = wl["gen"](0)
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    # the stored forces belong to exactly this network
    assert gold["n_nodes"] == len(nodes) and gold["n_segs"] == len(segs)
    assert gold["checks"]["sum_segs"] == int(segs.sum())
    assert abs(gold["checks"]["sum_nodes"] - nodes.sum()) <= 1e-9 * abs(nodes.sum())
    assert abs(gold["checks"]["sum_abs_b"] - np.abs(b).sum()) <= 1e-9 * np.abs(b).sum()
    ids = np.array(gold["node_ids"])
    assert np.allclose(nodes[ids], np.array(gold["node_xyz"]), rtol=0, atol=1e-12)
    return nodes, segs, b, wl, ids, np.array(gold["forces"])


def _forces(nodes, segs, b, wl, **over):
    import bench
    import paper_1712_07739_gb300 as gb

    kw = dict(p=wl["p"], levels=wl["levels"], precision=wl["precision"], h_mode=wl["h_mode"],
              circle_q=wl["circle_q"], **bench.m2l_options(wl))
    kw.update(over)
    if kw["precision"] != "mixed":  # the compressed M2L, Chebyshev nodes and the adaptive tree belong to the mixed pass
        kw.pop("nodes", None)
        kw.pop("m2l_svd_tol", None)
        kw.pop("refine_points", None)
    f = gb.FMM(**kw).set_material(wl["C"]())
    f.build(torch.tensor(nodes, device="cuda"), torch.tensor(segs, device="cuda"), torch.tensor(b, device="cuda"))
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    f.close()
    return F


@pytest.mark.parametrize("label,workload,over,tol", [
    pytest.param("bench configuration (adaptive tree)", "c3", {}, 1e-4, id="bench"),
    pytest.param("uniform 7-level tree", "c3u", {}, 1e-4, id="uniform"),
    pytest.param("Chebyshev, compressed M2L, p=8", "c3", {"p": 8}, 1e-4, id="p8"),
    pytest.param("equispaced, dense M2L", "c3legendre", {}, 1e-4, id="dense"),
    pytest.param("equispaced, compressed M2L", "c3svd", {}, 1e-4, id="svd"),
    pytest.param("dense M2L, FP64 interpolation stages", "c3legendre", {"precision": "mixed_f64t"}, 1e-4,
                 id="dense-f64t"),
    # order 6 on equispaced nodes is not enough for the slab walls: its interpolation error
    # alone (the FP64 pass at p = 6) is ~1.6e-4 against the direct sum
    pytest.param("dense M2L, p=6", "c3legendre", {"p": 6}, 3e-4, id="dense-p6"),
])
def test_full_size_sampled_nodes_match_direct_sum(c3_case, label, workload, over, tol):
    nodes, segs, b, _, ids, Fo = c3_case
    wl = _bench_workload(workload)
    F = _forces(nodes, segs, b, wl, **over)
    assert np.isfinite(F).all()
    err = np.linalg.norm(F[ids] - Fo) / np.linalg.norm(Fo)
    per = np.linalg.norm(F[ids] - Fo, axis=1) / np.linalg.norm(Fo, axis=1)
    print(f"1M segments, {label}: {len(ids)} sampled nodes vs direct sum: rel L2 {err:.3e}; "
          f"per node median {np.median(per):.2e}, max {per.max():.2e}")
    assert err < tol


def test_full_size_fp64_pass_matches_direct_sum(c3_case):
    """The plain FP64 pass at the bench's order and tree (the comparison arm
    bench.py times), against the same stored nodes."""
    nodes, segs, b, wl, ids, Fo = c3_case
    F = _forces(nodes, segs, b, wl, precision="fp64")
    err = np.linalg.norm(F[ids] - Fo) / np.linalg.norm(Fo)
    print(f"1M segments, FP64 pass p={wl['p']}: vs direct sum {err:.3e}")
    assert err < 1e-4


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


GOLDEN_Q = os.path.join(ROOT, "tests", "golden", "c3q_sampled_forces.json")


@pytest.mark.parametrize("p,prec", [(7, "mixed"), (8, "mixed"), (8, "mixed_f64t")])
def test_quarter_size_error_budget(p, prec):
    """250,000-segment slab network, 32 nodes against the direct sum (stored
    by tests/golden/make_c3q_sampled_forces.py): the FP64 pass shows the
    interpolation error of order p, the mixed pass adds the rounding error;
    both meet 1e-4 against the oracle."""
    wl = _bench_workload("c3q")
    nodes, segs, b = wl["gen"](0)
    with open(GOLDEN_Q) as fh:
        gold = json.load(fh)
    assert gold["n_segs"] == len(segs) and gold["checks"]["sum_segs"] == int(segs.sum())
    ids = np.array(gold["node_ids"])
    assert np.allclose(nodes[ids], np.array(gold["node_xyz"]), rtol=0, atol=1e-12)
    Fo = np.array(gold["forces"])
    Fd = _forces(nodes, segs, b, wl, p=p, precision="fp64", circle_q=32)
    Fm = _forces(nodes, segs, b, wl, p=p, precision=prec)
    e_d = np.linalg.norm(Fd[ids] - Fo) / np.linalg.norm(Fo)
    e_m = np.linalg.norm(Fm[ids] - Fo) / np.linalg.norm(Fo)
    print(f"250k segments, p={p}, {prec}: FP64 pass vs direct sum {e_d:.3e}, {prec} vs direct sum {e_m:.3e}")
    assert e_d < 1e-4 and e_m < 1e-4
