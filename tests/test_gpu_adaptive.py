"""The adaptive tree on the GPU (leaves holding more than ``refine_points``
points split once more; Sec. 3's adaptive octree) against the FP64 oracle.

* Small slab networks, cubic medium with the unit-circle h, Chebyshev nodes
  and the compressed M2L: the GPU's nodal forces against the oracle's
  ``adaptive_fmm`` (same split rule, same node set, the oracle's own SVD
  bases at the GPU's ranks), so the difference is rounding alone: 1e-4.
  Thresholds that split a few leaves, most leaves and every occupied leaf;
  at order 3 the adaptive and the uniform tree differ by 1e-4 to 1e-3 where
  many leaves split, and the GPU sits well inside that gap.
* A threshold above every leaf's count splits nothing: the pass equals the
  uniform tree's.
* Work counts: splitting removes near pairs (non-adjacent children of two
  split leaves) and adds M2L pairs one level down.
* The 1M-segment slab network of the bench with a refinement threshold,
  against the stored direct-sum forces at 32 nodes (1e-4).
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import oracle_b
from paper_1712_07739_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUB_C = synth.cubic_voigt()
Q = 16
P, LEV, TOL = 3, 4, 1e-4  # p = 3: the trees' approximations differ well above rounding


def _gpu(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _fmm(refine, **kw):
    import paper_1712_07739_gb300 as gb

    args = dict(p=P, levels=LEV, precision="mixed", h_mode="circle", circle_q=Q, nodes="chebyshev",
                m2l_svd_tol=TOL)
    args.update(kw)
    return gb.FMM(refine_points=refine, **args).set_material(CUB_C)


def _gpu_run(net, refine, **kw):
    xyz, segs, b = net
    f = _fmm(refine, **kw)
    f.build(_gpu(xyz), _gpu(segs), _gpu(b))
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    out = dict(F=F, ranks=f.m2l_ranks(), work=f.work_counts())
    f.close()
    return out


@pytest.fixture(scope="module")
def net():
    return synth.slab_loops(n_loops=40, segs_per_loop=16, n_slabs=3, seed=5)


@pytest.fixture(scope="module")
def leaf_counts(net):
    xyz, segs, b = net
    y, q, sid = oracle.quadrature(xyz, segs, b, 4)
    origin, H = oracle_b.root_box(y)
    n = 1 << (LEV - 1)
    sl = oracle_b.cell_of(y, origin, H, LEV - 1)
    cnt = np.bincount((sl[:, 0] * n + sl[:, 1]) * n + sl[:, 2], minlength=n ** 3)
    return cnt[cnt > 0]


@pytest.fixture(scope="module")
def oracle_side(net):
    """The oracle's medium, quadrature and SVD bases (at the GPU's ranks)."""
    xyz, segs, b = net
    mat = oracle.Material.aniso(CUB_C, Q=Q)
    ranks = _gpu_run(net, 0)["ranks"]
    U, R, _, _ = oracle_b.m2l_svd_bases(mat, P, "chebyshev", ranks=(ranks["r1"], ranks["r2"]))
    return mat, oracle.quadrature(xyz, segs, b, 4), (U, R), ranks


@pytest.mark.parametrize("refine", [100, 40, 1])
def test_adaptive_matches_oracle(net, leaf_counts, oracle_side, refine):
    xyz, segs, b = net
    mat, (y, q, sid), svd, ranks = oracle_side
    n_split = int((leaf_counts > refine).sum())
    assert 0 < n_split  # every case splits something
    if refine == 1:
        assert n_split == int((leaf_counts > 1).sum())
    g = _gpu_run(net, refine)
    assert g["ranks"]["r1"] == ranks["r1"] and g["ranks"]["r2"] == ranks["r2"]
    sig = oracle_b.adaptive_fmm(mat, y, q, sid, p=P, L=LEV, refine=refine, nodes="chebyshev", svd=svd)
    Fo = oracle.nodal_forces(xyz, segs, b, sig, 4)
    err = _rel(g["F"], Fo)
    # the adaptive tree is a different approximation than the uniform one
    sig_u = oracle_b.lagrange_fmm(mat, y, q, sid, p=P, L=LEV, nodes="chebyshev", svd=svd)
    gap = _rel(oracle.nodal_forces(xyz, segs, b, sig_u, 4), Fo)
    print(f"refine {refine}: {n_split}/{len(leaf_counts)} leaves split; GPU vs oracle {err:.2e}; "
          f"adaptive vs uniform {gap:.2e}")
    assert err <= 1e-4
    if gap > 5e-5:  # the GPU follows the adaptive tree, not the uniform one
        assert err < gap / 5


def test_no_split_equals_uniform_tree(net, leaf_counts):
    big = int(leaf_counts.max())
    a = _gpu_run(net, big)
    u = _gpu_run(net, 0)
    assert _rel(a["F"], u["F"]) <= 1e-6
    assert a["work"] == u["work"]


def test_work_counts_follow_the_split(net, leaf_counts):
    u = _gpu_run(net, 0)["work"]
    a = _gpu_run(net, 1)["work"]
    assert a["near_pairs"] < u["near_pairs"]
    assert a["m2l_pairs"] > u["m2l_pairs"]
    assert a["occupied_leaves"] == u["occupied_leaves"] and a["points"] == u["points"]


def test_refine_needs_compressed_circle_pass():
    import paper_1712_07739_gb300 as gb

    for kw in (dict(m2l_svd_tol=0.0, nodes="equispaced"), dict(h_mode="iso"), dict(refine=-1)):
        r = kw.pop("refine", 8)
        with pytest.raises(gb.GbfmmError):
            _fmm(r, **kw)


def test_fullsize_adaptive_against_direct_sum():
    """The 1M-segment slab network of the bench's headline (p = 7 on
    Chebyshev nodes, 7 levels with the leaves above the refinement threshold
    split, unit-circle Q = 16, cubic, compressed M2L), against the stored
    direct-sum forces at 32 nodes."""
    import sys

    sys.path.insert(0, ROOT)
    import bench
    import paper_1712_07739_gb300 as gb

    wl = bench.WORKLOADS["c3"]
    nodes, segs, b = wl["gen"](0)
    with open(os.path.join(ROOT, "tests", "golden", bench.GOLDEN["c3"])) as fh:
        gold = json.load(fh)
    ids = np.array(gold["node_ids"])
    f = gb.FMM(p=wl["p"], levels=wl["levels"], precision=wl["precision"], h_mode=wl["h_mode"],
               circle_q=wl["circle_q"], **bench.m2l_options(wl)).set_material(wl["C"]())
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    err = _rel(F[ids], np.array(gold["forces"]))
    print(f"1M slabs, adaptive tree (refine {wl['refine_points']}): {err:.3e} against the direct sum; "
          f"work {f.work_counts()}")
    assert err <= 1e-4
    f.close()
