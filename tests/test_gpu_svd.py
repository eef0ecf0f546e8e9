"""The SVD-compressed M2L (Sec. 3, the Chebyshev FMM's compression) on
equispaced and Chebyshev nodes, against the FP64 oracle.

* Small networks: the mixed pass with the compressed M2L against the
  oracle's Algorithm 2 with the same node set and the same compression (the
  oracle builds its own bases from the 316 operators, at the ranks the GPU
  reports), so the difference is rounding alone: bar 1e-4.
* The oracle's ranks at the GPU's tolerance are the GPU's counts above the
  tolerance (the same singular values, computed independently).
* The 1M-segment slab network with the compressed M2L at the bench's
  tolerance against the stored direct-sum forces at 32 nodes (1e-4).
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
ISO_C = synth.isotropic_voigt(1.0, 0.3)
CUB_C = synth.cubic_voigt()
ISO = oracle.Material.iso(1.0, 0.3)


def _gpu(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu_forces(xyz, segs, b, C, **kw):
    import paper_1712_07739_gb300 as gb

    f = gb.FMM(**kw).set_material(C)
    f.build(_gpu(xyz), _gpu(segs), _gpu(b))
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    ranks = f.m2l_ranks()
    f.close()
    return F, ranks


def _oracle_forces(xyz, segs, b, mat, p, L, node_set, svd):
    y, q, sid = oracle.quadrature(xyz, segs, b, 4)
    sig = oracle_b.lagrange_fmm(mat, y, q, sid, p=p, L=L, nodes=node_set, svd=svd)
    return oracle.nodal_forces(xyz, segs, b, sig, 4)


@pytest.fixture(scope="module")
def loops():
    return synth.slab_loops(n_loops=40, segs_per_loop=16, n_slabs=3, seed=5)


@pytest.mark.parametrize("node_set,tol", [("equispaced", 1e-3), ("chebyshev", 1e-3), ("chebyshev", 1e-5)])
def test_compressed_m2l_matches_oracle(loops, node_set, tol):
    xyz, segs, b = loops
    p, L = 4, 4
    F, ranks = _gpu_forces(xyz, segs, b, ISO_C, p=p, levels=L, precision="mixed", nodes=node_set, m2l_svd_tol=tol)
    P3 = p ** 3
    assert ranks["r1"] % 16 == 0 or ranks["r1"] == 6 * P3
    assert ranks["r2"] % 64 == 0 or ranks["r2"] == 9 * P3
    assert 0 < ranks["r1_raw"] <= ranks["r1"] <= 6 * P3 and 0 < ranks["r2_raw"] <= ranks["r2"] <= 9 * P3
    # the oracle's own bases: its counts above the tolerance are the GPU's
    U, R, st, ss = oracle_b.m2l_svd_bases(ISO, p, node_set, ranks=(ranks["r1"], ranks["r2"]))
    assert int((st > tol * st[0]).sum()) == ranks["r1_raw"]
    assert int((ss > tol * ss[0]).sum()) == ranks["r2_raw"]
    assert np.isclose(st[0], ranks["sigma"][0], rtol=1e-6) and np.isclose(ss[0], ranks["sigma"][2], rtol=1e-6)
    Fo = _oracle_forces(xyz, segs, b, ISO, p, L, node_set, (U, R))
    err = _rel(F, Fo)
    plain = _oracle_forces(xyz, segs, b, ISO, p, L, node_set, None)
    print(f"{node_set} tol {tol}: ranks {ranks['r1']}/{6 * P3}, {ranks['r2']}/{9 * P3}; GPU vs oracle {err:.2e}; "
          f"compression alone {_rel(Fo, plain):.2e}")
    assert err <= 1e-4


def test_chebyshev_needs_compressed_mixed_pass():
    import paper_1712_07739_gb300 as gb

    for kw in (dict(precision="fp64", nodes="chebyshev"), dict(precision="mixed", nodes="chebyshev"),
               dict(precision="fp64", m2l_svd_tol=1e-5)):
        with pytest.raises(gb.GbfmmError):
            gb.FMM(p=4, **kw)


def test_fullsize_compressed_m2l_against_direct_sum():
    """The 1M-segment slab network (bench.py c3: p = 7 on Chebyshev nodes, 7
    levels, unit-circle Q = 16, cubic) with the compressed M2L at the bench's
    tolerance, against the stored direct-sum forces at 32 nodes; the ranks
    kept are well below the 6 p^3 / 9 p^3 of the dense operators."""
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
    r = f.m2l_ranks()
    err = _rel(F[ids], np.array(gold["forces"]))
    print(f"1M slabs, compressed M2L {r}: {err:.3e} against the direct sum")
    assert err <= 1e-4
    P3 = wl["p"] ** 3
    assert r["r1"] * r["r2"] < 0.25 * (6 * P3) * (9 * P3)
    f.close()
