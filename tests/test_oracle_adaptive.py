"""Pins of the oracle's adaptive tree (the uniform tree of Algorithm 2 with
the leaves holding more than a threshold of points split once more).

* Nothing split: it is Algorithm 2 on the uniform tree, exactly.
* Every occupied leaf split: it is Algorithm 2 on one more level (same
  multipoles up to summation order, the same level-L interaction lists and
  the same near field, the 27 neighbours at level L), to rounding.  Both
  limits share no code path for the split leaves' near field and M2L with
  the uniform pass, so a pair counted twice or missed fails here.
* Part split: the pass converges to the direct sum of Eq. "stress3" as p
  grows, as the uniform pass does, and its error stays at the uniform
  passes' level.
"""
import numpy as np

import oracle
from oracle import oracle_b as ob
from paper_1712_07739_gb300 import synth

ISO = oracle.Material.iso(1.0, 0.3)


def _net():
    nodes, segs, b = synth.slab_loops(n_loops=40, segs_per_loop=16, n_slabs=3, seed=5)
    return oracle.quadrature(nodes, segs, b, 2)


def test_no_split_is_algorithm2():
    y, q, sid = _net()
    a = ob.adaptive_fmm(ISO, y, q, sid, p=3, L=4, refine=10 ** 9)
    b = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4)
    assert np.array_equal(a, b)


def test_all_split_is_algorithm2_one_level_deeper():
    y, q, sid = _net()
    a = ob.adaptive_fmm(ISO, y, q, sid, p=3, L=4, refine=0)
    b = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=5)
    assert oracle.rel_l2(a, b) < 1e-12
    # and it is not the uniform pass at L: the split changes the result
    c = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4)
    assert oracle.rel_l2(a, c) > 1e-6


def test_part_split_converges_to_direct_sum():
    y, q, sid = _net()
    origin, H = ob.root_box(y)
    sl = ob.cell_of(y, origin, H, 3)
    cnt = np.unique(sl[:, 0] * 64 + sl[:, 1] * 8 + sl[:, 2], return_counts=True)[1]
    refine = 20
    assert 0 < (cnt > refine).sum() < len(cnt)  # some leaves split, some not
    ref = oracle.direct_stress(ISO, y, sid, y, q, sid)
    errs = [oracle.rel_l2(ob.adaptive_fmm(ISO, y, q, sid, p=p, L=4, refine=refine), ref) for p in (2, 4, 6)]
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5, errs
    uni = max(oracle.rel_l2(ob.lagrange_fmm(ISO, y, q, sid, p=4, L=L), ref) for L in (4, 5))
    assert errs[1] < 2 * uni
