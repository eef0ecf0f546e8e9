"""Pins of the oracle's Lagrange FMM (Algorithm 2) and its building blocks.

* Lagrange basis (Section 4.1 footnote): delta property, partition of unity,
  exact reproduction of polynomials of degree <= p-1.
* M2M/L2L transfer: the parent basis restricted to a child is reproduced
  exactly by the child's interpolant.
* Tree sets (Section 4, Eq. "mem_cheb" footnote and App. B): 27 neighbours,
  189 interaction cells for an interior cell, 316 distinct offsets overall.
* Theorem 1: the node kernel matrix of an offset depends on l - m only, with
  (2p-1)^3 distinct 54-blocks; Eq. "mem_unif" gives ~300 MB at p = 7 (FP64).
* Algorithm 2 (with M2M/L2L) equals Algorithm 1 applied to every
  interaction pair (no M2M/L2L) to rounding.
* Convergence to the direct sum of Eq. "stress3" at a rate near 3^-p
  (Section 5.2), and to ~1e-12 for a single loop inside one cell with a far
  target (Section 5.2, single-loop configuration).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import oracle_b as ob
from paper_1712_07739_gb300 import synth

ISO = oracle.Material.iso(1.0, 0.3)


@pytest.mark.parametrize("p", [2, 3, 4, 6, 8])
def test_basis_delta_unity_reproduction(p):
    nodes = np.arange(p) / (p - 1)
    assert np.allclose(ob.basis_1d(nodes, p), np.eye(p), atol=1e-14)
    t = np.linspace(-0.3, 1.3, 37)
    B = ob.basis_1d(t, p)
    assert np.allclose(B.sum(1), 1.0, atol=1e-12)
    for deg in range(p):
        assert np.allclose(B @ nodes ** deg, t ** deg, atol=1e-11)
    # degree p is not reproduced: the check has teeth
    assert not np.allclose(B @ nodes ** p, t ** p, atol=1e-6)


@pytest.mark.parametrize("p", [3, 5])
def test_child_transfer_exact(p):
    M = ob.child_transfer(p)
    t = np.linspace(0, 1, 11)
    for c in (0, 1):
        # parent basis evaluated at child-local t equals child interpolant of it
        direct = ob.basis_1d((c + t) / 2, p)             # [t, a']
        via = ob.basis_1d(t, p) @ M[c].T                 # sum_a ell_a(t) ell_a'(child node a)
        assert np.allclose(direct, via, atol=1e-13)


def test_tree_set_counts():
    offs = set()
    for c in itertools.product((0, 1), repeat=3):
        lst = ob.interaction_offsets((4 + c[0], 4 + c[1], 4 + c[2]))
        assert len(lst) == 189
        offs.update(lst)
    assert len(offs) == 316
    assert len(list(itertools.product((-1, 0, 1), repeat=3))) == 27
    assert all(max(abs(x) for x in o) in (2, 3) for o in offs)


@pytest.mark.parametrize("p", [3, 4])
def test_theorem1_toeplitz(p):
    T = ob._node_kernels(ISO, p, 0.25, (2, -1, 3))  # [l, 6, m, 9]
    idx = list(itertools.product(range(p), repeat=3))
    seen = {}
    for li, l in enumerate(idx):
        for mi, m in enumerate(idx):
            key = tuple(np.subtract(l, m))
            blk = T[li, :, mi, :]
            if key in seen:
                assert np.allclose(blk, seen[key], rtol=1e-12, atol=1e-12 * np.abs(blk).max())
            else:
                seen[key] = blk
    assert len(seen) == (2 * p - 1) ** 3


def _printed_values():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                q, arg, val, unit, tol, where = [x.strip() for x in line.split("|")]
                rows.append((q, arg, float(val), unit, float(tol), where))
    return rows


def _oracle_counts():
    """Operator count and kernel components from the oracle's own structures:
    the distinct offsets over the 8 child positions, and the width of one
    node-kernel block."""
    offs = set()
    for c in itertools.product((0, 1), repeat=3):
        offs.update(ob.interaction_offsets((4 + c[0], 4 + c[1], 4 + c[2])))
    T = ob._node_kernels(ISO, 2, 0.25, (2, 0, 0))  # [l, 6, m, 9]
    return len(offs), T.shape[1] * T.shape[3]


def _unique_blocks(p):
    T = ob._node_kernels(ISO, p, 0.25, (3, 1, -2))
    idx = list(itertools.product(range(p), repeat=3))
    keys = {tuple(np.round(T[li, :, mi, :].ravel() / np.abs(T).max(), 11))
            for li in range(len(idx)) for mi in range(len(idx))}
    return len(keys)


def test_printed_values_reproduced():
    """Every value in tests/golden/paper_printed_values.txt follows from the
    oracle: operator counts from its interaction lists, unique blocks counted
    on its node-kernel matrices, memory from Eq. "mem_unif" with those, the
    operators left by the cube's symmetries from its orbits of offsets."""
    n_ops, n_comp = _oracle_counts()
    rows = _printed_values()
    assert len(rows) == 8
    n_orbits = len(ob.offset_orbits())
    for q, arg, val, unit, tol, where in rows:
        if q == "lagrange_m2l_memory_fp64":
            p = int(arg.split("=")[1])
            got = n_comp * n_ops * (2 * p - 1) ** 3 * 8 / 1e9
        elif q == "kernel_components":
            got = n_comp
        elif q == "precomputed_operators":
            got = n_ops
        elif q == "toeplitz_unique_blocks":
            got = _unique_blocks(int(arg.split("=")[1]))
        elif q == "unique_operators_by_symmetry":
            got = n_orbits
        elif q == "symmetry_memory_ratio":
            got = n_ops / n_orbits
        else:
            raise AssertionError(q)
        assert abs(got - val) <= tol, (q, arg, got, val, where)


def _tiny(seed=0, n_loops=6, per=10):
    nodes, segs, b = synth.hexagon_loops(n_loops=n_loops, segs_per_loop=per, r_range=(0.05, 0.15), seed=seed)
    return nodes, segs, b, *oracle.quadrature(nodes, segs, b, 2)


def test_algorithm2_equals_pairwise_algorithm1():
    nodes, segs, b, y, q, sid = _tiny()
    a = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4)
    c = ob.pairwise_far_field(ISO, y, q, sid, p=3, L=4)
    assert np.max(np.abs(a - c)) <= 1e-11 * np.abs(c).max()


def test_convergence_rate_iso():
    nodes, segs, b, y, q, sid = _tiny(1, 8, 12)
    ref = oracle.direct_stress(ISO, y, sid, y, q, sid)
    errs = []
    for p in (2, 4, 6):
        s = ob.lagrange_fmm(ISO, y, q, sid, p=p, L=3)
        errs.append(oracle.rel_l2(s, ref))
    # ~3^-p decay: two orders of p must gain well over a factor 9 on average
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5, errs
    assert errs[2] < 1e-3


def test_single_loop_far_target_high_order():
    """One small loop inside a single leaf, target a few cells away (the
    paper's single-loop configuration): high order reaches ~1e-12."""
    nodes, segs = np.zeros((0, 3)), None
    th = 2 * np.pi * np.arange(3) / 3
    nodes = np.stack([0.12 + 0.05 * np.cos(th), 0.12 + 0.05 * np.sin(th), 0.12 + 0.0 * th], 1)
    nodes = np.concatenate([nodes, [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])  # corner markers set the root
    segs = np.array([[0, 1], [1, 2], [2, 0]], np.int64)
    b = np.tile([[0.0, 0.0, 1.0]], (3, 1))
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    # two zero-strength source points pin the root box to the unit cube
    y = np.concatenate([y, [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])
    q = np.concatenate([q, np.zeros((2, 3, 3))])
    sid = np.concatenate([sid, [-2, -3]])
    xt = np.array([[0.85, 0.9, 0.8]])
    ref = oracle.direct_stress(ISO, xt, [-1], y, q, sid)
    s = ob.lagrange_fmm(ISO, y, q, sid, p=10, L=3, xt=xt, tseg=np.array([-1]))
    assert oracle.rel_l2(s, ref) < 1e-10
