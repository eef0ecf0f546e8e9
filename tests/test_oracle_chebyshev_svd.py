"""Pins of the oracle's Chebyshev-node FMM with SVD-compressed M2L (Sec. 3,
the Chebyshev FMM the paper compares against, Eq. "mem_cheb").

* Chebyshev nodes: the p zeros of T_p mapped to [0, 1] (checked with
  numpy's Chebyshev series, not with the cosine formula), and the 3-D basis
  on them reproduces every polynomial of degree <= p - 1 per axis.
* Transfers: Algorithm 2 on Chebyshev nodes equals the pairwise far field
  of Eq. "far-field" (no M2M/L2L), as on equispaced nodes, since the child
  interpolant reproduces the parent's polynomial exactly.
* Convergence: the Chebyshev-node FMM converges to the direct sum of
  Eq. "stress3" as p grows.
* SVD bases: the singular values equal those of a library SVD of the 316
  operators side by side (target side) and stacked (source side), and the
  energy the truncation drops equals the sum of the dropped squared
  singular values (Eckart-Young), computed from the operators themselves.
* Source null space: a strength q_wr = delta_wr (trace only) at any node
  produces no stress (the contraction of the antisymmetric epsilon with the
  symmetric C in the A tensor of Sec. 2 annihilates it), so the stacked
  operators have exactly p^3 zero singular values.
* Compressed M2L: at full rank it is the plain M2L; dropping only the null
  space changes nothing; at a tolerance of 1e-3 it stays within 1e-3 of it,
  while at 1e-2 it visibly does not.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import oracle
from oracle import oracle_b as ob
from paper_1712_07739_gb300 import synth

ISO = oracle.Material.iso(1.0, 0.3)


@pytest.mark.parametrize("p", [2, 3, 5, 8])
def test_chebyshev_nodes_are_zeros_of_Tp(p):
    t = ob.node_positions(p, "chebyshev")
    assert np.all(np.diff(t) > 0) and t[0] > 0 and t[-1] < 1
    Tp = npcheb.chebval(2.0 * t - 1.0, [0.0] * p + [1.0])
    assert np.max(np.abs(Tp)) < 1e-12
    # the roots of T_p from numpy, mapped to [0, 1]
    roots = np.sort((npcheb.chebroots([0.0] * p + [1.0]) + 1.0) / 2.0)
    assert np.allclose(t, roots, atol=1e-12)


@pytest.mark.parametrize("p", [3, 5])
def test_chebyshev_basis_reproduces_polynomials(p):
    rng = np.random.default_rng(p)
    c = rng.normal(size=(p, p, p))
    f = lambda x: np.einsum("ijk,ni,nj,nk->n", c, x[:, :1] ** np.arange(p), x[:, 1:2] ** np.arange(p),
                            x[:, 2:] ** np.arange(p))
    t = ob.node_positions(p, "chebyshev")
    grid = np.array([(a, b, cc) for a in t for b in t for cc in t])  # x slowest, as basis_3d flattens
    x = rng.uniform(-0.2, 1.2, size=(40, 3))
    got = ob.basis_3d(x, p, "chebyshev") @ f(grid)
    assert np.allclose(got, f(x), rtol=1e-10, atol=1e-10)
    # degree p in one variable is not reproduced
    g = lambda x: x[:, 1] ** p
    assert not np.allclose(ob.basis_3d(x, p, "chebyshev") @ g(grid), g(x), atol=1e-6)


def _tiny(seed=0, n_loops=6, per=10):
    nodes, segs, b = synth.hexagon_loops(n_loops=n_loops, segs_per_loop=per, r_range=(0.05, 0.15), seed=seed)
    return nodes, segs, b, *oracle.quadrature(nodes, segs, b, 2)


def test_chebyshev_algorithm2_equals_pairwise():
    nodes, segs, b, y, q, sid = _tiny()
    a = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4, nodes="chebyshev")
    c = ob.pairwise_far_field(ISO, y, q, sid, p=3, L=4, nodes="chebyshev")
    assert np.max(np.abs(a - c)) <= 1e-11 * np.abs(c).max()
    # and it is a different approximation than the equispaced one
    e = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4)
    assert np.max(np.abs(a - e)) > 1e-6 * np.abs(e).max()


def test_chebyshev_convergence():
    nodes, segs, b, y, q, sid = _tiny(1, 8, 12)
    ref = oracle.direct_stress(ISO, y, sid, y, q, sid)
    errs = [oracle.rel_l2(ob.lagrange_fmm(ISO, y, q, sid, p=p, L=3, nodes="chebyshev"), ref) for p in (2, 4, 6)]
    assert errs[1] < errs[0] / 5 and errs[2] < errs[1] / 5, errs
    assert errs[2] < 1e-3


@pytest.fixture(scope="module")
def bases_p3():
    U, R, st, ss = ob.m2l_svd_bases(ISO, 3, "chebyshev", ranks=(162, 243))
    return U, R, st, ss


def _operators(p, nodes):
    P3 = p ** 3
    return [ob._node_kernels(ISO, p, 1.0, o, nodes=nodes).reshape(6 * P3, 9 * P3) for o in ob.m2l_offsets()]


def test_svd_singular_values_match_library_svd(bases_p3):
    U, R, st, ss = bases_p3
    ops = _operators(3, "chebyshev")
    assert len(ops) == 316
    fat = np.concatenate(ops, axis=1)   # [T_1 ... T_316]
    thin = np.concatenate(ops, axis=0)  # T_1 over ... over T_316
    sf = np.linalg.svd(fat, compute_uv=False)
    sn = np.linalg.svd(thin, compute_uv=False)
    assert np.allclose(st[:40], sf[:40], rtol=1e-9)
    assert np.allclose(ss[:40], sn[:40], rtol=1e-9)
    # orthonormal bases
    assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-10)
    assert np.allclose(R.T @ R, np.eye(R.shape[1]), atol=1e-10)


@pytest.mark.parametrize("r1,r2", [(60, 80), (100, 120)])
def test_svd_truncation_energy(bases_p3, r1, r2):
    """sum_o ||(I - U U^T) T_o||_F^2 = sum_{i > r1} sigma_i^2 and the same on the source side."""
    U, R, st, ss = bases_p3
    Ur, Rr = U[:, :r1], R[:, :r2]
    ops = _operators(3, "chebyshev")
    left = sum(np.linalg.norm(T - Ur @ (Ur.T @ T)) ** 2 for T in ops)
    right = sum(np.linalg.norm(T - (T @ Rr) @ Rr.T) ** 2 for T in ops)
    assert np.isclose(left, np.sum(st[r1:] ** 2), rtol=1e-6)
    assert np.isclose(right, np.sum(ss[r2:] ** 2), rtol=1e-6)


def test_source_null_space_is_the_trace(bases_p3):
    U, R, st, ss = bases_p3
    P3 = 27
    # the Gram matrix squares the singular values: zeros come out near sqrt(eps) of the largest
    assert ss[9 * P3 - P3 - 1] > 1e-5 * ss[0] and np.all(ss[9 * P3 - P3:] < 1e-7 * ss[0])
    v = np.zeros((P3, 9))
    v[5, [0, 4, 8]] = 1.0  # q_wr = delta_wr at node 5
    ops = _operators(3, "chebyshev")
    assert max(np.abs(T @ v.reshape(-1)).max() for T in ops) < 1e-12 * max(np.abs(T).max() for T in ops)
    v[5, 1] = 1.0  # not a pure trace: some stress
    assert max(np.abs(T @ v.reshape(-1)).max() for T in ops) > 1e-3 * max(np.abs(T).max() for T in ops)


def test_compressed_m2l_full_rank_tight_and_loose():
    nodes, segs, b, y, q, sid = _tiny(2)
    plain = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4, nodes="chebyshev")
    full = ob.m2l_svd_bases(ISO, 3, "chebyshev", ranks=(162, 243))
    a = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4, nodes="chebyshev", svd=full[:2])
    assert np.max(np.abs(a - plain)) <= 1e-11 * np.abs(plain).max()
    null = ob.m2l_svd_bases(ISO, 3, "chebyshev", tol=1e-7)  # drops the trace null space only
    assert null[0].shape[1] == 162 and null[1].shape[1] == 243 - 27
    b_ = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4, nodes="chebyshev", svd=null[:2])
    assert oracle.rel_l2(b_, plain) < 1e-11
    mid = ob.m2l_svd_bases(ISO, 3, "chebyshev", tol=1e-3)
    assert mid[0].shape[1] < 162 and mid[1].shape[1] < 216
    assert oracle.rel_l2(ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4, nodes="chebyshev", svd=mid[:2]), plain) < 1e-3
    loose = ob.m2l_svd_bases(ISO, 3, "chebyshev", tol=1e-2)
    c = ob.lagrange_fmm(ISO, y, q, sid, p=3, L=4, nodes="chebyshev", svd=loose[:2])
    assert oracle.rel_l2(c, plain) > 1e-3
