"""Pins of the oracle's quadrature and force split against closed forms.

* Force split (Sec. 2: f = (sigma . b) x xi, integrated against the linear
  shape functions of the segment ends).  For a stress field that varies
  linearly along a segment, sigma = s0 + (2t - 1) s1 with t in [0, 1] from
  the first node to the second, the integrals of (1 - t) and t against it
  give, by hand,
      f1 = (1/2) (s0 b) x S - (1/6) (s1 b) x S,
      f2 = (1/2) (s0 b) x S + (1/6) (s1 b) x S,
  with S = x2 - x1.  Exchanging the two shape functions, or the order of the
  Gauss points along the segment, flips the sign of the 1/6 terms.  A
  quadratic variation (2t - 1)^2 s2 gives (1/6) (s2 b) x S at both ends.
* Straight-segment integral (Sec. 2, Eqs. "stress" and "k_iso").  In an
  isotropic medium h_vpq(T) / R^2 is a sum of d_i / R^3 and d_v d_p d_q / R^5
  terms (d = x - y), whose integrals along a straight line have closed-form
  antiderivatives in the distance rho from the line and the coordinate w
  along it:
      int dw / R^3 = w / (rho^2 R),            int w dw / R^3 = -1 / R,
      int dw / R^5 = w (2 w^2 + 3 rho^2) / (3 rho^4 R^3),
      int w dw / R^5 = -1 / (3 R^3),           int w^2 dw / R^5 = w^3 / (3 rho^2 R^3),
      int w^3 dw / R^5 = -(3 w^2 + 2 rho^2) / (3 R^3).
  The oracle's Gauss sum of Eq. "stress_discrete" at high order must
  converge to that exact segment field, which pins the quadrature points,
  the strengths q_wr = 1/2 b_w omega S_r and their contraction with the
  kernel; a dropped 1/2, a transposed q or a wrong point placement fails.
"""
import numpy as np

import oracle

MU, NU = 1.0, 0.3
ISO = oracle.Material.iso(MU, NU)


def _linear_field_forces(seed):
    rng = np.random.default_rng(seed)
    nodes = rng.normal(size=(2, 3))
    segs = np.array([[0, 1]], dtype=np.int64)
    b = rng.normal(size=(1, 3))
    s0, s1, s2 = (rng.normal(size=6) for _ in range(3))
    return nodes, segs, b, s0, s1, s2


def _t_of_points(nodes, y):
    """Position of each Gauss point along the segment: t = 0 at x1, 1 at x2."""
    S = nodes[1] - nodes[0]
    return (y - nodes[0]) @ S / (S @ S)


def test_force_split_linear_field_has_closed_form():
    for seed in range(5):
        nodes, segs, b, s0, s1, _ = _linear_field_forces(seed)
        for n_g in (2, 4, 7):
            y, _, _ = oracle.quadrature(nodes, segs, b, n_g)
            t = _t_of_points(nodes, y)
            sig = s0[None, :] + (2.0 * t - 1.0)[:, None] * s1[None, :]  # evaluated at the points' positions
            f1, f2 = oracle.segment_forces(nodes, segs, b, sig, n_g)
            S = nodes[1] - nodes[0]
            pk0 = np.cross(oracle.voigt_to_tensor(s0) @ b[0], S)
            pk1 = np.cross(oracle.voigt_to_tensor(s1) @ b[0], S)
            assert np.allclose(f1[0], 0.5 * pk0 - pk1 / 6.0, rtol=1e-13, atol=1e-14)
            assert np.allclose(f2[0], 0.5 * pk0 + pk1 / 6.0, rtol=1e-13, atol=1e-14)


def test_force_split_quadratic_field_has_closed_form():
    nodes, segs, b, _, _, s2 = _linear_field_forces(11)
    y, _, _ = oracle.quadrature(nodes, segs, b, 4)
    t = _t_of_points(nodes, y)
    sig = ((2.0 * t - 1.0) ** 2)[:, None] * s2[None, :]
    f1, f2 = oracle.segment_forces(nodes, segs, b, sig, 4)
    pk2 = np.cross(oracle.voigt_to_tensor(s2) @ b[0], nodes[1] - nodes[0])
    assert np.allclose(f1[0], pk2 / 6.0, rtol=1e-13, atol=1e-14)
    assert np.allclose(f2[0], pk2 / 6.0, rtol=1e-13, atol=1e-14)


def test_nodal_forces_assemble_end_forces_of_a_chain():
    """Three segments in a chain 0 -> 1 -> 2 -> 3 under a linear field: node 1
    gets f2 of segment 0 plus f1 of segment 1, and so on."""
    rng = np.random.default_rng(5)
    nodes = np.cumsum(rng.normal(size=(4, 3)), axis=0)
    segs = np.array([[0, 1], [1, 2], [2, 3]], dtype=np.int64)
    b = rng.normal(size=(3, 3))
    s0, s1 = rng.normal(size=6), rng.normal(size=6)
    y, _, _ = oracle.quadrature(nodes, segs, b, 4)
    sig = np.empty((len(y), 6))
    for k in range(3):
        t = _t_of_points(nodes[segs[k]], y[4 * k:4 * k + 4])
        sig[4 * k:4 * k + 4] = s0[None] + (k + 1.0) * (2.0 * t - 1.0)[:, None] * s1[None]
    F = oracle.nodal_forces(nodes, segs, b, sig, 4)
    want = np.zeros((4, 3))
    for k, (i, j) in enumerate(segs):
        S = nodes[j] - nodes[i]
        pk0 = np.cross(oracle.voigt_to_tensor(s0) @ b[k], S)
        pk1 = (k + 1.0) * np.cross(oracle.voigt_to_tensor(s1) @ b[k], S)
        want[i] += 0.5 * pk0 - pk1 / 6.0
        want[j] += 0.5 * pk0 + pk1 / 6.0
    assert np.allclose(F, want, rtol=1e-13, atol=1e-14)


def _segment_integrals(x, x1, x2):
    """J1[i] = int d_i / R^3 ds and J3[i, j, k] = int d_i d_j d_k / R^5 ds over
    the straight segment x1 -> x2, d = x - y(s), from the antiderivatives in w."""
    L = np.linalg.norm(x2 - x1)
    t = (x2 - x1) / L
    u = (x - x1) @ t
    rho_v = (x - x1) - u * t
    rho2 = rho_v @ rho_v
    # y(s) = x1 + s t, d = rho_v + (u - s) t; with w = u - s the integral over
    # s in [0, L] is the integral over w in [u - L, u]
    def F(w):
        R = np.sqrt(rho2 + w * w)
        F0 = w / (rho2 * R)
        F1 = -1.0 / R
        G0 = w * (2 * w * w + 3 * rho2) / (3 * rho2 * rho2 * R ** 3)
        G1 = -1.0 / (3 * R ** 3)
        G2 = w ** 3 / (3 * rho2 * R ** 3)
        G3 = -(3 * w * w + 2 * rho2) / (3 * R ** 3)
        return np.array([F0, F1]), np.array([G0, G1, G2, G3])
    Fa, Ga = F(u)
    Fb, Gb = F(u - L)
    I1 = Fa - Fb   # int w^n / R^3 dw, n = 0, 1
    I3 = Ga - Gb   # int w^n / R^5 dw, n = 0..3
    J1 = rho_v * I1[0] + t * I1[1]
    # (rho + w t)_i (rho + w t)_j (rho + w t)_k expanded in powers of w
    r, tt = rho_v, t
    J3 = (np.einsum("i,j,k->ijk", r, r, r) * I3[0]
          + (np.einsum("i,j,k->ijk", tt, r, r) + np.einsum("i,j,k->ijk", r, tt, r)
             + np.einsum("i,j,k->ijk", r, r, tt)) * I3[1]
          + (np.einsum("i,j,k->ijk", tt, tt, r) + np.einsum("i,j,k->ijk", tt, r, tt)
             + np.einsum("i,j,k->ijk", r, tt, tt)) * I3[2]
          + np.einsum("i,j,k->ijk", tt, tt, tt) * I3[3])
    return J1, J3, t


def _exact_segment_stress(x, x1, x2, b):
    """sigma_ab(x) = A_{ab,wr,vpq} b_w t_r int h_vpq(T) / R^2 ds, with the
    isotropic h_vpq / R^2 = c [-a delta_vp d_q / R^3 + delta_vq d_p / R^3
    + delta_pq d_v / R^3 - 3 d_v d_p d_q / R^5], c = 1 / (16 pi mu (1 - nu)),
    a = 3 - 4 nu (the gradient of Kelvin's Green's function, Eq. "k_iso")."""
    J1, J3, t = _segment_integrals(x, x1, x2)
    c = 1.0 / (16 * np.pi * MU * (1 - NU))
    a = 3 - 4 * NU
    d = np.eye(3)
    Hint = c * (-a * np.einsum("vp,q->vpq", d, J1) + np.einsum("vq,p->vpq", d, J1)
                + np.einsum("pq,v->vpq", d, J1) - 3.0 * J3)
    A = oracle.A_tensor(ISO.C)  # [ab, w, r, v, p, q]
    return np.einsum("awrvpq,w,r,vpq->a", A, b, t, Hint)


def test_high_order_gauss_sum_converges_to_exact_segment_field():
    rng = np.random.default_rng(8)
    x1, x2 = np.array([0.1, -0.2, 0.3]), np.array([0.9, 0.4, -0.2])
    nodes = np.stack([x1, x2])
    segs = np.array([[0, 1]], dtype=np.int64)
    b = np.array([[0.3, -0.5, 0.8]])
    mid, L = 0.5 * (x1 + x2), np.linalg.norm(x2 - x1)
    # targets at 0.5 to 5 segment lengths from the midpoint, off the line
    dirs = rng.normal(size=(12, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    xt = mid + (L * np.geomspace(0.5, 5.0, 12))[:, None] * dirs
    want = np.array([_exact_segment_stress(x, x1, x2, b[0]) for x in xt])
    y, q, sid = oracle.quadrature(nodes, segs, b, 48)
    got = oracle.direct_stress(ISO, xt, -np.ones(len(xt), np.int64), y, q, sid)
    err = np.abs(got - want).max(axis=1) / np.abs(want).max(axis=1)
    assert err.max() < 1e-12, err
    # the 4-point rule the pass uses: a few per cent at half a segment length,
    # converging fast with distance (1e-9 at five lengths)
    y4, q4, sid4 = oracle.quadrature(nodes, segs, b, 4)
    got4 = oracle.direct_stress(ISO, xt, -np.ones(len(xt), np.int64), y4, q4, sid4)
    err4 = np.abs(got4 - want).max(axis=1) / np.abs(want).max(axis=1)
    assert err4.max() < 5e-2 and err4[-1] < 1e-8


def test_exact_segment_field_detects_a_transposed_strength():
    """The check has teeth: swapping the roles of b and the line direction in
    q (q_rw instead of q_wr) changes the field by far more than the tolerance."""
    x1, x2 = np.array([0.0, 0.0, 0.0]), np.array([0.7, 0.2, -0.3])
    nodes = np.stack([x1, x2])
    segs = np.array([[0, 1]], dtype=np.int64)
    b = np.array([[0.2, 0.9, -0.4]])
    xt = np.array([[0.5, 1.1, 0.6], [-0.8, 0.3, 0.9]])
    want = np.array([_exact_segment_stress(x, x1, x2, b[0]) for x in xt])
    y, q, sid = oracle.quadrature(nodes, segs, b, 32)
    bad = oracle.direct_stress(ISO, xt, -np.ones(2, np.int64), y, q.transpose(0, 2, 1).copy(), sid)
    assert np.abs(bad - want).max() > 1e-3 * np.abs(want).max()
