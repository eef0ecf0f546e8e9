"""Pins of the oracle's stress sum (Eq. "stress3") and nodal forces.

* Textbook fields of infinite straight screw and edge dislocations
  (Hirth & Lothe), approached by a long closed loop: pins magnitude, the
  angular pattern and the nu dependence of Mura's formula (Section 2,
  Eq. "stress").  Eq. "stress" as printed gives the textbook field with the
  opposite overall sign for the same line sense and Burgers vector; the
  tests record that sign (it is a Burgers-circuit convention).
* Equilibrium: the exact field of a closed loop is divergence free; the
  Gauss sum of a closed polygon far from its segments is too, to quadrature
  error.  Checked by finite differences for isotropic and cubic media.
* Linearity in b, translation invariance, rotation covariance.
* Forces: constant stress on a closed loop gives zero net force, the two end
  forces of a segment add up to (sigma b) x S, and reversing line sense and
  b together changes nothing.
"""
import numpy as np
import pytest

import oracle
from paper_1712_07739_gb300 import synth

ISO = oracle.Material.iso(1.0, 0.3)


def _long_loop(L=1e5, s0=0.1, grow=1.15):
    z = [0.0]
    s = s0
    while z[-1] < L:
        z.append(min(L, z[-1] + s))
        s *= grow
    z = np.array(z)
    zz = np.concatenate([-z[::-1], z[1:]])
    line = np.stack([np.zeros_like(zz), np.zeros_like(zz), zz], 1)
    nodes = np.concatenate([line, np.array([[L, 0, L], [L, 0, -L]])])
    n = len(nodes)
    segs = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int64)
    return nodes, segs


def _loop_field(b, xt, mat=ISO):
    nodes, segs = _long_loop()
    B = np.repeat(np.asarray(b, float)[None], len(segs), 0)
    y, q, sid = oracle.quadrature(nodes, segs, B, 8)
    return oracle.direct_stress(mat, xt, -np.ones(len(xt), np.int64), y, q, sid)


XT = np.array([[0.6, 0.8, 0.0], [-1.0, 0.3, 0.0], [0.2, -1.7, 0.0]])


def test_infinite_screw_textbook_field():
    s = _loop_field([0, 0, 1.0], XT)
    for (x, y, _), si in zip(XT, s):
        r2 = x * x + y * y
        tb = np.zeros(6)
        tb[4] = -y / (2 * np.pi * r2)   # sigma_xz
        tb[3] = x / (2 * np.pi * r2)    # sigma_yz
        assert np.max(np.abs(si + tb)) <= 1e-4 * np.abs(tb).max()


def test_infinite_edge_textbook_field():
    nu = 0.3
    s = _loop_field([1.0, 0, 0], XT)
    D = 1.0 / (2 * np.pi * (1 - nu))
    for (x, y, _), si in zip(XT, s):
        r2 = x * x + y * y
        sxx = -D * y * (3 * x * x + y * y) / r2 ** 2
        syy = D * y * (x * x - y * y) / r2 ** 2
        sxy = D * x * (x * x - y * y) / r2 ** 2
        tb = np.array([sxx, syy, nu * (sxx + syy), 0.0, 0.0, sxy])
        assert np.max(np.abs(si + tb)) <= 1e-4 * np.abs(tb).max()


def _polygon_loop(n=24, r=1.0, normal=(0.2, 0.3, 1.0)):
    nrm = np.asarray(normal, float)
    nrm /= np.linalg.norm(nrm)
    e1 = np.cross(nrm, [1.0, 0, 0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nrm, e1)
    th = 2 * np.pi * np.arange(n) / n
    nodes = r * (np.cos(th)[:, None] * e1 + np.sin(th)[:, None] * e2)
    segs = np.stack([np.arange(n), (np.arange(n) + 1) % n], 1).astype(np.int64)
    return nodes, segs


@pytest.mark.parametrize("medium", ["iso", "cubic"])
def test_closed_loop_divergence_free(medium):
    mat = ISO if medium == "iso" else oracle.Material.aniso(synth.cubic_voigt(), Q=64)
    nodes, segs = _polygon_loop()
    b = np.repeat(np.array([[0.3, -0.5, 0.8]]), len(segs), 0)
    y, q, sid = oracle.quadrature(nodes, segs, b, 16)
    x0s = np.array([[0.2, -0.1, 0.6], [0.5, 0.4, -0.5]])
    hh = 1e-3
    for x0 in x0s:
        pts = [x0]
        for d in range(3):
            for k in (-2, -1, 1, 2):
                e = np.zeros(3)
                e[d] = k * hh
                pts.append(x0 + e)
        S = oracle.voigt_to_tensor(oracle.direct_stress(mat, np.array(pts), -np.ones(13, np.int64), y, q, sid))
        div = np.zeros(3)
        for d in range(3):
            f = {k: S[1 + 4 * d + i] for i, k in enumerate((-2, -1, 1, 2))}
            grad = (-f[2] + 8 * f[1] - 8 * f[-1] + f[-2]) / (12 * hh)
            div += grad[:, d]
        scale = np.abs(S[0]).max()
        assert np.max(np.abs(div)) <= 1e-7 * scale
        # a single open segment is not divergence free: the check has teeth
        y1, q1, s1 = oracle.quadrature(nodes, segs[:1], b[:1], 16)
        S1 = oracle.voigt_to_tensor(oracle.direct_stress(mat, np.array(pts), -np.ones(13, np.int64), y1, q1, s1))
        div1 = np.zeros(3)
        for d in range(3):
            f = {k: S1[1 + 4 * d + i] for i, k in enumerate((-2, -1, 1, 2))}
            div1 += ((-f[2] + 8 * f[1] - 8 * f[-1] + f[-2]) / (12 * hh))[:, d]
        assert np.max(np.abs(div1)) > 1e-3 * np.abs(S1[0]).max()


def _net(seed=0):
    return synth.hexagon_loops(n_loops=4, segs_per_loop=12, seed=seed)


def test_linear_in_b_and_translation_invariant():
    nodes, segs, b = _net()
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    s = oracle.direct_stress(ISO, y, sid, y, q, sid)
    y2, q2, _ = oracle.quadrature(nodes, segs, -2.5 * b, 4)
    assert np.allclose(oracle.direct_stress(ISO, y, sid, y2, q2, sid), -2.5 * s, rtol=1e-12, atol=1e-12 * np.abs(s).max())
    sh = np.array([0.3, -1.1, 2.0])
    y3, q3, _ = oracle.quadrature(nodes + sh, segs, b, 4)
    assert np.allclose(oracle.direct_stress(ISO, y3, sid, y3, q3, sid), s, rtol=0, atol=1e-9 * np.abs(s).max())


def test_isotropic_rotation_covariance():
    nodes, segs, b = _net(1)
    rng = np.random.default_rng(3)
    Rm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Rm) < 0:
        Rm[:, 0] *= -1
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    s = oracle.voigt_to_tensor(oracle.direct_stress(ISO, y, sid, y, q, sid))
    y2, q2, _ = oracle.quadrature(nodes @ Rm.T, segs, b @ Rm.T, 4)
    s2 = oracle.voigt_to_tensor(oracle.direct_stress(ISO, y2, sid, y2, q2, sid))
    want = np.einsum("ai,bj,nij->nab", Rm, Rm, s)
    assert np.max(np.abs(s2 - want)) <= 1e-10 * np.abs(s).max()


def test_forces_constant_stress_and_end_sum():
    nodes, segs, b = _net(2)
    sig = np.tile(np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.25]), (len(segs) * 4, 1))
    f1, f2 = oracle.segment_forces(nodes, segs, b, sig, 4)
    S = nodes[segs[:, 1]] - nodes[segs[:, 0]]
    sb = oracle.voigt_to_tensor(sig[0]) @ b.T
    want = np.cross(sb.T, S)
    assert np.allclose(f1 + f2, want, rtol=1e-13, atol=1e-17)
    assert np.allclose(f1, f2, rtol=1e-13, atol=1e-17)  # constant field splits evenly
    F = oracle.nodal_forces(nodes, segs, b, sig, 4)
    assert np.max(np.abs(F.sum(0))) <= 1e-13 * np.abs(F).max()


def test_forces_invariant_under_line_sense_reversal():
    nodes, segs, b = _net(3)
    F, _ = oracle.network_forces(ISO, nodes, segs, b)
    F2, _ = oracle.network_forces(ISO, nodes, segs[:, ::-1].copy(), -b)
    assert np.max(np.abs(F2 - F)) <= 1e-12 * np.abs(F).max()


def test_sampled_node_forces_match_full():
    nodes, segs, b = _net(4)
    F, _ = oracle.network_forces(ISO, nodes, segs, b)
    ids = np.array([0, 5, 17, 30])
    Fs, _ = oracle.sampled_node_forces(ISO, nodes, segs, b, ids)
    assert np.allclose(Fs, F[ids], rtol=1e-13, atol=1e-15 * np.abs(F).max())
