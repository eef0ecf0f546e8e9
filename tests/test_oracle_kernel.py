"""Pins of the oracle's Green's-function factor h and kernel K.

Each check compares the oracle with something other than itself: Kelvin's
closed-form Green's function (Section 2, Eq. "k_iso"), finite differences of
an independently computed G, symmetry of the cubic crystal, and the A = 1
reduction of a cubic medium to an isotropic one (Section 5.2: A = 1 is
equivalent to isotropic elasticity).
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1712_07739_gb300 import synth

MU, NU = 1.0, 0.3
CISO = oracle.voigt_to_cijkl(synth.isotropic_voigt(MU, NU))
CCUB = oracle.voigt_to_cijkl(synth.cubic_voigt())


def _dirs(n, seed=0):
    d = np.random.default_rng(seed).normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def kelvin_G(x, mu=MU, nu=NU):
    """Kelvin's solution written from Eq. "k_iso": R,ii = 2/R and
    R,vp = (delta_vp - T_v T_p)/R substituted into the printed bracket."""
    R = np.linalg.norm(x)
    T = x / R
    lap = 2.0 / R
    hess = (np.eye(3) - np.outer(T, T)) / R
    return (np.eye(3) * lap - hess / (2.0 * (1.0 - nu))) / (8.0 * np.pi * mu)


def test_circle_G_matches_kelvin():
    for t in _dirs(50):
        x = 0.37 * t
        G = oracle.G_circle(CISO, x, 64)
        assert np.allclose(G, kelvin_G(x), rtol=0, atol=1e-14 * np.abs(kelvin_G(x)).max())


def test_iso_h_matches_circle_h():
    for t in _dirs(200, 1):
        a = oracle.h_iso(t, MU, NU)
        b = oracle.h_circle(CISO, t, 64)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a))


def _fd_grad(f, x, step):
    """Fourth-order central differences of a matrix-valued f, one Richardson
    step on top (error O(step^6))."""
    def cd(hh):
        g = np.zeros((3, 3, 3))
        for q in range(3):
            e = np.zeros(3)
            e[q] = hh
            g[:, :, q] = (-f(x + 2 * e) + 8 * f(x + e) - 8 * f(x - e) + f(x - 2 * e)) / (12 * hh)
        return g
    g1, g2 = cd(step), cd(step / 2)
    return (16 * g2 - g1) / 15


@pytest.mark.parametrize("Cname", ["iso", "cubic"])
def test_h_is_gradient_of_G(Cname):
    C = CISO if Cname == "iso" else CCUB
    for t in _dirs(8, 2):
        x = 0.8 * t
        R = np.linalg.norm(x)
        g = _fd_grad(lambda y: oracle.G_circle(C, y, 128), x, 1e-2)
        h = oracle.h_circle(C, x / R, 128) / R ** 2
        assert np.max(np.abs(g - h)) <= 2e-9 * np.max(np.abs(h))


def test_iso_h_is_gradient_of_kelvin():
    for t in _dirs(8, 3):
        x = 1.3 * t
        R = np.linalg.norm(x)
        g = _fd_grad(kelvin_G, x, 1e-2)
        h = oracle.h_iso(t) / R ** 2
        assert np.max(np.abs(g - h)) <= 2e-9 * np.max(np.abs(h))


def test_h_odd_and_circle_basis_independent():
    for t in _dirs(20, 4):
        h = oracle.h_circle(CCUB, t, 64)
        assert np.max(np.abs(oracle.h_circle(CCUB, -t, 64) + h)) <= 1e-14 * np.abs(h).max()
        hr = oracle.h_circle(CCUB, t, 64, rot=0.4321)
        assert np.max(np.abs(hr - h)) <= 1e-13 * np.abs(h).max()
        # symmetric in (v, p), like G
        assert np.max(np.abs(h - h.transpose(1, 0, 2))) <= 1e-14 * np.abs(h).max()


def test_cubic_A1_equals_isotropic():
    lam, mu = 0.9, 0.7
    C = oracle.voigt_to_cijkl(synth.cubic_voigt(lam + 2 * mu, lam, mu))  # C11-C12 = 2 C44
    nu = lam / (2 * (lam + mu))
    for t in _dirs(50, 5):
        a = oracle.h_circle(C, t, 64)
        b = oracle.h_iso(t, mu, nu)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.abs(b).max()


def _cubic_rotations():
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((-1, 1), repeat=3):
            R = np.zeros((3, 3))
            for i in range(3):
                R[i, perm[i]] = signs[i]
            if np.linalg.det(R) > 0:
                out.append(R)
    assert len(out) == 24
    return out


def test_cubic_h_covariant_under_cube_rotations():
    for t in _dirs(5, 6):
        h = oracle.h_circle(CCUB, t, 64)
        for R in _cubic_rotations():
            hr = oracle.h_circle(CCUB, R @ t, 64)
            want = np.einsum("vi,pj,qk,ijk->vpq", R, R, R, h)
            assert np.max(np.abs(hr - want)) <= 1e-13 * np.abs(h).max()


def test_choose_Q_converged():
    Q = oracle.choose_Q(CCUB)
    for t in _dirs(20, 7):
        a = oracle.h_circle(CCUB, t, Q)
        b = oracle.h_circle(CCUB, t, 4 * Q)
        assert np.max(np.abs(a - b)) <= 1e-13 * np.abs(b).max()


def test_kernel_homogeneous_degree_minus_two():
    """K(alpha x) = alpha^-2 K(x) (Section 4.1 footnote)."""
    mat = oracle.Material.aniso(synth.cubic_voigt(), Q=64)
    d = _dirs(10, 8) * 0.3
    K1 = oracle.kernel(mat, d)
    K2 = oracle.kernel(mat, 2.5 * d)
    assert np.max(np.abs(K2 * 2.5 ** 2 - K1)) <= 1e-13 * np.abs(K1).max()
