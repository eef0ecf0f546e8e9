"""Pins of the oracle's symmetry reduction of the M2L operators (Sec. 6: the
symmetries of space and kernel leave 16 of the 316 operators).

* The group: 48 signed permutation matrices, closed under products, 24
  proper, containing -I.
* The orbits: 16 orbits partition the 316 offsets, every member is its map
  of the representative, and each orbit's size is 48 over the order of the
  representative's stabiliser (counted by brute force).
* The kernel: for media with the cube's symmetry (isotropic, cubic with axes
  along x, y, z) K(g d) = det(g) g g g g K(d) at random separations to
  rounding; without det(g) it fails for the improper maps, and a turned
  crystal breaks it.
* The operators: ``symmetric_operator`` rebuilds all 316 node-kernel
  matrices from the 16 representatives (equispaced and Chebyshev nodes,
  isotropic and cubic), and does not for a turned crystal.
* The transforms used by an M2L through the Toeplitz structure (Theorem 1):
  the discrete Fourier transform of an offset's embedded kernel equals
  det(g) g g g g times the representative's at the frequency g^T f (mod N),
  and a real kernel's transform at -f is the conjugate of the one at f, so
  the half spectrum of the 16 representatives gives every offset's.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import oracle_b as ob
from paper_1712_07739_gb300 import synth

ISO = oracle.Material.iso(1.0, 0.3)
CUB = oracle.Material.aniso(synth.cubic_voigt(), Q=48)
VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def _turned():
    a = 0.4
    R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
    return oracle.Material.aniso(synth.rotated_voigt(synth.cubic_voigt(), R), Q=48)


def _full(K):  # [6, 3, 3] -> [3, 3, 3, 3]
    T = np.zeros((3, 3, 3, 3))
    for i, (a, b) in enumerate(VOIGT):
        T[a, b] = K[i]
        T[b, a] = K[i]
    return T


def test_cube_group():
    G = ob.cube_group()
    assert len(G) == 48
    keys = {g.tobytes() for g in G}
    assert len(keys) == 48
    for g in G:
        assert np.array_equal(g @ g.T, np.eye(3, dtype=np.int64))
        assert np.count_nonzero(g) == 3
    for g in G:
        for h in G:
            assert (g @ h).tobytes() in keys
    dets = [round(np.linalg.det(g)) for g in G]
    assert dets.count(1) == 24 and dets.count(-1) == 24
    assert (-np.eye(3, dtype=np.int64)).tobytes() in keys


def test_offset_orbits_partition():
    orb = ob.offset_orbits()
    assert len(orb) == 16
    all_o = [o for _, mem in orb for o, _ in mem]
    assert len(all_o) == 316 and set(all_o) == set(ob.m2l_offsets())
    G = ob.cube_group()
    for rep, mem in orb:
        assert rep[0] >= rep[1] >= rep[2] >= 0 and max(rep) >= 2
        for o, g in mem:
            assert tuple(g @ np.array(rep)) == o
        stab = sum(1 for g in G if tuple(g @ np.array(rep)) == rep)
        assert len(mem) * stab == 48


@pytest.mark.parametrize("name", ["iso", "cubic"])
def test_kernel_covariance(name):
    mat = ISO if name == "iso" else CUB
    rng = np.random.default_rng(3)
    D = rng.normal(size=(6, 3))
    K = oracle.kernel(mat, D)
    for g in ob.cube_group():
        det = round(np.linalg.det(g))
        Kg = oracle.kernel(mat, D @ g.T)
        for n in range(len(D)):
            want = _full(Kg[n])
            rot = np.einsum("ai,bj,wk,rl,ijkl->abwr", g, g, g, g, _full(K[n]))
            assert np.abs(det * rot - want).max() <= 1e-13 * np.abs(want).max()
            if det < 0:  # the permutation symbol: without det(g) the improper maps fail
                assert np.abs(rot - want).max() > 0.5 * np.abs(want).max()


def test_turned_crystal_breaks_covariance():
    mat = _turned()
    D = np.array([[0.3, -0.7, 0.5]])
    K = oracle.kernel(mat, D)
    worst = 0.0
    for g in ob.cube_group():
        det = round(np.linalg.det(g))
        want = _full(oracle.kernel(mat, D @ g.T)[0])
        rot = det * np.einsum("ai,bj,wk,rl,ijkl->abwr", g, g, g, g, _full(K[0]))
        worst = max(worst, np.abs(rot - want).max() / np.abs(want).max())
    assert worst > 1e-2


@pytest.mark.parametrize("name,nodes", [("iso", "equispaced"), ("iso", "chebyshev"), ("cubic", "equispaced")])
def test_operators_from_16_representatives(name, nodes):
    mat = ISO if name == "iso" else CUB
    p = 3
    worst = 0.0
    for rep, mem in ob.offset_orbits():
        for o, g in mem:
            a = ob.symmetric_operator(mat, p, o, g, rep, nodes=nodes)
            b = ob._node_kernels(mat, p, 1.0, o, nodes=nodes)
            worst = max(worst, np.abs(a - b).max() / np.abs(b).max())
    assert worst <= 1e-13


def test_turned_crystal_operators_differ():
    mat = _turned()
    rep, mem = ob.offset_orbits()[5]
    o, g = [m for m in mem if m[0] != rep][3]
    a = ob.symmetric_operator(mat, 3, o, g, rep)
    b = ob._node_kernels(mat, 3, 1.0, o)
    assert np.abs(a - b).max() > 1e-2 * np.abs(b).max()


def _embedded_transform(mat, p, o):
    """DFT over (2p)^3 of the kernel on the node-difference lattice of offset o,
    K_o[d] = K(o (p - 1) + d) for d in [-(p - 1), p - 1]^3 placed at d mod 2p
    (index p unused): [N, N, N (x, y, z frequency), 6, 3, 3]."""
    N = 2 * p
    ds = np.array(list(itertools.product(range(-(p - 1), p), repeat=3)))
    K = oracle.kernel(mat, (np.array(o)[None, :] * (p - 1) + ds).astype(np.float64))
    E = np.zeros((N, N, N, 6, 3, 3))
    E[ds[:, 0] % N, ds[:, 1] % N, ds[:, 2] % N] = K
    return np.fft.fftn(E, axes=(0, 1, 2))


def test_fourier_form_of_the_reduction():
    """K^_o[f] = det(g) rho(g) K^_rep[g^T f mod N]: the relation an M2L through
    transforms applies to a table of the 16 representatives' half spectra."""
    p = 3
    N = 2 * p
    f = np.array(list(itertools.product(range(N), repeat=3)))
    for rep, mem in ob.offset_orbits():
        Fr = _embedded_transform(ISO, p, rep)
        # a real kernel: the transform at -f is the conjugate of the one at f
        neg = (-f) % N
        assert np.allclose(Fr[neg[:, 0], neg[:, 1], neg[:, 2]], np.conj(Fr[f[:, 0], f[:, 1], f[:, 2]]), atol=1e-12)
        for o, g in mem[:: max(1, len(mem) // 6)]:
            Fo = _embedded_transform(ISO, p, o)
            det = round(np.linalg.det(g))
            src = (f @ g) % N  # (g^T f)_j = sum_i g_ij f_i
            R = Fr[src[:, 0], src[:, 1], src[:, 2]]  # [n, 6, 3, 3]
            Rf = np.zeros((len(f), 3, 3, 3, 3), dtype=complex)
            for i, (a, b) in enumerate(VOIGT):
                Rf[:, a, b] = R[:, i]
                Rf[:, b, a] = R[:, i]
            got = det * np.einsum("ai,bj,wk,rl,nijkl->nabwr", g, g, g, g, Rf)
            want = Fo[f[:, 0], f[:, 1], f[:, 2]]
            for i, (a, b) in enumerate(VOIGT):
                assert np.abs(got[:, a, b] - want[:, i]).max() <= 1e-12 * np.abs(want).max()
