"""GPU FP64 Lagrange FMM vs the FP64 oracle, through the C ABI.

The FP64 pass must reproduce the oracle's Algorithm 2 (same tree, same
order p) to rounding: relative L2 <= 1e-10 on nodal forces and on free-target
stresses.  Against the direct sum of Eq. "stress3" the error is the FMM's
truncation error (about 3^-p, Section 5.2), reported and bounded loosely.
"""
import numpy as np
import pytest

import oracle
from oracle import oracle_b
from paper_1712_07739_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ISO_C = synth.isotropic_voigt(1.0, 0.3)
ISO = oracle.Material.iso(1.0, 0.3)
TOL_FP64 = 1e-10


def _gpu(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _fmm(nodes, segs, b, C, **kw):
    import paper_1712_07739_gb300 as gb

    f = gb.FMM(**kw).set_material(C)
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    return f


def _oracle_forces(mat, nodes, segs, b, p, L, n_g=4):
    y, q, sid = oracle.quadrature(nodes, segs, b, n_g)
    sig = oracle_b.lagrange_fmm(mat, y, q, sid, p=p, L=L)
    return oracle.nodal_forces(nodes, segs, b, sig, n_g), sig


@pytest.fixture(scope="module")
def c1():
    nodes, segs, b = synth.config("c1")
    return nodes, segs, b


def test_c1_forces_match_algorithm2(c1):
    nodes, segs, b = c1
    f = _fmm(nodes, segs, b, ISO_C, p=4, levels=3)
    F = f.nodal_forces().cpu().numpy()
    Fo, _ = _oracle_forces(ISO, nodes, segs, b, 4, 3)
    err = oracle.rel_l2(F, Fo)
    print("c1 FP64 vs Algorithm 2:", err)
    assert err <= TOL_FP64


def test_c1_forces_vs_direct_sum(c1):
    nodes, segs, b = c1
    f = _fmm(nodes, segs, b, ISO_C, p=4, levels=3)
    F = f.nodal_forces().cpu().numpy()
    Fd, _ = oracle.network_forces(ISO, nodes, segs, b)
    err = oracle.rel_l2(F, Fd)
    print("c1 FP64 p=4 vs direct sum:", err)
    assert err < 5e-2


def test_sigma_points_and_segment_forces_consistent(c1):
    nodes, segs, b = c1
    f = _fmm(nodes, segs, b, ISO_C, p=4, levels=3)
    fs = torch.empty((len(segs), 2, 3), dtype=torch.float64, device="cuda")
    sp = torch.empty((len(segs) * 4, 6), dtype=torch.float64, device="cuda")
    F = f.nodal_forces(f_seg=fs, sigma_pts=sp).cpu().numpy()
    _, sig = _oracle_forces(ISO, nodes, segs, b, 4, 3)
    assert oracle.rel_l2(sp.cpu().numpy(), sig) <= TOL_FP64
    f1, f2 = oracle.segment_forces(nodes, segs, b, sig)
    assert oracle.rel_l2(fs.cpu().numpy(), np.stack([f1, f2], 1)) <= TOL_FP64
    Fn = np.zeros_like(F)
    np.add.at(Fn, segs[:, 0], fs.cpu().numpy()[:, 0])
    np.add.at(Fn, segs[:, 1], fs.cpu().numpy()[:, 1])
    assert np.allclose(Fn, F, rtol=1e-12, atol=1e-14 * np.abs(F).max())


@pytest.mark.parametrize("p,L", [(2, 3), (3, 4), (6, 4)])
def test_orders_and_depths_match_algorithm2(p, L):
    nodes, segs, b = synth.polygon_loops(n_segs=600, n_loops=20, seed=11)
    f = _fmm(nodes, segs, b, ISO_C, p=p, levels=L)
    F = f.nodal_forces().cpu().numpy()
    Fo, _ = _oracle_forces(ISO, nodes, segs, b, p, L)
    assert oracle.rel_l2(F, Fo) <= TOL_FP64


def test_free_target_stress_matches_algorithm2(c1):
    nodes, segs, b = c1
    f = _fmm(nodes, segs, b, ISO_C, p=4, levels=3)
    rng = np.random.default_rng(5)
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    lo, hi = y.min(0), y.max(0)
    xt = lo + (hi - lo) * rng.uniform(0.02, 0.98, (300, 3))
    s = f.stress(_gpu(xt)).cpu().numpy()
    so = oracle_b.lagrange_fmm(ISO, y, q, sid, p=4, L=3, xt=xt, tseg=-np.ones(len(xt), np.int64))
    assert oracle.rel_l2(s, so) <= TOL_FP64


def test_cubic_circle_matches_algorithm2():
    nodes, segs, b = synth.polygon_loops(n_segs=300, n_loops=10, seed=12)
    C6 = synth.cubic_voigt()
    mat = oracle.Material.aniso(C6, Q=64)
    f = _fmm(nodes, segs, b, C6, p=3, levels=3, h_mode="circle", circle_q=64)
    F = f.nodal_forces().cpu().numpy()
    Fo, _ = _oracle_forces(mat, nodes, segs, b, 3, 3)
    assert oracle.rel_l2(F, Fo) <= TOL_FP64


def test_single_segment_and_two_gauss_points():
    nodes = np.array([[0.1, 0.2, 0.3], [0.4, 0.1, 0.35]])
    segs = np.array([[0, 1]], np.int64)
    b = np.array([[0.0, 0.5, 0.5]])
    f = _fmm(nodes, segs, b, ISO_C, p=3, levels=3, n_gauss=2)
    F = f.nodal_forces().cpu().numpy()
    # The two Gauss points span the root cube, so they sit in non-adjacent
    # leaves: Algorithm 2 then approximates the segment's own interaction in
    # the far field (only same-leaf-neighbourhood pairs are excluded).  The
    # oracle follows the same algorithm.
    Fo, _ = _oracle_forces(ISO, nodes, segs, b, 3, 3, n_g=2)
    assert oracle.rel_l2(F, Fo) <= TOL_FP64
    xt = np.array([[0.3, 0.5, 0.1], [0.2, 0.15, 0.32]])
    s = f.stress(_gpu(xt)).cpu().numpy()
    y, q, sid = oracle.quadrature(nodes, segs, b, 2)
    # targets outside the root cube are clamped to boundary leaves on both sides
    so = oracle_b.lagrange_fmm(ISO, y, q, sid, p=3, L=3, xt=xt, tseg=np.array([-1, -1]))
    assert oracle.rel_l2(s, so) <= TOL_FP64


def test_errors_are_reported():
    import paper_1712_07739_gb300 as gb

    f = gb.FMM(p=3, levels=3)
    with pytest.raises(gb.GbfmmError):
        f.nodal_forces(out=torch.empty((2, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(gb.GbfmmError):
        f.set_material(-np.eye(6))
    with pytest.raises(gb.GbfmmError):
        f.set_material(synth.cubic_voigt())  # iso mode needs an isotropic medium
    f.set_material(ISO_C)
    nodes = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [0.5, 0.5, 0.5]])
    segs = np.array([[0, 1], [1, 2]], np.int64)
    with pytest.raises(gb.GbfmmError):
        f.build(_gpu(nodes), _gpu(segs), _gpu(np.ones((2, 3))))
    # the context stays usable after an error
    nodes[1] = [0.3, 0.2, 0.1]
    f.build(_gpu(nodes), _gpu(segs), _gpu(np.ones((2, 3))))
    assert np.isfinite(f.nodal_forces().cpu().numpy()).all()


# ---------------------------------------------------------------- M2L through transforms
# The Toeplitz form (Sec. 4.1, Theorem 1) computes the same Algorithm 2: each
# offset's node-to-node map is a convolution, applied through discrete
# Fourier transforms of size (2p)^3.  It must meet the same 1e-10 bar against
# the oracle, and agree with the dense FP64 pass to rounding.

@pytest.mark.parametrize("p,L", [(2, 3), (3, 4), (6, 4)])
def test_fft_m2l_matches_algorithm2(p, L):
    nodes, segs, b = synth.polygon_loops(n_segs=600, n_loops=20, seed=11)
    f = _fmm(nodes, segs, b, ISO_C, p=p, levels=L, m2l_fft=1)
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    Fo, _ = _oracle_forces(ISO, nodes, segs, b, p, L)
    err = oracle.rel_l2(F, Fo)
    print(f"FFT M2L p={p} L={L} vs Algorithm 2: {err:.3e}")
    assert err <= TOL_FP64


def test_fft_m2l_free_targets_match_algorithm2(c1):
    nodes, segs, b = c1
    f = _fmm(nodes, segs, b, ISO_C, p=4, levels=3, m2l_fft=1)
    rng = np.random.default_rng(5)
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    lo, hi = y.min(0), y.max(0)
    xt = lo + (hi - lo) * rng.uniform(0.02, 0.98, (300, 3))
    s = f.stress(_gpu(xt)).cpu().numpy()
    so = oracle_b.lagrange_fmm(ISO, y, q, sid, p=4, L=3, xt=xt, tseg=-np.ones(len(xt), np.int64))
    assert oracle.rel_l2(s, so) <= TOL_FP64


@pytest.mark.parametrize("p,L", [(5, 4), (7, 4), (8, 3)])
def test_fft_m2l_equals_dense_pass(p, L):
    """Cubic medium (unit-circle h), nodal forces and free-target stresses:
    the transform form and the dense node-pair sums agree to rounding."""
    nodes, segs, b = synth.polygon_loops(n_segs=800, n_loops=25, seed=13)
    C6 = synth.cubic_voigt()
    kw = dict(p=p, levels=L, h_mode="circle", circle_q=32)
    fd = _fmm(nodes, segs, b, C6, m2l_fft=0, **kw)
    ff = _fmm(nodes, segs, b, C6, m2l_fft=1, **kw)
    Fd, Ff = fd.nodal_forces().cpu().numpy(), ff.nodal_forces().cpu().numpy()
    rng = np.random.default_rng(6)
    xt = nodes.min(0) + (nodes.max(0) - nodes.min(0)) * rng.uniform(0.05, 0.95, (200, 3))
    sd, sf = fd.stress(_gpu(xt)).cpu().numpy(), ff.stress(_gpu(xt)).cpu().numpy()
    e_f, e_s = oracle.rel_l2(Ff, Fd), oracle.rel_l2(sf, sd)
    print(f"FFT vs dense M2L p={p} L={L}: forces {e_f:.3e}, stresses {e_s:.3e}")
    assert e_f <= 1e-12 and e_s <= 1e-12
