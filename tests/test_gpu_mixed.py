"""Mixed-precision pass (FP32 stages, tensor-core M2L in FP16 with per-level
scaling or BF16 with split correction, FP32 near field with FP64 close
pairs) vs the FP64 oracle.

Tolerance: relative L2 nodal-force error <= 1e-4 against the oracle's
Algorithm 2 at the same order and tree (the mixed-precision bar of the
method's accuracy target), and the device status word stays clean.
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
TOL_MIXED = 1e-4


def _gpu(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _run(nodes, segs, b, C, **kw):
    import paper_1712_07739_gb300 as gb

    f = gb.FMM(**kw).set_material(C)
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    F = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    return f, F


def _oracle_forces(mat, nodes, segs, b, p, L):
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    sig = oracle_b.lagrange_fmm(mat, y, q, sid, p=p, L=L)
    return oracle.nodal_forces(nodes, segs, b, sig, 4)


def test_mixed_c1_matches_algorithm2():
    nodes, segs, b = synth.config("c1")
    _, F = _run(nodes, segs, b, ISO_C, p=4, levels=3, precision="mixed")
    Fo = _oracle_forces(ISO, nodes, segs, b, 4, 3)
    err = oracle.rel_l2(F, Fo)
    print("mixed c1 vs Algorithm 2:", err)
    assert err <= TOL_MIXED


@pytest.mark.parametrize("p,L", [(3, 4), (4, 4), (6, 4)])
def test_mixed_orders_depths(p, L):
    nodes, segs, b = synth.polygon_loops(n_segs=800, n_loops=25, seed=21)
    _, F = _run(nodes, segs, b, ISO_C, p=p, levels=L, precision="mixed")
    Fo = _oracle_forces(ISO, nodes, segs, b, p, L)
    err = oracle.rel_l2(F, Fo)
    print(f"mixed p={p} L={L} vs Algorithm 2:", err)
    assert err <= TOL_MIXED


def test_mixed_rotated_crystal_general_rule():
    """A cubic crystal turned off the x, y, z axes: the near field takes the
    general unit-circle rule (all 81 stiffness entries), evaluated once per
    point pair for both directions."""
    nodes, segs, b = synth.polygon_loops(n_segs=600, n_loops=16, seed=27)
    C6 = synth.rotated_voigt(synth.cubic_voigt(), synth.rotation())
    _, F = _run(nodes, segs, b, C6, p=4, levels=4, precision="mixed", h_mode="circle", circle_q=48)
    Fo = _oracle_forces(oracle.Material.aniso(C6, Q=48), nodes, segs, b, 4, 4)
    err = oracle.rel_l2(F, Fo)
    print("mixed rotated crystal vs Algorithm 2:", err)
    assert err <= TOL_MIXED


def test_mixed_fp64_interpolation_stages():
    """GBFMM_MIXED_F64T: P2M, M2M, L2L and L2P in FP64 around the tensor-core
    M2L and the FP32 near field, against Algorithm 2 at p = 6."""
    nodes, segs, b = synth.polygon_loops(n_segs=800, n_loops=25, seed=21)
    _, F = _run(nodes, segs, b, ISO_C, p=6, levels=4, precision="mixed_f64t")
    Fo = _oracle_forces(ISO, nodes, segs, b, 6, 4)
    err = oracle.rel_l2(F, Fo)
    print("mixed with FP64 interpolation stages, p=6 L=4 vs Algorithm 2:", err)
    assert err <= TOL_MIXED


def test_mixed_cubic_circle():
    nodes, segs, b = synth.polygon_loops(n_segs=400, n_loops=12, seed=23)
    C6 = synth.cubic_voigt()
    _, F = _run(nodes, segs, b, C6, p=3, levels=4, precision="mixed", h_mode="circle", circle_q=64)
    Fo = _oracle_forces(oracle.Material.aniso(C6, Q=64), nodes, segs, b, 3, 4)
    err = oracle.rel_l2(F, Fo)
    print("mixed cubic vs Algorithm 2:", err)
    assert err <= TOL_MIXED


@pytest.mark.parametrize("m2l", [dict(m2l_split=2, m2l_basis=0, m2l_split_kblocks=0, m2l_chunks=1),
                                 dict(m2l_split=6, m2l_basis=0, m2l_split_kblocks=0, m2l_chunks=7), {}])
def test_mixed_free_targets(m2l):
    """Free points see mostly far field, where the M2L operands' rounding
    shows: residual passes on every offset (node values), or the default
    Legendre-moment operands, meet 1e-4 against Algorithm 2."""
    nodes, segs, b = synth.polygon_loops(n_segs=800, n_loops=25, seed=24)
    import paper_1712_07739_gb300 as gb

    f = gb.FMM(p=4, levels=4, precision="mixed", **m2l).set_material(ISO_C)
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    rng = np.random.default_rng(9)
    lo, hi = y.min(0), y.max(0)
    xt = lo + (hi - lo) * rng.uniform(0.02, 0.98, (400, 3))
    s = f.stress(_gpu(xt)).cpu().numpy()
    assert f.device_status() == 0
    so = oracle_b.lagrange_fmm(ISO, y, q, sid, p=4, L=4, xt=xt, tseg=-np.ones(len(xt), np.int64))
    err = oracle.rel_l2(s, so)
    print(f"mixed free targets {m2l}:", err)
    assert err <= TOL_MIXED


def test_bounded_wait_reports_timeout_and_context_recovers():
    """Failure detection without a fault: the injected pass leaves one
    pipeline stage unfilled, the consumer's wait gives up after ~10 s, the
    status word reports GBFMM_ERR_TIMEOUT, and the next pass is correct."""
    import paper_1712_07739_gb300 as gb

    nodes, segs, b = synth.polygon_loops(n_segs=600, n_loops=20, seed=25)
    f = gb.FMM(p=3, levels=3, precision="mixed").set_material(ISO_C)
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    good = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    f.inject_fault(1)
    f.nodal_forces()
    assert f.device_status() == -5
    again = f.nodal_forces().cpu().numpy()
    assert f.device_status() == 0
    assert np.allclose(again, good, rtol=0, atol=1e-12 * np.abs(good).max())


@pytest.fixture(scope="module")
def cubic_slabs_oracle():
    nodes, segs, b = synth.slab_loops(n_loops=40, segs_per_loop=20, n_slabs=3, seed=26)
    C6 = synth.cubic_voigt()
    return nodes, segs, b, C6, _oracle_forces(oracle.Material.aniso(C6, Q=64), nodes, segs, b, 5, 4)


@pytest.mark.parametrize("q", [16, 20, 32])
def test_mixed_cubic_quadrature_points(cubic_slabs_oracle, q):
    """Points of the unit-circle rule in the near field (spectral convergence:
    2.7e-5 at Q = 16, 1.5e-6 at Q = 20 in h): the mixed pass with Q points
    against Algorithm 2 with Q = 64 meets 1e-4 from Q = 16 on."""
    nodes, segs, b, C6, Fo = cubic_slabs_oracle
    _, F = _run(nodes, segs, b, C6, p=5, levels=4, precision="mixed", h_mode="circle", circle_q=q)
    err = oracle.rel_l2(F, Fo)
    print(f"circle Q={q} vs Algorithm 2 (Q=64): {err:.3e}")
    assert err <= TOL_MIXED
