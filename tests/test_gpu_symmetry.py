"""The symmetry-reduced M2L table of the FP64 pass (Sec. 6: 16 of the 316
operators; gbfmm_options.m2l_symmetry) against the full table and the oracle.

* Isotropic medium (closed-form h, covariant to rounding): nodal forces and
  free-target stresses with the 16-representative table equal the full
  table's to rounding (1e-12) and the oracle's Algorithm 2 to 1e-10, at
  orders 3, 5 and 7.
* Cubic medium with axes along x, y, z (unit-circle h, Q = 64): the same
  against the full table and Algorithm 2 with the oracle's cubic medium.
* A turned crystal lacks the symmetries: the evaluation reports INVALID_ARG
  and the context stays usable with the full table; the option needs the
  FP64 pass through transforms.
* The table's device memory shrinks by (343 - 16) offset slots at p = 7
  (free device memory before and after each context's first pass).
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
CUB_C = synth.cubic_voigt()
TOL_FP64 = 1e-10


def _gpu(a):
    return torch.tensor(np.asarray(a), device="cuda")


def _fmm(net, C, **kw):
    import paper_1712_07739_gb300 as gb

    nodes, segs, b = net
    f = gb.FMM(precision="fp64", m2l_fft=1, **kw).set_material(C)
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    return f


@pytest.fixture(scope="module")
def net():
    return synth.polygon_loops(n_segs=600, n_loops=20, seed=11)


def _targets(nodes, n=200, seed=6):
    rng = np.random.default_rng(seed)
    return nodes.min(0) + (nodes.max(0) - nodes.min(0)) * rng.uniform(0.05, 0.95, (n, 3))


@pytest.mark.parametrize("p,L", [(3, 4), (5, 4), (7, 3)])
def test_iso_reduced_table(net, p, L):
    nodes, segs, b = net
    xt = _targets(nodes)
    fs = _fmm(net, ISO_C, p=p, levels=L, m2l_symmetry=1)
    ff = _fmm(net, ISO_C, p=p, levels=L, m2l_symmetry=0)
    Fs, Ff = fs.nodal_forces().cpu().numpy(), ff.nodal_forces().cpu().numpy()
    ss, sf = fs.stress(_gpu(xt)).cpu().numpy(), ff.stress(_gpu(xt)).cpu().numpy()
    assert fs.device_status() == 0
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    sig = oracle_b.lagrange_fmm(ISO, y, q, sid, p=p, L=L)
    Fo = oracle.nodal_forces(nodes, segs, b, sig, 4)
    e_full, e_s, e_o = oracle.rel_l2(Fs, Ff), oracle.rel_l2(ss, sf), oracle.rel_l2(Fs, Fo)
    print(f"iso p={p} L={L}: 16-operator table vs full {e_full:.2e} (stresses {e_s:.2e}), vs Algorithm 2 {e_o:.2e}")
    assert e_full <= 1e-12 and e_s <= 1e-12
    assert e_o <= TOL_FP64


def test_cubic_reduced_table(net):
    nodes, segs, b = net
    kw = dict(p=4, levels=4, h_mode="circle", circle_q=64)
    fs = _fmm(net, CUB_C, m2l_symmetry=1, **kw)
    ff = _fmm(net, CUB_C, m2l_symmetry=0, **kw)
    Fs, Ff = fs.nodal_forces().cpu().numpy(), ff.nodal_forces().cpu().numpy()
    mat = oracle.Material.aniso(CUB_C, Q=64)
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    Fo = oracle.nodal_forces(nodes, segs, b, oracle_b.lagrange_fmm(mat, y, q, sid, p=4, L=4), 4)
    e_full, e_o = oracle.rel_l2(Fs, Ff), oracle.rel_l2(Fs, Fo)
    print(f"cubic Q=64: 16-operator table vs full {e_full:.2e}, vs Algorithm 2 {e_o:.2e}")
    assert e_full <= 1e-12
    assert e_o <= TOL_FP64


def test_turned_crystal_is_refused(net):
    import paper_1712_07739_gb300 as gb

    a = 0.4
    R = np.array([[np.cos(a), -np.sin(a), 0.0], [np.sin(a), np.cos(a), 0.0], [0.0, 0.0, 1.0]])
    C_t = synth.rotated_voigt(CUB_C, R)
    f = _fmm(net, C_t, p=3, levels=3, h_mode="circle", circle_q=32, m2l_symmetry=1)
    with pytest.raises(gb.GbfmmError):
        f.nodal_forces()
    # the aligned crystal on the same context works
    f.set_material(CUB_C)
    nodes, segs, b = net
    f.build(_gpu(nodes), _gpu(segs), _gpu(b))
    assert np.isfinite(f.nodal_forces().cpu().numpy()).all()
    for kw in (dict(precision="mixed"), dict(m2l_fft=0), dict(m2l_symmetry=2)):
        args = dict(p=3, precision="fp64", m2l_fft=1, m2l_symmetry=1)
        args.update(kw)
        with pytest.raises(gb.GbfmmError):
            gb.FMM(**args)


def test_table_memory(net):
    p = 7
    NF = (2 * p) ** 2 * (p + 1)
    used = {}
    warm = _fmm(net, ISO_C, p=p, levels=3, m2l_symmetry=0)  # modules and library state loaded once
    warm.nodal_forces()
    warm.close()
    for sym in (0, 1):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        f = _fmm(net, ISO_C, p=p, levels=3, m2l_symmetry=sym)
        f.nodal_forces()
        torch.cuda.synchronize()
        used[sym] = free0 - torch.cuda.mem_get_info()[0]
        f.close()
    saved = used[0] - used[1]
    expect = (343 - 16) * 54 * NF * 16
    print(f"p=7 operator table: full {343 * 54 * NF * 16 / 1e6:.0f} MB, reduced {16 * 54 * NF * 16 / 1e6:.1f} MB; "
          f"device memory saved {saved / 1e6:.0f} MB")
    assert abs(saved - expect) <= 0.05 * expect
