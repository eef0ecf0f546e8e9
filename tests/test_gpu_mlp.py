"""The learned angular factor: GPU BF16 training and inference kernels vs the
FP64 CPU reference network, and the trained network vs the plain evaluator.
"""
import numpy as np
import pytest

import oracle
from oracle import oracle_b
from oracle import mlp_ref
from paper_1712_07739_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CUB = synth.cubic_voigt()


def _bf16(a):
    t = torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


def _ctx():
    import paper_1712_07739_gb300 as gb

    return gb.FMM(p=3, levels=3, precision="mixed", h_mode="circle", circle_q=64).set_material(CUB)


def _params(seed=0):
    rng = np.random.default_rng(seed)
    th = np.zeros(mlp_ref.N_PARAMS)
    o = 0
    for name, shp in mlp_ref.SIZES:
        n = int(np.prod(shp))
        fan = shp[1] if len(shp) == 2 else 128
        th[o:o + n] = rng.normal(scale=np.sqrt(2.0 / fan), size=n) if len(shp) == 2 else rng.normal(scale=0.1, size=n)
        o += n
    d = mlp_ref.unpack(th)
    d["W4"][27:] = 0.0
    d["b4"][27:] = 0.0
    return mlp_ref.pack(d).astype(np.float32), rng.uniform(0.02, 0.08, 27).astype(np.float32)


def _rounded(theta):
    """CPU view of the GPU's parameters: BF16 weight matrices, FP32 biases."""
    d = mlp_ref.unpack(theta.astype(np.float64))
    for k in ("W1", "W2", "W3", "W4"):
        d[k] = _bf16(d[k])
    return mlp_ref.pack(d)


def test_labels_match_oracle():
    f = _ctx()
    dirs = synth.directions(500, seed=5)
    y = f.mlp_labels(torch.tensor(dirs, device="cuda")).cpu().numpy()
    C = oracle.voigt_to_cijkl(CUB)
    ref = np.array([oracle.h_circle(C, t.astype(np.float64), 64).reshape(27) for t in dirs])
    assert np.max(np.abs(y - ref)) <= 1e-6 * np.abs(ref).max()


def test_forward_matches_cpu_reference():
    f = _ctx()
    theta, scale = _params(1)
    f.mlp_set(theta, scale)
    dirs = synth.directions(2000, seed=6)
    h = f.mlp_eval(torch.tensor(dirs, device="cuda")).cpu().numpy()
    ref, _ = mlp_ref.forward(_rounded(theta), dirs.astype(np.float64), scale)
    err = np.linalg.norm(h - ref) / np.linalg.norm(ref)
    print("forward GPU vs CPU:", err)
    assert err < 2e-2  # BF16 activations between layers


def test_gradients_match_cpu_reference():
    f = _ctx()
    theta, scale = _params(2)
    f.mlp_set(theta, scale)
    dirs = synth.directions(1024, seed=7)
    rng = np.random.default_rng(8)
    y = rng.normal(scale=0.05, size=(1024, 27)).astype(np.float32)
    g, loss = f.mlp_grad(torch.tensor(dirs, device="cuda"), torch.tensor(y, device="cuda"))
    g = g.cpu().numpy().astype(np.float64)
    l_ref, g_ref = mlp_ref.loss_and_grad(_rounded(theta), dirs.astype(np.float64), y.astype(np.float64), scale)
    assert abs(loss - l_ref) <= 2e-2 * l_ref
    o = 0
    for name, shp in mlp_ref.SIZES:
        n = int(np.prod(shp))
        a, b = g[o:o + n], g_ref[o:o + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        print(f"grad {name}: {rel:.3e}")
        assert rel < 5e-2, name
        o += n


def test_training_reduces_error():
    f = _ctx()
    dirs = torch.tensor(synth.directions(400_000, seed=9), device="cuda")
    loss = f.mlp_train(dirs, epochs=25, batch=4096, lr=3e-3, seed=1)
    test = torch.tensor(synth.directions(20_000, seed=10), device="cuda")
    h = f.mlp_eval(test).cpu().numpy()
    y = f.mlp_labels(test).cpu().numpy()
    err = np.sqrt(np.mean((h - y) ** 2)) / np.sqrt(np.mean(y ** 2))
    print("trained network relative RMS error:", err, "loss", loss)
    assert err < 5e-2
    # odd by construction
    h2 = f.mlp_eval(-test).cpu().numpy()
    assert np.array_equal(h2, -h)


def test_network_in_near_field_vs_algorithm2():
    """Mixed pass with the learned h in the near field (pairs beyond
    mlp_min_dist segment lengths, bins the plain evaluator accepted at
    5e-2 x RMS(h)) against the oracle's Lagrange FMM (Algorithm 2) on the same
    tree: the network's error in h (~1 % RMS, BF16) shows in the forces."""
    import paper_1712_07739_gb300 as gb

    nodes, segs, b = synth.slab_loops(n_loops=40, segs_per_loop=20, n_slabs=3, seed=33)
    dn, ds, db = (torch.tensor(a, device="cuda") for a in (nodes, segs, b))
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    Fo = oracle.nodal_forces(nodes, segs, b,
                             oracle_b.lagrange_fmm(oracle.Material.aniso(CUB, Q=32), y, q, sid, p=4, L=4), 4)
    f = gb.FMM(p=4, levels=4, precision="mixed", h_mode="mlp", circle_q=32, mlp_min_dist=8.0).set_material(CUB)
    f.mlp_train(torch.tensor(synth.directions(400_000, seed=34), device="cuda"), epochs=20, batch=4096, lr=3e-3,
                seed=2)
    frac = f.mlp_calibrate(5e-2)
    f.build(dn, ds, db)
    Fm = f.nodal_forces().cpu().numpy()
    err = oracle.rel_l2(Fm, Fo)
    print(f"network near field vs Algorithm 2: rel L2 {err:.3e}, bins on the plain rule {frac:.3f}")
    assert frac < 1.0  # the network serves part of the pairs
    assert np.isfinite(Fm).all()
    assert err < 1e-2
    # with every bin on the plain rule the pass meets the mixed-precision bar
    f.mlp_calibrate(1e-12)
    Fa = f.nodal_forces().cpu().numpy()
    err_plain = oracle.rel_l2(Fa, Fo)
    print(f"every bin on the plain rule vs Algorithm 2: {err_plain:.3e}")
    assert err_plain < 1e-4


def _near_ms(f, dn, ds, db, reps=3):
    f.build(dn, ds, db)
    f.set_timing(True)
    f.nodal_forces()  # warm-up
    t = []
    for _ in range(reps):
        F = f.nodal_forces()
        t.append(f.stage_times()[4])
    f.set_timing(False)
    return min(t), F.cpu().numpy()


def test_network_gain_rotated_crystal():
    """What the trained network gains: in a cubic crystal whose axes are not
    along x, y, z the plain evaluator is the general unit-circle rule (zz and
    zT from all 81 stiffness entries at Q = 32 points per pair); the network
    costs the same whatever the medium.  Same pass with the network (pairs
    beyond mlp_min_dist segment lengths, bins the plain evaluator accepted)
    against the plain evaluator everywhere: the network's near field must be
    faster, and both are measured against the oracle's direct-sum forces at
    16 stored nodes (tests/golden/rotated100k_sampled_forces.json)."""
    import json
    import os

    import paper_1712_07739_gb300 as gb

    C = synth.rotated_voigt(CUB, synth.rotation())
    nodes, segs, b = synth.slab_loops(n_loops=2000, segs_per_loop=50, n_slabs=8, seed=35)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                           "rotated100k_sampled_forces.json")) as fh:
        gold = json.load(fh)
    assert gold["n_segs"] == len(segs) and gold["checks"]["sum_segs"] == int(segs.sum())
    ids = np.array(gold["node_ids"])
    assert np.allclose(nodes[ids], np.array(gold["node_xyz"]), rtol=0, atol=1e-12)
    Fo = np.array(gold["forces"])
    dn, ds, db = (torch.tensor(a, device="cuda") for a in (nodes, segs, b))
    kw = dict(p=5, levels=5, precision="mixed", circle_q=32)
    plain = gb.FMM(h_mode="circle", **kw).set_material(C)
    t_plain, Fp = _near_ms(plain, dn, ds, db)
    f = gb.FMM(h_mode="mlp", mlp_min_dist=4.0, **kw).set_material(C)
    f.mlp_train(torch.tensor(synth.directions(1_000_000, seed=36), device="cuda"), epochs=15, batch=8192, lr=3e-3,
                seed=3)
    frac = f.mlp_calibrate(5e-2)
    t_mlp, Fm = _near_ms(f, dn, ds, db)
    e_plain = np.linalg.norm(Fp[ids] - Fo) / np.linalg.norm(Fo)
    e_mlp = np.linalg.norm(Fm[ids] - Fo) / np.linalg.norm(Fo)
    print(f"rotated cubic crystal, 100k segments: near field plain {t_plain:.1f} ms, network {t_mlp:.1f} ms "
          f"(gain {t_plain / t_mlp:.2f}x), bins on the plain rule {frac:.3f}; vs direct sum: plain {e_plain:.2e}, "
          f"network {e_mlp:.2e}")
    assert np.isfinite(Fm).all()
    assert t_plain / t_mlp > 1.0
    assert e_mlp < 2e-2
