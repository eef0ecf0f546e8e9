"""Batched evaluation of independent networks: results equal separate
contexts at the same depth, the recorded graph replays identically, and the
autotuner picks a depth per network from measured costs."""
import numpy as np
import pytest

from paper_1712_07739_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CUB = synth.cubic_voigt()


def _nets():
    return [synth.polygon_loops(n_segs=n, n_loops=max(5, n // 45), seed=70 + i, box=0.5 + 0.2 * i)
            for i, n in enumerate((1200, 5000, 2500, 9000))]


def _gpu(a):
    return torch.tensor(np.asarray(a), device="cuda")


def test_batch_equals_separate_contexts():
    import paper_1712_07739_gb300 as gb

    nets = _nets()
    bt = gb.Batch(len(nets), p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
    for k, (n, s, b) in enumerate(nets):
        bt.build(k, _gpu(n), _gpu(s), _gpu(b))
    F1 = [f.cpu().numpy().copy() for f in bt.nodal_forces()]
    F2 = [f.cpu().numpy().copy() for f in bt.nodal_forces()]  # graph replay
    for k, (n, s, b) in enumerate(nets):
        f = gb.FMM(p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
        f.build(_gpu(n), _gpu(s), _gpu(b))
        Fs = f.nodal_forces().cpu().numpy()
        assert np.array_equal(F1[k], Fs), k
        assert np.array_equal(F2[k], Fs), k


def test_batch_autotuned_depths():
    import paper_1712_07739_gb300 as gb

    nets = _nets()
    bt = gb.Batch(len(nets), p=4, levels=0, leaf_segments=32, precision="mixed", h_mode="circle",
                  circle_q=24).set_material(CUB)
    for k, (n, s, b) in enumerate(nets):
        bt.build(k, _gpu(n), _gpu(s), _gpu(b))
    F = bt.nodal_forces()
    torch.cuda.synchronize()
    info = [bt.info(k) for k in range(len(nets))]
    print("autotuned depths:", [i["levels"] for i in info], "c_near", info[0]["c_near"], "c_far", info[0]["c_far"])
    assert all(3 <= i["levels"] <= 8 for i in info)
    assert info[0]["c_near"] > 0 and info[0]["c_far"] > 0
    assert all(np.isfinite(f.cpu().numpy()).all() for f in F)
    # each network at its chosen depth alone gives the same forces
    for k, (n, s, b) in enumerate(nets):
        f = gb.FMM(p=4, levels=info[k]["levels"], precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
        f.build(_gpu(n), _gpu(s), _gpu(b))
        assert np.array_equal(F[k].cpu().numpy(), f.nodal_forces().cpu().numpy())


def test_batch_rebuild_with_another_network_rerecords():
    """Replacing one network (other size, other buffers) invalidates the
    recorded graph: the next evaluation records a new one and matches a
    separate context; rebuilding the same network keeps results identical."""
    import paper_1712_07739_gb300 as gb

    nets = _nets()
    bt = gb.Batch(len(nets), p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
    for k, (n, s, b) in enumerate(nets):
        bt.build(k, _gpu(n), _gpu(s), _gpu(b))
    F0 = [f.cpu().numpy().copy() for f in bt.nodal_forces()]
    other = synth.polygon_loops(n_segs=14000, n_loops=300, seed=99, box=0.8)
    bt.build(1, _gpu(other[0]), _gpu(other[1]), _gpu(other[2]))
    F1 = [f.cpu().numpy().copy() for f in bt.nodal_forces()]
    f = gb.FMM(p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
    f.build(_gpu(other[0]), _gpu(other[1]), _gpu(other[2]))
    assert np.array_equal(F1[1], f.nodal_forces().cpu().numpy())
    for k in (0, 2, 3):
        assert np.array_equal(F1[k], F0[k]), k


def _moved(n, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    return np.asarray(n) + amp * rng.normal(size=np.shape(n))


def test_step_equals_separate_builds_and_follows_moved_nodes():
    """A step (every tree rebuilt on the device and every network evaluated,
    one graph replay) gives the forces of separate contexts built from the same
    nodes; after the nodes move in place the next replay follows them, although
    the graph was recorded before the move (the leaf occupancy changes, the
    buffer sizes do not)."""
    import paper_1712_07739_gb300 as gb

    nets = _nets()
    bt = gb.Batch(len(nets), p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
    for k, (n, s, b) in enumerate(nets):
        bt.build(k, _gpu(n), _gpu(s), _gpu(b))
    launches0 = bt.info(0)["launches"]
    F1 = [f.cpu().numpy().copy() for f in bt.step()]
    launches1 = bt.info(0)["launches"]
    F2 = [f.cpu().numpy().copy() for f in bt.step()]
    per_step = bt.info(0)["launches"] - launches1
    assert per_step > 0 and launches1 - launches0 == per_step  # every replay counts its kernels
    assert bt.status() == (-1, 0)
    for k, (n, s, b) in enumerate(nets):
        f = gb.FMM(p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
        f.build(_gpu(n), _gpu(s), _gpu(b))
        Fs = f.nodal_forces().cpu().numpy()
        assert np.array_equal(F1[k], Fs), k
        assert np.array_equal(F2[k], Fs), k
    moved = [_moved(n, 200 + k) for k, (n, _, _) in enumerate(nets)]
    for k in range(len(nets)):
        bt.nodes(k).copy_(_gpu(moved[k]))
    F3 = [f.cpu().numpy().copy() for f in bt.step()]
    assert bt.status() == (-1, 0)
    for k, (_, s, b) in enumerate(nets):
        f = gb.FMM(p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
        f.build(_gpu(moved[k]), _gpu(s), _gpu(b))
        assert np.array_equal(F3[k], f.nodal_forces().cpu().numpy()), k
        assert not np.array_equal(F3[k], F1[k])


def test_step_status_reports_a_collapsed_segment():
    """The recorded builds skip the host checks: a segment collapsed in place
    (both ends on one point) shows in the status read afterwards, and the
    other networks' slots are not blamed."""
    import paper_1712_07739_gb300 as gb

    nets = _nets()[:3]
    bt = gb.Batch(len(nets), p=4, levels=4, precision="mixed", h_mode="circle", circle_q=24).set_material(CUB)
    for k, (n, s, b) in enumerate(nets):
        bt.build(k, _gpu(n), _gpu(s), _gpu(b))
    bt.step()
    assert bt.status() == (-1, 0)
    i, j = (int(x) for x in nets[1][1][0])
    x = bt.nodes(1)
    x[j] = x[i]
    bt.step()
    assert bt.status() == (1, -6)  # GBFMM_ERR_DEGENERATE
    x.copy_(_gpu(nets[1][0]))
    bt.step()
    assert bt.status() == (-1, 0)


def test_step_autotuned_tile_form():
    """Created with m2l_kernel=2 the batch times both M2L tile forms on the
    calibration network and keeps the faster; the forces equal a separate
    context using the chosen form at the chosen depth."""
    import paper_1712_07739_gb300 as gb

    nets = _nets()
    bt = gb.Batch(len(nets), p=5, levels=0, leaf_segments=32, precision="mixed", h_mode="circle", circle_q=24,
                  m2l_kernel=2).set_material(CUB)
    for k, (n, s, b) in enumerate(nets):
        bt.build(k, _gpu(n), _gpu(s), _gpu(b))
    F = [f.cpu().numpy().copy() for f in bt.step()]
    t = bt.tuning()
    print("tile form", t)
    assert t["m2l_kernel"] in (0, 1) and min(t["m2l_ms"]) > 0
    assert t["m2l_ms"][t["m2l_kernel"]] <= t["m2l_ms"][1 - t["m2l_kernel"]]
    for k, (n, s, b) in enumerate(nets):
        f = gb.FMM(p=5, levels=bt.info(k)["levels"], precision="mixed", h_mode="circle", circle_q=24,
                   m2l_kernel=t["m2l_kernel"]).set_material(CUB)
        f.build(_gpu(n), _gpu(s), _gpu(b))
        assert np.array_equal(F[k], f.nodal_forces().cpu().numpy()), k
