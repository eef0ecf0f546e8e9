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
