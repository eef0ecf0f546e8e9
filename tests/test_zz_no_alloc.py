"""The allocation-free network evaluation (fmm_mlp_eval_noalloc).

Callers such as a dislocation-dynamics time step replayed from its own
memory pool cannot let the library allocate device memory.  This entry
point keeps its scratch in a static device array; its results must equal
those of the allocating fmm_mlp_eval, call after call, and sizes beyond its
stated maximum must be refused with an error.  The file sorts last so that a
stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

from paper_1712_07739_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # same kernels and summation order: expected bit-identical


def _net():
    import paper_1712_07739_gb300 as gb

    f = gb.FMM(p=3, levels=3, precision="mixed", h_mode="circle", circle_q=32).set_material(synth.cubic_voigt())
    rng = np.random.default_rng(31)
    theta = rng.normal(scale=0.08, size=gb.MLP_PARAMS).astype(np.float32)
    scale = rng.uniform(0.02, 0.08, 27).astype(np.float32)
    f.mlp_set(theta, scale)
    return f


def test_noalloc_matches_allocating_eval_twice():
    f = _net()
    for seed, n in ((41, 10_000), (42, 3_333)):
        d = torch.tensor(synth.directions(n, seed=seed), device="cuda")
        ref = f.mlp_eval(d)
        out = torch.full((n, 27), float("nan"), dtype=torch.float32, device="cuda")
        f.mlp_eval_noalloc(d, out)
        torch.cuda.synchronize()
        ref, got = ref.cpu().numpy(), out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.max(np.abs(got - ref)) <= TOL * np.abs(ref).max()


def test_noalloc_rejects_oversize():
    import paper_1712_07739_gb300 as gb

    f = _net()
    d = torch.zeros((1, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros((1, 27), dtype=torch.float32, device="cuda")
    rc = f._lib.fmm_mlp_eval_noalloc(f._h, (1 << 24) + 1, gb._ptr(d), gb._ptr(out))
    assert rc == -1
    assert "maximum" in f._lib.fmm_last_error(f._h).decode()
