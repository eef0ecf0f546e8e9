"""Writes c3q_sampled_forces.json: FP64 oracle nodal forces at 32 sampled
nodes of the 250,000-segment cubic slab network (5,000 loops x 50 segments
in 32 Gaussian slabs, seed 2), by the direct sum of Eq. "stress3" against all
1,000,000 source points with the unit-circle h at Q = 32 (Section 2,
Eq. "k_aniso" read as the unit-circle integral).

Calls only the oracle and the seeded input generator.  Takes about 5 min on
8 cores:  python tests/golden/make_c3q_sampled_forces.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1712_07739_gb300 import synth  # noqa: E402

N_SAMPLE = 32
Q = 32


def main():
    nodes, segs, b = synth.slab_loops(n_loops=5000, seed=2)
    ids = np.sort(np.random.default_rng(2025).choice(len(nodes), N_SAMPLE, replace=False))
    mat = oracle.Material.aniso(synth.cubic_voigt(), Q=Q)
    t0 = time.time()
    F, used = oracle.sampled_node_forces(mat, nodes, segs, b, ids)
    out = {
        "what": "FP64 oracle nodal forces, direct sum against all source points, unit-circle h",
        "network": "synth.slab_loops(n_loops=5000, seed=2): 250,000 segments, cubic C11=1.684 C12=1.214 C44=0.754",
        "Q": Q, "n_gauss": 4, "threads": int(used), "seconds": round(time.time() - t0, 1),
        "n_nodes": int(len(nodes)), "n_segs": int(len(segs)),
        "checks": {"sum_nodes": float(nodes.sum()), "sum_abs_b": float(np.abs(b).sum()),
                   "sum_segs": int(segs.sum())},
        "node_ids": ids.tolist(),
        "node_xyz": nodes[ids].tolist(),
        "forces": F.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3q_sampled_forces.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "in", out["seconds"], "s")


if __name__ == "__main__":
    main()
