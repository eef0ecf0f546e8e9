"""Writes rotated100k_sampled_forces.json: FP64 oracle nodal forces at 16
sampled nodes of the 100,000-segment slab network (2,000 loops x 50 segments
in 8 Gaussian slabs, seed 35) in the cubic crystal turned off the coordinate
axes (synth.rotated_voigt(cubic, synth.rotation())), by the direct sum of
Eq. "stress3" against all source points, unit-circle h with the general
81-entry stiffness at Q = 32 (Section 2).

Calls only the oracle and the seeded input generator.  A few minutes on 8
cores:  python tests/golden/make_rotated100k_sampled_forces.py
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

N_SAMPLE = 16
Q = 32


def main():
    nodes, segs, b = synth.slab_loops(n_loops=2000, segs_per_loop=50, n_slabs=8, seed=35)
    ids = np.sort(np.random.default_rng(3535).choice(len(nodes), N_SAMPLE, replace=False))
    mat = oracle.Material.aniso(synth.rotated_voigt(synth.cubic_voigt(), synth.rotation()), Q=Q)
    t0 = time.time()
    F, used = oracle.sampled_node_forces(mat, nodes, segs, b, ids)
    out = {
        "what": "FP64 oracle nodal forces, direct sum against all source points, unit-circle h (general medium)",
        "network": "synth.slab_loops(n_loops=2000, segs_per_loop=50, n_slabs=8, seed=35): 100,000 segments, "
                   "cubic C11=1.684 C12=1.214 C44=0.754 turned by synth.rotation()",
        "Q": Q, "n_gauss": 4, "threads": int(used), "seconds": round(time.time() - t0, 1),
        "n_nodes": int(len(nodes)), "n_segs": int(len(segs)),
        "checks": {"sum_nodes": float(nodes.sum()), "sum_abs_b": float(np.abs(b).sum()),
                   "sum_segs": int(segs.sum())},
        "node_ids": ids.tolist(), "node_xyz": nodes[ids].tolist(), "forces": F.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rotated100k_sampled_forces.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "in", out["seconds"], "s")


if __name__ == "__main__":
    main()
