"""Writes c2_forces.json for the 50,000-segment cubic network (1,000
polygonal loops of 10-80 segments, log-uniform radii 0.005-0.05, seed 1;
C11 = 1.684, C12 = 1.214, C44 = 0.754): FP64 oracle nodal forces by the
oracle's Lagrange FMM (Sec. 4, Algorithm 2; p = 5, 5-level octree, unit-circle
h at Q = 32) at 200 sampled nodes, and by the direct sum of Eq. "stress3" at
32 of them.

Calls only the oracle and the seeded input generator.  Several minutes on 8
cores:  python tests/golden/make_c2_forces.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import oracle_b  # noqa: E402
from paper_1712_07739_gb300 import synth  # noqa: E402

P, L, Q = 5, 5, 32


def main():
    nodes, segs, b = synth.config("c2")
    rng = np.random.default_rng(2222)
    ids = np.sort(rng.choice(len(nodes), 200, replace=False))
    ids_d = ids[np.sort(rng.choice(len(ids), 32, replace=False))]
    mat = oracle.Material.aniso(synth.cubic_voigt(), Q=Q)
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    t0 = time.time()
    F2 = oracle.nodal_forces(nodes, segs, b, oracle_b.lagrange_fmm(mat, y, q, sid, p=P, L=L), 4)
    t1 = time.time()
    Fd, used = oracle.sampled_node_forces(mat, nodes, segs, b, ids_d)
    out = {
        "what": "FP64 oracle nodal forces: Lagrange FMM (Algorithm 2) at p=5 on the 5-level octree at 200 nodes, "
                "and the direct sum of Eq. stress3 at 32 of them; unit-circle h, Q=32",
        "network": "synth.config('c2') = synth.polygon_loops(seed=1): 50,000 segments, cubic",
        "p": P, "levels": L, "Q": Q, "n_gauss": 4, "threads": int(used),
        "seconds": {"algorithm2": round(t1 - t0, 1), "direct": round(time.time() - t1, 1)},
        "n_nodes": int(len(nodes)), "n_segs": int(len(segs)),
        "checks": {"sum_nodes": float(nodes.sum()), "sum_abs_b": float(np.abs(b).sum()),
                   "sum_segs": int(segs.sum())},
        "node_ids": ids.tolist(), "node_xyz": nodes[ids].tolist(), "forces_algorithm2": F2[ids].tolist(),
        "direct_node_ids": ids_d.tolist(), "forces_direct": Fd.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_forces.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "in", out["seconds"], "s")


if __name__ == "__main__":
    main()
