"""Writes slab6k_algorithm2_forces.json: FP64 oracle nodal forces of the
6,000-segment slab network (300 loops x 20 segments in 6 Gaussian slabs,
seed 22; isotropic mu = 1, nu = 0.3) by the Lagrange FMM of the oracle
(Sec. 4, Algorithm 2; p = 6, 5-level octree) and by the direct sum of
Eq. "stress3", at 400 sampled nodes.

The GPU passes run the same method on the same tree, so the difference from
the Algorithm-2 forces is their rounding error alone (the mixed-precision
bar is 1e-4); the direct-sum forces give the interpolation error of order 6.

Calls only the oracle and the seeded input generator.  About 3 min on 8
cores:  python tests/golden/make_slab6k_algorithm2_forces.py
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

N_SAMPLE = 400
P, L = 6, 5


def main():
    nodes, segs, b = synth.slab_loops(n_loops=300, segs_per_loop=20, n_slabs=6, seed=22)
    ids = np.sort(np.random.default_rng(606).choice(len(nodes), N_SAMPLE, replace=False))
    mat = oracle.Material.iso(1.0, 0.3)
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    t0 = time.time()
    F2 = oracle.nodal_forces(nodes, segs, b, oracle_b.lagrange_fmm(mat, y, q, sid, p=P, L=L), 4)
    t1 = time.time()
    Fd, used = oracle.sampled_node_forces(mat, nodes, segs, b, ids)
    out = {
        "what": "FP64 oracle nodal forces: Lagrange FMM (Algorithm 2) at p=6 on the 5-level octree, and the "
                "direct sum of Eq. stress3, isotropic closed-form h",
        "network": "synth.slab_loops(n_loops=300, segs_per_loop=20, n_slabs=6, seed=22): 6,000 segments",
        "p": P, "levels": L, "n_gauss": 4, "threads": int(used),
        "seconds": {"algorithm2": round(t1 - t0, 1), "direct": round(time.time() - t1, 1)},
        "n_nodes": int(len(nodes)), "n_segs": int(len(segs)),
        "checks": {"sum_nodes": float(nodes.sum()), "sum_abs_b": float(np.abs(b).sum()),
                   "sum_segs": int(segs.sum())},
        "node_ids": ids.tolist(),
        "node_xyz": nodes[ids].tolist(),
        "forces_algorithm2": F2[ids].tolist(),
        "forces_direct": Fd.tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "slab6k_algorithm2_forces.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "in", out["seconds"], "s")


if __name__ == "__main__":
    main()
