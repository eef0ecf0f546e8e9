"""Writes c5_sampled_forces.json: FP64 oracle nodal forces at 8 sampled nodes
of three networks of the 64-network cubic ensemble (synth.ensemble, seed 4):
the smallest, the one nearest the median size and the largest, by the direct
sum of Eq. "stress3" against all source points of each network, unit-circle
h at Q = 32 (Section 2, Eq. "k_aniso" read as the unit-circle integral).

Calls only the oracle and the seeded input generator.  A few minutes on 8
cores:  python tests/golden/make_c5_sampled_forces.py
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

N_SAMPLE = 8
Q = 32


def main():
    nets = synth.ensemble(seed=4)
    sizes = np.array([len(s) for _, s, _ in nets])
    order = np.argsort(sizes)
    pick = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    mat = oracle.Material.aniso(synth.cubic_voigt(), Q=Q)
    out = {
        "what": "FP64 oracle nodal forces, direct sum against all source points of each network, unit-circle h",
        "ensemble": "synth.ensemble(seed=4): 64 cubic networks, C11=1.684 C12=1.214 C44=0.754",
        "Q": Q, "n_gauss": 4, "networks": [],
    }
    t0 = time.time()
    for k in pick:
        nodes, segs, b = nets[k]
        ids = np.sort(np.random.default_rng(5000 + k).choice(len(nodes), N_SAMPLE, replace=False))
        F, used = oracle.sampled_node_forces(mat, nodes, segs, b, ids)
        out["networks"].append({
            "index": k, "n_nodes": int(len(nodes)), "n_segs": int(len(segs)),
            "checks": {"sum_nodes": float(nodes.sum()), "sum_abs_b": float(np.abs(b).sum()),
                       "sum_segs": int(segs.sum())},
            "node_ids": ids.tolist(), "node_xyz": nodes[ids].tolist(), "forces": F.tolist(),
        })
        out["threads"] = int(used)
    out["seconds"] = round(time.time() - t0, 1)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c5_sampled_forces.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "in", out["seconds"], "s")


if __name__ == "__main__":
    main()
