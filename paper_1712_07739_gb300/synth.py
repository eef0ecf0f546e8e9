"""Seeded synthetic dislocation networks.

This module only draws geometry: closed planar polygonal glide loops with
Burgers vectors of the 1/2<111> family, the kind of network the paper's
multiple-loops benchmark uses (Section 5.2, "Multiple-loops configuration":
closed loops inside a cubic box, some of them crossing cells).  It contains
none of the stress or FMM arithmetic, so both the CUDA path and the FP64
oracle can take their inputs from here.

Every generator returns ``(nodes, segs, burgers)``:

* ``nodes``   float64 [n_nodes, 3]   node positions
* ``segs``    int64   [n_segs, 2]    node indices (line sense n0 -> n1)
* ``burgers`` float64 [n_segs, 3]    Burgers vector of each segment

Loops are closed, so every node has exactly two incident segments.
"""
from __future__ import annotations

import numpy as np

_B111 = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=np.float64)


def _unit(v):
    return v / np.linalg.norm(v)


def _glide_basis(rng, bdir):
    """Random {110} plane containing b, with a random in-plane rotation.

    For b along <111> the three {110} planes containing it have normals
    b x e_k (k = x, y, z) normalised; one is drawn uniformly.
    """
    k = rng.integers(3)
    e = np.zeros(3)
    e[k] = 1.0
    n = _unit(np.cross(bdir, e))
    e1 = _unit(np.cross(n, bdir))
    e2 = np.cross(n, e1)
    th = rng.uniform(0.0, 2.0 * np.pi)
    return n, np.cos(th) * e1 + np.sin(th) * e2, -np.sin(th) * e1 + np.cos(th) * e2


def _burgers(rng, bmag):
    d = _B111[rng.integers(4)] * (1.0 if rng.random() < 0.5 else -1.0)
    d = d / np.sqrt(3.0)
    return d, d * bmag


def _emit_loop(verts, b, nodes, segs, burg):
    base = sum(len(x) for x in nodes)
    m = len(verts)
    nodes.append(verts)
    idx = base + np.arange(m, dtype=np.int64)
    segs.append(np.stack([idx, np.roll(idx, -1)], axis=1))
    burg.append(np.repeat(b[None, :], m, axis=0))


def _pack(nodes, segs, burg):
    return (np.concatenate(nodes).astype(np.float64),
            np.concatenate(segs).astype(np.int64),
            np.concatenate(burg).astype(np.float64))


def hexagon_loops(n_loops=50, segs_per_loop=40, r_range=(0.02, 0.1),
                  bmag=1e-3, seed=0):
    """Hexagonal glide loops, each side split into sub-segments.

    40 segments per hexagon are split 7,7,7,7,6,6 over the six sides (40 is
    not a multiple of 6).  Centres uniform in the unit cube, radii uniform.
    """
    rng = np.random.default_rng(seed)
    per_side = [segs_per_loop // 6 + (1 if s < segs_per_loop % 6 else 0) for s in range(6)]
    nodes, segs, burg = [], [], []
    for _ in range(n_loops):
        c = rng.uniform(0.0, 1.0, 3)
        r = rng.uniform(*r_range)
        bdir, b = _burgers(rng, bmag)
        _, e1, e2 = _glide_basis(rng, bdir)
        corners = [c + r * (np.cos(np.pi * k / 3) * e1 + np.sin(np.pi * k / 3) * e2) for k in range(7)]
        verts = []
        for s in range(6):
            for t in range(per_side[s]):
                f = t / per_side[s]
                verts.append((1 - f) * corners[s] + f * corners[s + 1])
        _emit_loop(np.array(verts), b, nodes, segs, burg)
    return _pack(nodes, segs, burg)


def _polygon(rng, c, r, n, bdir, jitter):
    _, e1, e2 = _glide_basis(rng, bdir)
    ang = 2.0 * np.pi * (np.arange(n) + jitter * rng.uniform(-0.5, 0.5, n)) / n
    rad = r * (1.0 + jitter * rng.uniform(-0.5, 0.5, n))
    return c + rad[:, None] * (np.cos(ang)[:, None] * e1 + np.sin(ang)[:, None] * e2)


def _split_counts(rng, total, n_loops, lo, hi):
    """Loop sizes drawn U[lo, hi], then adjusted round-robin to sum to total."""
    n = rng.integers(lo, hi + 1, n_loops)
    i = 0
    while n.sum() != total:
        k = i % n_loops
        if n.sum() < total and n[k] < hi:
            n[k] += 1
        elif n.sum() > total and n[k] > lo:
            n[k] -= 1
        i += 1
    return n


def polygon_loops(n_segs=50_000, n_loops=1000, seg_range=(10, 80),
                  r_range=(0.005, 0.05), bmag=1e-3, jitter=0.1, seed=1,
                  box=1.0, origin=(0.0, 0.0, 0.0)):
    """Random polygonal loops with log-uniform radii, centres uniform in a box."""
    rng = np.random.default_rng(seed)
    counts = _split_counts(rng, n_segs, n_loops, *seg_range)
    nodes, segs, burg = [], [], []
    o = np.asarray(origin, dtype=np.float64)
    for m in counts:
        c = o + rng.uniform(0.0, box, 3)
        r = np.exp(rng.uniform(np.log(r_range[0]), np.log(r_range[1])))
        bdir, b = _burgers(rng, bmag)
        _emit_loop(_polygon(rng, c, r, int(m), bdir, jitter), b, nodes, segs, burg)
    return _pack(nodes, segs, burg)


def slab_loops(n_loops=20_000, segs_per_loop=50, n_slabs=32, sigma=0.02,
               r_range=(0.005, 0.05), bmag=1e-3, jitter=0.1, seed=2):
    """Loops clustered in Gaussian slabs that mimic dense dislocation walls.

    Each slab has a normal uniform on the sphere and passes through a point
    uniform in the unit cube; a loop centre is uniform on the slab plane
    (clipped to the cube by rejection) plus N(0, sigma^2) along the normal.
    """
    rng = np.random.default_rng(seed)
    normals = rng.normal(size=(n_slabs, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    anchors = rng.uniform(0.0, 1.0, (n_slabs, 3))
    nodes, segs, burg = [], [], []
    for _ in range(n_loops):
        s = rng.integers(n_slabs)
        n = normals[s]
        while True:
            c = rng.uniform(0.0, 1.0, 3)
            c = c - np.dot(c - anchors[s], n) * n + rng.normal(0.0, sigma) * n
            if np.all(c >= 0.0) and np.all(c <= 1.0):
                break
        r = np.exp(rng.uniform(np.log(r_range[0]), np.log(r_range[1])))
        bdir, b = _burgers(rng, bmag)
        _emit_loop(_polygon(rng, c, r, segs_per_loop, bdir, jitter), b, nodes, segs, burg)
    return _pack(nodes, segs, burg)


def ensemble(n_configs=64, ns_range=(10_000, 200_000), density_range=(0.2, 5.0), seed=4):
    """Independent configurations of uneven size for the batched pass.

    Returns a list of ``(nodes, segs, burgers)``; configuration k has
    N_s log-uniform in ns_range and a loop density (loops per unit volume)
    scaled by a factor uniform in density_range relative to 1,000 loops per
    unit cube, which sets its box edge.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_configs):
        ns = int(np.exp(rng.uniform(np.log(ns_range[0]), np.log(ns_range[1]))))
        n_loops = max(1, ns // 45)
        dens = 1000.0 * rng.uniform(*density_range)
        box = (n_loops / dens) ** (1.0 / 3.0)
        lo = max(10, min(80, ns // n_loops - 10))
        hi = max(lo, min(80, ns // n_loops + 10))
        n_loops = max(n_loops, -(-ns // hi))
        n_loops = min(n_loops, ns // lo)
        out.append(polygon_loops(n_segs=ns, n_loops=n_loops, seg_range=(lo, hi),
                                 r_range=(0.005 * box, 0.05 * box), seed=1000 + k,
                                 box=box))
    return out


def directions(n=2_000_000, near_frac=0.2, spread_deg=5.0, seed=3):
    """Unit directions for training the angular network: a fraction uniform on
    the sphere, the rest scattered (angular Gaussian, spread_deg) about the
    6 <100> and 8 <111> axes of the cubic crystal.  float32 [n, 3]."""
    rng = np.random.default_rng(seed)
    n_near = int(round(n * near_frac))
    u = rng.normal(size=(n - n_near, 3))
    axes = np.concatenate([np.eye(3), -np.eye(3),
                           np.array([[a, b, c] for a in (-1, 1) for b in (-1, 1) for c in (-1, 1)]) / np.sqrt(3.0)])
    pick = axes[rng.integers(len(axes), size=n_near)]
    v = pick + rng.normal(scale=np.deg2rad(spread_deg), size=(n_near, 3))
    d = np.concatenate([u, v])
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d[rng.permutation(n)].astype(np.float32)


def config(name: str):
    """Named workloads: c1 (2,000 iso), c2 (50,000 cubic), c3 (1M slabs)."""
    if name == "c1":
        return hexagon_loops()
    if name == "c2":
        return polygon_loops()
    if name == "c3":
        return slab_loops()
    raise ValueError(name)


def cubic_voigt(c11=1.684, c12=1.214, c44=0.754):
    """6x6 Voigt stiffness of a cubic crystal with axes along x, y, z."""
    C = np.zeros((6, 6))
    C[:3, :3] = c12
    for i in range(3):
        C[i, i] = c11
        C[3 + i, 3 + i] = c44
    return C


def isotropic_voigt(mu=1.0, nu=0.3):
    """6x6 Voigt stiffness of an isotropic medium (Lame lambda, mu)."""
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    return cubic_voigt(lam + 2.0 * mu, lam, mu)


def rotation(axis=(1.0, 2.0, 3.0), angle=0.7):
    """Proper rotation matrix about a unit axis (Rodrigues)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def rotated_voigt(C6, R):
    """Voigt stiffness of the medium C6 turned by the rotation R
    (C'_ijkl = R_ia R_jb R_kc R_ld C_abcd): a crystal whose axes are not
    along x, y, z."""
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    C = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(pairs):
        for J, (k, l) in enumerate(pairs):
            for a, b in ((i, j), (j, i)):
                for c, d in ((k, l), (l, k)):
                    C[a, b, c, d] = C6[I][J]
    Cr = np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C)
    out = np.zeros((6, 6))
    for I, (i, j) in enumerate(pairs):
        for J, (k, l) in enumerate(pairs):
            out[I, J] = Cr[i, j, k, l]
    return out
