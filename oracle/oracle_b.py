"""The Lagrange FMM by its definition, in plain NumPy, for tiny inputs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The method (arXiv:1712.07739, Sec. 4) replaces the kernel between two
well-separated cells by its tensor-product Lagrange interpolant on p
equispaced nodes per axis in each cell (Sec. 4.1, Eq. "interpolant"), so the
far-field sum at a target factors (Sec. 4.3, Eq. "far-field") into: the
source strengths weighted by the source cell's basis functions at the
source points (the multipole weights W of each node), the node-to-node
kernel matrix of the cell pair (Eq. "m2l") applied to them, and the target
cell's basis functions at the target.  On a uniform octree with levels
0 .. L-1 (Algorithm 2) the weights of a parent follow from its children's by
evaluating the parent's basis at the child nodes (exact: the child
interpolant is a polynomial of the same degree), each cell receives the
node-kernel sums of its interaction list, a child receives its parent's
local values interpolated to its nodes, and a leaf's targets get the local
values interpolated to them plus the direct sum of Eq. "stress3" over the
neighbouring leaves.

The Chebyshev FMM the paper compares against (Sec. 3, the kernel-independent
method of Fong and Darve it implements) is the same algorithm on Chebyshev
nodes with the M2L compressed by the singular value decomposition: the node
set is a parameter here (``nodes``), and ``m2l_svd_bases`` gives the two
orthonormal bases of the compression, which ``lagrange_fmm`` applies when
given them.

The symmetry reduction the paper points to (Sec. 6): for a medium with the
cube's symmetries (isotropic, or cubic with axes along x, y, z) every one of
the 316 operators is a signed permutation of rows and columns of one of 16
(``cube_group``, ``offset_orbits``, ``symmetric_operator``).

``lagrange_fmm`` computes that result level by level.
``pairwise_far_field`` evaluates Eq. "far-field" separately for every
(target cell, interaction-list cell) pair at every level, with no
child/parent transfers; the two agree to rounding because the transfers are
exact, which is a pin.

Conventions (readings of the paper where it is silent):
* root cube: edge H = s (1 + 2^-10), s the largest extent of the source
  points (1 if they coincide), centred on their bounding box; a point goes to
  cell floor((y - origin) * (2^l / H)), clamped to [0, 2^l - 1];
* nodes: p equispaced nodes per dimension including the cell faces,
  t_a = a / (p - 1), a = 0..p-1 (Section 4.1); Chebyshev nodes are the
  zeros of the Chebyshev polynomial T_p mapped to [0, 1] (first kind),
  t_a = (1 - cos((2a + 1) pi / (2p))) / 2, in increasing order;
* SVD compression (Sec. 3, Eq. "mem_cheb"; the paper gives the compression
  ratio, not the construction, which is the cited black-box FMM's): with
  T_o the node-kernel matrix of offset o on a unit cell (rows (target node,
  stress component), columns (source node, strength component)), the target
  basis U holds the leading left singular vectors of [T_1 ... T_316] side by
  side and the source basis R the leading right singular vectors of the 316
  stacked; a vector is kept while its singular value exceeds tol times the
  largest.  The compressed M2L applies U (U^T T_o R) R^T in place of T_o;
  the kernel's homogeneity makes the bases one for all levels;
* basis: "owner cell's basis at node l, evaluated at the point" for all of
  P2M, M2M, L2L and L2P (the argument order of L_p is inconsistent between
  Algorithms 1 and 2);
* C(.), I(.), P(.), N(.) are the standard uniform-octree sets; M2L runs at
  levels >= 2; the near sum skips source points of the target's own segment.
"""
from __future__ import annotations

import itertools

import numpy as np

from . import direct_stress, kernel


def root_box(y):
    lo = y.min(axis=0)
    hi = y.max(axis=0)
    s = float(np.max(hi - lo))
    if s == 0.0:
        s = 1.0
    H = s * (1.0 + 2.0 ** -10)
    origin = 0.5 * (lo + hi) - 0.5 * H
    return origin, H


def cell_of(y, origin, H, level):
    n = 1 << level
    idx = np.floor((y - origin) * (n / H)).astype(np.int64)
    return np.clip(idx, 0, n - 1)


def node_positions(p, nodes="equispaced"):
    """The p interpolation nodes of a unit cell, in [0, 1], increasing."""
    if nodes == "equispaced":
        return np.arange(p) / (p - 1)
    if nodes == "chebyshev":
        return 0.5 * (1.0 - np.cos((2 * np.arange(p) + 1) * np.pi / (2 * p)))
    raise ValueError(nodes)


def basis_1d(t, p, nodes="equispaced"):
    """ell_a(t) = prod_{b != a} (t - t_b) / (t_a - t_b) on the node set's t_a."""
    nodes = node_positions(p, nodes)
    t = np.asarray(t, dtype=np.float64)
    out = np.ones(t.shape + (p,))
    for a in range(p):
        for b in range(p):
            if b != a:
                out[..., a] *= (t - nodes[b]) / (nodes[a] - nodes[b])
    return out


def basis_3d(t, p, nodes="equispaced"):
    """L_p(xbar_l, x) for local coordinates t [n, 3] -> [n, p^3], l = (a, b, c)
    flattened with a (x) slowest."""
    bx, by, bz = basis_1d(t[:, 0], p, nodes), basis_1d(t[:, 1], p, nodes), basis_1d(t[:, 2], p, nodes)
    return np.einsum("na,nb,nc->nabc", bx, by, bz).reshape(len(t), p ** 3)


def child_transfer(p, nodes="equispaced"):
    """M[c][a', a] = ell_a'((c + t_a) / 2): parent basis a' at child node a."""
    t = node_positions(p, nodes)
    return [basis_1d((c + t) / 2.0, p, nodes).T for c in (0, 1)]


def interaction_offsets(cell):
    """Offsets o = B - A of the interaction list I(B) for a cell B at
    integer coordinates ``cell``: children of the parent's neighbours that
    are not neighbours of B."""
    par = np.asarray(cell) // 2
    out = []
    for dp in itertools.product((-1, 0, 1), repeat=3):
        for c in itertools.product((0, 1), repeat=3):
            a = 2 * (par + np.asarray(dp)) + np.asarray(c)
            o = np.asarray(cell) - a
            if np.max(np.abs(o)) >= 2:
                out.append(tuple(o))
    return out


def _node_kernels(mat, p, h, o, rows=None, nodes="equispaced"):
    """T_o[l, :, m, :] = K(xbar_l - ybar_m) for one offset o, with the node
    difference (o + (t_l - t_m)) h; returns [len(rows), 6, p^3, 9] for the
    requested target-node rows l (all rows by default)."""
    t = node_positions(p, nodes)
    g = np.array(list(itertools.product(t, t, t)))  # [p^3, 3], x slowest
    if rows is None:
        rows = np.arange(len(g))
    diff = g[rows][:, None, :] - g[None, :, :]       # [l, m, 3]
    d = (np.asarray(o, dtype=np.float64)[None, None, :] + diff) * h
    K = kernel(mat, d.reshape(-1, 3)).reshape(len(rows), len(g), 6, 9)
    return np.ascontiguousarray(K.transpose(0, 2, 1, 3))


def _apply_offset(mat, p, h, o, Wstack, chunk=64, nodes="equispaced"):
    """sum_m K(xbar_l - ybar_m) W_m for a stack of source weights [n, p^3, 9]
    -> [n, p^3, 6], building the node kernel a block of rows at a time."""
    P3 = p ** 3
    out = np.zeros((Wstack.shape[0], P3, 6))
    for r0 in range(0, P3, chunk):
        rows = np.arange(r0, min(P3, r0 + chunk))
        T = _node_kernels(mat, p, h, o, rows, nodes)
        out[:, rows, :] = np.einsum("lamw,nmw->nla", T, Wstack)
    return out


def m2l_offsets():
    """The 316 offsets o = B - A over all interaction lists: o in [-3, 3]^3 with
    max |o_i| >= 2 (the 7^3 - 3^3 of Sec. 3's count of pre-computed operators)."""
    return [o for o in itertools.product(range(-3, 4), repeat=3) if max(abs(x) for x in o) >= 2]


def cube_group():
    """The 48 orthogonal maps of a cube onto itself (Sec. 6: the symmetries of
    space the operator count 316 -> 16 relies on): the signed permutation
    matrices g, g[i, pi(i)] = s_i, 24 of them proper (det +1)."""
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            g = np.zeros((3, 3), dtype=np.int64)
            for i in range(3):
                g[i, perm[i]] = signs[i]
            out.append(g)
    return out


def offset_orbits():
    """The 316 offsets grouped into orbits of ``cube_group``: a list of
    (rep, members), members = [(o, g)] with o = g rep for every offset of the
    orbit, rep the member with non-negative components in decreasing order."""
    G = cube_group()
    seen, out = set(), []
    for o in m2l_offsets():
        rep = tuple(sorted((abs(x) for x in o), reverse=True))
        if rep in seen:
            continue
        seen.add(rep)
        members = {}
        for g in G:
            img = tuple(int(x) for x in g @ np.array(rep))
            members.setdefault(img, g)  # one map per image
        out.append((rep, sorted(members.items())))
    return out


def symmetric_operator(mat, p, o, g, rep, nodes="equispaced"):
    """T_o [p^3, 6, p^3, 9] (layout of ``_node_kernels``) built from the
    operator of its orbit's representative, o = g rep.

    For a medium with C_ijkl invariant under g the kernel obeys
    K(g d)_{ab,wr} = det(g) g_ai g_bj g_wk g_rl K(d)_{ij,kl} (the factor det(g)
    comes from the permutation symbol in the kernel of Sec. 2, a pseudo-tensor).
    The cell maps onto itself by x -> g (x - c) + c about its centre c, which
    takes node l (positions t_l) to the node l' with l'_i = l_pi(i) where
    s_i = +1 and p - 1 - l_pi(i) where s_i = -1 (the node sets are symmetric
    under t -> 1 - t); node differences then map by g, so
    T_o[l', ab, m', wr] = det(g) s_a s_b s_w s_r T_rep[l, pi(a)pi(b), m, pi(w)pi(r)]."""
    g = np.asarray(g)
    assert tuple(int(x) for x in g @ np.array(rep)) == tuple(o)
    P3 = p ** 3
    T = _node_kernels(mat, p, 1.0, rep, nodes=nodes)  # [l, ab, m, wr]
    perm = [int(np.nonzero(g[i])[0][0]) for i in range(3)]
    sgn = [int(g[i, perm[i]]) for i in range(3)]
    det = int(round(np.linalg.det(g)))
    # node map l -> l' (index (lx p + ly) p + lz, x slowest)
    idx = np.array(list(itertools.product(range(p), repeat=3)))
    img = np.empty_like(idx)
    for i in range(3):
        col = idx[:, perm[i]]
        img[:, i] = col if sgn[i] > 0 else p - 1 - col
    lmap = (img[:, 0] * p + img[:, 1]) * p + img[:, 2]
    voigt = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    out = np.zeros((P3, 6, P3, 9))
    for ab, (a, b) in enumerate(pairs):
        src_ab = voigt[(perm[a], perm[b])]
        for w in range(3):
            for r in range(3):
                s = det * sgn[a] * sgn[b] * sgn[w] * sgn[r]
                out[np.ix_(lmap, [ab], lmap, [3 * w + r])] = s * T[:, [src_ab], :, :][:, :, :, [3 * perm[w] + perm[r]]]
    return out


def m2l_svd_bases(mat, p, nodes="equispaced", tol=None, ranks=None):
    """Bases of the SVD-compressed M2L on a unit cell (module header): U [6 p^3, r1]
    and R [9 p^3, r2] with orthonormal columns, and the singular values of the
    side-by-side (target side) and stacked (source side) operator matrices, in
    decreasing order.  Their squares are the eigenvalues of the Gram matrices
    sum_o T_o T_o^T and sum_o T_o^T T_o, whose eigenvectors are the singular
    vectors.  The ranks come from ``tol`` (relative to the largest singular
    value) or are given as ``ranks`` = (r1, r2)."""
    P3 = p ** 3
    Gt = np.zeros((6 * P3, 6 * P3))
    Gs = np.zeros((9 * P3, 9 * P3))
    for o in m2l_offsets():
        T = _node_kernels(mat, p, 1.0, o, nodes=nodes).reshape(6 * P3, 9 * P3)
        Gt += T @ T.T
        Gs += T.T @ T
    lt, Ut = np.linalg.eigh(Gt)
    ls, Us = np.linalg.eigh(Gs)
    st, Ut = np.sqrt(np.maximum(lt[::-1], 0.0)), Ut[:, ::-1]
    ss, Us = np.sqrt(np.maximum(ls[::-1], 0.0)), Us[:, ::-1]
    if ranks is None:
        ranks = (int((st > tol * st[0]).sum()), int((ss > tol * ss[0]).sum()))
    r1, r2 = ranks
    return np.ascontiguousarray(Ut[:, :r1]), np.ascontiguousarray(Us[:, :r2]), st, ss


def _near(mat, xt, tseg, tleaf, ys, qs, sseg, sleaf, n):
    out = np.zeros((len(xt), 6))
    for key in np.unique(tleaf[:, 0] * n * n + tleaf[:, 1] * n + tleaf[:, 2]):
        B = np.array([key // (n * n), (key // n) % n, key % n])
        ti = np.nonzero((tleaf == B).all(axis=1))[0]
        lo = np.maximum(B - 1, 0)
        hi = np.minimum(B + 1, n - 1)
        m = ((sleaf >= lo) & (sleaf <= hi)).all(axis=1)
        sj = np.nonzero(m)[0]
        if len(sj) == 0:
            continue
        out[ti] = direct_stress(mat, xt[ti], tseg[ti], ys[sj], qs[sj], sseg[sj])
    return out


def _m2l_level(mat, p, H, lev, W, src_occ, tgt_occ, nodes, svd):
    """Node-kernel sums of one level's interaction lists (Algorithm 2, M2L), pairs
    grouped by offset: S[B] = sum over A in I(B) of T_(B - A) W[A] for the target
    cells tgt_occ and the source cells src_occ (boolean grids); with svd the
    compressed M2L (sources projected onto R, each cell's sum onto U)."""
    n = 1 << lev
    h = H / n
    P3 = p ** 3
    S = np.zeros((n, n, n, P3, 6))
    groups = {}
    for B in itertools.product(range(n), repeat=3):
        if not tgt_occ[B]:
            continue  # no target below B: its local values are never used
        for o in interaction_offsets(B):
            A = tuple(B[d] - o[d] for d in range(3))
            if all(0 <= A[d] < n for d in range(3)) and src_occ[A]:
                groups.setdefault(o, []).append((B, A))
    for o, pairs in groups.items():
        Ws = np.stack([W[A] for _, A in pairs])
        if svd is not None:  # R R^T W: the source weights seen through the compression
            R = svd[1]
            Ws = ((Ws.reshape(len(pairs), 9 * P3) @ R) @ R.T).reshape(len(pairs), P3, 9)
        res = _apply_offset(mat, p, h, o, Ws, nodes=nodes)
        for (B, _), r in zip(pairs, res):
            S[B] += r
    if svd is not None:  # U U^T of each cell's M2L sum
        U = svd[0]
        S = ((S.reshape(-1, 6 * P3) @ U) @ U.T).reshape(S.shape)
    return S


def lagrange_fmm(mat, ys, qs, sseg, p, L, xt=None, tseg=None, nodes="equispaced", svd=None):
    """Stress [n_t, 6] at targets by the multilevel Lagrange FMM (Algorithm 2; targets
    default to sources), on the given node set; with svd = (U, R) from
    ``m2l_svd_bases`` the M2L is the compressed one: every source cell's weights
    are projected onto R's columns and every cell's M2L sum onto U's."""
    ys = np.asarray(ys, dtype=np.float64)
    qs = np.asarray(qs, dtype=np.float64).reshape(-1, 9)
    if xt is None:
        xt, tseg = ys, sseg
    origin, H = root_box(ys)
    S, sl, tl = _far_levels(mat, ys, qs, p, L, xt, origin, H, nodes, svd)
    lf = L - 1
    nL = 1 << lf
    hL = H / nL
    out = np.zeros((len(xt), 6))
    if lf >= 2:
        tt = (xt - (origin + tl * hL)) / hL
        out += np.einsum("nl,nls->ns", basis_3d(tt, p, nodes), S[lf][tl[:, 0], tl[:, 1], tl[:, 2]])
    out += _near(mat, xt, np.asarray(tseg), tl, ys, qs, np.asarray(sseg), sl, nL)
    return out


def _far_levels(mat, ys, qs, p, L, xt, origin, H, nodes, svd):
    """P2M at the leaves, M2M up, M2L at every level >= 2 and L2L down (Algorithm 2):
    the local values S[level] of every cell, and the leaf cell of each source
    and target."""
    lf = L - 1
    nL = 1 << lf
    P3 = p ** 3
    # multipole weights of the leaves: source strengths times the leaf basis at the points
    W = {lf: np.zeros((nL, nL, nL, P3, 9))}
    sl = cell_of(ys, origin, H, lf)
    hL = H / nL
    t = (ys - (origin + sl * hL)) / hL
    Lb = basis_3d(t, p, nodes)
    np.add.at(W[lf], (sl[:, 0], sl[:, 1], sl[:, 2]), Lb[:, :, None] * qs[:, None, :])
    # weights of the parents: the parent basis at the child nodes (upward)
    M = child_transfer(p, nodes)
    for lev in range(lf - 1, 1, -1):
        n = 1 << lev
        Wp = np.zeros((n, n, n, P3, 9))
        Wc = W[lev + 1]
        for c in itertools.product((0, 1), repeat=3):
            ch = Wc[c[0]::2, c[1]::2, c[2]::2].reshape(n, n, n, p, p, p, 9)
            Wp += np.einsum("Aa,Bb,Cc,xyzabcw->xyzABCw", M[c[0]], M[c[1]], M[c[2]], ch).reshape(
                n, n, n, P3, 9)
        W[lev] = Wp
    # node-kernel sums over the interaction lists at every level >= 2
    S = {}
    for lev in range(2, lf + 1):
        n = 1 << lev
        occ = np.zeros((n, n, n), dtype=bool)
        c = cell_of(ys, origin, H, lev)
        occ[c[:, 0], c[:, 1], c[:, 2]] = True
        tocc = np.zeros((n, n, n), dtype=bool)
        c = cell_of(xt, origin, H, lev)
        tocc[c[:, 0], c[:, 1], c[:, 2]] = True
        S[lev] = _m2l_level(mat, p, H, lev, W[lev], occ, tocc, nodes, svd)
    # local values of the children: the parent's interpolated to the child nodes (downward)
    for lev in range(3, lf + 1):
        n = 1 << (lev - 1)
        Sp = S[lev - 1].reshape(n, n, n, p, p, p, 6)
        for c in itertools.product((0, 1), repeat=3):
            add = np.einsum("Aa,Bb,Cc,xyzABCs->xyzabcs", M[c[0]], M[c[1]], M[c[2]], Sp)
            S[lev][c[0]::2, c[1]::2, c[2]::2] += add.reshape(n, n, n, P3, 6)
    return S, sl, cell_of(xt, origin, H, lf)


def adaptive_fmm(mat, ys, qs, sseg, p, L, refine, nodes="equispaced", svd=None):
    """Stress [n, 6] at the source points by the Lagrange FMM on an adaptive tree:
    the uniform tree of Algorithm 2 (leaves at level L - 1) in which every leaf
    holding more than ``refine`` points is split once more.  Two adjacent split
    leaves interact through their children: adjacent children by the direct sum
    of Eq. "stress3", the others by an M2L at level L (the children's interaction
    lists, restricted to children of split leaves); every other pair of adjacent
    leaves by the direct sum as in Algorithm 2.  The points of a split leaf take
    the local values of their child: the parent's interpolated to it plus the
    level-L M2L sum.  With every occupied leaf split this is Algorithm 2 on L + 1
    levels."""
    ys = np.asarray(ys, dtype=np.float64)
    qs = np.asarray(qs, dtype=np.float64).reshape(-1, 9)
    sseg = np.asarray(sseg)
    origin, H = root_box(ys)
    S, sl, _ = _far_levels(mat, ys, qs, p, L, ys, origin, H, nodes, svd)
    lf = L - 1
    nL, nF = 1 << lf, 2 << lf
    hL, hF = H / nL, H / nF
    P3 = p ** 3
    cnt = np.zeros((nL, nL, nL), dtype=np.int64)
    np.add.at(cnt, (sl[:, 0], sl[:, 1], sl[:, 2]), 1)
    split = cnt > refine
    in_split = split[sl[:, 0], sl[:, 1], sl[:, 2]]
    sf = cell_of(ys, origin, H, lf + 1)
    # children of split leaves: multipole weights, M2L among themselves at level L, L2L from the parent
    idx = np.nonzero(in_split)[0]
    Wf = np.zeros((nF, nF, nF, P3, 9))
    tf = (ys[idx] - (origin + sf[idx] * hF)) / hF
    np.add.at(Wf, (sf[idx, 0], sf[idx, 1], sf[idx, 2]), basis_3d(tf, p, nodes)[:, :, None] * qs[idx][:, None, :])
    focc = np.zeros((nF, nF, nF), dtype=bool)
    focc[sf[idx, 0], sf[idx, 1], sf[idx, 2]] = True
    Sf = _m2l_level(mat, p, H, lf + 1, Wf, focc, focc, nodes, svd)
    if lf >= 2:
        M = child_transfer(p, nodes)
        Sp = S[lf].reshape(nL, nL, nL, p, p, p, 6)
        for c in itertools.product((0, 1), repeat=3):
            add = np.einsum("Aa,Bb,Cc,xyzABCs->xyzabcs", M[c[0]], M[c[1]], M[c[2]], Sp)
            Sf[c[0]::2, c[1]::2, c[2]::2] += add.reshape(nL, nL, nL, P3, 6)
    # far field at the points: the leaf's local values, or the child's for points of split leaves
    out = np.zeros((len(ys), 6))
    co = np.nonzero(~in_split)[0]
    if lf >= 2 and len(co):
        tt = (ys[co] - (origin + sl[co] * hL)) / hL
        out[co] += np.einsum("nl,nls->ns", basis_3d(tt, p, nodes), S[lf][sl[co, 0], sl[co, 1], sl[co, 2]])
    if len(idx):
        out[idx] += np.einsum("nl,nls->ns", basis_3d(tf, p, nodes), Sf[sf[idx, 0], sf[idx, 1], sf[idx, 2]])
    # near field: adjacent leaves, except non-adjacent children of two different split leaves
    for key in np.unique(sl[:, 0] * nL * nL + sl[:, 1] * nL + sl[:, 2]):
        B = np.array([key // (nL * nL), (key // nL) % nL, key % nL])
        ti = np.nonzero((sl == B).all(axis=1))[0]
        near = ((sl >= B - 1) & (sl <= B + 1)).all(axis=1)
        if not split[tuple(B)]:
            sj = np.nonzero(near)[0]
            out[ti] += direct_stress(mat, ys[ti], sseg[ti], ys[sj], qs[sj], sseg[sj])
            continue
        other_split = near & in_split & ~(sl == B).all(axis=1)
        for fc in np.unique(sf[ti], axis=0):
            tc = ti[(sf[ti] == fc).all(axis=1)]
            keep = near & ~(other_split & (np.abs(sf - fc).max(axis=1) >= 2))
            sj = np.nonzero(keep)[0]
            out[tc] += direct_stress(mat, ys[tc], sseg[tc], ys[sj], qs[sj], sseg[sj])
    return out


def pairwise_far_field(mat, ys, qs, sseg, p, L, xt=None, tseg=None, nodes="equispaced"):
    """Far field of the same tree by Eq. "far-field" for each (B, A) pair with
    A in I(B), at each level >= 2: the weights of A's points on A's nodes, the
    node kernel of the pair, B's basis at B's points.  Near sum included."""
    ys = np.asarray(ys, dtype=np.float64)
    qs = np.asarray(qs, dtype=np.float64).reshape(-1, 9)
    if xt is None:
        xt, tseg = ys, sseg
    origin, H = root_box(ys)
    lf = L - 1
    out = np.zeros((len(xt), 6))
    for lev in range(2, lf + 1):
        n = 1 << lev
        h = H / n
        sc = cell_of(ys, origin, H, lev)
        tc = cell_of(xt, origin, H, lev)
        for B in {tuple(r) for r in tc}:
            ti = np.nonzero((tc == B).all(axis=1))[0]
            LB = basis_3d((xt[ti] - (origin + np.asarray(B) * h)) / h, p, nodes)
            for o in interaction_offsets(B):
                A = tuple(B[d] - o[d] for d in range(3))
                sj = np.nonzero((sc == A).all(axis=1))[0]
                if len(sj) == 0:
                    continue
                LA = basis_3d((ys[sj] - (origin + np.asarray(A) * h)) / h, p, nodes)
                Wm = LA.T @ qs[sj]                                   # weights on A's nodes
                sl = _apply_offset(mat, p, h, o, Wm[None], nodes=nodes)[0]  # node kernel of (B, A)
                out[ti] += LB @ sl                                    # B's basis at the targets
    nL = 1 << lf
    out += _near(mat, xt, np.asarray(tseg), cell_of(xt, origin, H, lf), ys, qs,
                 np.asarray(sseg), cell_of(ys, origin, H, lf), nL)
    return out
