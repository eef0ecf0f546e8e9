"""FP64 CPU oracle for the Lagrange-FMM dislocation stress path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_1712_07739_gb300``)
and never imports it; both take their inputs from
``paper_1712_07739_gb300.synth``, which holds no stress arithmetic.

Contents (arXiv:1712.07739):

* ``voigt_to_cijkl``, ``A_tensor``    -- stiffness and the contraction of
  Section 2, Eq. "kernel".
* ``h_iso``, ``h_circle``, ``G_circle`` -- Green's-function derivative factor
  h_vpq(T) = R^2 dG_vp/dx_q (Section 2, Eqs. "k_iso" and the unit-circle
  integral used in place of Eq. "k_aniso").
* ``quadrature``                       -- Gauss points y and strengths
  q_wr = 1/2 b_w omega S_r (Section 2, Eq. "stress_discrete").
* ``direct_stress``                    -- the N-body sum of Eq. "stress3".
* ``nodal_forces``                     -- Peach-Koehler force f = (sigma.b) x xi
  (Section 2) integrated with linear shape functions at the segment ends.
* ``oracle_b``                         -- the Lagrange FMM result by its
  definition (Algorithms 1 and 2): near sum plus, for every level and every
  interaction-list pair, anterpolation / node kernel / interpolation.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, textbook fields, invariants or brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lib = None

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def build(force=False):
    """Compile oracle.c with gcc (-O2, OpenMP) into oracle/_lib/liboracle.so."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.POINTER(ctypes.c_int64)
        L.orc_A_tensor.argtypes = [d, d]
        L.orc_h_iso.argtypes = [ctypes.c_double, ctypes.c_double, d, d]
        L.orc_G_circle_rot.argtypes = [d, d, ctypes.c_int, ctypes.c_double, d]
        L.orc_h_circle_rot.argtypes = [d, d, ctypes.c_int, ctypes.c_double, d]
        L.orc_kernel_batch.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, d, ctypes.c_int, d,
                                       ctypes.c_int64, d, d, ctypes.c_int]
        L.orc_direct_stress.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, d, ctypes.c_int, d,
                                        ctypes.c_int64, d, i64, ctypes.c_int64, d, d, i64, d, ctypes.c_int]
        L.orc_direct_stress.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pi(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _c(a, dt=np.float64):
    return np.ascontiguousarray(a, dtype=dt)


# --------------------------------------------------------------------------
# Material
# --------------------------------------------------------------------------

def voigt_to_cijkl(C6):
    """6x6 Voigt stiffness -> C[i,j,k,l] (Voigt order 11,22,33,23,13,12)."""
    C6 = np.asarray(C6, dtype=np.float64)
    idx = {}
    for a, (i, j) in enumerate(VOIGT):
        idx[(i, j)] = a
        idx[(j, i)] = a
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = C6[idx[(i, j)], idx[(k, l)]]
    return C


def A_tensor(C):
    """A[ab, w, r, v, p, q] = sum_{n,g} eps_ngr C_abvg C_pqwn (Eq. "kernel")."""
    A = np.zeros(6 * 9 * 27)
    lib().orc_A_tensor(_p(_c(C)), _p(A))
    return A.reshape(6, 3, 3, 3, 3, 3)


class Material:
    """Kernel evaluation settings.

    ``Material.iso(mu, nu)`` uses the closed-form isotropic h.
    ``Material.aniso(C6, Q)`` uses the unit-circle integral with Q points on
    the half circle; ``Q=None`` picks it with ``choose_Q``.
    """

    def __init__(self, mode, C, mu=0.0, nu=0.0, Q=0):
        self.mode, self.mu, self.nu, self.Q = mode, float(mu), float(nu), int(Q)
        self.C = _c(C)
        self.A = _c(A_tensor(self.C).reshape(54, 27))

    @classmethod
    def iso(cls, mu=1.0, nu=0.3):
        lam = 2 * mu * nu / (1 - 2 * nu)
        C6 = np.zeros((6, 6))
        C6[:3, :3] = lam
        for i in range(3):
            C6[i, i] = lam + 2 * mu
            C6[3 + i, 3 + i] = mu
        return cls(0, voigt_to_cijkl(C6), mu, nu)

    @classmethod
    def aniso(cls, C6, Q=None):
        C = voigt_to_cijkl(C6)
        if Q is None:
            Q = choose_Q(C)
        return cls(1, C, Q=Q)

    def _args(self):
        return (self.mode, self.mu, self.nu, _p(self.C), self.Q, _p(self.A))


def h_iso(T, mu=1.0, nu=0.3):
    T = _c(np.asarray(T, dtype=np.float64) / np.linalg.norm(T))
    h = np.zeros(27)
    lib().orc_h_iso(mu, nu, _p(T), _p(h))
    return h.reshape(3, 3, 3)


def h_circle(C, T, Q, rot=0.0):
    h = np.zeros(27)
    lib().orc_h_circle_rot(_p(_c(C)), _p(_c(T)), int(Q), float(rot), _p(h))
    return h.reshape(3, 3, 3)


def G_circle(C, x, Q, rot=0.0):
    G = np.zeros(9)
    lib().orc_G_circle_rot(_p(_c(C)), _p(_c(x)), int(Q), float(rot), _p(G))
    return G.reshape(3, 3)


def choose_Q(C, n_dirs=200, seed=12345, tol=1e-14, q0=8, qmax=1024):
    """Smallest Q (doubling from q0) whose doubling changes max|h| by < tol*max|h|
    over seeded directions; the trapezoid sum is spectrally convergent for a
    periodic analytic integrand."""
    rng = np.random.default_rng(seed)
    dirs = rng.normal(size=(n_dirs, 3))
    Q = q0
    prev = np.array([h_circle(C, t, Q) for t in dirs])
    while Q < qmax:
        cur = np.array([h_circle(C, t, 2 * Q) for t in dirs])
        if np.max(np.abs(cur - prev)) < tol * np.max(np.abs(cur)):
            return Q
        Q *= 2
        prev = cur
    return Q


def kernel(mat: Material, d, nthreads=0):
    """K[n, ab, w, r] at separation vectors d[n, 3] (Eq. "kernel")."""
    d = _c(np.atleast_2d(d))
    K = np.zeros((d.shape[0], 54))
    lib().orc_kernel_batch(*mat._args(), d.shape[0], _p(d), _p(K), int(nthreads))
    return K.reshape(-1, 6, 3, 3)


# --------------------------------------------------------------------------
# Discretisation (Eq. "stress_discrete")
# --------------------------------------------------------------------------

def quadrature(nodes, segs, burgers, n_g=4):
    """Gauss points y [N_s*n_g, 3], strengths q [N_s*n_g, 3, 3] and segment ids.

    Point k of segment i is y = (x1+x2)/2 + xi_k (x2-x1)/2 and
    q_wr = 1/2 b_w omega_k S_r with S = x2 - x1 (Gauss-Legendre on [-1, 1],
    numpy's leggauss)."""
    xi, om = np.polynomial.legendre.leggauss(n_g)
    x1 = nodes[segs[:, 0]]
    x2 = nodes[segs[:, 1]]
    S = x2 - x1
    mid = 0.5 * (x1 + x2)
    y = mid[:, None, :] + xi[None, :, None] * 0.5 * S[:, None, :]
    q = 0.5 * burgers[:, None, :, None] * om[None, :, None, None] * S[:, None, None, :]
    segid = np.repeat(np.arange(len(segs), dtype=np.int64), n_g)
    return y.reshape(-1, 3), q.reshape(-1, 3, 3), segid


def direct_stress(mat: Material, xt, tseg, ys, qs, sseg, nthreads=0, return_threads=False):
    """Voigt stress [n_t, 6] by the direct sum of Eq. "stress3", excluding
    source points whose segment id equals the target's (use -1 for free
    targets)."""
    xt, ys = _c(np.atleast_2d(xt)), _c(ys)
    qs = _c(np.asarray(qs).reshape(-1, 9))
    tseg, sseg = _c(tseg, np.int64), _c(sseg, np.int64)
    out = np.zeros((xt.shape[0], 6))
    used = lib().orc_direct_stress(*mat._args(), xt.shape[0], _p(xt), _pi(tseg),
                                   ys.shape[0], _p(ys), _p(qs), _pi(sseg), _p(out), int(nthreads))
    return (out, used) if return_threads else out


def voigt_to_tensor(s):
    s = np.asarray(s)
    out = np.zeros(s.shape[:-1] + (3, 3))
    for a, (i, j) in enumerate(VOIGT):
        out[..., i, j] = s[..., a]
        out[..., j, i] = s[..., a]
    return out


def segment_forces(nodes, segs, burgers, sigma_pts, n_g=4):
    """Peach-Koehler end forces f1, f2 [N_s, 3] of each segment.

    f = (sigma . b) x xi per unit length (Section 2), integrated against the
    linear shape functions (1-t) and t along the segment with the same Gauss
    rule: f1 = sum_k (omega_k/2) (1-xi_k)/2 (sigma_k b) x S, f2 likewise
    with (1+xi_k)/2."""
    xi, om = np.polynomial.legendre.leggauss(n_g)
    S = nodes[segs[:, 1]] - nodes[segs[:, 0]]
    sig = voigt_to_tensor(np.asarray(sigma_pts).reshape(len(segs), n_g, 6))
    sb = np.einsum("skij,sj->ski", sig, burgers)
    pk = np.cross(sb, S[:, None, :])
    w1 = 0.5 * om * 0.5 * (1 - xi)
    w2 = 0.5 * om * 0.5 * (1 + xi)
    f1 = np.einsum("k,ski->si", w1, pk)
    f2 = np.einsum("k,ski->si", w2, pk)
    return f1, f2


def nodal_forces(nodes, segs, burgers, sigma_pts, n_g=4):
    """Node forces [n_nodes, 3]: sum of incident segments' end forces."""
    f1, f2 = segment_forces(nodes, segs, burgers, sigma_pts, n_g)
    F = np.zeros((len(nodes), 3))
    np.add.at(F, segs[:, 0], f1)
    np.add.at(F, segs[:, 1], f2)
    return F


def network_stress(mat, nodes, segs, burgers, n_g=4, nthreads=0):
    """Stress at every Gauss point of the network, direct sum."""
    y, q, sid = quadrature(nodes, segs, burgers, n_g)
    return direct_stress(mat, y, sid, y, q, sid, nthreads)


def network_forces(mat, nodes, segs, burgers, n_g=4, nthreads=0):
    sig = network_stress(mat, nodes, segs, burgers, n_g, nthreads)
    return nodal_forces(nodes, segs, burgers, sig, n_g), sig


def sampled_node_forces(mat, nodes, segs, burgers, node_ids, n_g=4, nthreads=0):
    """Forces at selected nodes only: the stress is evaluated by direct sum at
    the Gauss points of the segments incident to those nodes, against all
    sources.  Returns (forces [len(node_ids), 3], threads used)."""
    node_ids = np.asarray(node_ids, dtype=np.int64)
    inc = np.nonzero(np.isin(segs[:, 0], node_ids) | np.isin(segs[:, 1], node_ids))[0]
    y, q, sid = quadrature(nodes, segs, burgers, n_g)
    tgt = (inc[:, None] * n_g + np.arange(n_g)[None, :]).reshape(-1)
    sig, used = direct_stress(mat, y[tgt], sid[tgt], y, q, sid, nthreads, return_threads=True)
    f1, f2 = segment_forces(nodes, segs[inc], burgers[inc], sig, n_g)
    F = np.zeros((len(nodes), 3))
    np.add.at(F, segs[inc, 0], f1)
    np.add.at(F, segs[inc, 1], f2)
    return F[node_ids], used


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
