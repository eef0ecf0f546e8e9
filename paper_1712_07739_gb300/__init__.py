"""gbfmm: Lagrange FMM for dislocation stresses and Peach-Koehler forces on GB300.

Thin ctypes binding over the C ABI declared in ``include/gbfmm.h``.  Every
step of the pass runs in the library's CUDA kernels; this module only
marshals torch CUDA tensors (for device memory) and the current torch CUDA
stream.  Importing it does not need a GPU; constructing ``FMM`` loads the
compiled library and raises if it is missing -- there is no CPU fallback.

Method: Chen, Aubry, Oppelstrup, Arsenlis, Darve, arXiv:1712.07739
(Sec. 2 for the stress formula and kernel, Sec. 4 / Algorithm 2 for the pass).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgbfmm.so")

FP64, MIXED, MIXED_F64T = 0, 1, 2  # gbfmm_options.precision
H_ISO, H_CIRCLE, H_MLP = 0, 1, 2
_PREC = {"fp64": FP64, "mixed": MIXED, "mixed_f64t": MIXED_F64T}
_HMODE = {"iso": H_ISO, "circle": H_CIRCLE, "mlp": H_MLP}

# exported names the header declares (checked by the CPU test suite)
EXPORTS = [
    "fmm_default_options", "fmm_create", "fmm_destroy", "fmm_last_error",
    "fmm_set_material", "fmm_build_tree", "fmm_eval_stress", "fmm_eval_nodal_forces",
    "fmm_tree_info", "fmm_m2l_ranks", "fmm_set_timing", "fmm_stage_times", "fmm_launch_count", "fmm_work_counts",
    "fmm_device_status", "fmm_inject_fault", "fmm_probe_fma",
    "fmm_mlp_train", "fmm_mlp_get", "fmm_mlp_set", "fmm_mlp_eval", "fmm_mlp_grad", "fmm_mlp_labels",
    "fmm_mlp_eval_noalloc", "fmm_mlp_calibrate",
    "fmm_batch_create", "fmm_batch_destroy", "fmm_batch_last_error", "fmm_batch_set_material", "fmm_batch_build",
    "fmm_batch_eval_nodal_forces", "fmm_batch_info", "fmm_batch_step", "fmm_batch_status", "fmm_batch_tuning",
]
MLP_PARAMS = 37664


class Options(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int), ("n_gauss", ctypes.c_int), ("levels", ctypes.c_int),
        ("precision", ctypes.c_int), ("h_mode", ctypes.c_int), ("circle_q", ctypes.c_int),
        ("leaf_segments", ctypes.c_int), ("near_fp64", ctypes.c_double), ("m2l_split", ctypes.c_int),
        ("mlp_min_dist", ctypes.c_double), ("m2l_fft", ctypes.c_int), ("m2l_chunks", ctypes.c_int),
        ("m2l_basis", ctypes.c_int), ("m2l_split_levels", ctypes.c_int), ("m2l_split_kblocks", ctypes.c_int),
        ("m2l_kernel", ctypes.c_int), ("nodes", ctypes.c_int), ("m2l_svd_tol", ctypes.c_double),
        ("refine_points", ctypes.c_int), ("m2l_symmetry", ctypes.c_int),
    ]


class GbfmmError(RuntimeError):
    pass


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgbfmm.so (built by ``build.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise GbfmmError(f"CUDA library not built: {path} (run paper_1712_07739_gb300.build.build())")
    L = ctypes.CDLL(path)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
    L.fmm_default_options.argtypes = [ctypes.POINTER(Options)]
    L.fmm_default_options.restype = None
    L.fmm_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options), vp]
    L.fmm_destroy.argtypes = [vp]
    L.fmm_destroy.restype = None
    L.fmm_last_error.argtypes = [vp]
    L.fmm_last_error.restype = ctypes.c_char_p
    L.fmm_set_material.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fmm_build_tree.argtypes = [vp, i64, dp, i64, dp, dp]
    L.fmm_eval_stress.argtypes = [vp, i64, dp, dp]
    L.fmm_eval_nodal_forces.argtypes = [vp, dp, dp, dp]
    L.fmm_tree_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.fmm_m2l_ranks.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.fmm_set_timing.argtypes = [vp, ctypes.c_int]
    L.fmm_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fmm_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
    L.fmm_work_counts.argtypes = [vp, ctypes.POINTER(i64)]
    L.fmm_device_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.fmm_inject_fault.argtypes = [vp, ctypes.c_int]
    L.fmm_probe_fma.argtypes = [ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]
    L.fmm_probe_fma.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    L.fmm_mlp_train.argtypes = [vp, i64, dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint64, fp]
    L.fmm_mlp_get.argtypes = [vp, fp, fp]
    L.fmm_mlp_set.argtypes = [vp, fp, fp]
    L.fmm_mlp_eval.argtypes = [vp, i64, dp, dp]
    L.fmm_mlp_grad.argtypes = [vp, ctypes.c_int, dp, dp, dp, fp]
    L.fmm_mlp_labels.argtypes = [vp, i64, dp, dp]
    L.fmm_mlp_eval_noalloc.argtypes = [vp, i64, dp, dp]
    L.fmm_mlp_calibrate.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.fmm_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Options), ctypes.c_int, vp]
    L.fmm_batch_destroy.argtypes = [vp]
    L.fmm_batch_destroy.restype = None
    L.fmm_batch_last_error.argtypes = [vp]
    L.fmm_batch_last_error.restype = ctypes.c_char_p
    L.fmm_batch_set_material.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.fmm_batch_build.argtypes = [vp, ctypes.c_int, i64, dp, i64, dp, dp]
    L.fmm_batch_eval_nodal_forces.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p)]
    L.fmm_batch_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.fmm_batch_step.argtypes = [vp, ctypes.POINTER(ctypes.c_void_p)]
    L.fmm_batch_status.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.fmm_batch_tuning.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    for name in ("fmm_batch_create", "fmm_batch_set_material", "fmm_batch_build", "fmm_batch_eval_nodal_forces",
                 "fmm_batch_info", "fmm_batch_step", "fmm_batch_status", "fmm_batch_tuning"):
        getattr(L, name).restype = ctypes.c_int
    for name in ("fmm_mlp_calibrate", "fmm_mlp_eval_noalloc", "fmm_mlp_train", "fmm_mlp_get", "fmm_mlp_set", "fmm_mlp_eval", "fmm_mlp_grad", "fmm_mlp_labels",
                 "fmm_inject_fault", "fmm_device_status", "fmm_launch_count", "fmm_work_counts", "fmm_create", "fmm_set_material", "fmm_build_tree", "fmm_eval_stress",
                 "fmm_eval_nodal_forces", "fmm_tree_info", "fmm_m2l_ranks", "fmm_set_timing", "fmm_stage_times"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def probe_fma(kind, stream=None):
    """Measured FMA throughput of the current device in TFLOP/s: kind "fp32",
    "fp32x2" (packed pairs) or "fp64" (self-checking chains, ~0.5 s)."""
    import torch

    lib = load_library()
    k = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    st = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double()
    rc = lib.fmm_probe_fma(k, ctypes.c_void_p(st.cuda_stream), ctypes.byref(v))
    if rc != 0:
        raise GbfmmError(f"fmm_probe_fma({kind}) failed ({rc})")
    return v.value


_NODES = {"equispaced": 0, "chebyshev": 1}


def _set_nodes_svd(o, nodes, m2l_svd_tol, refine_points=None):
    if refine_points is not None:
        o.refine_points = int(refine_points)
    if nodes is not None:
        o.nodes = _NODES[nodes] if isinstance(nodes, str) else int(nodes)
    if m2l_svd_tol is not None:
        o.m2l_svd_tol = float(m2l_svd_tol)


class FMM:
    """One Lagrange-FMM context on the current CUDA device and stream.

    ``FMM(p=4).set_material(C).build(nodes, segs, b).nodal_forces()``; inputs
    are torch CUDA tensors: nodes float64 [n, 3], segs int64 [m, 2],
    burgers float64 [m, 3].  The context keeps references to them.
    """

    def __init__(self, p=4, n_gauss=4, levels=0, precision="fp64", h_mode="iso", circle_q=0,
                 leaf_segments=0, near_fp64=0.0, m2l_split=None, mlp_min_dist=0.0, m2l_fft=None, m2l_chunks=None,
                 m2l_basis=None, m2l_split_levels=None, m2l_split_kblocks=None, m2l_kernel=None, nodes=None,
                 m2l_svd_tol=None, refine_points=None, m2l_symmetry=None, stream=None):
        import torch

        self._torch = torch
        self._lib = load_library()
        o = Options()
        self._lib.fmm_default_options(ctypes.byref(o))
        _set_nodes_svd(o, nodes, m2l_svd_tol, refine_points)
        if m2l_symmetry is not None:
            o.m2l_symmetry = int(m2l_symmetry)
        o.p, o.n_gauss, o.levels = p, n_gauss, levels
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.h_mode = _HMODE[h_mode] if isinstance(h_mode, str) else int(h_mode)
        o.circle_q, o.leaf_segments, o.near_fp64 = circle_q, leaf_segments, near_fp64
        if m2l_split is not None:
            o.m2l_split = int(m2l_split)
        o.mlp_min_dist = mlp_min_dist
        if m2l_fft is not None:
            o.m2l_fft = int(m2l_fft)
        if m2l_chunks is not None:
            o.m2l_chunks = int(m2l_chunks)
        if m2l_basis is not None:
            o.m2l_basis = int(m2l_basis)
        if m2l_split_levels is not None:
            o.m2l_split_levels = int(m2l_split_levels)
        if m2l_split_kblocks is not None:
            o.m2l_split_kblocks = int(m2l_split_kblocks)
        if m2l_kernel is not None:
            o.m2l_kernel = int(m2l_kernel)
        self.options = o
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self._lib.fmm_create(ctypes.byref(h), ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise GbfmmError(f"fmm_create failed ({rc})")
        self._h = h
        self._keep = ()
        self.n_nodes = self.n_segs = 0

    def _check(self, rc, what):
        if rc != 0:
            msg = self._lib.fmm_last_error(self._h).decode()
            raise GbfmmError(f"{what} failed ({rc}): {msg}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_material(self, C_voigt):
        C = np.ascontiguousarray(np.asarray(C_voigt, dtype=np.float64).reshape(36))
        self._check(self._lib.fmm_set_material(self._h, C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "fmm_set_material")
        return self

    def build(self, nodes, segs, burgers):
        t = self._torch
        nodes = nodes.to(dtype=t.float64).contiguous()
        segs = segs.to(dtype=t.int64).contiguous()
        burgers = burgers.to(dtype=t.float64).contiguous()
        for x in (nodes, segs, burgers):
            if not x.is_cuda:
                raise GbfmmError("build: inputs must be CUDA tensors")
        self._keep = (nodes, segs, burgers)
        self.n_nodes, self.n_segs = nodes.shape[0], segs.shape[0]
        self._check(self._lib.fmm_build_tree(self._h, nodes.shape[0], _ptr(nodes), segs.shape[0], _ptr(segs),
                                             _ptr(burgers)), "fmm_build_tree")
        return self

    def nodal_forces(self, out=None, f_seg=None, sigma_pts=None):
        t = self._torch
        if out is None:
            dev = self._keep[0].device if self._keep else t.device("cuda", t.cuda.current_device())
            out = t.empty((max(self.n_nodes, 0), 3), dtype=t.float64, device=dev)
        self._check(self._lib.fmm_eval_nodal_forces(self._h, _ptr(out), _ptr(f_seg), _ptr(sigma_pts)),
                    "fmm_eval_nodal_forces")
        return out

    def stress(self, x, out=None):
        t = self._torch
        x = x.to(dtype=t.float64).contiguous()
        if out is None:
            out = t.empty((x.shape[0], 6), dtype=t.float64, device=x.device)
        self._check(self._lib.fmm_eval_stress(self._h, x.shape[0], _ptr(x), _ptr(out)), "fmm_eval_stress")
        return out

    def tree_info(self):
        lv, nl, npt = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.fmm_tree_info(self._h, ctypes.byref(lv), ctypes.byref(nl), ctypes.byref(npt)),
                    "fmm_tree_info")
        return {"levels": lv.value, "n_leaves": nl.value, "n_points": npt.value}

    def m2l_ranks(self):
        """Compressed M2L: coefficients per cell as run and above the tolerance, and the
        largest / smallest kept singular values (zeros when not compressed)."""
        r, sg = (ctypes.c_int * 4)(), (ctypes.c_double * 4)()
        self._check(self._lib.fmm_m2l_ranks(self._h, r, sg), "fmm_m2l_ranks")
        return {"r1": r[0], "r2": r[1], "r1_raw": r[2], "r2_raw": r[3], "sigma": list(sg)}

    def launch_count(self):
        c = ctypes.c_int64()
        self._check(self._lib.fmm_launch_count(self._h, ctypes.byref(c)), "fmm_launch_count")
        return c.value

    def work_counts(self):
        """near point pairs, M2L cell pairs, occupied leaves, points (synchronises)."""
        a = (ctypes.c_int64 * 4)()
        self._check(self._lib.fmm_work_counts(self._h, a), "fmm_work_counts")
        return {"near_pairs": a[0], "m2l_pairs": a[1], "occupied_leaves": a[2], "points": a[3]}

    def device_status(self):
        """0, or GBFMM_ERR_TIMEOUT (-5) if a bounded device wait gave up (synchronises, clears)."""
        v = ctypes.c_int()
        self._check(self._lib.fmm_device_status(self._h, ctypes.byref(v)), "fmm_device_status")
        return v.value

    def inject_fault(self, kind=1):
        """Test hook: make the next tensor-core M2L's bounded wait run out."""
        self._check(self._lib.fmm_inject_fault(self._h, int(kind)), "fmm_inject_fault")
        return self

    # ---------------------------------------------------------- learned h
    def _f32(self, x):
        return x.to(dtype=self._torch.float32).contiguous()

    def mlp_labels(self, dirs):
        """Plain-evaluator h (27 components) at unit directions [n, 3] (device)."""
        dirs = self._f32(dirs)
        y = self._torch.empty((dirs.shape[0], 27), dtype=self._torch.float32, device=dirs.device)
        self._check(self._lib.fmm_mlp_labels(self._h, dirs.shape[0], _ptr(dirs), _ptr(y)), "fmm_mlp_labels")
        return y

    def mlp_train(self, dirs, epochs=10, batch=4096, lr=2e-3, seed=0):
        """Train the network on the plain evaluator's values at dirs; returns the last batch loss."""
        dirs = self._f32(dirs)
        loss = ctypes.c_float()
        self._check(self._lib.fmm_mlp_train(self._h, dirs.shape[0], _ptr(dirs), int(epochs), int(batch), float(lr),
                                            int(seed), ctypes.byref(loss)), "fmm_mlp_train")
        return loss.value

    def mlp_calibrate(self, bin_tol=2e-2):
        """Flag the angular bins where the network's error exceeds bin_tol x RMS(h);
        returns the flagged fraction."""
        fr = ctypes.c_double()
        self._check(self._lib.fmm_mlp_calibrate(self._h, float(bin_tol), ctypes.byref(fr)), "fmm_mlp_calibrate")
        return fr.value

    def mlp_get(self):
        th = np.zeros(MLP_PARAMS, np.float32)
        sc = np.zeros(27, np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self._lib.fmm_mlp_get(self._h, th.ctypes.data_as(fp), sc.ctypes.data_as(fp)), "fmm_mlp_get")
        return th, sc

    def mlp_set(self, theta, scale):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        sc = np.ascontiguousarray(scale, dtype=np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        self._check(self._lib.fmm_mlp_set(self._h, th.ctypes.data_as(fp), sc.ctypes.data_as(fp)), "fmm_mlp_set")
        return self

    def mlp_eval(self, dirs):
        dirs = self._f32(dirs)
        h = self._torch.empty((dirs.shape[0], 27), dtype=self._torch.float32, device=dirs.device)
        self._check(self._lib.fmm_mlp_eval(self._h, dirs.shape[0], _ptr(dirs), _ptr(h)), "fmm_mlp_eval")
        return h

    def mlp_eval_noalloc(self, dirs, out):
        """Network h into a caller-provided tensor, with no device allocation
        in the library (scratch is a static device array)."""
        dirs = self._f32(dirs)
        self._check(self._lib.fmm_mlp_eval_noalloc(self._h, dirs.shape[0], _ptr(dirs), _ptr(out)),
                    "fmm_mlp_eval_noalloc")
        return out

    def mlp_grad(self, dirs, y):
        dirs, y = self._f32(dirs), self._f32(y)
        g = self._torch.empty(MLP_PARAMS, dtype=self._torch.float32, device=dirs.device)
        loss = ctypes.c_float()
        self._check(self._lib.fmm_mlp_grad(self._h, dirs.shape[0], _ptr(dirs), _ptr(y), _ptr(g),
                                           ctypes.byref(loss)), "fmm_mlp_grad")
        return g, loss.value

    def set_timing(self, on=True):
        self._check(self._lib.fmm_set_timing(self._h, int(bool(on))), "fmm_set_timing")
        return self

    def stage_times(self):
        a = (ctypes.c_double * 8)()
        self._check(self._lib.fmm_stage_times(self._h, a), "fmm_stage_times")
        return list(a)


class Batch:
    """Independent segment networks evaluated together (shared medium tables,
    autotuned depth per network with levels=0, graph-recorded evaluation)."""

    def __init__(self, n_configs, p=6, n_gauss=4, levels=0, precision="mixed", h_mode="circle", circle_q=0,
                 leaf_segments=0, near_fp64=0.0, m2l_split=None, m2l_basis=None, m2l_chunks=None,
                 m2l_split_levels=None, m2l_split_kblocks=None, m2l_kernel=None, nodes=None, m2l_svd_tol=None,
                 stream=None):
        import torch

        self._torch = torch
        self._lib = load_library()
        o = Options()
        self._lib.fmm_default_options(ctypes.byref(o))
        _set_nodes_svd(o, nodes, m2l_svd_tol)
        o.p, o.n_gauss, o.levels = p, n_gauss, levels
        o.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
        o.h_mode = _HMODE[h_mode] if isinstance(h_mode, str) else int(h_mode)
        o.circle_q, o.leaf_segments, o.near_fp64 = circle_q, leaf_segments, near_fp64
        for name, v in (("m2l_split", m2l_split), ("m2l_basis", m2l_basis), ("m2l_chunks", m2l_chunks), ("m2l_split_levels", m2l_split_levels),
                        ("m2l_split_kblocks", m2l_split_kblocks), ("m2l_kernel", m2l_kernel)):
            if v is not None:
                setattr(o, name, int(v))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self._lib.fmm_batch_create(ctypes.byref(h), ctypes.byref(o), int(n_configs),
                                        ctypes.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise GbfmmError(f"fmm_batch_create failed ({rc})")
        self._h = h
        self.n = int(n_configs)
        self._keep = [None] * self.n
        self._out = [None] * self.n

    def _check(self, rc, what):
        if rc != 0:
            raise GbfmmError(f"{what} failed ({rc}): {self._lib.fmm_batch_last_error(self._h).decode()}")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_material(self, C_voigt):
        C = np.ascontiguousarray(np.asarray(C_voigt, dtype=np.float64).reshape(36))
        self._check(self._lib.fmm_batch_set_material(self._h, C.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
                    "fmm_batch_set_material")
        return self

    def build(self, k, nodes, segs, burgers):
        t = self._torch
        nodes = nodes.to(dtype=t.float64).contiguous()
        segs = segs.to(dtype=t.int64).contiguous()
        burgers = burgers.to(dtype=t.float64).contiguous()
        self._keep[k] = (nodes, segs, burgers)
        if self._out[k] is None or self._out[k].shape[0] != nodes.shape[0]:
            self._out[k] = t.empty((nodes.shape[0], 3), dtype=t.float64, device=nodes.device)
        self._check(self._lib.fmm_batch_build(self._h, int(k), nodes.shape[0], _ptr(nodes), segs.shape[0],
                                              _ptr(segs), _ptr(burgers)), "fmm_batch_build")
        return self

    def nodes(self, k):
        """Network k's node array as the library reads it (the tensor given to
        build, or its float64 copy): move nodes in place, then call step()."""
        return self._keep[k][0]

    def nodal_forces(self):
        """Evaluate every network; returns the list of [n_nodes_k, 3] tensors (reused between calls)."""
        arr = (ctypes.c_void_p * self.n)(*[o.data_ptr() for o in self._out])
        self._check(self._lib.fmm_batch_eval_nodal_forces(self._h, arr), "fmm_batch_eval_nodal_forces")
        return self._out

    def step(self):
        """Rebuild every network from its current node positions and evaluate all
        of them as one graph replay (the inputs' sizes and addresses must be the
        ones of the last build); returns the list of force tensors."""
        arr = (ctypes.c_void_p * self.n)(*[o.data_ptr() for o in self._out])
        self._check(self._lib.fmm_batch_step(self._h, arr), "fmm_batch_step")
        return self._out

    def status(self):
        """(slot, code) of the first network whose last build or pass reported a
        problem, or (-1, 0) (synchronises)."""
        k, c = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.fmm_batch_status(self._h, ctypes.byref(k), ctypes.byref(c)), "fmm_batch_status")
        return k.value, c.value

    def tuning(self):
        """M2L tile form in use and, when the autotuner chose it, each form's M2L
        time on the calibration network (ms)."""
        form, ms = ctypes.c_int(), (ctypes.c_double * 2)()
        self._check(self._lib.fmm_batch_tuning(self._h, ctypes.byref(form), ms), "fmm_batch_tuning")
        return {"m2l_kernel": form.value, "m2l_ms": [ms[0], ms[1]]}

    def info(self, k):
        lv, la = ctypes.c_int(), ctypes.c_int64()
        cn, cf = ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.fmm_batch_info(self._h, int(k), ctypes.byref(lv), ctypes.byref(la), ctypes.byref(cn),
                                             ctypes.byref(cf)), "fmm_batch_info")
        return {"levels": lv.value, "launches": la.value, "c_near": cn.value, "c_far": cf.value}
