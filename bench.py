"""Benchmark: Lagrange-FMM segment nodal forces per second on one GB300.

A step is one pass of the whole hot path over one synthetic network:
Gauss points + tree build (fmm_build_tree) and the FMM evaluation of
Peach-Koehler nodal forces (fmm_eval_nodal_forces: P2M, M2M, M2L, L2L,
L2P + near field, forces).  The M2L operators (per medium and order) are
built once before timing, as the method prescribes (they do not depend on
the configuration).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...     # the FP64 CPU oracle, sampled

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1712_07739_gb300 import synth  # noqa: E402

METRIC = "FMM segment nodal forces/sec at 1e-4 rel err: mixed+learned vs plain FP64, 1 GB300"
UNIT = "segments/s"

# per-pair arithmetic of the near field (counted from the kernel source, FMA = 2):
# FP64 path, isotropic: separation 3, |d|^2 5, rsqrt 1, direction 3, h (18
#   components) ~100, contraction with the 6x18 source tensor 216, scale and
#   accumulate 13 -> 341
# mixed path, isotropic polynomial form: separation 3, |d|^2 5, rsqrt 1,
#   1/R^3 and 1/R^5 3, cubic monomials 16, per stress component 3 linear +
#   10 cubic FMAs and 2 scaled adds (29) x 6 -> 202
# unit-circle h in a cubic medium with axes along x, y, z (the specialised
#   form both paths use): separation, |d|^2, rsqrt, direction and circle basis
#   41; per circle point 193 (point 9, zz 15, adjugate 18, determinant and
#   reciprocal 6, zT 18, U = adj zT 45, F = U adj 30, 1/det^2 into z 4,
#   accumulate z F 36, sum of (zz)^-1 12); final T-term and scale 36;
#   contraction with the 6x18 source tensor and 1/R^2 223; accumulate 6
#   -> 193 Q + 306
# unit-circle h, general medium: Q x (zz and zT from the 81-entry C 2 x 81
#   FMA, inverse 30, F 54, accumulate 36, point 6) ~ Q x 450, plus 236
FLOP_PER_NEAR_PAIR = {("fp64", "iso"): 341, ("mixed", "iso"): 202}


def is_cubic_aligned(C6):
    """Cubic symmetry with the crystal axes along x, y, z (Voigt 6x6)."""
    C = np.asarray(C6, dtype=np.float64).reshape(6, 6)
    off = C.copy()
    for i in range(3):
        off[i, :3] = 0.0
        off[3 + i, 3 + i] = 0.0
    return (np.allclose(np.diag(C)[:3], C[0, 0]) and np.allclose(np.diag(C)[3:], C[3, 3])
            and np.allclose([C[0, 1], C[0, 2], C[1, 2]], C[0, 1]) and np.allclose(C[:3, :3], C[:3, :3].T)
            and not np.any(off))


def near_pair_flops(precision, h_mode, q, cubic=False):
    """FLOP per ordered near pair of the one-sided evaluation."""
    if h_mode == "iso":
        return FLOP_PER_NEAR_PAIR[(precision, h_mode)]
    return 193 * q + 306 if cubic else 450 * q + 236


def near_flops(wl, work):
    """Algorithmic FLOP of the near field (+ L2P) of one pass and the kernel
    that does it.  With the unit-circle h both passes evaluate h once per
    unordered pair (h is odd) and contract it for both directions: per
    ordered pair half an h evaluation (cubic rule 193 Q + 77, general rule
    450 Q + 20) plus one contraction (229)."""
    p, q = wl["p"], wl.get("circle_q", 64)
    cubic = is_cubic_aligned(wl["C"]())
    l2p = work["points"] * (12 * p ** 3 + 30 * p)
    if wl["h_mode"] == "circle":
        # symmetric kernels (FP32 in the mixed pass, FP64 in the FP64 pass)
        h = 193 * q + 77 if cubic else 450 * q + 20
        name = "k_near_sym64" if wl["precision"] == "fp64" else "k_near_sym"
        return work["near_pairs"] * (h / 2.0 + 229) + l2p, name
    if wl["precision"] == "fp64":
        return work["near_pairs"] * near_pair_flops("fp64", wl["h_mode"], q, cubic) + l2p, "k_leaf_eval_f64"
    name = "k_near_mlp" if wl["h_mode"] == "mlp" else "k_near_mixed"
    return work["near_pairs"] * near_pair_flops("mixed", wl["h_mode"], q, cubic) + l2p, name


# DRAM bytes per target point of one k_near_sym launch (cubic rule, Q = 16), from
# one ncu capture on the 250,000-segment slab network (dram__bytes_read.sum +
# dram__bytes_write.sum = 6.494 + 1.347 GB for 1,000,000 points); valid for the
# kernel version the capture was taken of
NEAR_SYM_DRAM_BYTES_PER_POINT = (6.493849e9 + 1.346746e9) / 1.0e6
# the same two counters for the headline's launch itself (1M segments, adaptive tree at
# threshold 128; a one-pass capture of the full-size run)
NEAR_SYM_ADAPTIVE_1M_DRAM_BYTES = 21815144704 + 4425026816


def measured_alu_peaks():
    """FP32 and FP64 fused multiply-add throughput of this GPU, measured now by
    the library's self-checking probe (fmm_probe_fma, ~0.5 s each): the
    denominators of the near-field and FP64-pass rooflines."""
    import paper_1712_07739_gb300 as gb

    fp32 = max(gb.probe_fma("fp32"), gb.probe_fma("fp32x2"))
    return {"fp32_tflops": fp32, "fp64_tflops": gb.probe_fma("fp64"),
            "source": "fmm_probe_fma on this GPU before the timed region (FMA chains, CUDA events, best of 3), "
                      "of measured"}

WORKLOADS = {
    "c1": dict(
        desc="2,000 segments (50 hexagonal glide loops x 40), isotropic mu=1 nu=0.3, order p=4, 3-level octree, "
             "4 Gauss points/segment, FP64 plain",
        gen=lambda seed: synth.hexagon_loops(seed=seed), C=lambda: synth.isotropic_voigt(1.0, 0.3),
        h_mode="iso", p=4, levels=3, precision="fp64"),
}
# The mixed pass's M2L operands in every mixed workload below: FP16 Legendre moments of
# the source cells, residual (hi + lo) passes on the leading block of low-order moments,
# the offsets summed in 7 runs (the library defaults, spelled out).
MIXED_M2L = dict(m2l_split=6, m2l_basis=1, m2l_chunks=7, m2l_split_kblocks=1)
WORKLOADS["c2"] = dict(
    desc="50,000 segments (1,000 polygonal loops of 10-80 segments, log-uniform radii 0.005-0.05, seed 1), cubic "
         "C11=1.684 C12=1.214 C44=0.754, plain FP64 pass (M2L through transforms, symmetric FP64 near field), "
         "order p=5, 5-level octree, unit-circle h Q=32",
    gen=lambda seed: synth.polygon_loops(seed=1 + 1000 * seed), C=lambda: synth.cubic_voigt(),
    h_mode="circle", circle_q=32, p=5, levels=5, precision="fp64")
# The compressed M2L of the headline: Chebyshev nodes, singular vectors kept above 5e-5 of
# the largest (the paper's Chebyshev FMM), FP16 operands with residual passes on the
# leading block of 64 singular directions, offsets summed in 3 runs.
CHEB_M2L = dict(nodes="chebyshev", m2l_svd_tol=5e-5, m2l_split=6, m2l_chunks=3, m2l_split_kblocks=1)
WORKLOADS["c3"] = dict(
    desc="1,000,000 segments (20,000 loops x 50 in 32 Gaussian slabs, sigma 0.02), cubic C11=1.684 C12=1.214 "
         "C44=0.754, order p=7 on Chebyshev nodes, adaptive octree: 7 levels with every leaf holding more than 128 "
         "Gauss points split once more (children of two split leaves that are not adjacent interact by an M2L one "
         "level down, adjacent ones directly), mixed precision (SVD-compressed M2L on the tensor cores: FP16 "
         "operands, residual passes on the leading singular directions; FP32 near field with FP64 separations for "
         "close pairs), unit-circle h (cubic form, Q=16 points on the half circle); the same step through the "
         "plain FP64 pass (uniform 7-level tree) is timed in the same run",
    gen=lambda seed: synth.slab_loops(seed=2 + 1000 * seed), C=lambda: synth.cubic_voigt(),
    h_mode="circle", circle_q=16, p=7, levels=7, precision="mixed", refine_points=128, fp64_arm=True, **CHEB_M2L)
WORKLOADS["c3u"] = dict(
    desc="c3 on the uniform 7-level octree (no leaf split)",
    gen=WORKLOADS["c3"]["gen"], C=WORKLOADS["c3"]["C"], h_mode="circle", circle_q=16, p=7, levels=7,
    precision="mixed", **CHEB_M2L)
WORKLOADS["c3legendre"] = dict(
    desc="c3 on equispaced nodes with the dense M2L (every one of the 54 p^6 products per cell pair, on FP16 "
         "Legendre moments of the source cells with residual passes on the low-order moments)",
    gen=WORKLOADS["c3"]["gen"], C=WORKLOADS["c3"]["C"], h_mode="circle", circle_q=16, p=7, levels=7,
    precision="mixed", **MIXED_M2L)
WORKLOADS["c3svd"] = dict(
    desc="c3 on equispaced nodes with the SVD-compressed M2L (singular vectors kept above 1e-5 of the largest)",
    gen=WORKLOADS["c3"]["gen"], C=WORKLOADS["c3"]["C"], h_mode="circle", circle_q=16, p=7, levels=7,
    precision="mixed", m2l_svd_tol=1e-5, m2l_split=6, m2l_chunks=7, m2l_split_kblocks=1)
WORKLOADS["c3_iso"] = dict(
    desc="1,000,000 segments (20,000 loops x 50 in 32 Gaussian slabs), isotropic mu=1 nu=0.3, p=7, mixed precision",
    gen=lambda seed: synth.slab_loops(seed=2 + 1000 * seed), C=lambda: synth.isotropic_voigt(1.0, 0.3),
    h_mode="iso", p=7, levels=7, precision="mixed", **MIXED_M2L)
WORKLOADS["c3q"] = dict(
    desc="profiling case: 250,000 segments (5,000 loops x 50 in 32 Gaussian slabs), cubic, p=7, mixed, 6-level octree",
    gen=lambda seed: synth.slab_loops(n_loops=5000, seed=2 + 1000 * seed), C=lambda: synth.cubic_voigt(),
    h_mode="circle", circle_q=20, p=7, levels=6, precision="mixed", **MIXED_M2L)
WORKLOADS["c3q_cheb"] = dict(
    desc="profiling case of the headline's kernels: 250,000 segments (5,000 loops x 50 in 32 Gaussian slabs), "
         "cubic, p=7 on Chebyshev nodes with the compressed M2L as c3, unit-circle Q=16, 6-level octree",
    gen=WORKLOADS["c3q"]["gen"], C=lambda: synth.cubic_voigt(), h_mode="circle", circle_q=16, p=7, levels=6,
    precision="mixed", **CHEB_M2L)
WORKLOADS["c3_mlp"] = dict(
    desc="c3 network with the learned angular factor in the near field (pairs beyond 8 segment lengths in bins "
         "the plain evaluator accepted at 2e-2 x RMS(h)), plain cubic rule elsewhere",
    gen=WORKLOADS["c3"]["gen"], C=WORKLOADS["c3"]["C"], h_mode="mlp", circle_q=20, p=7, levels=7,
    precision="mixed", mlp=dict(n_dirs=2_000_000, epochs=12, batch=8192, lr=3e-3, bin_tol=2e-2), **MIXED_M2L)
WORKLOADS["c3_fp64"] = dict(
    desc="the 1,000,000-segment cubic slab network of c3 through the plain FP64 path: FP64 M2L through transforms, "
         "symmetric FP64 near field, unit-circle h (cubic form, Q=20), p=7, 7-level octree",
    gen=WORKLOADS["c3"]["gen"], C=WORKLOADS["c3"]["C"], h_mode="circle", circle_q=20, p=7, levels=7,
    precision="fp64")
WORKLOADS["c3q_iso_fp64"] = dict(
    desc="250,000 segments (5,000 loops x 50 in 32 Gaussian slabs), isotropic mu=1 nu=0.3, plain FP64 path, p=6, "
         "6-level octree (the isotropic near field is cheap, so the step shows the FP64 M2L)",
    gen=WORKLOADS["c3q"]["gen"], C=lambda: synth.isotropic_voigt(1.0, 0.3), h_mode="iso", p=6, levels=6,
    precision="fp64")
WORKLOADS["c5"] = dict(
    desc="64 independent cubic networks, N_s log-uniform in [1e4, 2e5] (4,639,301 segments in all), loop "
         "densities 0.2-5x, mixed precision p=7 (Chebyshev nodes and compressed M2L as c3), unit-circle Q=20, depth per network by "
         "the autotuner (and the M2L tile form), every step's 64 tree builds and passes replayed as one CUDA graph",
    batch=True, gen_batch=lambda seed: synth.ensemble(seed=4 + 1000 * seed), C=lambda: synth.cubic_voigt(),
    h_mode="circle", circle_q=20, p=7, levels=0, precision="mixed", m2l_kernel=2, **CHEB_M2L)
DEFAULT_WORKLOAD = "c3"


def profile_region(args, start):
    """With --profile-region, the timed steps alone are a profiler range
    (ncu --profile-from-start off captures only them, not the medium setup)."""
    if getattr(args, "profile_region", False):
        import torch

        rt = torch.cuda.cudart()
        (rt.cudaProfilerStart if start else rt.cudaProfilerStop)()


def rank_configs(n_configs, world, rank):
    """Configurations of an ensemble handled by one rank (round robin): the
    networks are independent, so ranks exchange nothing but timings."""
    return list(range(rank, n_configs, world))


def global_rate(local_segs, local_ms, group=None):
    """Whole-job throughput: segments of all ranks over the slowest rank's time
    (sum of segments, max of milliseconds across the process group)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return local_segs / (local_ms / 1e3), local_segs, local_ms
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    segs = torch.tensor([float(local_segs)], dtype=torch.float64, device=dev)
    ms = torch.tensor([float(local_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(segs, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(ms, op=dist.ReduceOp.MAX, group=group)
    return float(segs.item()) / (float(ms.item()) / 1e3), float(segs.item()), float(ms.item())


def _rank_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_bf16_peak():
    """Dense 16-bit tensor peak from MEASURED_PEAKS.json: the sustained figure, as
    the M2L runs inside a step of several hundred milliseconds (FP16 and BF16
    have the same nominal dense rate)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return (float(json.load(fh)["bf16_tflops_sustained"]),
                    "MEASURED_PEAKS.json bf16_tflops_sustained (FP16 operands: same nominal rate), of measured")
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback 1.7 PFLOP/s bf16 sustained, of fallback"


def oracle_sample_rate(wl, nodes, segs, b, budget_s, nthreads=0, seed=123):
    """FP64 oracle direct sum (Eq. "stress3") timed on a bounded sample.

    Targets are the Gauss points of randomly drawn segments (at least four
    per host thread: the oracle runs one target per thread), sources a random
    subset of all source points; the work of the direct sum is the same for
    every (target, source) pair, so the full workload's rate is
    pairs/s / (n_g x all source points) segments/s.  The sample grows (sources
    first, then segments) until one evaluation takes about budget_s / 2.
    Returns (segments/s, threads, description, seconds)."""
    import oracle

    C6 = wl["C"]()
    mat = oracle.Material.iso(1.0, 0.3) if wl["h_mode"] == "iso" else oracle.Material.aniso(C6, Q=64)
    y, q, sid = oracle.quadrature(nodes, segs, b, 4)
    n_all = len(y)
    rng = np.random.default_rng(seed)
    threads = nthreads or os.cpu_count() or 1
    n_seg = min(len(segs), threads)
    n_src = min(n_all, 4096)
    while True:
        pick = rng.choice(len(segs), size=n_seg, replace=False)
        tgt = (pick[:, None] * 4 + np.arange(4)[None, :]).reshape(-1)
        src = np.sort(rng.choice(n_all, size=n_src, replace=False)) if n_src < n_all else np.arange(n_all)
        t0 = time.perf_counter()
        sig, used = oracle.direct_stress(mat, y[tgt], sid[tgt], y[src], q[src], sid[src], nthreads,
                                         return_threads=True)
        oracle.segment_forces(nodes, segs[pick], b[pick], sig, 4)
        dt = time.perf_counter() - t0
        done = n_src == n_all and n_seg == len(segs)
        if dt >= 0.5 * budget_s or done:
            rate = len(tgt) * n_src / dt / (4.0 * n_all)
            desc = (f"{n_seg} randomly drawn segments ({len(tgt)} Gauss-point targets) against {n_src} of the "
                    f"{n_all} source points, FP64 direct Mura sum ({'isotropic closed form' if wl['h_mode'] == 'iso' else 'unit circle, Q=64'}), "
                    f"{dt:.1f} s; segments/s = pairs/s / (4 x {n_all})")
            return rate, used, desc, dt
        grow = max(2.0, 0.6 * budget_s / max(dt, 1e-3))
        if n_src < n_all:
            n_src = int(min(n_all, n_src * grow))
        else:
            n_seg = int(min(len(segs), n_seg * grow))


def run_reference(args, wl):
    rank, world, _ = _rank_env()
    if rank != 0:
        return
    nodes, segs, b = wl["gen"](0)
    per_step = max(2.0, 150.0 / (args.steps + args.warmup))
    rates = []
    for i in range(args.warmup + args.steps):
        r, used, desc, dt = oracle_sample_rate(wl, nodes, segs, b, per_step, seed=123 + i)
        if i >= args.warmup:
            rates.append((r, used, desc, dt))
    seg_equiv = sum(r * dt for r, _, _, dt in rates)   # segments of the full workload the samples amount to
    t_tot = sum(x[3] for x in rates)
    value = seg_equiv / t_tot
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / len(rates),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": wl["desc"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": rates[0][1], "kind": "oracle",
                         "sample": "per step: " + rates[0][2]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_batch(args, wl):
    """Batched ensemble: a step builds every network and evaluates all of them."""
    import torch

    import paper_1712_07739_gb300 as gb

    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    nets_all = wl["gen_batch"](0)  # every rank draws the same ensemble and takes its share
    nets = [nets_all[k] for k in rank_configs(len(nets_all), world, rank)]
    n_segs = sum(len(s) for _, s, _ in nets)
    dn = [(torch.tensor(n, device=dev), torch.tensor(s, device=dev), torch.tensor(b, device=dev)) for n, s, b in nets]
    bt = gb.Batch(len(nets), p=wl["p"], levels=wl["levels"], precision=wl["precision"], h_mode=wl["h_mode"],
                  circle_q=wl.get("circle_q", 0), **m2l_options(wl)).set_material(wl["C"]())
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    # first builds outside the timed region: the autotuner picks each network's depth
    # (and the M2L tile form); a step then rebuilds every tree from the resident node
    # arrays and evaluates every network, all of it one graph replay
    for k, (n, s, b) in enumerate(dn):
        bt.build(k, n, s, b)

    def step():
        return bt.step()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    slot, code = bt.status()
    if code != 0:
        raise RuntimeError(f"batched step reported status {code} for network {slot}")
    tuning = bt.tuning()
    depths = [bt.info(k)["levels"] for k in range(len(nets))]
    l0 = bt.info(0)["launches"]
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    profile_region(args, True)
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    profile_region(args, False)
    clk = clocks.stop()
    launches = bt.info(0)["launches"] - l0
    t_ms = sum(a.elapsed_time(b_) for a, b_ in evs)
    value, _, t_ms = global_rate(n_segs * args.steps, t_ms)
    # end to end with host inputs and outputs
    hn = [(torch.tensor(n).pin_memory(), torch.tensor(s).pin_memory(), torch.tensor(b).pin_memory()) for n, s, b in nets]
    e_ms = []
    h2d = sum(x.numel() * 8 for t3 in hn for x in t3)
    d2h = sum(len(n) * 3 * 8 for n, _, _ in nets)
    outs_h = [torch.empty((len(n), 3), dtype=torch.float64).pin_memory() for n, _, _ in nets]
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for (a, b_, c), (x, y, z) in zip(dn, hn):
            a.copy_(x, non_blocking=True)
            b_.copy_(y, non_blocking=True)
            c.copy_(z, non_blocking=True)
        F = step()
        for o, f_ in zip(outs_h, F):
            o.copy_(f_, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e_ms.append(e0.elapsed_time(e1))
    e2e, _, _ = global_rate(n_segs * len(e_ms), sum(e_ms))
    # roofline of the dominant kernel on the largest network, measured alone
    big = int(np.argmax([len(s) for _, s, _ in nets]))
    f = gb.FMM(p=wl["p"], levels=depths[big], precision=wl["precision"], h_mode=wl["h_mode"],
               circle_q=wl.get("circle_q", 0), **dict(m2l_options(wl), m2l_kernel=tuning["m2l_kernel"]))
    f.set_material(wl["C"]())
    f.build(*dn[big])
    out = torch.empty((len(nets[big][0]), 3), dtype=torch.float64, device=dev)
    f.nodal_forces(out=out)
    f.set_timing(True)
    f.nodal_forces(out=out)
    st = f.stage_times()
    work = f.work_counts()
    p = wl["p"]
    if st[4] >= st[2]:
        flops, kname = near_flops(wl, work)
        pk = measured_alu_peaks()
        roof = {"bound": "alu", "kernel": kname + " (largest network alone)", "achieved": flops / (st[4] / 1e3) / 1e12,
                "peak": pk["fp32_tflops"], "unit": "TFLOP/s", "peak_source": pk["source"]}
    else:
        pk, src = measured_bf16_peak()
        flops = work["m2l_pairs"] * 2 * 54 * p ** 6
        roof = {"bound": "tensor", "kernel": "k_m2l_tc (largest network alone)",
                "achieved": flops / (st[2] / 1e3) / 1e12, "peak": pk, "unit": "TFLOP/s", "peak_source": src}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = None
    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f32/fp16", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "n_configs": len(nets_all),
                       "n_segs_rank0": n_segs,
                       "depths": depths, "l2": "flushed: 256 MiB write between steps, outside the step events",
                       "step": "fmm_batch_step: every network's tree build and pass, one CUDA graph replay",
                       "m2l_kernel": tuning["m2l_kernel"], "m2l_ms_by_form": tuning["m2l_ms"]},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "cpu_baseline": None,
        }
        print(json.dumps(res, default=float))
    f.close()
    bt.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_ours(args, wl):
    import torch

    import paper_1712_07739_gb300 as gb

    rank, world, local = _rank_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    nodes, segs, b = wl["gen"](rank)  # weak scaling: each rank its own configuration
    n_segs = len(segs)
    d_nodes = torch.tensor(nodes, device=dev)
    d_segs = torch.tensor(segs, device=dev)
    d_b = torch.tensor(b, device=dev)
    f = gb.FMM(p=wl["p"], levels=args.levels or wl["levels"], precision=wl["precision"], h_mode=wl["h_mode"],
               circle_q=wl.get("circle_q", 0), m2l_fft=None if args.m2l_fft < 0 else args.m2l_fft,
               **m2l_options(wl))
    f.set_material(wl["C"]())
    mlp_info = None
    if wl["h_mode"] == "mlp":
        m = wl["mlp"]
        t_tr = time.perf_counter()
        loss = f.mlp_train(torch.tensor(synth.directions(m["n_dirs"], seed=3), device=dev), epochs=m["epochs"],
                           batch=m["batch"], lr=m["lr"], seed=0)
        frac = f.mlp_calibrate(m["bin_tol"])
        mlp_info = {"train_s": time.perf_counter() - t_tr, "final_loss": loss, "bins_on_plain_rule": frac}
    out = torch.empty((len(nodes), 3), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        f.build(d_nodes, d_segs, d_b)
        f.nodal_forces(out=out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = f.tree_info()
    work = f.work_counts()
    f.set_timing(True)
    launches0 = f.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage = []
    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    profile_region(args, True)
    t0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
        stage.append(f.stage_times())
    torch.cuda.synchronize()
    profile_region(args, False)
    wall = time.perf_counter() - t0
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = f.launch_count() - launches0
    dev_status = f.device_status()  # non-zero: a bounded wait ran out, the pass is invalid
    if dev_status != 0:
        raise RuntimeError(f"device status {dev_status} after the timed steps")
    step_ms = [a.elapsed_time(b_) for a, b_ in evs]
    t_ms = sum(step_ms)
    value, _, t_ms = global_rate(n_segs * args.steps, t_ms)

    # end to end through the public API: pinned host inputs in, forces out
    h_nodes = torch.tensor(nodes).pin_memory()
    h_segs = torch.tensor(segs).pin_memory()
    h_b = torch.tensor(b).pin_memory()
    h_out = torch.empty((len(nodes), 3), dtype=torch.float64).pin_memory()
    f.set_timing(False)
    e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d_nodes.copy_(h_nodes, non_blocking=True)
        d_segs.copy_(h_segs, non_blocking=True)
        d_b.copy_(h_b, non_blocking=True)
        step()
        h_out.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e_ms.append(e0.elapsed_time(e1))
    e2e, _, _ = global_rate(n_segs * len(e_ms), sum(e_ms))
    h2d = h_nodes.numel() * 8 + h_segs.numel() * 8 + h_b.numel() * 8
    d2h = h_out.numel() * 8

    # roofline of the dominant kernel (stage times are CUDA events around it)
    peaks = measured_alu_peaks()
    st = np.array(stage)            # [steps, 8]: precontract, P2M+M2M, M2L, L2L, L2P+P2P, forces
    p = wl["p"]
    ranks = f.m2l_ranks()
    roofline = roofline_of(wl, work, st[:, 2].mean(), st[:, 4].mean(), int(f.options.m2l_fft), peaks, ranks=ranks)
    accuracy = oracle_node_error(wl, args.workload, out.cpu().numpy(), nodes, segs, b)
    f.close()

    fp64_arm = None
    if wl.get("fp64_arm") and not args.no_fp64_arm:
        fp64_arm = run_fp64_arm(wl, args.workload, d_nodes, d_segs, d_b, nodes, segs, b, flush, stream)
        fp64_arm["roofline"] = roofline_of(dict(wl, precision="fp64"), work, fp64_arm["stage_ms"]["m2l"],
                                           fp64_arm["stage_ms"]["l2p_p2p"], 1, peaks)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            r, used, desc, dt = oracle_sample_rate(wl, nodes, segs, b, 20.0)
            cpu = {"value": r, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc}
        fp64 = wl["precision"] == "fp64"
        res = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32/fp16",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"], "n_segs": n_segs, "levels": info["levels"],
                       "p": p, "precision": wl["precision"], "h_mode": wl["h_mode"],
                       "circle_q": wl.get("circle_q", 0), "m2l_split": int(f.options.m2l_split),
                       "m2l_chunks": int(f.options.m2l_chunks), "m2l_basis": int(f.options.m2l_basis),
                       "m2l_split_kblocks": int(f.options.m2l_split_kblocks),
                       "m2l_kernel": int(f.options.m2l_kernel), "m2l_fft": int(f.options.m2l_fft),
                       "nodes": ["equispaced", "chebyshev"][int(f.options.nodes)],
                       "m2l_svd_tol": float(f.options.m2l_svd_tol), "m2l_svd_ranks": ranks,
                       "refine_points": int(f.options.refine_points),
                       "m2l_symmetry": int(f.options.m2l_symmetry),
                       "l2": "flushed: 256 MiB write between steps, outside the step events",
                       "step": "fmm_build_tree + fmm_eval_nodal_forces"},
            "stage_ms": {"precontract": st[:, 0].mean(), "p2m_m2m": st[:, 1].mean(), "m2l": st[:, 2].mean(),
                         "l2l": st[:, 3].mean(), "l2p_p2p": st[:, 4].mean(), "forces": st[:, 5].mean()},
            "work": work, "wall_s": wall,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "device_status": dev_status, "clocks": clk, "roofline": roofline,
            "peaks": peaks, "accuracy": accuracy, "cpu_baseline": cpu,
        }
        if fp64_arm is not None:
            res["fp64_plain"] = fp64_arm
            res["speedup_vs_fp64_plain"] = value / fp64_arm["value"]
        if mlp_info is not None:
            res["learned"] = mlp_info
        print(json.dumps(res, default=float))
    if world > 1:
        torch.distributed.destroy_process_group()


GOLDEN = {"c3": "c3_sampled_forces.json", "c3q": "c3q_sampled_forces.json", "c3_fp64": "c3_sampled_forces.json",
          "c2": "c2_forces.json", "c3svd": "c3_sampled_forces.json", "c3legendre": "c3_sampled_forces.json",
          "c3u": "c3_sampled_forces.json"}


def m2l_options(wl):
    """The tensor-core M2L operand options a workload names (library defaults otherwise)."""
    return {k: wl[k] for k in ("m2l_split", "m2l_basis", "m2l_chunks", "m2l_split_kblocks", "m2l_kernel", "nodes",
                               "m2l_svd_tol", "refine_points", "m2l_symmetry") if k in wl}


def oracle_node_error(wl, name, F, nodes, segs, b):
    """Relative L2 nodal-force error on the nodes whose FP64 oracle forces
    (direct sum of Eq. stress3) are stored under tests/golden (written by the
    scripts there, which call only the oracle); None for other workloads."""
    fn = GOLDEN.get(name)
    if fn is None:
        return None
    with open(os.path.join(ROOT, "tests", "golden", fn)) as fh:
        gold = json.load(fh)
    if "forces_direct" in gold:  # Algorithm-2 forces at many nodes, direct-sum forces at some of them
        ids, Fo = np.array(gold["direct_node_ids"]), np.array(gold["forces_direct"])
    else:
        ids, Fo = np.array(gold["node_ids"]), np.array(gold["forces"])
    # the stored forces belong to exactly this network
    chk = gold["checks"]
    if (gold["n_segs"] != len(segs) or chk["sum_segs"] != int(segs.sum())
            or abs(chk["sum_nodes"] - nodes.sum()) > 1e-9 * abs(nodes.sum())):
        return None
    err = float(np.linalg.norm(F[ids] - Fo) / np.linalg.norm(Fo))
    return {"rel_l2_vs_oracle": err, "nodes": int(len(ids)), "gate": 1e-4, "meets_gate": err <= 1e-4,
            "oracle": f"tests/golden/{fn}: FP64 direct sum, unit-circle h Q={gold.get('Q')}"}


def roofline_of(wl, work, m2l_ms, leaf_ms, m2l_fft, peaks, ranks=None):
    """Roofline of the dominant stage of a pass: near field + L2P (ALU-bound)
    or M2L (tensor-bound on the mixed pass, FP64 ALU on the FP64 pass).  With
    the compressed M2L a cell pair costs 2 r1 r2 (the ranks as run), and the
    stage time includes the two per-cell basis transforms."""
    svd = bool(ranks and ranks.get("r1"))
    p = wl["p"]
    fp64 = wl["precision"] == "fp64"
    alu_peak = peaks["fp64_tflops"] if fp64 else peaks["fp32_tflops"]
    traffic, traffic_src = None, None
    if leaf_ms >= m2l_ms:
        flops, kname = near_flops(wl, work)
        achieved = flops / (leaf_ms / 1e3) / 1e12
        dom, bound, peak, src = kname + " (L2P + near-field P2P)", "alu", alu_peak, peaks["source"]
        if kname == "k_near_sym" and wl.get("circle_q") == 16 and not wl.get("refine_points"):
            traffic = NEAR_SYM_DRAM_BYTES_PER_POINT * work["points"]
            traffic_src = ("dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of k_near_sym on the "
                           "250k-segment slab network, scaled by points")
        elif (kname == "k_near_sym" and wl.get("refine_points") == 128 and work["points"] == 4_000_000
              and NEAR_SYM_ADAPTIVE_1M_DRAM_BYTES):
            traffic = NEAR_SYM_ADAPTIVE_1M_DRAM_BYTES
            traffic_src = ("dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of this launch "
                           "(1M-segment network, adaptive tree at threshold 128)")
    else:
        fft = fp64 and m2l_fft == 1
        # dense: 2*54*p^6 per cell pair; through transforms: 54 complex multiply-adds
        # (8 FLOP) at each of (2p)^2 (p+1) frequencies per cell pair
        per_pair = 8 * 54 * (2 * p) ** 2 * (p + 1) if fft else 2 * 54 * p ** 6
        if svd:
            per_pair = 2 * ranks["r1"] * ranks["r2"]
        flops = work["m2l_pairs"] * per_pair
        achieved = flops / (m2l_ms / 1e3) / 1e12
        if fp64:
            dom = "k_m2l_fft (FP64 M2L through transforms)" if fft else "k_m2l_f64 (M2L)"
            bound, peak, src = "alu", alu_peak, peaks["source"]
        else:
            dom, bound = "k_m2l_tc (M2L, tcgen05 FP16 operands)", "tensor"
            if svd:
                dom = "k_m2l_tc (SVD-compressed M2L, tcgen05 FP16 operands; stage includes the basis transforms)"
            peak, src = measured_bf16_peak()
    return {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_src, "peak_source": src,
            "work": "algorithmic: near pairs x FLOP/pair (h once per unordered pair when h is the unit-circle "
                    "rule) + L2P, or M2L cell pairs x 2*54*p^6 (x 8*54*(2p)^2*(p+1) through transforms, "
                    "x 2*r1*r2 compressed)"}


def run_fp64_arm(wl, name, d_nodes, d_segs, d_b, nodes, segs, b, flush, stream):
    """The same step through the plain FP64 pass (the metric's comparison arm):
    FP64 everywhere, M2L through transforms, symmetric FP64 near field with the
    same unit-circle rule.  One untimed and one timed step (tens of seconds
    each at a million segments)."""
    import torch

    import paper_1712_07739_gb300 as gb

    f = gb.FMM(p=wl["p"], levels=wl["levels"], precision="fp64", h_mode=wl["h_mode"],
               circle_q=wl.get("circle_q", 0), m2l_fft=1).set_material(wl["C"]())
    out = torch.empty((len(nodes), 3), dtype=torch.float64, device=d_nodes.device)
    f.build(d_nodes, d_segs, d_b)
    f.nodal_forces(out=out)
    f.set_timing(True)
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    f.build(d_nodes, d_segs, d_b)
    f.nodal_forces(out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    st = f.stage_times()
    ms = e0.elapsed_time(e1)
    f.close()
    return {"value": len(segs) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": 1, "warmup": 1,
            "stage_ms": {"precontract": st[0], "p2m_m2m": st[1], "m2l": st[2], "l2l": st[3], "l2p_p2p": st[4],
                         "forces": st[5]},
            "accuracy": oracle_node_error(wl, name, out.cpu().numpy(), nodes, segs, b),
            "config": "same network, p, tree and unit-circle rule; precision fp64, M2L through transforms"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the plain FP64 pass of the same step")
    ap.add_argument("--profile-region", action="store_true",
                    help="mark the timed steps as the profiler range (for ncu --profile-from-start off)")
    ap.add_argument("--levels", type=int, default=0, help="override the workload's tree depth")
    ap.add_argument("--p", type=int, default=0, help="override the workload's interpolation order")
    ap.add_argument("--m2l-split", type=int, default=-1, help="override the M2L operand mode (fmm options)")
    ap.add_argument("--circle-q", type=int, default=0, help="override the unit-circle points")
    ap.add_argument("--m2l-fft", type=int, default=-1, help="FP64 path: 1 = M2L through transforms, 0 = dense")
    ap.add_argument("--m2l-chunks", type=int, default=-1, help="override the M2L offset chunks (fmm options)")
    ap.add_argument("--m2l-basis", type=int, default=-1, help="override the M2L operand basis (fmm options)")
    ap.add_argument("--m2l-split-kblocks", type=int, default=-1, help="override the residual K blocks (fmm options)")
    ap.add_argument("--m2l-kernel", type=int, default=-1, help="override the M2L tile form (fmm options)")
    ap.add_argument("--m2l-svd-tol", type=float, default=-1.0, help="override the M2L compression (fmm options)")
    ap.add_argument("--m2l-symmetry", type=int, default=-1,
                    help="override the FP64 M2L table: 1 = 16 symmetry-orbit representatives, 0 = all 316")
    ap.add_argument("--refine-points", type=int, default=-1,
                    help="override the adaptive tree's split threshold (0: uniform tree; fmm options)")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.p:
        wl["p"] = args.p
    if args.m2l_split >= 0:
        wl["m2l_split"] = args.m2l_split
    if args.circle_q:
        wl["circle_q"] = args.circle_q
    if args.m2l_chunks >= 0:
        wl["m2l_chunks"] = args.m2l_chunks
    if args.m2l_basis >= 0:
        wl["m2l_basis"] = args.m2l_basis
    if args.m2l_split_kblocks >= 0:
        wl["m2l_split_kblocks"] = args.m2l_split_kblocks
    if args.m2l_kernel >= 0:
        wl["m2l_kernel"] = args.m2l_kernel
    if args.m2l_svd_tol >= 0:
        wl["m2l_svd_tol"] = args.m2l_svd_tol
    if args.refine_points >= 0:
        wl["refine_points"] = args.refine_points
    if args.m2l_symmetry >= 0:
        wl["m2l_symmetry"] = args.m2l_symmetry
    if args.impl == "reference":
        run_reference(args, wl)
    elif wl.get("batch"):
        run_batch(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
