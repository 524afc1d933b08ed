#!/usr/bin/env python3
"""Benchmark of the half-plane Robin FMM on GB300.

One step = the whole evaluation path on one synthetic point set: validation,
bounding square, Morton keys and sort, leaf offsets, translation tables
(hpfmm_update_points), then the FMM passes and the near field with
potentials and fields for one charge vector (hpfmm_eval).  Inputs stay
resident in HBM; L2 is flushed (a 512 MiB write) between timed steps.

Metric: particle interactions per second = N^2 / t_step at N = 1e6 (uniform
points in [0,1) x (0,1], charges U[-1,1), kappa = 1 lossless), fast path
(FP32, fields included) at a truncation order whose relative L2 error against
the FP64 oracle (sampled targets) is at most 1e-6; the plain FP64 FMM on the
same workload is timed beside it.

--impl reference runs the oracle (the CPU direct sum with the quadrature
reaction kernel) on a bounded sample of the same workload.
Multi-GPU (torchrun, one process per GPU): independent replicas, no
collective on the data path ("replicas only").
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "particle interactions/sec at N=1e6, rel err ≤1e-6, vs plain FP64 FMM on GB300"
UNIT = "interactions/s"

# The timed configuration of the headline line.  tests/test_gpu_headline.py
# checks the accuracy gate (relative L2 error <= 1e-6 of the potential and of
# the gradient against the oracle, 256 sampled targets) at exactly these
# settings.  p = 13, the smallest order that meets the gate with margin: at
# p = 12 the truncation error of the gradient alone is 8.6e-7 (FP64 run) and
# the single-precision total 9.3e-7; at p = 13 the measured errors are 6.2e-7
# (potential) and 5.6e-7 (gradient).
HEADLINE = dict(n=1_000_000, kappa=1.0, p=13, levels=8, prec="fp32", async_update=True)
GATE = 1e-6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--points", dest="n", type=int, default=HEADLINE["n"])
    ap.add_argument("--kappa", type=float, default=HEADLINE["kappa"])
    ap.add_argument("--p", type=int, default=HEADLINE["p"])
    ap.add_argument("--levels", type=int, default=HEADLINE["levels"])
    ap.add_argument("--prec", default=HEADLINE["prec"], choices=["fp32", "mixed", "fp64"])
    ap.add_argument("--p64", type=int, default=0,
                    help="order of the FP64 comparison run (0: chosen by hpfmm_autotune at the "
                         "same 1e-6 tolerance)")
    ap.add_argument("--levels64", type=int, default=0)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--check-targets", type=int, default=256)
    ap.add_argument("--cpu-targets", type=int, default=8)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the clustered / adjoint / multi-RHS / batched lines")
    return ap.parse_args()


# --------------------------------------------------------------------------
# oracle pieces (CPU baseline, error check); spawn pool so no fork after CUDA
def _oracle_chunk(args):
    xs, ys, qs, idx, kappa = args
    import oracle as o
    return o.direct_closed(xs, ys, qs, idx, kappa)


def oracle_sampled(x, y, q, idx, kappa):
    import multiprocessing as mp
    procs = min(16, os.cpu_count() or 1, len(idx))
    chunks = [c for c in np.array_split(np.asarray(idx), procs) if len(c)]
    with mp.get_context("spawn").Pool(len(chunks)) as pool:
        res = pool.map(_oracle_chunk, [(x, y, q, c, kappa) for c in chunks])
    return np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res])


def cpu_baseline(x, y, q, kappa, ntargets):
    """The oracle (C, OpenMP, quadrature reaction kernel) as it stands, timed on
    ntargets sampled targets x all sources; returns interactions/s."""
    import oracle
    idx = workloads.sample_targets(len(x), ntargets, seed=1)
    nthreads = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.direct(x, y, q, x[idx], y[idx], kappa, self_index=idx, grad=True)
    dt = time.perf_counter() - t0
    pairs = len(idx) * len(x)
    return {"value": pairs / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": "%d sampled targets x %d sources, potentials and fields, %.1f s"
                      % (len(idx), len(x), dt)}


# --------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_index):
        self.proc = None
        self.dev = dev_index

    def start(self):
        try:
            import torch
            sel = ["-i", str(torch.cuda.get_device_properties(self.dev).uuid)]
            sel[1] = sel[1] if sel[1].startswith("GPU-") else "GPU-" + sel[1]
        except Exception:
            sel = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", *sel, "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [s.strip() for s in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def leaf_pairs(keys, H):
    """Near-field pair counts of the uniform level-H tree: free pairs (3x3
    neighbourhood, j != i) and mirror pairs (bottom-row neighbours)."""
    nx = 1 << H
    leaf = (keys >> np.uint64(60 - 2 * H)).astype(np.int64)
    ix = np.zeros_like(leaf); iy = np.zeros_like(leaf)
    for b in range(H):
        ix |= ((leaf >> (2 * b)) & 1) << b
        iy |= ((leaf >> (2 * b + 1)) & 1) << b
    grid = np.zeros((nx + 2, nx + 2), np.int64)
    np.add.at(grid, (iy + 1, ix + 1), 1)
    c = grid[1:-1, 1:-1]
    nb = sum(grid[1 + dy:nx + 1 + dy, 1 + dx:nx + 1 + dx] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    free = int(np.sum(c * nb) - len(keys))
    row = grid[1, :]
    mirror = int(np.sum(row[1:-1] * (row[:-2] + row[1:-1] + row[2:])))
    return free, mirror


def vlist_translations(H):
    """Exact number of free-space M2L translations on the uniform tree: per box
    of level l >= 2 and child type (a, b), the offsets (dx, dy) in
    [-2-a, 3-a] x [-2-b, 3-b] minus the 3x3 near ones, inside the grid."""
    tot = 0
    for l in range(2, H + 1):
        n = 1 << l
        i = np.arange(n)
        a = i & 1
        far = np.zeros(n); near = np.zeros(n)
        for d in range(-3, 4):
            ok = (i + d >= 0) & (i + d < n) & (d >= -2 - a) & (d <= 3 - a)
            far += ok
            near += ok & (abs(d) <= 1)
        tot += int(np.sum(np.outer(far, far) - np.outer(near, near)))
    return tot


# the kernels of each pass whose work bench.py can count (the candidates for
# the dominant-kernel roofline); a pass may take several launches per step (the
# leaf-level M2L runs apart from the coarser levels, the tree build is six
# kernels), and its work per launch is then the step's work over its launches
PASS_KERNELS = {"eval": ("k_near32", "k_eval64"), "m2l_free": ("k_m2l_free_patch", None),
                "m2l_mirror": ("k_m2l_mirror_all", "k_m2l_mirror_all"),
                "p2m": ("k_s2m_tile", "k_p2m"), "near_mirror": ("k_mirror32", None),
                "tree": ("k_tb_* (tree build: bbox, keys, scan, scatter, sort, big-leaf sort)",) * 2,
                "l2l": ("k_downward<float, true>", "k_downward<double, false>")}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel as it is now, from one ncu capture of the configuration it was taken
# on (kernel, n, p, levels, precision); null for any other configuration
NCU_TRAFFIC = {}


def _traffic(name, args, H):
    return NCU_TRAFFIC.get((name, args.n, args.p, H, args.prec))


def roofline_entries(passes_ms, launches, args, npairs, H, alu, hbm_gbs):
    """Roofline entries of the passes with countable work: achieved = the
    pass's algorithmic work per step / its CUDA-event device time per step
    (equal to work per launch / average launch duration), against the peak of
    the pipe (or memory) that bounds it, measured on this device
    (hpfmm_measure_alu_peaks; HBM from the copy bandwidth in MEASURED_PEAKS.json)."""
    n, P1 = args.n, args.p + 1
    out = {}
    for dom, names in PASS_KERNELS.items():
        if launches.get(dom, 0) <= 0 or passes_ms.get(dom, 0) <= 0:
            continue
        name = names[0 if args.prec != "fp64" else 1]
        if name is None:
            continue
        t = passes_ms[dom] / 1e3  # seconds per step
        e = {"kernel": name, "per_launch_ms": t * 1e3 / launches[dom],
             "launches_per_step": launches[dom]}
        if dom == "eval" and args.prec != "fp64":
            ops = 2.0 * npairs
            e.update(bound="alu", unit="TOP/s", achieved=ops / t / 1e12,
                     peak=alu["mufu_ops_per_s"] / 1e12,
                     work="2 SFU ops (lg2, rcp) per free-space near-field pair, %d pairs" % npairs,
                     peak_source="measured: lg2.approx + rcp.approx throughput on %d SMs at "
                                 "%.0f MHz (hpfmm_measure_alu_peaks)" % (alu["sms"],
                                                                        alu["mufu_mhz"]))
        elif dom == "m2l_free":
            ntrans = vlist_translations(H)
            flops = 8.0 * P1 * P1 * ntrans
            e.update(bound="alu", unit="TFLOP/s", achieved=flops / t / 1e12,
                     peak=alu["ffma_flops_per_s"] / 1e12,
                     work="8 (p+1)^2 flops per V-list translation, %d translations" % ntrans,
                     peak_source="measured: FP32 FMA throughput on %d SMs at %.0f MHz "
                                 "(hpfmm_measure_alu_peaks)" % (alu["sms"], alu["ffma_mhz"]))
        elif dom == "tree" and hbm_gbs:
            # read x, y once; write keys, permutation and the tree-order
            # coordinates (single precision: hi and lo leaf frames, y; double:
            # x, y), and the leaf offsets
            per = 16 + 8 + 8 + (20 if args.prec != "fp64" else 16)
            byts = per * n + 4 * (4 ** H + 1)
            e.update(bound="hbm", unit="GB/s", achieved=byts / t / 1e9, peak=hbm_gbs,
                     work="%d B per point (x, y in; keys, permutation, tree-order coordinates "
                          "out) + leaf offsets" % per,
                     peak_source="MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)")
        elif dom == "l2l" and args.prec != "fp64" and hbm_gbs:
            # the fused downward pass + L2P: near sums, leaf frames and
            # permutation in, potential and gradient (complex128) out
            per = 16 + 8 + 8 + 48
            byts = per * n
            e.update(bound="hbm", unit="GB/s", achieved=byts / t / 1e9, peak=hbm_gbs,
                     work="%d B per point (near sums, leaf frame, permutation in; potential "
                          "and gradient out)" % per,
                     peak_source="MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)")
        else:
            e.update(bound="alu", unit="ms", achieved=t * 1e3 / launches[dom], peak=None)
        e["frac"] = e["achieved"] / e["peak"] if e.get("peak") else None
        e["traffic"] = _traffic(name, args, H)
        out[dom] = e
    return out


def roofline(passes_ms, launches, args, npairs, H, alu, hbm_gbs):
    """The contract's roofline object: the single-kernel pass with the largest
    device time per step, plus every other entry under "others"."""
    ent = roofline_entries(passes_ms, launches, args, npairs, H, alu, hbm_gbs)
    dom = max(ent, key=lambda k: passes_ms[k])
    r = dict(ent[dom])
    r["others"] = {k: v for k, v in ent.items() if k != dom}
    return r


def ranks():
    """(world, rank, local rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init_replicas(backend="nccl"):
    """Process group of the replicas (None for a single process).  The data
    path has no collective: the group only carries the barriers around the
    timed region and the max-over-ranks reduction of the timings."""
    import torch
    world, _, local = ranks()
    if world <= 1:
        return None
    import torch.distributed as dist
    if backend == "nccl":
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)
    return dist


def max_over_ranks(v, dist, device=None):
    """Maximum of a per-rank float over all ranks (the slowest replica)."""
    if dist is None:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, n, seconds_per_step):
    """Whole-job interactions/s: every replica evaluates its own N-point
    problem (N^2 interactions) per step; the step time is the slowest rank's."""
    return world * float(n) * float(n) / seconds_per_step


# --------------------------------------------------------------------------
# the other workloads: each timed on its own (CUDA events, W warm-ups), inputs
# resident, potentials and fields
def _event_time(fn, k, w, flush):
    import torch
    for _ in range(w):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for i in range(k):
        flush.fill_(i & 0xff)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        tot += a.elapsed_time(b)
    return tot / k


def extra_workloads(args, dev, flush, check):
    import torch
    import paper_2507_21913_gb300 as hp
    t = lambda a: torch.tensor(a, device=dev)
    out = {}
    k, w = 3, 2

    # clustered: 4e6 points, kappa = 1 + 0.5i, mixed precision, p = 20
    n = 4_000_000
    x, y, q = workloads.clustered(n, seed=0)
    xd, yd, qd = t(x), t(y), t(q)
    kap = 1.0 + 0.5j
    pot = torch.empty(n, dtype=torch.complex128, device=dev)
    grad = torch.empty((n, 2), dtype=torch.complex128, device=dev)
    if check:
        near = np.flatnonzero(y < 0.06)
        far = np.flatnonzero(y >= 0.06)
        g0 = np.random.Generator(np.random.PCG64(1))
        idx = np.sort(np.concatenate([g0.choice(near, 128, replace=False),
                                      g0.choice(far, 128, replace=False)]))
        u_ref, g_ref = oracle_sampled(x, y, q, idx, kap)
    e = {}
    # the configured mixed-precision path on the adaptive tree (the line's
    # value), then single precision throughout and the uniform tree of depth
    # 11 for comparison
    for tag, prec, adaptive in (("", "mixed", True), ("fp32_", "fp32", True),
                                ("uniform_", "mixed", False), ("uniform_fp32_", "fp32", False)):
        plan = hp.hpfmm_create(xd, yd, kappa=kap, p=20, leaf_size=32, prec=prec,
                               levels=0 if adaptive else 11, adaptive=adaptive)

        def step():
            hp.hpfmm_update_points(plan, xd, yd)
            hp.hpfmm_eval(plan, qd, out=(pot, grad))
        ms = _event_time(step, k, w, flush)
        if not tag:
            e = {"workload": "clustered N=4e6 (80% in 64 clusters sigma 0.01 near y=0), "
                             "kappa=1+0.5i, mixed precision, p=20, adaptive tree (leaves of at "
                             "most 32 points), tree rebuilt every step",
                 "ms_per_step": ms, "value": float(n) * n / (ms / 1e3), "unit": UNIT}
            boxes, leaves, depth = hp.hpfmm_get_adaptive_counts(plan)
            e["tree"] = {"boxes": int(boxes.sum()), "leaves": int(leaves.sum()), "depth": depth}
        else:
            e[tag + "ms_per_step"] = ms
        if check:
            ee = errors(pot.cpu().numpy()[idx], grad.cpu().numpy()[idx], u_ref, g_ref)
            e[tag + "rel_err_pot"] = ee["pot"]
            e[tag + "rel_err_grad"] = ee["grad"]
            e["check_targets"] = "%d (half with y < 0.06)" % len(idx)
        del plan
    out["clustered"] = e
    del pot, grad, xd, yd, qd

    # adjoint: N = 1e6, kappa = 2, p = 16, single precision; forward (with field)
    # then backward for E = w . u
    n = 1_000_000
    x, y, q, wv = workloads.uniform(n, seed=0, with_w=True)
    xd, yd, qd = t(x), t(y), t(q)
    g = t(wv.astype(np.complex128))
    plan = hp.hpfmm_create(xd, yd, kappa=2.0, p=16, leaf_size=64, prec="fp32")
    pot = torch.empty(n, dtype=torch.complex128, device=dev)
    grad = torch.empty((n, 2), dtype=torch.complex128, device=dev)
    ms_f = _event_time(lambda: hp.hpfmm_eval(plan, qd, out=(pot, grad)), k, w, flush)
    ms_b = _event_time(lambda: hp.hpfmm_eval_adjoint(plan, qd, g, grad_q=grad), k, w, flush)
    out["adjoint"] = {"workload": "uniform N=1e6, kappa=2, p=16, fp32; E = w.u, dE/dq and dE/dr",
                      "forward_ms": ms_f, "backward_ms": ms_b,
                      "backward_over_forward": ms_b / ms_f}
    del plan, pot, grad

    # many charge vectors on one tree: 64 RHS on N = 5e5, p = 16, single precision
    n = 500_000
    x, y, _ = workloads.uniform(n, seed=0)
    Q = t(np.random.Generator(np.random.PCG64(8)).uniform(-1.0, 1.0, (64, n)))
    plan = hp.hpfmm_create(t(x), t(y), kappa=1.0, p=16, leaf_size=32, prec="fp32")
    pot = torch.empty((64, n), dtype=torch.complex128, device=dev)
    grad = torch.empty((64, n, 2), dtype=torch.complex128, device=dev)
    ms_m = _event_time(lambda: hp.hpfmm_eval(plan, Q, out=(pot, grad)), k, w, flush)

    def looped():
        for r in range(64):
            hp.hpfmm_eval(plan, Q[r], out=(pot[r], grad[r]))
    ms_l = _event_time(looped, 2, 1, flush)
    out["multi_rhs"] = {"workload": "64 charge vectors on uniform N=5e5, kappa=1, p=16, fp32, "
                                    "potentials and fields", "ms_shared_passes": ms_m,
                        "ms_one_at_a_time": ms_l, "speedup": ms_l / ms_m,
                        "value": 64.0 * n * n / (ms_m / 1e3), "unit": UNIT}
    del plan, pot, grad, Q

    # independent problems of uneven size as one CUDA graph
    sizes, kappas = workloads.batched_sizes(32, seed=0)
    plans, qs = [], []
    for i, (nn, kk) in enumerate(zip(sizes, kappas)):
        xx, yy, qq = workloads.uniform(int(nn), seed=100 + i)
        plans.append(hp.hpfmm_create(t(xx), t(yy), kappa=float(kk), p=16, leaf_size=32,
                                     prec="fp32"))
        qs.append(t(qq))
    outs = [(torch.empty(p_.n, dtype=torch.complex128, device=dev),
             torch.empty((p_.n, 2), dtype=torch.complex128, device=dev)) for p_ in plans]
    batch = hp.hpfmm_batch_create(plans)
    ms_g = _event_time(lambda: hp.hpfmm_eval_batched(batch, qs), k, w, flush)

    def one_by_one():
        for p_, q_, o_ in zip(plans, qs, outs):
            hp.hpfmm_eval(p_, q_, out=o_)
    ms_o = _event_time(one_by_one, k, w, flush)
    pairs = float(np.sum(sizes.astype(np.float64) ** 2))
    out["batched"] = {"workload": "32 problems, N=floor(10^U[4,log10 4e5]) (sum %d), "
                                  "kappa=U[0.1,10], p=16, fp32, one CUDA graph" % int(sizes.sum()),
                      "ms_graph": ms_g, "ms_one_by_one": ms_o, "speedup": ms_o / ms_g,
                      "value": pairs / (ms_g / 1e3), "unit": UNIT,
                      "graph_captures": batch.captures()}
    del batch, plans

    # separate targets: the Example 2 geometry (8 charged circles, field mesh
    # including y = 0) at 2e5 sources and 1.25e5 field points
    xs, ys, qs, xt, yt = workloads.example2(n_source=25_000, nfx=512, nfy=245)
    plan = hp.hpfmm_create(t(xs), t(ys), kappa=1.0, p=16, leaf_size=32, prec="fp32", levels=8,
                           root=(-4.4, 8.8))
    qd, xtd, ytd = t(qs), t(xt), t(yt)
    ms_t = _event_time(lambda: hp.hpfmm_eval_targets(plan, qd, xtd, ytd), k, w, flush)
    e = {"workload": "Example 2 geometry: 8 circles x 25000 sources (charge 2pi/25000), "
                     "512 x 245 field mesh on [-4.4,4.4]x[0,4.2], kappa=1, fp32 plan p=16, L=8",
         "ms_per_eval": ms_t, "value": float(len(xs)) * len(xt) / (ms_t / 1e3), "unit": UNIT}
    if check:
        pot, _ = hp.hpfmm_eval_targets(plan, qd, xtd, ytd, grad=False)
        idx = np.linspace(0, len(xt) - 1, 256).astype(np.int64)
        import oracle
        u_ref, _ = oracle.direct(xs, ys, qs, xt=xt[idx], yt=yt[idx], kappa=1.0, grad=False)
        u = pot.cpu().numpy()[idx]
        e["rel_err_pot"] = float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref))
        e["check_targets"] = len(idx)
    out["targets"] = e
    del plan

    # the autotuner on the headline workload: its pick for single precision at 1e-6
    n = 1_000_000
    x, y, _ = workloads.uniform(n, seed=0)
    t0 = time.perf_counter()
    tun = hp.hpfmm_autotune(t(x), t(y), kappa=1.0, prec="fp32", tol=GATE, nsample=256)
    tun["tuning_seconds"] = time.perf_counter() - t0
    tun["workload"] = ("uniform N=1e6, kappa=1, fp32, tol 1e-6 on potential and gradient (probe "
                       "charges, 256 sampled targets)")
    out["autotune"] = tun

    # the configuration sweep of the uniform 1e6 workload: kappa x p in both
    # precisions, tree rebuilt every step; the leaf level of each cell is the
    # faster of 7 and 8 (mean leaf 61 and 15); errors at 256 sampled targets
    # (one oracle reference per kappa, shared by the orders and precisions)
    xd, yd = t(x), t(y)
    q = workloads.uniform(n, seed=0)[2]
    qd = t(q)
    pot = torch.empty(n, dtype=torch.complex128, device=dev)
    grad = torch.empty((n, 2), dtype=torch.complex128, device=dev)
    idx = workloads.sample_targets(n, 256, seed=1)
    rows = []
    for kap in (0.1, 1.0, 10.0):
        ref = oracle_sampled(x, y, q, idx, kap) if check else None
        for prec in ("fp32", "fp64"):
            for p in (8, 16, 24, 32):
                cells = []
                for lev in (7, 8):
                    plan = hp.hpfmm_create(xd, yd, kappa=kap, p=p, leaf_size=32, prec=prec,
                                           levels=lev, async_update=True)

                    def step():
                        hp.hpfmm_update_points(plan, xd, yd)
                        hp.hpfmm_eval(plan, qd, out=(pot, grad))
                    ms = _event_time(step, 3, 2, flush)
                    hp.hpfmm_sync(plan)
                    row = {"kappa": kap, "prec": prec, "p": p, "levels": lev,
                           "ms_per_step": ms, "value": float(n) * n / (ms / 1e3)}
                    if check:
                        ee = errors(pot.cpu().numpy()[idx], grad.cpu().numpy()[idx], *ref)
                        row["rel_err_pot"] = ee["pot"] if np.isfinite(ee["pot"]) else None
                        row["rel_err_grad"] = ee["grad"] if np.isfinite(ee["grad"]) else None
                    cells.append(row)
                    del plan
                best = min(cells, key=lambda r: r["ms_per_step"])
                best["other_level_ms"] = [r["ms_per_step"] for r in cells if r is not best][0]
                rows.append(best)
    out["sweep"] = {"workload": "uniform N=1e6, kappa in {0.1, 1, 10}, p in {8, 16, 24, 32}, fp32 "
                                "and fp64, leaf level the faster of 7 and 8, potentials and "
                                "fields, tree rebuilt every step", "unit": UNIT,
                    "check_targets": len(idx) if check else 0, "rows": rows}

    # O(N): uniform N from 1e5 to 4e6 at the headline order, the leaf level
    # the faster of the two nearest a mean leaf of 16
    rows = []
    for nn in (100_000, 250_000, 500_000, 1_000_000, 2_000_000, 4_000_000):
        xx, yy, qq = workloads.uniform(nn, seed=0)
        xd2, yd2, qd2 = t(xx), t(yy), t(qq)
        pot2 = torch.empty(nn, dtype=torch.complex128, device=dev)
        grad2 = torch.empty((nn, 2), dtype=torch.complex128, device=dev)
        l_mid = math.log(nn / 16.0, 4)
        cells = []
        for lev in sorted({int(math.floor(l_mid)), int(math.ceil(l_mid))}):
            plan = hp.hpfmm_create(xd2, yd2, kappa=1.0, p=HEADLINE["p"], leaf_size=32,
                                   prec="fp32", levels=lev, async_update=True)

            def step():
                hp.hpfmm_update_points(plan, xd2, yd2)
                hp.hpfmm_eval(plan, qd2, out=(pot2, grad2))
            ms = _event_time(step, 5, 3, flush)
            hp.hpfmm_sync(plan)
            cells.append({"n": nn, "levels": lev, "ms_per_step": ms,
                          "us_per_point": 1e3 * ms / nn})
            del plan
        rows.append(min(cells, key=lambda r: r["ms_per_step"]))
        del xd2, yd2, qd2, pot2, grad2
    upp = [r["us_per_point"] for r in rows]
    out["scaling_n"] = {"workload": "uniform N in [1e5, 4e6], kappa=1, fp32, p=%d, potentials "
                                    "and fields, tree rebuilt every step" % HEADLINE["p"],
                        "rows": rows, "max_over_min_us_per_point": max(upp) / min(upp),
                        "max_over_min_us_per_point_from_5e5":
                            max(upp[2:]) / min(upp[2:])}
    return out


def errors(u, g, u_ref, g_ref):
    """Relative L2 errors of the potential and the gradient over the sampled
    targets, and the largest per-target error relative to the rms value."""
    rms_u = np.sqrt(np.mean(np.abs(u_ref) ** 2))
    rms_g = np.sqrt(np.mean(np.sum(np.abs(g_ref) ** 2, axis=1)))
    return {"pot": float(np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)),
            "grad": float(np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)),
            "pot_max_over_rms": float(np.max(np.abs(u - u_ref)) / rms_u),
            "grad_max_over_rms": float(np.max(np.linalg.norm(g - g_ref, axis=1)) / rms_g)}


def run_ours(args):
    import torch
    import paper_2507_21913_gb300 as hp

    world, rank, local = ranks()
    dist = init_replicas("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    hp.lib(build_if_missing=True)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_gbs = peaks.get("hbm_gbs")
    # the arithmetic pipes' throughput on this device (SFU, FP32 and FP64 FMA)
    alu = hp.hpfmm_measure_alu_peaks(dev)

    n = args.n
    x, y, q = workloads.uniform(n, seed=0)
    xd = torch.tensor(x, device=dev); yd = torch.tensor(y, device=dev)
    qd = torch.tensor(q, device=dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make_plan(prec, p, levels, subtree=0):
        return hp.hpfmm_create(xd, yd, kappa=args.kappa, p=p, leaf_size=32, prec=prec,
                               levels=levels, subtree_levels=subtree,
                               async_update=HEADLINE["async_update"])

    def timed_steps(plan, k, w, timing):
        """k timed steps (rebuild + evaluation), CUDA events on the launching
        stream, L2 flushed between steps outside the events; with timing the
        plan also records per-pass events."""
        pot = torch.empty(n, dtype=torch.complex128, device=dev)
        grad = torch.empty((n, 2), dtype=torch.complex128, device=dev)
        for _ in range(w):
            hp.hpfmm_update_points(plan, xd, yd)
            hp.hpfmm_eval(plan, qd, out=(pot, grad))
        hp.hpfmm_sync(plan)
        hp.hpfmm_read_timing(plan)
        hp.hpfmm_set_timing(plan, timing)
        _, l0 = hp.hpfmm_read_timing(plan)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(k)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        for i in range(k):
            flush.fill_(i & 0xff)  # evict L2 between steps (outside the events)
            ev[i][0].record(stream)
            hp.hpfmm_update_points(plan, xd, yd)
            hp.hpfmm_eval(plan, qd, out=(pot, grad))
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        pms, l1 = hp.hpfmm_read_timing(plan)
        hp.hpfmm_set_timing(plan, False)
        hp.hpfmm_sync(plan)  # raises on invalid input or a device timeout
        launches = {kk: l1[kk] - l0[kk] for kk in l1}
        return ms, pms, launches, pot, grad

    # fast path, timed (without per-pass events), then once more with them
    # for the per-pass breakdown and the rooflines
    plan = make_plan(args.prec, args.p, args.levels)
    info = plan.info()
    clock = ClockSampler(local)
    clock.start()
    ms, _, launches, pot, grad = timed_steps(plan, args.steps, args.warmup, False)
    clocks = clock.stop()
    ms = max_over_ranks(ms, dist, dev)
    ms_step = ms / args.steps
    value = replica_throughput(world, n, ms_step / 1e3)
    ms_t, pms, launches, _, _ = timed_steps(plan, args.steps, 1, True)

    keys, _ = hp.hpfmm_get_order(plan)
    npairs, mpairs = leaf_pairs(keys, info["levels"])
    launches_per_step = {k: v / args.steps for k, v in launches.items()}
    pass_ms_step = {k: v / args.steps for k, v in pms.items()}
    roof = roofline(pass_ms_step, launches_per_step, args, npairs, info["levels"], alu, hbm_gbs)

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32" if args.prec != "fp64" else "f64",
              "data": "synthetic (seeded uniform points, PCG64 seed 0)",
              "config": {"workload": "uniform N=%d in [0,1)x(0,1], q~U[-1,1), kappa=%g lossless, "
                                     "potential+field, one RHS, tree rebuilt every step" %
                                     (n, args.kappa),
                         "n": n, "kappa": args.kappa, "p": args.p, "levels": info["levels"],
                         "mean_leaf": n / 4 ** info["levels"], "precision": args.prec,
                         "rebuild": "asynchronous (async_update)" if HEADLINE["async_update"]
                         else "synchronous",
                         "l2": "flushed between steps (512 MiB write)",
                         "parallelism": "replicas" if world > 1 else "single GPU"},
              "gpu_launches": int(sum(launches.values())),
              "passes_ms_per_step": pass_ms_step,
              "ms_per_step_with_pass_events": ms_t / args.steps,
              "launches_per_step": launches_per_step,
              "near_field_pairs": {"free": npairs, "mirror": mpairs},
              "roofline": roof, "clocks": clocks,
              "alu_peaks_measured": alu}

    # accuracy of the timed configuration
    idx = workloads.sample_targets(n, args.check_targets, seed=1)
    u_ref = g_ref = None
    if not args.no_check and rank == 0:
        u_ref, g_ref = oracle_sampled(x, y, q, idx, args.kappa)
        e = errors(pot.cpu().numpy()[idx], grad.cpu().numpy()[idx], u_ref, g_ref)
        e.update(targets=len(idx), reference="oracle (E1 closed form), seed-1 sample")
        result["rel_err"] = e
        result["meets_gate"] = bool(e["pot"] <= GATE and e["grad"] <= GATE)

    # the plain FP64 FMM on the same workload, at the configuration the
    # autotuner picks for the same tolerance (potential and gradient)
    if not args.no_fp64:
        if args.p64 > 0:
            tun64 = {"p": args.p64, "levels": args.levels64, "subtree_levels": 0,
                     "picked_by": "command line"}
        else:
            t0 = time.perf_counter()
            tun64 = hp.hpfmm_autotune(xd, yd, kappa=args.kappa, prec="fp64", tol=GATE,
                                      nsample=256)
            tun64["tuning_seconds"] = time.perf_counter() - t0
            tun64["picked_by"] = "hpfmm_autotune(prec=fp64, tol=1e-6)"
        plan64 = make_plan("fp64", tun64["p"], tun64["levels"], tun64["subtree_levels"])
        k64 = max(2, min(args.steps, 5))
        ms64, pms64, _, pot64, grad64 = timed_steps(plan64, k64, 2, True)
        ms64 = max_over_ranks(ms64, dist, dev)
        e = {"value": replica_throughput(world, n, ms64 / k64 / 1e3), "unit": UNIT,
             "ms_per_step": ms64 / k64, "p": tun64["p"], "levels": plan64.info()["levels"],
             "tuning": tun64, "passes_ms_per_step": {k: v / k64 for k, v in pms64.items()}}
        if u_ref is not None:
            e["rel_err"] = errors(pot64.cpu().numpy()[idx], grad64.cpu().numpy()[idx], u_ref,
                                  g_ref)
        result["fp64_fmm"] = e
        result["speedup_vs_fp64_fmm"] = e["ms_per_step"] / ms_step
        del plan64

    # end to end through the C ABI with host buffers (pinned), copies included
    if not args.no_e2e:
        xh = torch.tensor(x).pin_memory(); yh = torch.tensor(y).pin_memory()
        qh = torch.tensor(q).pin_memory()
        poth = torch.empty(n, dtype=torch.complex128).pin_memory()
        gradh = torch.empty((n, 2), dtype=torch.complex128).pin_memory()
        for _ in range(2):
            hp.hpfmm_update_points(plan, xh, yh)
            hp.hpfmm_eval(plan, qh, out=(poth, gradh))
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        k = args.steps
        for _ in range(k):
            hp.hpfmm_update_points(plan, xh, yh)
            hp.hpfmm_eval(plan, qh, out=(poth, gradh))  # synchronises (host outputs)
        dt = max_over_ranks((time.perf_counter() - t0) / k, dist, dev)
        hp.hpfmm_sync(plan)
        result["e2e"] = {"value": replica_throughput(world, n, dt), "unit": UNIT,
                         "ms_per_step": dt * 1e3,
                         "h2d_bytes_per_step": 3 * 8 * n, "d2h_bytes_per_step": (16 + 32) * n}

    # the extra lines are single-GPU measurements of other configurations: at
    # N = 1 only, so that a multi-GPU run holds its GPUs for the headline alone
    if not args.no_extra and world == 1:
        result["extra"] = extra_workloads(args, dev, flush, check=not args.no_check and rank == 0)

    if rank == 0 and not args.no_cpu_baseline and world == 1:
        result["cpu_baseline"] = cpu_baseline(x, y, q, args.kappa, args.cpu_targets)
    if rank == 0:
        print(json.dumps(result))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args):
    _, rank, _ = ranks()
    if rank != 0:
        return
    import oracle
    n = args.n
    x, y, q = workloads.uniform(n, seed=0)
    ntarg = max(1, args.cpu_targets // 4)
    idx_all = workloads.sample_targets(n, ntarg * (args.steps + args.warmup), seed=1)
    nthreads = oracle.max_threads()
    times = []
    for s in range(args.warmup + args.steps):
        idx = idx_all[s * ntarg:(s + 1) * ntarg]
        t0 = time.perf_counter()
        oracle.direct(x, y, q, x[idx], y[idx], args.kappa, self_index=idx, grad=True)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    t = float(np.sum(times))
    pairs = ntarg * n * args.steps
    value = pairs / t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded uniform points, PCG64 seed 0)",
        "config": {"workload": "uniform N=%d, kappa=%g; each step %d sampled targets x all sources"
                               % (n, args.kappa, ntarg), "n": n, "kappa": args.kappa},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                         "sample": "%d targets x %d sources per step" % (ntarg, n)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
