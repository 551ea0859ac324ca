#!/usr/bin/env python
"""Benchmark: QBX layer-potential targets/s of GIGAQBX on one GB300 per rank.

Workload: 16 x 16 grid of starfish curves (64 panels x 16 nodes each,
262,144 base nodes, 1,048,576 quadrature nodes, 524,288 QBX centres),
1,048,576 off-surface targets uniform in the bounding box + 1,048,576
on-surface targets (the quadrature nodes, two-sided), p_qbx = 8, p_fmm = 15,
n_max = 32, single-layer potential S in FP64.

One step = the whole hot path for one geometry and density: centres, target
association, root, keys, quadtree, the six interaction lists (gq_build) and
upsampling, Stages 2-8 and the final QBX evaluation (gq_eval).  Inputs are
resident in device memory when the timed region starts; an L2 flush (256 MB
write) separates timed steps.  `e2e` repeats the step through the same C ABI
from pinned host buffers, host<->device copies included.

Multi-GPU: one independent replica per rank (the method has no exchange
step between independent problems); value = all ranks' targets / max time.
`--impl reference` times the CPU FP64 oracle (plain serial C) on a bounded
sample of the workload instead.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QBX layer-potential targets/sec at stated rel. error vs FP64 oracle; % roofline"
UNIT = "targets/s"
NOMINAL_FP64_TFLOPS = 1.25   # GB300 nominal FP64, used only if the probe fails
SAMPLE_GRID = (8, 6)         # CPU baseline: 48 of the 256 curves, same per-curve sizes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gigaqbx", choices=["gigaqbx", "reference"])
    ap.add_argument("--kernel", default="S", choices=["S", "D"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false",
                    help="skip the FP64 vs MIXED evaluation sweep at eps = 1e-4 ... 1e-12 (orders from eps)")
    ap.add_argument("--no-learned", dest="learned", action="store_false",
                    help="skip the learned order selection (training on the oracle labels, deployment at eps 1e-8)")
    ap.add_argument("--learned-curves", type=int, default=2000,
                    help="training curves (of tests/golden/order_labels.npz) for the learned order selection")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the 64 geometries of uneven size (2k-200k quadrature nodes, log-uniform) x 8 "
                         "densities: the persistent launch and the graph branches against one gq_eval after "
                         "another, and the batched exterior Neumann solves")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2],
                    help="precision of the timed step: 0 FP64 (the benchmark), 1 MIXED, 2 MIXED_FMM at --eps "
                         "with the workload's orders (profiling cases)")
    ap.add_argument("--eps", type=float, default=1e-6, help="requested accuracy for --precision 1 or 2")
    ap.add_argument("--grid", type=int, nargs=2, default=[16, 16],
                    help="curves per row / column (the benchmark workload is 16 16; smaller grids are "
                         "profiling cases with the same per-curve sizes)")
    return ap.parse_args()


def workload(n_off=1 << 20, grid=(16, 16)):
    import workloads
    return workloads.starfish_grid(grid[0], grid[1], 64, n_off=n_off, on_surface="up", seed=1)


# ---------------------------------------------------------------- distributed plumbing
def dist_init(args):
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch.distributed as dist
        import torch
        if args.impl == "gigaqbx":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group("gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(step_ms, units, world, device=None):
    """Whole-job throughput of independent replicas: every rank processed
    `units` per step; the job time is the slowest rank's total.  Returns
    (ms per step, units/s over all ranks)."""
    tot_ms = max_over_ranks(sum(step_ms), world, device)
    return tot_ms / len(step_ms), world * units * len(step_ms) / (tot_ms * 1e-3)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.device)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.25)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic work model
LOG_FLOPS = 7   # FP64 flops of one table-driven logarithm as the kernels run it: 3 FMAs + 1 add


def work_model(geo, p, q, kernel="S"):
    """Units per launch of each stage (pairs), from the exported lists.  Flop
    weights: direct to centres 14q + 20 per (source, centre) pair, direct to
    points 10 per pair plus, for S, one logarithm (LOG_FLOPS), M2L 8(p+1)^2 per
    List 2 pair, List 3 far to centres 8(p+1)(q+1) per (box, centre)."""
    bx = geo.boxes()
    L = geo.lists()
    nsrc, nctr, ntgt = bx["nsrc"].astype(np.int64), bx["nctr"].astype(np.int64), bx["ntgt"].astype(np.int64)

    def per_box_sum(name):
        off, idx = L[name]
        v = np.zeros(len(off) - 1, np.int64)
        box = np.repeat(np.arange(len(off) - 1), np.diff(off))
        np.add.at(v, box, nsrc[idx])
        return v

    near = per_box_sum("U") + per_box_sum("WC") + per_box_sum("XC")
    wf = np.diff(L["WF"][0]).astype(np.int64)
    pairs_ctr = int((near * nctr).sum())
    pairs_pt = int((near * ntgt).sum())
    v_pairs = int(len(L["V"][1]))
    wf_ctr = int((wf * nctr).sum())
    return {
        5: dict(name="k_near_centres", units=pairs_ctr, flops_per_unit=14 * q + 20, unit="(source, centre) pair"),
        6: dict(name="k_near_points", units=pairs_pt, flops_per_unit=10 + (LOG_FLOPS if kernel == "S" else 0),
                unit="(source, point) pair"),
        2: dict(name="k_m2l_tc" if p <= 15 else "k_m2l", units=v_pairs, flops_per_unit=8 * (p + 1) ** 2,
                unit="List 2 pair (FP64-equivalent flops of the translation)"),
        7: dict(name="k_w_centres_tc" if (p <= 16 and q <= 15 and math.comb(q + p - 1, p - 1) < 1 << 24)
                else "k_w_centres_q", units=wf_ctr, flops_per_unit=8 * (p + 1) * (q + 1),
                unit="(List 3 far box, centre) pair (FP64-equivalent flops of the translation)"),
    }


STAGE_NAMES = ["upsample", "p2m_m2m", "m2l", "p2l", "l2l", "near_centres", "near_points", "wfar_centres",
               "wfar_points", "l2qbxl_l2p", "final"]


# ---------------------------------------------------------------- CPU oracle sample
def cpu_model():
    """The host CPU's model name (lscpu), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_sample(kernel, reps=1, grid=SAMPLE_GRID, threads=1, g=None):
    """The CPU oracle (plain C, FP64) on a grid of the workload (a sub-grid
    has the same per-curve discretisation, density recipe and target density:
    its share of the curves and of the off-surface targets).  Build +
    evaluation timed.  threads > 1 runs the oracle's evaluation loops on that
    many cores (the same results bit for bit; the tree build stays serial)."""
    import oracle
    if g is None:
        n_off = (1 << 20) * grid[0] * grid[1] // 256
        g = workload(n_off=n_off, grid=grid)
    used = oracle.set_threads(threads)
    times = []
    vals = None
    try:
        for _ in range(reps):
            t0 = time.perf_counter()
            o = oracle.Oracle(g, oracle.default_params(g))
            vals = o.eval(kernel, g["density"])
            times.append(time.perf_counter() - t0)
            del o
    finally:
        oracle.set_threads(1)
    nt = len(g["tgt_xy"])
    return g, vals, nt, times, used


def host_cores():
    import oracle
    return max(1, min(os.cpu_count() or 1, oracle.max_threads()))


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    # the oracle on all host cores: the full workload takes about 7-11 s a step
    # (serial tree build + parallel evaluation); smaller sub-grids when many steps are
    # asked for, so that the whole run stays within a few minutes (targets/s is per target)
    cores = host_cores()
    n = args.steps + args.warmup
    grid = (16, 16) if n <= 10 else SAMPLE_GRID if n <= 24 else (4, 3)
    g = workload(n_off=(1 << 20) * grid[0] * grid[1] // 256, grid=grid)
    for _ in range(args.warmup):
        oracle_sample(args.kernel, threads=cores, g=g)
    g, _, nt, times, used = oracle_sample(args.kernel, reps=args.steps, threads=cores, g=g)
    tot = sum(times)
    value = nt * args.steps / tot
    full = grid == (16, 16)
    sample = (f"oracle build (serial) + {args.kernel} evaluation ({used} OpenMP threads) of "
              f"{'the whole workload' if full else f'a {grid[0]}x{grid[1]} sub-grid'} "
              f"({nt} targets, {len(g['up_w'])} quadrature nodes) per step")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": g["name"] + ("" if full else " (sub-grid sample)"),
                       "kernel": args.kernel, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched workload
def batched_workloads(n_geom=64, n_dens=8, seed=4):
    """n_geom starfish arrays with quadrature-node counts log-uniform in
    [2k, 200k] (64 nodes per panel, 64 panels per curve; the smallest are one
    curve with fewer panels), on-surface targets at the base nodes plus as many
    off-surface targets, n_dens random-Fourier densities each."""
    import workloads
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_geom):
        ns = float(np.exp(rng.uniform(np.log(2000), np.log(200000))))
        curves = max(1, int(round(ns / 4096)))
        panels = 64 if curves > 1 else max(8, int(round(ns / 64)))
        nx = int(np.ceil(np.sqrt(curves)))
        ny = int(np.ceil(curves / nx))
        g = workloads.starfish_grid(nx, ny, panels, n_off=nx * ny * panels * 16, on_surface="base", seed=100 + i)
        dens = np.stack([workloads.starfish.fourier_density(g, rng) for _ in range(n_dens)])
        out.append((g, dens))
    return out


def run_batched(args, dev, stream):
    import torch

    from paper_1801_04070_gb300 import Batch, Geometry, params_default
    items = batched_workloads()
    geos, dens, outs = [], [], []
    for g, d in items:
        geo = Geometry(g, params_default(p_qbx=8, p_fmm=15, n_max=32), device=dev.index)
        geo.build()
        geos.append(geo)
        dens.append(torch.tensor(d, dtype=torch.float64, device=dev))
        outs.append(torch.empty((d.shape[0], len(g["tgt_xy"])), dtype=torch.float64, device=dev))
    ntot = sum(o.numel() for o in outs)
    nsrc = [int(len(g["up_w"])) for g, _ in items]
    kern = args.kernel

    def sequential():
        for geo, d, o in zip(geos, dens, outs):
            for j in range(d.shape[0]):
                geo.eval(kern, d[j], o[j])

    b = Batch(geos)
    b.eval(kern, dens, outs)            # eager pass, autotune, capture (persistent launch)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    sequential()
    torch.cuda.synchronize()
    diff = max(float((a - c).abs().max() / c.abs().max()) for a, c in zip(ref, outs))
    res = {}

    def timed3(fn):
        fn()
        torch.cuda.synchronize()
        t = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.mean(t)

    res["auto"] = timed3(lambda: b.eval(kern, dens, outs))
    auto_pick = "persistent" if b.persistent_tile() > 0 else "graph"
    b.mode(0)
    res["persistent"] = timed3(lambda: b.eval(kern, dens, outs))
    tile, streams, ctas = b.persistent_tile(), b.streams(), b.persistent_ctas()
    b.mode(1)
    res["graph"] = timed3(lambda: b.eval(kern, dens, outs))
    graph_streams = b.streams()
    res["sequential"] = timed3(sequential)
    b.close()
    for geo in geos:
        geo.close()

    # exterior Neumann solves -mu/2 + S' mu = g on the same geometries (base nodes
    # as targets), g the normal derivative of Re 1/(z - z0), z0 inside the first curve
    ggeos, rhs, mus, refs = [], [], [], []
    for g, _ in items:
        geo = Geometry(g, params_default(p_qbx=8, p_fmm=15, n_max=32), device=dev.index)
        geo.set_targets(g["base_xy"], np.arange(len(g["base_xy"]), dtype=np.int32))
        geo.build()
        ggeos.append(geo)
        x = g["base_xy"][:, 0] + 1j * g["base_xy"][:, 1]
        z0 = x[g["base_curve"] == 0].mean()
        nrm = g["base_n"][:, 0] + 1j * g["base_n"][:, 1]
        rhs.append(torch.tensor((nrm * (-1.0 / (x - z0) ** 2)).real, dtype=torch.float64, device=dev))
        mus.append(torch.zeros_like(rhs[-1]))
        refs.append(torch.zeros_like(rhs[-1]))
    gb = Batch(ggeos)
    tol, maxit, restart = 1e-10, 100, 30
    gb.gmres(rhs, mus, tol=tol, maxit=maxit, restart=restart)   # capture and autotune the S' graph
    torch.cuda.synchronize()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    ms_b, (its, res_b) = timed(lambda: gb.gmres(rhs, mus, tol=tol, maxit=maxit, restart=restart))

    def seq():
        return [geo.gmres(r, tol=tol, maxit=maxit, restart=restart, mu=m)[1:] for geo, r, m in zip(ggeos, rhs, refs)]
    ms_s, seq_out = timed(seq)
    diff = max(float((m - r).abs().max() / r.abs().max()) for m, r in zip(mus, refs))
    gmres = {"tol": tol, "restart": restart, "maxit": maxit, "unknowns": int(sum(r.numel() for r in rhs)),
             "batched_ms": ms_b, "sequential_ms": ms_s, "iterations_max": int(max(its)),
             "iterations_total": int(sum(its)), "max_rel_residual": float(max(res_b)),
             "converged": int(sum(r <= 2 * tol for r in res_b)), "geometries": len(ggeos),
             "max_rel_diff_vs_sequential": diff,
             "same_iterations_as_sequential": bool(all(a == c[0] for a, c in zip(its, seq_out)))}
    gb.close()
    for geo in ggeos:
        geo.close()
    return {"workload": f"{len(items)} starfish arrays, {min(nsrc)}-{max(nsrc)} quadrature nodes "
                        f"(log-uniform), {dens[0].shape[0]} densities each, p_qbx 8, p_fmm 15, {kern}",
            "targets_x_densities": ntot, "auto_ms": res["auto"], "auto_pick": auto_pick,
            "auto_targets_per_s": ntot / (res["auto"] * 1e-3),
            "persistent_ms": res["persistent"], "graph_ms": res["graph"],
            "sequential_ms": res["sequential"],
            "persistent_targets_per_s": ntot / (res["persistent"] * 1e-3),
            "graph_targets_per_s": ntot / (res["graph"] * 1e-3),
            "sequential_targets_per_s": ntot / (res["sequential"] * 1e-3),
            "persistent_tile": tile, "persistent_ctas": ctas, "persistent_streams": streams,
            "graph_streams": graph_streams,
            "max_rel_diff_vs_sequential": diff, "gmres": gmres}


# ---------------------------------------------------------------- learned order selection
LABELS = os.path.join(ROOT, "tests", "golden", "order_labels.npz")
LEARNED_EPS = 1e-8


def order_labels():
    """Oracle labels of the order-selection training set (written by
    tests/golden/make_order_labels.py): [n_centres, 2] float32 and metadata."""
    with np.load(LABELS) as f:
        meta = json.loads(str(f["meta"]))
        y = -f["codes"].astype(np.float32) / meta["codes_per_decade"]
    return y, meta


def run_learned(args, dev, g, flush):
    """Train the order-selection network on the oracle labels (features on the
    GPU, one geometry per training curve), then evaluate the workload at eps =
    1e-8 with the bound-driven orders, the learned FMM order (one p_fmm for
    the tree, the bound-driven order as cap and fallback; p_qbx from eps), the
    same with the mixed-precision tier of that eps, and per-centre learned
    QBX orders on top (the labels are one-sided truncation errors at the
    centre's base node, which overstate the two-sided on-surface error, so
    these orders are conservative).  Returns
    the report and, per mode, the outputs at a sample of targets of each kind
    (the CPU leg compares them with the oracle's direct QBX)."""
    import workloads
    from paper_1801_04070_gb300 import MLP, Geometry, params_default
    y, meta = order_labels()
    per = int(meta["centres_per_curve"])
    ncur = min(args.learned_curves, int(meta["n_curves"]))
    curves = workloads.order_training_curves(int(meta["n_curves"]), int(meta["curve_seed"]))
    t0 = time.perf_counter()
    X = []
    for i in range(ncur):
        gi = workloads.order_training_problem(curves[i], i)
        geo = Geometry(gi, params_default(p_qbx=int(meta["q_ref"]), p_fmm=int(meta["p_ref"]), n_max=32),
                       device=dev.index)
        geo.build()
        X.append(geo.features())
        geo.close()
    t_feat = time.perf_counter() - t0
    hold = max(1, ncur // 20)
    ntr = ncur - hold
    Xtr = np.concatenate(X[:ntr]).astype(np.float32)
    Ytr = y[:ntr * per]
    Xs = X[ntr:]
    Ys = [y[i * per:(i + 1) * per] for i in range(ntr, ncur)]
    geo0 = Geometry(workloads.order_training_problem(curves[0], 0), device=dev.index)
    m = MLP(geo0, seed=7)
    t0 = time.perf_counter()
    epochs = 20
    loss = m.train(Xtr, Ytr, epochs=epochs, batch=1024, lr=1e-3, seed=0)
    t_train = time.perf_counter() - t0
    Xv, Yv = np.concatenate(Xs), np.concatenate(Ys)
    pv = m.predict(Xv)
    r2 = [float(1 - ((pv[:, k] - Yv[:, k]) ** 2).mean() / Yv[:, k].var()) for k in (0, 1)]
    # margins from the held-out curves: the upper tail of the QBX residuals (per
    # centre); for the one FMM order, the largest excess of a curve's worst
    # measured error over its worst prediction
    margin_q = float(np.quantile(Yv[:, 0] - pv[:, 0], 0.995)) + 0.25
    margin_f = max(float(yy[:, 1].max() - m.predict(xx)[:, 1].max()) for xx, yy in zip(Xs, Ys)) + 0.5

    nt = len(g["tgt_xy"])
    rng = np.random.default_rng(12)
    modes = {}
    sample = {}
    mask = None
    for mode in ("bound", "learned", "learned+mixed", "learned per-centre"):
        prec = 1 if mode == "learned+mixed" else 0
        geo = Geometry(g, params_default(p_qbx=0, p_fmm=0, n_max=int(g["n_max"]), eps=LEARNED_EPS, precision=prec),
                       device=dev.index)
        geo.build()
        pb, qb = geo.params.p_fmm, geo.params.p_qbx
        sel_ms = None
        if mode == "bound":
            p, q = pb, qb
            kind, _ = geo.association()
            mask = np.zeros(nt, np.int32)
            for k in (0, 1, 2):
                ids = np.nonzero(kind == k)[0]
                if len(ids):
                    mask[rng.choice(ids, min(200, len(ids)), replace=False)] = 1
        else:
            ts = time.perf_counter()
            # "learned": the tree's FMM order from the network, the QBX order from eps;
            # "learned per-centre": each centre's QBX order from the network as well
            q_ref = int(meta["q_ref"]) if mode == "learned per-centre" else 0
            p, q = geo.learned_orders(m, LEARNED_EPS, margin_qbx=margin_q, margin_fmm=margin_f,
                                      q_ref=q_ref, p_ref=int(meta["p_ref"]), p_bound=pb)
            sel_ms = 1e3 * (time.perf_counter() - ts)
        import torch
        dmu = torch.tensor(g["density"], dtype=torch.float64, device=dev)
        out = torch.empty(nt, dtype=torch.float64, device=dev)
        for _ in range(2):
            geo.eval(args.kernel, dmu, out)
        ms = []
        for _ in range(3):
            flush.zero_()
            _, st = geo.eval(args.kernel, dmu, out, stats=True)
            ms.append(st.ms_total)
        torch.cuda.synchronize()
        vals = out.cpu().numpy()
        sample[mode] = vals[mask.astype(bool)]
        modes[mode] = {"p_fmm": int(p), "p_qbx_max": int(q), "eval_ms": statistics.median(ms),
                       "eval_targets_per_s": nt / (statistics.median(ms) * 1e-3),
                       "order_selection_ms": sel_ms, "precision": "MIXED" if prec else "FP64"}
        geo.close()
    geo0.close()
    m.close()
    rep = {"eps": LEARNED_EPS, "kernel": args.kernel, "training_curves": ntr, "held_out_curves": hold,
           "training_centres": int(len(Xtr)), "labels": "oracle (tests/golden/order_labels.npz)",
           "epochs": epochs, "final_loss": loss, "held_out_r2": {"qbx": r2[0], "fmm": r2[1]},
           "margins": {"qbx": margin_q, "fmm": margin_f}, "features_s": t_feat, "train_s": t_train,
           "inference": "BF16 mma.sync m16n8k16 (tensor cores), FP32 accumulation",
           "modes": modes, "qbx_labels": "one-sided truncation error at the centre's base node",
           "speedup_learned_vs_bound": modes["bound"]["eval_ms"] / modes["learned"]["eval_ms"],
           "speedup_learned_mixed_vs_bound": modes["bound"]["eval_ms"] / modes["learned+mixed"]["eval_ms"]}
    return rep, mask, sample


# ---------------------------------------------------------------- GPU arm
def run_gpu(args, rank, world, local):
    import torch

    from paper_1801_04070_gb300 import Geometry, lib, params_default
    from paper_1801_04070_gb300._lib import GeometryDesc, Stats, TreeInfo, _ptr

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = lib()
    grid = tuple(args.grid)
    g = workload(n_off=(1 << 20) * grid[0] * grid[1] // 256, grid=grid)
    nt = len(g["tgt_xy"])
    P, Q = int(g["p_fmm"]), int(g["p_qbx"])
    if args.precision == 0:
        prm = params_default(p_qbx=Q, p_fmm=P, n_max=int(g["n_max"]))
    else:
        prm = params_default(p_qbx=Q, p_fmm=P, n_max=int(g["n_max"]), eps=args.eps, precision=args.precision)
    stream = torch.cuda.current_stream(dev)

    # device-resident inputs
    keys = ("ref_b", "ref_u", "base_xy", "base_n", "up_xy", "up_n", "up_w", "panel_len")
    dg = {k: torch.tensor(np.ascontiguousarray(g[k], np.float64), device=dev) for k in keys}
    d_txy = torch.tensor(g["tgt_xy"], dtype=torch.float64, device=dev)
    d_ton = torch.tensor(g["tgt_onsurf"], dtype=torch.int32, device=dev)
    d_mu = torch.tensor(g["density"], dtype=torch.float64, device=dev)
    d_out = torch.empty(nt, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    ctx = C.c_void_p()
    assert L.gq_create(local, C.c_void_p(stream.cuda_stream), C.byref(ctx)) == 0
    desc = GeometryDesc(int(g["npanels"]), int(g["nb"]), int(g["nu"]), *[dg[k].data_ptr() for k in keys])
    geom = C.c_void_p()

    def chk(s):
        if s != 0:
            raise RuntimeError(L.gq_last_error(ctx).decode())

    chk(L.gq_geometry_create(ctx, C.byref(desc), C.byref(prm), C.byref(geom)))
    kern = 0 if args.kernel == "S" else 1
    st = Stats()

    def step():
        chk(L.gq_targets_set(geom, nt, d_txy.data_ptr(), d_ton.data_ptr()))
        chk(L.gq_build(geom))
        chk(L.gq_eval(geom, kern, d_mu.data_ptr(), d_out.data_ptr(), C.byref(st)))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    n0 = C.c_int64()
    chk(L.gq_context_launches(ctx, C.byref(n0)))
    step_ms, eval_ms, stage_ms = [], [], np.zeros(11)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            eval_ms.append(st.ms_total)
            stage_ms += np.array(st.ms_stage[:11])
    torch.cuda.synchronize()
    barrier(world)
    n1 = C.c_int64()
    chk(L.gq_context_launches(ctx, C.byref(n1)))
    launches = int(n1.value - n0.value)
    ms_step, value = replica_throughput(step_ms, nt, world, dev)
    stage_ms /= args.steps

    # ---- roofline of the dominant kernel (longest stage), FP64 ALU bound
    wrap = Geometry.__new__(Geometry)
    wrap.L, wrap._ctx, wrap._geom, wrap.nt = L, ctx, geom, nt
    info = TreeInfo()
    chk(L.gq_tree_info_get(geom, C.byref(info)))
    tp = (C.c_int(), C.c_int())
    chk(L.gq_tensor_paths(geom, C.byref(tp[0]), C.byref(tp[1])))
    tensor_paths = {"m2l": bool(tp[0].value), "m2qbxl": bool(tp[1].value)}
    wrap.info, wrap.nbox, wrap.nc, wrap.npt, wrap.nsrc = info, info.nbox, info.ncentres, info.npoint_targets, info.nsources
    model = work_model(wrap, P, Q, args.kernel)
    wrap._geom = wrap._ctx = None     # borrowed handles: released below, not by the wrapper
    dom = int(np.argmax(stage_ms))
    peak = C.c_double()
    peak_src = "measured (FP64 FMA probe, gq_probe_fma_peak)"
    if L.gq_probe_fma_peak(ctx, 0, C.byref(peak)) != 0 or not peak.value > 0:
        peak.value, peak_src = NOMINAL_FP64_TFLOPS, "nominal GB300 FP64"
    roof = None
    if dom in model:
        m = model[dom]
        flops = m["units"] * m["flops_per_unit"]
        achieved = flops / (stage_ms[dom] * 1e-3) / 1e12
        traffic = None
        tf = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tf):
            traffic = json.load(open(tf)).get(m["name"])
        # the other measured rates on this GPU: FP32 FMA, and the FP64 tensor cores (an FP64
        # contraction would belong there only if they beat the FP64 FMA rate)
        others = {}
        for what, name in ((1, "fp32_fma"), (2, "fp64_tensor_mma"), (3, "fp64_fma_and_mma_together")):
            v = C.c_double()
            if L.gq_probe_fma_peak(ctx, what, C.byref(v)) == 0:
                others[name] = v.value
        per_kernel = {}
        # FP64 instructions per unit measured by ncu (profiles/fp64_inst.json): the FP64 pipe
        # issues one instruction per slot whatever its kind, at the measured FMA peak / 2
        fi = os.path.join(ROOT, "profiles", "fp64_inst.json")
        inst = json.load(open(fi)) if os.path.exists(fi) else {}
        for i, mm in model.items():
            a = mm["units"] * mm["flops_per_unit"] / (stage_ms[i] * 1e-3) / 1e12
            per_kernel[mm["name"]] = {"achieved": a, "frac": a / peak.value, "ms_per_launch": float(stage_ms[i]),
                                      "units_per_launch": mm["units"], "flops_per_unit": mm["flops_per_unit"],
                                      "unit_of_work": mm["unit"]}
            if args.kernel == "S" and mm["name"] in inst:
                rate = mm["units"] * inst[mm["name"]] / (stage_ms[i] * 1e-3) / 1e12
                per_kernel[mm["name"]]["fp64_inst_per_unit"] = inst[mm["name"]]
                per_kernel[mm["name"]]["fp64_issue_frac"] = rate / (peak.value / 2)
        roof = {"bound": "alu", "kernel": m["name"], "achieved": achieved, "peak": peak.value,
                "unit": "TFLOP/s", "frac": achieved / peak.value, "traffic": traffic,
                "peak_source": peak_src, "units_per_launch": m["units"], "unit_of_work": m["unit"],
                "flops_per_unit": m["flops_per_unit"], "ms_per_launch": stage_ms[dom],
                "other_measured_tflops": others, "kernels": per_kernel}
    stage_report = {STAGE_NAMES[i]: round(float(stage_ms[i]), 4) for i in range(11)}
    for i, m in model.items():
        stage_report[STAGE_NAMES[i] + "_tflops"] = m["units"] * m["flops_per_unit"] / (stage_ms[i] * 1e-3) / 1e12

    # ---- end to end through the same ABI from pinned host memory
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.tensor(np.ascontiguousarray(g[k], np.float64)).pin_memory() for k in keys}
        h_txy = torch.tensor(g["tgt_xy"], dtype=torch.float64).pin_memory()
        h_ton = torch.tensor(g["tgt_onsurf"], dtype=torch.int32).pin_memory()
        h_mu = torch.tensor(g["density"], dtype=torch.float64).pin_memory()
        h_out = torch.empty(nt, dtype=torch.float64).pin_memory()
        hdesc = GeometryDesc(int(g["npanels"]), int(g["nb"]), int(g["nu"]), *[pin[k].data_ptr() for k in keys])
        h2d = sum(pin[k].numel() * 8 for k in keys) + h_txy.numel() * 8 + h_ton.numel() * 4 + h_mu.numel() * 8
        d2h = h_out.numel() * 8

        def step_e2e():
            hg = C.c_void_p()
            chk(L.gq_geometry_create(ctx, C.byref(hdesc), C.byref(prm), C.byref(hg)))
            chk(L.gq_targets_set(hg, nt, h_txy.data_ptr(), h_ton.data_ptr()))
            chk(L.gq_build(hg))
            chk(L.gq_eval(hg, kern, h_mu.data_ptr(), h_out.data_ptr(), None))
            L.gq_geometry_destroy(hg)

        step_e2e()
        torch.cuda.synchronize()
        barrier(world)
        t = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            step_e2e()
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        tot = max_over_ranks(sum(t), world, dev)
        e2e = {"value": world * nt * args.steps / tot, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": 1e3 * tot / args.steps}

    learned, l_mask, l_sample = None, None, None
    if args.learned and rank == 0 and args.precision == 0 and os.path.exists(LABELS):
        learned, l_mask, l_sample = run_learned(args, dev, g, flush)

    # ---- CPU oracle baseline (rank 0, N = 1): the whole workload on all host cores,
    # and a single-core figure on a sub-grid; the GPU result is compared with the
    # oracle at every target of the whole workload
    cpu = None
    rel_err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = host_cores()
        _, ref, nts, times, used = oracle_sample(args.kernel, threads=cores, g=g)
        gpu_vals = np.empty(nt)
        geo_full = C.c_void_p()
        chk(L.gq_geometry_create(ctx, C.byref(desc), C.byref(prm), C.byref(geo_full)))
        chk(L.gq_targets_set(geo_full, nt, d_txy.data_ptr(), d_ton.data_ptr()))
        chk(L.gq_build(geo_full))
        chk(L.gq_eval(geo_full, kern, d_mu.data_ptr(), d_out.data_ptr(), None))
        torch.cuda.synchronize()
        gpu_vals[:] = d_out.cpu().numpy()
        L.gq_geometry_destroy(geo_full)
        rel_err = float(np.abs(gpu_vals - ref).max() / np.abs(ref).max())
        if learned is not None:
            # the acceleration error (the Theorem's quantity, Sec. 4.5) of the modes
            # with one QBX order: their outputs against the oracle's unaccelerated QBX
            # (O1) of that order at the sampled targets of every kind
            import oracle
            t0 = time.perf_counter()
            qg = learned["modes"]["bound"]["p_qbx_max"]
            oracle.set_threads(cores)
            try:
                o1 = oracle.Oracle(g, oracle.default_params(g, p_qbx=qg))
                ref1 = o1.direct(args.kernel, g["density"], target_mask=l_mask)[l_mask.astype(bool)]
            finally:
                oracle.set_threads(1)
            sc = np.abs(ref1).max()
            for mode, v in l_sample.items():
                if learned["modes"][mode]["p_qbx_max"] != qg or mode == "learned per-centre":
                    continue
                err = float(np.abs(v - ref1).max() / sc)
                learned["modes"][mode]["err_vs_oracle_O1"] = err
                learned["modes"][mode]["meets_eps"] = err <= LEARNED_EPS
            learned["oracle_check"] = {"targets": int(l_mask.sum()), "s": time.perf_counter() - t0,
                                       "reference": f"oracle O1 (unaccelerated QBX) at p_qbx {qg}"}
        gs, _, nts1, times1, _ = oracle_sample(args.kernel)
        cpu = {"value": nts / times[0], "unit": UNIT, "cores": used, "kind": "oracle",
               "nproc": os.cpu_count(), "cpu_model": cpu_model(),
               "sample": (f"C oracle, build (serial) + {args.kernel} evaluation ({used} OpenMP threads) of the whole "
                          f"workload ({nts} targets), {times[0]:.1f} s"),
               "single_core": {"value": nts1 / times1[0], "unit": UNIT, "cores": 1,
                               "sample": (f"the same oracle on one core, a {SAMPLE_GRID[0]}x{SAMPLE_GRID[1]} sub-grid "
                                          f"({nts1} targets), {times1[0]:.1f} s")}}

    # ---- accuracy sweep: orders from eps, FP64 vs MIXED (FP64 translations) vs
    # MIXED_FMM (translations in FP32 pairs too) evaluation throughput
    sweep = None
    if args.sweep and rank == 0:
        sweep = []
        for eps in (1e-4, 1e-6, 1e-8, 1e-10, 1e-12):
            row = {"eps": eps}
            ref = None
            for prec, name in ((0, "fp64"), (1, "mixed"), (2, "mixed_fmm")):
                pr = params_default(p_qbx=0, p_fmm=0, n_max=int(g["n_max"]), eps=eps, precision=prec)
                sg = C.c_void_p()
                chk(L.gq_geometry_create(ctx, C.byref(desc), C.byref(pr), C.byref(sg)))
                chk(L.gq_targets_set(sg, nt, d_txy.data_ptr(), d_ton.data_ptr()))
                chk(L.gq_build(sg))
                sst = Stats()
                for _ in range(2):
                    chk(L.gq_eval(sg, kern, d_mu.data_ptr(), d_out.data_ptr(), C.byref(sst)))
                ms, sms = [], np.zeros(11)
                for _ in range(3):
                    flush.zero_()
                    chk(L.gq_eval(sg, kern, d_mu.data_ptr(), d_out.data_ptr(), C.byref(sst)))
                    ms.append(sst.ms_total)
                    sms += np.array(sst.ms_stage[:11]) / 3
                rp = params_default()
                chk(L.gq_geometry_params(sg, C.byref(rp)))
                row["p_qbx"], row["p_fmm"] = rp.p_qbx, rp.p_fmm
                row[name + "_eval_targets_per_s"] = nt / (statistics.mean(ms) * 1e-3)
                row[name + "_stage_ms"] = {STAGE_NAMES[i]: round(float(sms[i]), 3) for i in range(11)}
                out = d_out.clone()
                if ref is None:
                    ref = out
                else:
                    row[name + "_rel_err_vs_fp64_path"] = float((out - ref).abs().max() / ref.abs().max())
                L.gq_geometry_destroy(sg)
            sweep.append(row)

    # ---- level-restricted tree (Sec. 4.6 remark): the same workload with the
    # balanced tree; build and evaluation times, tree size and List 3 sizes of
    # leaves against the plain tree
    restricted = None
    if args.sweep and rank == 0 and args.precision == 0:
        def tree_stats(gh):
            bx = gh.boxes()
            Lh = gh.lists()
            leaf = np.ones(len(bx["level"]), bool)
            leaf[bx["parent"][bx["parent"] >= 0]] = False
            w3 = np.diff(Lh["WC"][0]) + np.diff(Lh["WF"][0])
            return int(len(bx["level"])), int(w3[leaf].max()), int(sum(len(Lh[k][1]) for k in Lh))

        out_plain = d_out.clone()
        res = {}
        # 0: the plain tree, 1: level-restricted, 2: disk-shaped TCR (appendix corrigendum)
        for lr in (0, 1, 2):
            pr = params_default(p_qbx=Q, p_fmm=P, n_max=int(g["n_max"]), level_restrict=1 if lr == 1 else 0,
                                tcr_shape=1 if lr == 2 else 0)
            sg = C.c_void_p()
            chk(L.gq_geometry_create(ctx, C.byref(desc), C.byref(pr), C.byref(sg)))
            chk(L.gq_targets_set(sg, nt, d_txy.data_ptr(), d_ton.data_ptr()))
            bms = []
            for _ in range(3):
                b0 = torch.cuda.Event(enable_timing=True)
                b1 = torch.cuda.Event(enable_timing=True)
                b0.record(stream)
                chk(L.gq_build(sg))
                b1.record(stream)
                b1.synchronize()
                bms.append(b0.elapsed_time(b1))
            sst = Stats()
            ems = []
            for _ in range(3):
                flush.zero_()
                chk(L.gq_eval(sg, kern, d_mu.data_ptr(), d_out.data_ptr(), C.byref(sst)))
                ems.append(sst.ms_total)
            gh = Geometry.__new__(Geometry)
            gh.L, gh._ctx, gh._geom, gh.nt = L, ctx, sg, nt
            ti = TreeInfo()
            chk(L.gq_tree_info_get(sg, C.byref(ti)))
            gh.info, gh.nbox, gh.nc, gh.npt, gh.nsrc = ti, ti.nbox, ti.ncentres, ti.npoint_targets, ti.nsources
            nb, w3max, nlist = tree_stats(gh)
            gh._geom = gh._ctx = None
            res[lr] = {"build_ms": statistics.median(bms), "eval_ms": statistics.median(ems), "boxes": nb,
                       "list3_max_per_leaf": w3max, "list_entries": nlist,
                       "stages_ms": {STAGE_NAMES[i]: round(float(sst.ms_stage[i]), 3) for i in range(11)}}
            if lr >= 1:
                res[lr]["max_rel_diff_vs_plain_tree"] = float((d_out - out_plain).abs().max() / out_plain.abs().max())
            L.gq_geometry_destroy(sg)
        restricted = {"plain": res[0], "level_restricted": res[1],
                      "eval_targets_per_s": nt / (res[1]["eval_ms"] * 1e-3),
                      "disk_tcr": res[2], "disk_tcr_eval_targets_per_s": nt / (res[2]["eval_ms"] * 1e-3)}
        d_out.copy_(out_plain)

    batched = run_batched(args, dev, stream) if args.batched else None

    L.gq_geometry_destroy(geom)
    L.gq_destroy(ctx)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "f64/f32 mixed", "data": "synthetic",
        "config": {"workload": g["name"], "kernel": args.kernel, "targets": nt,
                   "quadrature_nodes": int(len(g["up_w"])), "centres": int(info.ncentres),
                   "point_targets": int(info.npoint_targets), "boxes": int(info.nbox),
                   "p_qbx": Q, "p_fmm": P, "n_max": int(g["n_max"]), "t_f": 0.9,
                   "step": "gq_targets_set + gq_build + gq_eval", "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"replicas x{world}",
                   **({} if args.precision == 0 else {"precision": ("MIXED", "MIXED_FMM")[args.precision - 1],
                                                      "eps": args.eps})},
        "eval_only": {"value": world * nt / (statistics.mean(eval_ms) * 1e-3), "unit": UNIT,
                      "ms": statistics.mean(eval_ms)},
        "stages_ms": stage_report,
        "rel_err_vs_oracle": rel_err,
        "precision_sweep": sweep,
        "tree_variants": restricted,
        "batched": batched,
        "learned_orders": learned,
        "tensor_core_translations": tensor_paths,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_gpu(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
