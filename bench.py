"""Benchmark: one step = the whole hot path (transport, splat, DAS, envelope/log, loss, image
VJP, transposed DAS, splat adjoint, path adjoint) on the inclusion phantom (200k triangles in
12 regions, 1e5 scatterers, 128 elements, 16 plane waves, 1e6 rays per transmit, <= 8
interactions, 4096 samples, 256 x 1024 B-mode), synthetic data, FP32.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "path-segments/s"
UNIT = "segments/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="record", choices=["record", "recompute"])
    ap.add_argument("--rays", type=int, default=7813, help="rays per element and transmit")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU oracle sample budget")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-stages", action="store_true")
    ap.add_argument("--nee-stream", type=int, default=-1,
                    help="frame: US_OPT_NEE_STREAM (secondary rays on a second stream, %% of their grid; -1: default)")
    ap.add_argument("--rough", type=float, default=0.0,
                    help="frame: GGX roughness of every inclusion's interface (0: smooth, the default workload)")
    ap.add_argument("--shape-grad", action="store_true",
                    help="frame: the adjoint also returns dL/d(triangle vertices) (us_adjoint_shape)")
    ap.add_argument("--acq-grad", action="store_true",
                    help="frame: the adjoint also returns dL/d(c_bf, pitch, steering angles) (us_adjoint_acq)")
    ap.add_argument("--config", default="frame", choices=["frame", "batch", "serve", "optim", "cylinder"],
                    help="frame: one fwd+adj frame per step (the metric line); batch: a batch of scenes of "
                         "uneven size, batched vs one by one; serve: Poisson arrivals through the serving loop; "
                         "optim: iterations of the micro-batched inverse problem (Alg. 1)")
    ap.add_argument("--batch-n", type=int, default=256, help="scenes in the batch")
    ap.add_argument("--scale", type=float, default=1.0, help="ray/scatterer scale of batch and serve scenes")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: Poisson arrival rate, requests/s")
    ap.add_argument("--serve-seconds", type=float, default=60.0, help="serve: arrival window, s")
    ap.add_argument("--serve-scenes", type=int, default=32, help="serve: resident scenes requests draw from")
    ap.add_argument("--lanes", type=int, default=4, help="serve: concurrent lanes")
    ap.add_argument("--frame-only", action="store_true", help="frame config: skip the embedded batch and serve modes")
    ap.add_argument("--default-serve-seconds", type=float, default=20.0,
                    help="frame config: arrival window of the embedded serve measurement")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Replicas (one process per GPU, independent frames, no data-path collective): each rank
# renders its own realisation, the slowest rank's time sets the whole job's throughput.
def replica_seed(base, rank):
    return base + 1000 * rank


def max_over_ranks(x, world, device):
    """The largest x over the ranks (a collective on the process group; x itself with one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_rate(units_per_rank, world, seconds):
    return units_per_rank * world / seconds


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.stop = threading.Event()
        self.t = None

    def _run(self):
        while not self.stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0:
                    self.samples.append([v.strip() for v in out.stdout.strip().split(",")])
            except Exception:
                pass
            self.stop.wait(0.2)

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if len(s) > 3 + k and
                          s[3 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# algorithmic work per unit of each stage: a closest-hit query is a log-depth search over the
# scene's primitives (box tests per node visit plus a few primitive tests), counted in FP32 flop
FMA_LANES_PER_SM = 128  # FP32 lanes per SM (sm_100-class)


def alu_peak_tflops(pk, n_sms):
    mhz = pk.get("sm_max_mhz", 2070.0)
    return n_sms * FMA_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def traverse_flops_per_query(n_prims):
    # 2 log2(N) node visits x 2 box tests x 12 flop + 4 triangle tests x 30 flop
    return 2 * math.ceil(math.log2(max(2, n_prims))) * 2 * 12 + 4 * 30


def stage_work(stage, w, stats, n_prims):
    """(bound, algorithmic work per step in flop or bytes) of a stage."""
    acq, img = w["acq"], w["img"]
    taps = img["n_lines"] * img["n_depth"] * acq["n_elem"] * len(acq["angles"])
    rows = acq["n_elem"] * len(acq["angles"])
    if stage == "traverse":
        return "alu", stats["segments"] * traverse_flops_per_query(n_prims)
    if stage == "nee":
        return "alu", stats["nee_queries"] * traverse_flops_per_query(w["tris"].shape[0])
    if stage in ("path_adj", "nee_adj"):
        return "alu", 300 * stats["segments"] + 57 * 30 * stats["arrivals"]
    if stage in ("das", "das_adj"):
        return "alu", 25 * taps
    if stage in ("splat_sort", "splat_rows"):
        return "hbm", 16 * stats["arrivals"] + 4 * rows * acq["n_samples"]
    if stage == "interact":
        return "hbm", 96 * stats["segments"]
    return "hbm", 8 * img["n_lines"] * img["n_depth"]


def profile_traffic(name):
    """DRAM bytes per launch from the committed ncu summary `profiles/<name>.md`, or None when
    the kernels' sources changed since the capture (the summary records their hash)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    vals = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    srcs = vals.get("sources", "").split()
    h = hashlib.sha256()
    for f in srcs:
        fp = os.path.join(ROOT, "paper_2604_15017_gb300", "csrc", f)
        if not os.path.exists(fp):
            return None
        h.update(open(fp, "rb").read())
    if h.hexdigest()[:16] != vals.get("sources_sha256", ""):
        return None
    try:
        return float(vals["dram_bytes_per_step"]) / float(vals["launches_per_step"])
    except Exception:
        return None


# --------------------------------------------------------------------------------------------
def cpu_baseline(w, seconds, seed):
    """The FP64 oracle as it stands on the host cores: transport + splat of a contiguous sample
    of paths, grown until about `seconds` of work; path-segments/s."""
    from oracle import oracle as O

    nth = O.default_threads()
    sc = O.Scene.from_workload(w)
    n = 2000
    spent = 0.0
    segs = 0
    total_paths = 0
    lo = 0
    while spent < seconds:
        t0 = time.perf_counter()
        run = O.Run(sc, w["theta"], w["M"], w["acq"], seed, nth, lo, lo + n)
        run.rf()
        dt = time.perf_counter() - t0
        c = run.counters()
        spent += dt
        segs += c["segments"] + c["nee"]
        total_paths += n
        lo += n
        if dt < seconds / 8:
            n *= 2
    return dict(value=segs / spent, unit=UNIT, cores=nth, kind="oracle",
                sample="%d contiguous paths of the first transmit (of %d), transport + splat, %.1f s" %
                (total_paths, w["acq"]["n_rays"] * w["acq"]["n_elem"] * len(w["acq"]["angles"]), spent))


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O

    nth = O.default_threads()
    sc = O.Scene.from_workload(w)
    per_step = max(1.0, 20.0 / max(1, args.steps + args.warmup))
    # size the per-step sample from a probe
    n = 1000
    t0 = time.perf_counter()
    O.Run(sc, w["theta"], w["M"], w["acq"], w["seed"], nth, 0, n).rf()
    n = max(500, int(n * per_step / max(time.perf_counter() - t0, 1e-3)))
    lo = 0
    for _ in range(args.warmup):
        O.Run(sc, w["theta"], w["M"], w["acq"], w["seed"], nth, lo, lo + n).rf()
        lo += n
    segs = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = O.Run(sc, w["theta"], w["M"], w["acq"], w["seed"], nth, lo, lo + n)
        r.rf()
        c = r.counters()
        segs += c["segments"] + c["nee"]
        lo += n
    dt = time.perf_counter() - t0
    val = segs / dt
    sample = "%d paths per step (transport + splat) of the inclusion workload" % n
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "inclusions-200k-tris-1e5-scatterers-16tx-1e6rays"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": nth, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# --------------------------------------------------------------------------------------------
def _prepare_items(ctx, ws):
    """Upload the scenes and make each odd-index request a fwd+adj step against a target image
    rendered at perturbed parameters (outside any timed region)."""
    items = []
    for w in ws:
        sid = ctx.upload_workload(w)
        it = dict(scene=sid, theta=w["theta"], acq=w["acq"], img=w["img"], seed=w["seed"])
        if w["adjoint"]:
            _, bref = ctx.forward(sid, w["theta_target"], w["acq"], w["img"], seed=w["seed"])
            it["bref"] = bref.clone()
        items.append(it)
    return items


def _plain(ctx, it):
    """One request through the plain per-call API on the current stream."""
    if it.get("bref") is None:
        return ctx.forward(it["scene"], it["theta"], it["acq"], it["img"], seed=it["seed"])
    rf, b = ctx.forward(it["scene"], it["theta"], it["acq"], it["img"], seed=it["seed"], keep_record=True)
    loss, gb = ctx.loss(it["img"], b, it["bref"])
    return ctx.adjoint(it["scene"], it["theta"], it["acq"], it["img"], it["seed"], rf, gb)


def run_batch(args):
    print(json.dumps(measure_batch(args, args.steps, args.warmup)))


def measure_batch(args, steps, warmup, frame_rate=None):
    """Batched (lanes + CUDA graph, autotuned) vs one-by-one: path-segments/s over the batch.
    frame_rate (path-segments/s of the full single frame, fwd + adj) gives the reasoned bound on
    any launch organisation of these kernels, a persistent whole-batch launch included: the
    batch's segments at the rate the kernels reach when one frame fills the GPU."""
    import torch
    from paper_2604_15017_gb300 import phantoms as P, usrt

    ws = P.batch_workloads(n=args.batch_n, seed=4, scale=args.scale)
    ctx = usrt.Context(0)
    items = _prepare_items(ctx, ws)
    segs = 0
    for it in items:  # per-request work counts (also the plain path's warm-up)
        _plain(ctx, it)
        st_ = ctx.stats()
        segs += st_["segments"] + st_["nee_queries"]
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_plain = timed(lambda: [_plain(ctx, it) for it in items])
    batch = usrt.Batch(ctx, items)
    lanes, trav = batch.autotune()
    launches0 = ctx.launch_count()
    with ClockSampler(0) as clk:
        ms_batch = timed(batch.run)
    launches = (ctx.launch_count() - launches0) // (steps + warmup)
    side = torch.cuda.Stream()
    side.wait_stream(st)
    with torch.cuda.stream(side):
        batch.run(stream=side)
    st.wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        batch.run()
    ms_graph = timed(g.replay)
    n_paths = sum(w["acq"]["n_rays"] * w["acq"]["n_elem"] * len(w["acq"]["angles"]) for w in ws)
    best = min(ms_batch, ms_graph)
    out = {"metric": METRIC, "value": segs / (best * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": steps,
           "warmup": warmup, "ms_per_step": best, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch-%d-scenes-seed4-scale%g" % (args.batch_n, args.scale),
                      "step": "whole batch (even fwd, odd fwd+loss+adj)", "paths_per_step": n_paths,
                      "segments_per_step": segs, "autotuned_lanes": lanes, "autotuned_trav_blocks_per_sm": trav,
                      "l2": "per-step working set exceeds L2"},
           "plain": {"ms_per_step": ms_plain, "value": segs / (ms_plain * 1e-3)},
           "batched": {"ms_per_step": ms_batch, "value": segs / (ms_batch * 1e-3)},
           "graph": {"ms_per_step": ms_graph, "value": segs / (ms_graph * 1e-3)},
           "speedup_vs_plain": ms_plain / best, "gpu_launches": launches * steps, "clocks": clk.summary()}
    if frame_rate:
        out["full_gpu_bound_ms"] = segs / frame_rate * 1e3
        out["fraction_of_full_gpu_rate"] = out["full_gpu_bound_ms"] / best
    for it in items:
        ctx.release_scene(it["scene"])
    ctx.close()
    return out


def run_serve(args):
    print(json.dumps(measure_serve(args, args.serve_seconds)))


def measure_serve(args, seconds):
    """Poisson arrivals of requests on resident scenes (70 % fwd B-mode, 30 % fwd+loss+adj), served
    by the continuous-batching loop under a memory budget, against the plain sequential path."""
    import torch
    from paper_2604_15017_gb300 import phantoms as P, serve, usrt

    ws = P.batch_workloads(n=args.serve_scenes, seed=5, scale=args.scale)
    ctx = usrt.Context(0)
    items = _prepare_items(ctx, ws)
    for w, it in zip(ws, items):
        if it.get("bref") is None:  # every scene can take both kinds of request
            _, bref = ctx.forward(it["scene"], P.perturbed_theta(w["theta"], 99), w["acq"], w["img"], seed=w["seed"])
            it["bref_fa"] = bref.clone()
        else:
            it["bref_fa"] = it["bref"]
    torch.cuda.synchronize()
    times = serve.poisson_arrivals(args.rate, seconds, seed=5)
    rng = np.random.default_rng(5)
    arrivals = []
    n_adj = 0
    for t in times:
        it = dict(items[int(rng.integers(len(items)))])
        adj = rng.random() < 0.3
        n_adj += adj
        it["bref"] = it["bref_fa"] if adj else None
        it.pop("bref_fa")
        arrivals.append((t, it))
    srv = serve.Server(ctx, n_lanes=args.lanes, mem_budget_bytes=120 << 30)
    srv.warmup([a[1] for a in arrivals])
    with ClockSampler(0) as clk:
        served = srv.run(arrivals)
    seq = serve.run_sequential(ctx, arrivals)
    out = {"metric": "requests/s", "value": served["throughput"], "unit": "requests/s", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "serve-poisson-%grps-%gs-%d-scenes-seed5-scale%g" %
                      (args.rate, seconds, args.serve_scenes, args.scale), "lanes": args.lanes,
                      "requests": len(arrivals), "fwd_adj_requests": int(n_adj), "mem_budget_gb": 120},
           "served": served, "sequential": seq, "max_running": srv.max_running, "clocks": clk.summary()}
    for it in items:
        ctx.release_scene(it["scene"])
    ctx.close()
    return out


def run_optim(args):
    """Iterations of the micro-batched inverse problem (Alg. 1) on the differentiation workload
    (inclusion phantom, one 0-deg plane wave, K_max 4, 1e5 rays): two ray micro-batches per
    iteration, each forward + loss + adjoint in record mode, then one Adam step; every
    parameter free within +-20 %, target at theta0 +-5 %."""
    import torch
    from paper_2604_15017_gb300 import phantoms as P, optim, usrt

    w = P.differentiation()
    ctx = usrt.Context(0)
    sid = ctx.upload_workload(w)
    th0 = np.asarray(w["theta"], np.float64)
    prob = optim.InverseProblem(ctx, sid, th0, 0.8 * th0, 1.2 * th0, 0.01, optim.split_rays(w["acq"], 2), w["img"],
                                seed=w["seed"])
    prob.set_targets(w["theta_target"])
    for _ in range(args.warmup):
        prob.step()
    torch.cuda.synchronize()
    segs = 0
    for b, acq in enumerate(prob.batches):  # work per iteration (the realisations are fixed)
        ctx.forward(sid, prob.physical(), acq, w["img"], seed=prob.seed + b)
        st_ = ctx.stats()
        segs += st_["segments"] + st_["nee_queries"]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        losses = prob.run(args.steps)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
    out = {"metric": "optimiser iterations/s", "value": 1.0 / dt, "unit": "iterations/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "differentiation-inclusions-1tx-1e5rays-kmax4", "micro_batches": 2,
                      "parameters": int(th0.size), "segments_per_iteration": segs,
                      "step": "2 x (fwd + loss + adj, record mode) + Adam"},
           "path_segments_per_s": segs / dt, "loss_first": losses[0], "loss_last": losses[-1],
           "clocks": clk.summary()}
    print(json.dumps(out))
    ctx.close()


def run_cylinder(args):
    """Iterations of the shape-aware inverse problem on the hollow cylinder (the paper's
    experiment over R and Z, the wall rough with alpha 0.2 held fixed): radius 5.0 -> 5.15 mm and
    the wall density +8 %, two ray micro-batches of 750 rays per element; every iteration
    rebuilds and uploads the mesh, runs forward + loss + adjoint with the vertex gradient,
    contracts it with d tris / dR and takes an Adam step."""
    import torch
    from paper_2604_15017_gb300 import phantoms as P, optim, usrt

    w = P.with_roughness(P.hollow_cylinder(n_rays=1500), [0.0, 0.2, 0.0])
    ctx = usrt.Context(0)
    n_mat = len(w["theta"])
    shape = optim.ShapeModel(lambda q: (lambda m: (m[0], m[2][None]))(P.hollow_cylinder_mesh(radius=q[0])), w,
                             [w["radius"]])
    th0 = np.concatenate([w["theta"], [w["radius"]]])
    tgt = th0.copy()
    tgt[4] *= 1.08
    tgt[n_mat] = 5.15e-3
    lo, hi = th0.copy(), th0.copy()
    lo[4], hi[4] = 0.85 * th0[4], 1.15 * th0[4]
    lo[n_mat], hi[n_mat] = 4.7e-3, 5.3e-3
    prob = optim.InverseProblem(ctx, None, th0, lo, hi, 0.02, optim.split_rays(w["acq"], 2), w["img"],
                                seed=w["seed"], shape=shape)
    prob.set_targets(tgt)
    for _ in range(args.warmup):
        prob.step()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        losses = prob.run(args.steps)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
    th = prob.physical()
    out = {"metric": "optimiser iterations/s", "value": 1.0 / dt, "unit": "iterations/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": "hollow-cylinder-R5mm-at-15mm-rough-wall-0.2", "micro_batches": 2,
                      "free": ["wall density", "radius"], "triangles": int(len(w["tris"])),
                      "step": "mesh rebuild + 2 x (fwd + loss + adj with vertex gradient) + Adam"},
           "loss_first": losses[0], "loss_last": losses[-1], "radius_mm": float(th[n_mat]) * 1e3,
           "wall_density": float(th[4]), "clocks": clk.summary()}
    print(json.dumps(out))
    ctx.close()


def main():
    args = parse()
    from paper_2604_15017_gb300 import phantoms as P

    if args.impl == "ours" and args.config == "batch":
        run_batch(args)
        return
    if args.impl == "ours" and args.config == "serve":
        run_serve(args)
        return
    if args.impl == "ours" and args.config == "optim":
        run_optim(args)
        return
    if args.impl == "ours" and args.config == "cylinder":
        run_cylinder(args)
        return

    w = P.inclusions(n_rays=args.rays)
    if args.rough > 0.0:
        w = P.with_roughness(w, [0.0] + [args.rough] * (w["M"] - 1))
    if args.impl == "reference":
        run_reference(args, w)
        return
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2604_15017_gb300 import usrt

    ctx = usrt.Context(local)
    if args.nee_stream >= 0:
        ctx.set_option(usrt.OPT_NEE_STREAM, args.nee_stream)
    sid = ctx.upload_workload(w)
    acq, img = w["acq"], w["img"]
    seed = replica_seed(w["seed"], rank)  # independent frames per rank
    mode = usrt.MODE_RECORD if args.mode == "record" else usrt.MODE_RECOMPUTE
    # target image at the perturbed parameters (outside the timed region)
    _, bref = ctx.forward(sid, P.perturbed_theta(w["theta"], 7), acq, img, seed=seed)
    bref = bref.clone()
    theta = w["theta"]
    st = torch.cuda.current_stream()

    n_tris = int(w["tris"].shape[0])

    def adjoint(rf, gb):
        if args.acq_grad:
            return ctx.adjoint_acq(sid, theta, acq, img, seed, rf, gb, mode=mode)
        if args.shape_grad:
            return ctx.adjoint_shape(sid, theta, acq, img, seed, rf, gb, n_tris, mode=mode)
        return ctx.adjoint(sid, theta, acq, img, seed, rf, gb, mode=mode)[0], None

    def step():
        rf, b = ctx.forward(sid, theta, acq, img, seed=seed, keep_record=(mode == usrt.MODE_RECORD))
        loss, gb = ctx.loss(img, b, bref)
        gth, gacq = adjoint(rf, gb)
        return loss, gth

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats = ctx.stats()
    segs_per_step = stats["segments"] + stats["nee_queries"]

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = ctx.launch_count()
    ctx.profile(True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            loss, gth = step()
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    stages = ctx.profile_read()
    ctx.profile(False)
    gpu_launches = ctx.launch_count() - launches0
    ms = max_over_ranks(ms, world, "cuda")
    value = whole_job_rate(segs_per_step, world, ms * 1e-3)

    # forward only (transport, splat, DAS, envelope/log: the B-mode frame), same frame
    for _ in range(args.warmup):
        ctx.forward(sid, theta, acq, img, seed=seed)
    torch.cuda.synchronize()
    barrier()
    e0.record(st)
    for _ in range(args.steps):
        ctx.forward(sid, theta, acq, img, seed=seed)
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    ms_fwd = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    fwd = {"ms_per_step": ms_fwd, "value": whole_job_rate(segs_per_step, world, ms_fwd * 1e-3), "unit": UNIT,
           "frames_per_s": world * 1e3 / ms_fwd, "step": "fwd (transport + splat + DAS + envelope/log)"}

    # end to end through the public API with host buffers: B_ref host -> device each step,
    # loss and gradient device -> host each step
    bref_h = bref.cpu().pin_memory()
    gth_h = torch.empty(len(theta), dtype=torch.float32).pin_memory()
    gacq_h = torch.empty((n_tris, 9) if args.shape_grad else (2 + len(acq["angles"]),),
                         dtype=torch.float32).pin_memory()
    loss_h = torch.empty(1, dtype=torch.float32).pin_memory()
    bref_d = torch.empty_like(bref)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bref_d.copy_(bref_h, non_blocking=True)
        rf, b = ctx.forward(sid, theta, acq, img, seed=seed, keep_record=(mode == usrt.MODE_RECORD))
        loss, gb = ctx.loss(img, b, bref_d)
        gth, gacq = adjoint(rf, gb)
        gth_h.copy_(gth, non_blocking=True)
        if gacq is not None:
            gacq_h.copy_(gacq, non_blocking=True)
        loss_h.copy_(loss, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, "cuda")
    e2e = {"value": whole_job_rate(segs_per_step, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": bref_h.numel() * 4,
           "d2h_bytes_per_step": 4 * (len(theta) + 1 + (gacq_h.numel() if (args.acq_grad or args.shape_grad) else 0))}

    # roofline of the dominant stage, from its live CUDA-event time over the timed region
    n_prims = int(w["tris"].shape[0] + w["scat_pos"].shape[0])
    pk = peaks()
    dom = max(stages, key=lambda k: stages[k][0])
    dom_ms = stages[dom][0] / args.steps
    dom_launches = max(1, stages[dom][1] // args.steps)
    bound, work = stage_work(dom, w, stats, n_prims)
    if bound == "alu":
        achieved = work / (dom_ms * 1e-3) / 1e12
        peak = alu_peak_tflops(pk, torch.cuda.get_device_properties(local).multi_processor_count)
        unit = "TFLOP/s"
    else:
        achieved = work / (dom_ms * 1e-3) / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        unit = "GB/s"
    kernel_of = {"traverse": "k_traverse+k_march", "path_adj": "k_path_adjoint", "nee": "k_nee", "das": "k_das",
                 "splat_rows": "k_row_splat", "nee_adj": "k_nee_adjoint"}
    kern = kernel_of.get(dom, dom)
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": profile_traffic(kern.replace("+", "_") + "_inclusions"), "kernel": kern,
                "stage_ms_per_step": dom_ms, "launches_per_step": dom_launches,
                "work_per_step": work, "peak_source": "measured" if bound == "hbm" else
                "derived: SMs x 128 FP32 lanes x 2 x max SM clock (MEASURED_PEAKS sm_max_mhz)"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "inclusions-200k-tris-1e5-scatterers-16tx-1e6rays",
                      "step": "fwd+adj" + ("+acq" if args.acq_grad else ("+shape" if args.shape_grad else "")),
                      "roughness": args.rough,
                      "adjoint_mode": args.mode, "paths_per_step": stats["n_paths"],
                      "segments_per_step": stats["segments"], "nee_queries_per_step": stats["nee_queries"],
                      "arrivals_per_step": stats["arrivals"],
                      "paths_per_round": stats["live"][:w["acq"]["k_max"] + 1], "frames_per_s": world * 1e3 / ms,
                      "l2": "per-step working set (path queues + arrivals, ~4 GB) exceeds L2; scene BVH resident"},
           "clocks": clk.summary(), "e2e": e2e, "gpu_launches": gpu_launches, "roofline": roofline,
           "stages_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in stages.items() if v[1]}}
    out["fwd"] = fwd
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds, seed)
    ctx.release_scene(sid)
    ctx.close()
    if rank == 0 and world == 1 and not args.frame_only:
        # the batched (many scenes of uneven size) and served (Poisson arrivals) modes of the
        # metric, at their own configurations; one GPU
        out["batch"] = measure_batch(args, 2, 1, frame_rate=value)
        out["serve"] = measure_serve(args, args.default_serve_seconds)
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
