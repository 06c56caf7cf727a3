"""Benchmark of the SBR hot path.  Default workload: the large city.

Large city (seeded, synthetic): 60 x 60 blocks of extruded convex polygons (6-12 sides,
lognormal heights with median 25 m) on a 700 x 700 heightfield terrain (~1.07M triangles),
4 Tx x 4096 Rx, equiangular division n = 2200 (48,400,002 rays per Tx), up to 8
reflections, reception cone sqrt(3) * theta_launch, 16 refinement iterations with 9
sub-rays.  One step = ray generation + persistent trace with reception + double-count
removal + batched refinement + validity test + outputs, replayed as one captured CUDA
graph (one GPU).  Under torchrun (N GPUs) each rank traces a contiguous ray-id range of
every Tx, the ranks all-gather their reception records, and each removes double counts and
refines the paths of the (Tx, Rx) pairs it owns.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload instead.  `--workload canyon|office|shoebox|grad|...`
selects the other configurations.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-bounces/s and refined paths/s at <=0.01 deg AOD/AOA error; % of roofline"
SQ3 = float(np.sqrt(3.0))
# Per workload: the launch, the refinement, and two oracle samples: every `cpu_stride`-th
# ray id of every Tx for the CPU baseline line (about 10-30 s on 16 cores) and every
# `ref_stride`-th (from a per-step offset) for each step of the reference arm (a few seconds).
WORKLOADS = {
    "city": dict(workload="large city: 60x60 extruded polygons + 700^2 terrain (~1.07M tris), 4 Tx x 4096 Rx, "
                          "n=2200, order 8, alpha=sqrt(3), 16 refinement iterations, K=9",
                 gen="large_city", n_div=2200, max_order=8, alpha=SQ3, iters=16, K=9, target=0.0,
                 cpu_stride=7919, ref_stride=61027, steps=10),
    "canyon": dict(workload="urban canyon: 20x20 box city + ground (~10k tris), 1 Tx x 256 Rx, n=700, order 6, "
                            "alpha=sqrt(3), 6 refinement iterations, K=9",
                   gen="urban_canyon", n_div=700, max_order=6, alpha=SQ3, iters=6, K=9, target=0.0,
                   cpu_stride=4, ref_stride=4999, steps=300),
    "office": dict(workload="office: 40x30x4 m shell + 400 boxes (~55k tris), 16 Tx x 1024 Rx, n=128, order 6, "
                            "alpha=sqrt(3), refinement K=16 with early stop at 0.01 deg, cap 8",
                   gen="office", n_div=128, max_order=6, alpha=SQ3, iters=8, K=16, target=float(np.radians(0.01)),
                   cpu_stride=211, ref_stride=3001, steps=5),
    "shoebox": dict(workload="shoebox: 10x8x3 m room (12 tris), 1 Tx x 1 Rx, n=64, order 3, alpha=sqrt(3), "
                             "K=9, early stop at 0.01 deg (AOD and AOA), cap 8",
                    gen="shoebox_config", n_div=64, max_order=3, alpha=SQ3, iters=8, K=9,
                    target=float(np.radians(0.01)), cpu_stride=1, ref_stride=7, steps=300),
}
# the office at a quarter of its pairs (4 Tx x 1024 Rx, ~0.94M paths, the same many-path
# refinement kernels): the size the per-kernel ncu captures of the refinement run on
WORKLOADS["office_quarter"] = dict(WORKLOADS["office"], gen_kw={"ntx": 4}, steps=5,
                                   workload=WORKLOADS["office"]["workload"].replace("16 Tx", "4 Tx"))
WORKLOADS["canyon_diffraction"] = dict(WORKLOADS["canyon"], diffraction=True,
                                       workload=WORKLOADS["canyon"]["workload"] + ", plus order-1 diffraction")
DEFAULT_WORKLOAD = "city"
ACC_DEG = 0.01
# FLOPs per unit of the trace kernel (counted from the kernel source): a 4-wide node visit
# (four child slab tests of 6 FMA each), one watertight triangle test, one receiver
# candidate test
FLOP_NODE, FLOP_TRI, FLOP_RX = 48, 40, 20
L2_FLUSH_BYTES = 256 << 20

TRACE_SOURCES = ["paper_2208_10009_gb300/csrc/kernels_trace.cu", "paper_2208_10009_gb300/csrc/lattice_order.cuh",
                 "paper_2208_10009_gb300/csrc/sbr_device.cuh", "paper_2208_10009_gb300/csrc/sbr_internal.h"]
TRAFFIC_FILES = {"canyon": os.path.join(ROOT, "profiles", "trace_kernel_traffic.json"),
                 "city": os.path.join(ROOT, "profiles", "trace_kernel_traffic_large_city.json")}
UNFOLD_SOURCES = ["paper_2208_10009_gb300/csrc/kernels_unfold.cu", "paper_2208_10009_gb300/csrc/sbr_device.cuh",
                  "paper_2208_10009_gb300/csrc/sbr_internal.h"]
UNFOLD_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "unfold_bwd_traffic.json")


def source_hash(sources) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def trace_source_hash() -> str:
    return source_hash(TRACE_SOURCES)


def recorded_traffic(path, sources):
    """DRAM bytes per launch from a committed ncu record, or None when the kernel sources
    have changed since it was captured."""
    try:
        rec = json.load(open(path))
    except Exception:
        return None, None
    if rec.get("source_sha256") != source_hash(sources):
        return None, rec
    return rec["dram_bytes_per_launch"], rec


def fp32_peak(device: int):
    """The FP32 FMA rate of this GPU from the microbenchmark library (scalar fma.rn.f32 and
    packed fma.rn.f32x2, best of three launches each); None if it is not built."""
    import ctypes

    from paper_2208_10009_gb300 import build as _b
    if not os.path.exists(_b.SO_PROBE):
        return None
    lib = ctypes.CDLL(_b.SO_PROBE)
    lib.sbr_probe_fp32.restype = ctypes.c_int
    lib.sbr_probe_fp32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)]
    best = {}
    for packed in (0, 1):
        r = []
        for _ in range(3):
            f, ms = ctypes.c_double(), ctypes.c_float()
            if lib.sbr_probe_fp32(device, packed, 8, 200000, ctypes.byref(f), ctypes.byref(ms)) != 0:
                return None
            r.append(f.value / 1e12)
        best[packed] = max(r)
    form = "packed fma.rn.f32x2" if best[1] > best[0] else "scalar fma.rn.f32"
    return {"tflops": max(best.values()), "scalar_tflops": best[0], "packed_tflops": best[1], "form": form}


def recorded_issue(workload):
    """Issue-slot utilisation (sm__issue_active) of the trace kernel from the committed ncu
    record of this workload, while the kernel sources are unchanged since the capture."""
    path = TRAFFIC_FILES.get(workload)
    if not path:
        return None, None
    val, rec = recorded_traffic(path, TRACE_SOURCES)
    if val is None or rec is None or "issue_active_pct" not in rec:
        return None, rec
    return rec["issue_active_pct"], rec


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms during the timed region."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == len(self.FIELDS):
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time (every rank gets it); the time itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- oracle legs
def cpu_oracle_sample(W, sc, tx, rx, stride, offset=0):
    """The oracle (as it stands) on every `stride`-th ray id (from `offset`) of every Tx of
    the workload: trace, double-count removal, refinement, validity and outputs.  Returns
    (ray-bounces, accurate refined paths, seconds, rays, threads)."""
    import oracle
    S = oracle.Scene.from_generated(sc)
    n = W["n_div"]
    ids = np.arange(offset, 10 * n * n + 2, stride, dtype=np.int64)
    t0 = time.perf_counter()
    res = oracle.sbr_pipeline(S, tx, rx, n, W["max_order"], W["alpha"], W["K"], W["iters"], target=W["target"],
                              ray_ids=ids, diffraction=bool(W.get("diffraction", False)))
    dt = time.perf_counter() - t0
    good = sum(1 for p in res.paths if p["valid"] and p["ref_err"] <= np.radians(ACC_DEG))
    return res.nsegments, good, dt, len(ids) * len(tx), oracle.num_threads()


def oracle_accuracy(sc, tx, rx, recs):
    """Valid refined paths whose AOD and AOA are both within 0.01 deg of the exact path the
    oracle computes in FP64 for the same face sequence (the image method through the
    fixed-face unfolding; the exact diffraction point for diffraction paths).  Every valid
    path is checked."""
    import oracle
    S = oracle.Scene.from_generated(sc)
    v = recs[recs["valid"] == 1]
    refl = v[~((v["order"] == 1) & (v["faces"][:, 0] < 0))]
    diff = v[(v["order"] == 1) & (v["faces"][:, 0] < 0)]

    def unit(az, el):
        return np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)], -1)

    def angle(a, b):
        return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, -1))

    aod_err, aoa_err = [], []
    if len(refl):
        ex = oracle.unfold_many(S, refl["order"], refl["faces"], np.asarray(tx, np.float64)[refl["tx"]],
                                np.asarray(rx, np.float64)[refl["rx"]])
        aod_err.append(angle(refl["dir"], unit(ex[:, 4], ex[:, 5])))
        e = angle(unit(refl["aoa"][:, 0].astype(np.float64), refl["aoa"][:, 1].astype(np.float64)),
                  unit(ex[:, 6], ex[:, 7]))
        aoa_err.append(e)
    for r in diff:
        im = oracle.wedge_image(S, tx[r["tx"]], rx[r["rx"]], -1 - int(r["faces"][0]))
        aod_err.append(np.array([angle(r["dir"], im["aod_dir"])]))
        aoa_err.append(np.array([angle(unit(*r["aoa"].astype(np.float64)), unit(*im["aoa"]))]))
    if not aod_err:
        return dict(checked=0, accurate=0, worst_aod_deg=None, worst_aoa_deg=None)
    a, b = np.concatenate(aod_err), np.concatenate(aoa_err)
    ok = (a <= np.radians(ACC_DEG)) & (b <= np.radians(ACC_DEG))
    return dict(checked=int(len(a)), accurate=int(ok.sum()), worst_aod_deg=float(np.degrees(a.max())),
                worst_aoa_deg=float(np.degrees(b.max())))


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return
    from paper_2208_10009_gb300 import scenes
    W = WORKLOADS[args.workload]
    sc, tx, rx = getattr(scenes, W["gen"])(**W.get("gen_kw", {}))
    stride = W["ref_stride"]
    for w in range(args.warmup):
        cpu_oracle_sample(W, sc, tx, rx, stride, offset=w)
    segs = good = 0
    secs = 0.0
    nr = cores = 0
    for k in range(args.steps):
        s, g, dt, nrays, cores = cpu_oracle_sample(W, sc, tx, rx, stride, offset=args.warmup + k)
        segs += s
        good += g
        secs += dt
        nr += nrays
    value = segs / secs
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "ray-bounces/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": _config(W, sc, tx, rx, 1),
           "cpu_baseline": {"value": value, "unit": "ray-bounces/s", "cores": cores, "kind": "oracle",
                            "sample": f"every {stride}th ray id of every Tx per step ({nr // max(args.steps, 1)} "
                                      f"rays), brute-force FP64 trace + refine"},
           "refined_paths_per_s": good / secs,
           "e2e": {"value": value, "unit": "ray-bounces/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def _config(W, sc, tx, rx, world):
    n = W["n_div"]
    return dict({k: v for k, v in W.items() if k not in ("gen", "gen_kw", "cpu_stride", "ref_stride", "steps")},
                triangles=int(sc.nt), ntx=int(len(tx)), nrx=int(len(rx)), rays=int(len(tx) * (10 * n * n + 2)),
                l2="flushed (256 MiB write) between timed steps, outside the event-timed region",
                parallelism=f"ray-range shards x{world} (records all-gathered)" if world > 1 else "single GPU")


# ----------------------------------------------------------------------------- GPU arm
def _size_containers(ctx, api, scene, tx_dev, rxs, n, order, alpha, opts):
    """Record and path capacities from one synchronous launch (grown on overflow)."""
    cap_r, cap_p = 1 << 20, 1 << 18
    while True:
        probe = ctx.paths_create(cap_r, cap_p)
        try:
            ctx.launch(scene, tx_dev, rxs, probe, n, order, rx_angle_scale=alpha, **opts, sync=True)
            st = ctx.launch_stats(probe)
            break
        except api.SbrError as e:
            if e.status != 5:
                raise
            st = ctx.launch_stats(probe)
            cap_r = max(cap_r, 2 * st["records"], int(st["diffraction_candidates"] / 1.25) + 1)
            cap_p = max(cap_p, 2 * st["paths"])
        finally:
            probe.close()
    rec_cap = max(2 * st["records"], int(st["diffraction_candidates"] / 1.25) + 1, 1024)
    return ctx.paths_create(rec_cap, max(2 * st["paths"], 256)), st


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2208_10009_gb300 import api, autotune, scenes, shard

    rank, world, local = _dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = WORKLOADS[args.workload]
    opts = {"diffraction": bool(W.get("diffraction", False))}
    sc, tx, rx = getattr(scenes, W["gen"])(**W.get("gen_kw", {}))
    n, order, alpha, iters, K, target = (W[k] for k in ("n_div", "max_order", "alpha", "iters", "K", "target"))
    n_rays = 10 * n * n + 2
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = api.Context(local, stream=stream)
    scene = ctx.scene_from(sc)
    rxs = ctx.rx_upload(rx)
    tx_dev = torch.as_tensor(tx.astype(np.float32), device=dev)
    paths, st0 = _size_containers(ctx, api, scene, tx_dev, rxs, n, order, alpha, opts)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    recbuf = torch.empty(paths.record_cap * 64, dtype=torch.uint8, device=dev) if world > 1 else None

    def relaunch():
        if world > 1:
            shard.sharded_launch(ctx, scene, tx_dev, rxs, paths, n, order, rank, world, buf=recbuf,
                                 rx_angle_scale=alpha, **opts)
        else:
            ctx.launch(scene, tx_dev, rxs, paths, n, order, rx_angle_scale=alpha, **opts)

    # pick the batched kernel's launch shape on these paths (autotuner)
    if args.batch_shape:
        b, l, sm = (int(x) for x in args.batch_shape.split(","))
        tuned = {"block_threads": b, "lanes_per_path": l, "blocks_per_sm": sm, "ms": None}
    else:
        tuned = autotune.tune_batch_refine(ctx, scene, paths, relaunch, iters, K, target=target)
    shape = {k: tuned[k] for k in ("block_threads", "lanes_per_path", "blocks_per_sm")}

    def step():
        relaunch()
        ctx.batch_refine(scene, paths, iters, K, target=target, **shape)

    # one event-timed launch to split the step into kernels
    for _ in range(2):
        step()
    rng_kw = {"ray_range": shard.ray_range(n_rays, rank, world)} if world > 1 else {}
    ctx.launch(scene, tx_dev, rxs, paths, n, order, rx_angle_scale=alpha, **opts, **rng_kw, timing=True)
    st_t = ctx.launch_stats(paths)
    relaunch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.batch_refine(scene, paths, iters, K, target=target, **shape)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_refine = e0.elapsed_time(e1)

    # one GPU: the whole step as one CUDA graph; shards: eager steps (the record exchange
    # sizes its buffers on the host)
    if world == 1:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="thread_local"):
            step()
        run_step = graph.replay
    else:
        run_step = step
    for _ in range(args.warmup):
        flush.zero_()
        run_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t_wall = time.perf_counter()
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            run_step()
            b.record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), dev)
    clocks = clk.summary()
    st = ctx.launch_stats(paths)
    recs = ctx.query(paths)
    bounces = sum_over_ranks(st["segments"], dev)
    secs = ms / 1e3
    value = bounces * args.steps / secs
    # roofline of the dominant kernel (trace): algorithmic FP32 FLOPs / its event time
    flops = FLOP_NODE * st_t["node_visits"] + FLOP_TRI * st_t["tri_tests"] + FLOP_RX * st_t["rx_tests"]
    peaks, src = _peaks()
    sms = ctx.num_sms
    derived_tflops = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    probe = fp32_peak(local)
    peak_tflops = probe["tflops"] if probe else derived_tflops
    achieved = flops / (st_t["ms_trace"] / 1e3) / 1e12
    issue, issue_rec = recorded_issue(args.workload)
    traffic, traffic_rec = (recorded_traffic(TRAFFIC_FILES[args.workload], TRACE_SOURCES)
                            if args.workload in TRAFFIC_FILES and world == 1 else (None, None))

    # the three refinement forms on the same fresh rough paths: one plain launch over all
    # paths, one launch per (Tx, Rx) pair, and the batched persistent form as a graph
    forms = _refine_forms(ctx, scene, paths, relaunch, stream, iters, K, target, shape, len(tx), len(rx))
    e2e = _e2e(ctx, scene, tx, rx, n, order, alpha, iters, K, paths, args, shape, target, opts, rank, world, recbuf)

    nvalid = int(sum_over_ranks(int(np.sum(recs["valid"] == 1)), dev))
    out = {"metric": METRIC, "value": value, "unit": "ray-bounces/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
           "dtype": "f32 (f64 in final refinement iterations)", "data": "synthetic",
           "config": _config(W, sc, tx, rx, world),
           "paths": int(sum_over_ranks(len(recs), dev)), "valid_paths": nvalid,
           "refine_iters_hist": np.bincount(recs["iters"], minlength=iters + 1).tolist(),
           "fp64_paths": int(np.sum((recs["flags"] & 2) != 0)),
           "ray_bounces_per_step": int(bounces),
           "kernel_ms": {"raygen": st_t["ms_raygen"], "trace": st_t["ms_trace"], "dedup": st_t["ms_dedup"],
                         "diffract": st_t["ms_diffract"], "batch_refine": ms_refine},
           "diffraction": {"records": st_t["diffraction_records"], "wedge_tests": st_t["wedge_tests"],
                           "candidates": st_t["diffraction_candidates"],
                           "paths": int(np.sum((recs["order"] == 1) & (recs["faces"][:, 0] < 0))),
                           "valid_paths": int(np.sum((recs["order"] == 1) & (recs["faces"][:, 0] < 0) &
                                                     (recs["valid"] == 1)))} if opts["diffraction"] else None,
           "trace_counters": {k: st_t[k] for k in ("node_visits", "tri_tests", "rx_tests", "records", "segments")},
           "refine_forms": forms,
           "batch_refine_shape": dict(shape, tuned_ms=tuned["ms"]),
           "roofline": {"bound": "alu", "kernel": "trace_kernel", "achieved": achieved, "peak": peak_tflops,
                        "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                        "traffic_source": None if traffic is None else traffic_rec.get("capture"),
                        "peak_source": ("measured: FP32 FMA microbenchmark in this run (" + probe["form"] + "), "
                                        f"{probe['scalar_tflops']:.1f} TF/s scalar, {probe['packed_tflops']:.1f} packed"
                                        if probe else f"derived: {sms} SMs x 128 FP32 lanes x 2 x sm_max_mhz ({src} "
                                        "MEASURED_PEAKS.json)"),
                        "derived_peak": derived_tflops, "flops_per_launch": flops, "trace_ms": st_t["ms_trace"],
                        "issue_active": issue, "issue_source": None if issue is None else issue_rec.get("capture")},
           "clocks": clocks, "gpu_launches": _launches_per_step(opts, world) * args.steps,
           "wall_s": t_wall, "e2e": e2e}
    if rank == 0 and not args.no_cpu_baseline:
        acc = oracle_accuracy(sc, tx, rx, recs) if world == 1 else None
        if acc is not None:
            out["refined_paths_accurate"] = acc["accurate"]
            out["refined_paths_per_s"] = acc["accurate"] * args.steps / secs
            out["accuracy"] = dict(acc, judge="oracle FP64 exact path (image method) per face sequence, "
                                              "AOD and AOA both within 0.01 deg, every valid path")
            for f in forms.values():
                if isinstance(f, dict) and f.get("ms"):
                    f["refined_paths_per_s"] = acc["accurate"] / (f["ms"] / 1e3)
        stride = W["cpu_stride"]
        s, g, dt, nr, cores = cpu_oracle_sample(W, sc, tx, rx, stride)
        out["cpu_baseline"] = {"value": s / dt, "unit": "ray-bounces/s", "cores": cores, "kind": "oracle",
                               "sample": f"every {stride}th ray id of every Tx ({nr} rays, {s} ray-bounces): "
                                         f"brute-force FP64 trace, dedup, refine, validity; {dt:.1f} s",
                               "refined_paths_per_s": g / dt}
    if rank == 0:
        print(json.dumps(out), flush=True)
    for h in (paths, rxs, scene):
        h.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def _launches_per_step(opts, world):
    """Library kernels per step: raygen, trace (+3 diffraction: candidates, receivers,
    occlusion), 4 dedup, 4 batched refinement; shards add the record-count reset kernel."""
    return 10 + (3 if opts["diffraction"] else 0) + (1 if world > 1 else 0)


def _refine_forms(ctx, scene, paths, relaunch, stream, iters, K, target, shape, ntx, nrx, trials=3):
    """Host-timed refinement of the same fresh rough paths in three forms (each trial
    starts from a new launch): `plain` = one sbr_refine launch over all paths (one thread
    per path, static schedule); `per_pair` = one sbr_refine_pair launch per (Tx, Rx) pair
    from the host (asynchronous; the pair grouping and its one host read-back happen
    before the timed region); `batched_graph` = the persistent work-queue form replayed
    as a CUDA graph.  Results are identical across the forms."""
    import torch
    out = {}

    def timed(fn, prep=None):
        ts = []
        for _ in range(trials if ntx * nrx <= 4096 else 1):
            relaunch()
            if prep:
                prep()
            torch.cuda.synchronize()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(1e3 * (time.perf_counter() - t))
        return float(np.median(ts))

    out["plain"] = {"ms": timed(lambda: ctx.refine(scene, paths, iters, K, target=target))}

    def per_pair():
        for t in range(ntx):
            for r in range(nrx):
                ctx.refine_pair(scene, paths, t, r, iters, K, target=target)

    # grouping by pair (one synchronising read-back per launch) outside the timed region
    out["per_pair"] = {"ms": timed(per_pair, prep=lambda: ctx.refine_pair(scene, paths, 0, 0, 0, K)),
                       "launches": ntx * nrx}
    relaunch()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
        ctx.batch_refine(scene, paths, iters, K, target=target, **shape)
    out["batched_graph"] = {"ms": timed(g.replay)}
    return out


def _e2e(ctx, scene, tx, rx, n, order, alpha, iters, K, paths, args, shape, target, opts, rank, world, recbuf):
    """Same step through the public API with host inputs: Tx/Rx from pinned host memory (the
    receiver BVH is rebuilt from them), results read back to pinned host memory."""
    import torch

    from paper_2208_10009_gb300 import _binding as B
    from paper_2208_10009_gb300 import shard
    tx_h = torch.as_tensor(np.asarray(tx, np.float32)).pin_memory().numpy()
    rx_h = torch.as_tensor(np.asarray(rx, np.float32)).pin_memory().numpy()
    out_h = torch.empty(paths.path_cap * 128, dtype=torch.uint8).pin_memory().numpy().view(B.PATH_DTYPE)
    nbytes_out = 0

    def one():
        nonlocal nbytes_out
        rxs = ctx.rx_upload(rx_h)
        if world > 1:
            shard.sharded_launch(ctx, scene, tx_h, rxs, paths, n, order, rank, world, buf=recbuf,
                                 rx_angle_scale=alpha, **opts)
        else:
            ctx.launch(scene, tx_h, rxs, paths, n, order, rx_angle_scale=alpha, **opts)
        ctx.batch_refine(scene, paths, iters, K, target=target, **shape)
        got = ctx.query(paths, out_h)
        nbytes_out = len(got) * 128
        rxs.close()
        return ctx.launch_stats(paths)["segments"]

    for _ in range(max(1, args.warmup)):
        one()
    torch.cuda.synchronize()
    t = time.perf_counter()
    segs = 0
    for _ in range(args.steps):
        segs += one()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    dev = torch.device("cuda", ctx.device)
    dt = max_over_ranks(dt, dev)
    segs = sum_over_ranks(segs, dev)
    return {"value": segs / dt, "unit": "ray-bounces/s", "h2d_bytes_per_step": int(tx_h.nbytes + rx_h.nbytes),
            "d2h_bytes_per_step": int(nbytes_out), "note": "h2d counts the Tx/Rx coordinates handed over; the "
            "receiver BVH built from them is uploaded too"}


def run_grad(args):
    """Gradient workload: 1M fixed face-sequence paths (orders 1-6 from the canyon's refined
    paths, Tx/Rx jittered by +-1 m); one step = unfolding forward + adjoint (vector-Jacobian
    product) through the autograd Function.  HBM bound: per path 68 B read (Tx, Rx, az/el,
    order, 8 face ids) + 32 B written forward, 100 B read (+ the output gradient) + 32 B
    written (three input gradients) backward; the face-plane table stays in L2."""
    import torch

    from paper_2208_10009_gb300 import api, scenes
    from paper_2208_10009_gb300.autograd import unfold
    dev = torch.device("cuda", 0)
    sc, tx, rx = scenes.urban_canyon()
    ctx = api.Context(0)
    scene = ctx.scene_from(sc)
    rxs = ctx.rx_upload(rx)
    paths = ctx.paths_create(1 << 16, 1 << 14)
    ctx.launch(scene, tx, rxs, paths, 700, 6, rx_angle_scale=SQ3, sync=True)
    ctx.batch_refine(scene, paths, 6, 9)
    got = ctx.query(paths)
    base = got[(got["valid"] == 1) & (got["order"] >= 1)]
    P = 1 << 20
    rng = np.random.default_rng(4)
    b = base[rng.integers(0, len(base), P)]
    T = torch.tensor(scenes.jitter(rng, tx[b["tx"]], 1.0), dtype=torch.float32, device=dev, requires_grad=True)
    R = torch.tensor(scenes.jitter(rng, rx[b["rx"]], 1.0), dtype=torch.float32, device=dev, requires_grad=True)
    d = b["dir"]
    AE = torch.tensor(np.stack([np.arctan2(d[:, 1], d[:, 0]), np.arctan2(d[:, 2], np.hypot(d[:, 0], d[:, 1]))], -1),
                      dtype=torch.float32, device=dev, requires_grad=True)
    F = torch.tensor(b["faces"], dtype=torch.int32, device=dev)
    O = torch.tensor(b["order"], dtype=torch.int32, device=dev)
    G = torch.randn((P, 8), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        T.grad = R.grad = AE.grad = None
        out = unfold(ctx, scene, T, R, AE, F, O)
        out.backward(G)

    for _ in range(args.warmup):
        step()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for a, e in evs:
        flush.zero_()
        a.record()
        step()
        e.record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(e) for a, e in evs) / args.steps
    # kernel-only timing of the adjoint (the HBM-bound kernel): one ABI call per launch into
    # preallocated gradients, each behind an L2 flush and between its own pair of events,
    # with no host synchronisation inside the loop (the host queues ahead of the device, so
    # no host time falls between a launch's events); median of 10
    from paper_2208_10009_gb300.api import _ptr
    Td, Rd, AEd = T.detach(), R.detach(), AE.detach()
    gt, gr, ga = torch.empty_like(Td), torch.empty_like(Rd), torch.empty_like(AEd)

    def bwd_call():
        st = ctx.lib.sbr_unfold_bwd(ctx.handle, scene.handle, P, _ptr(Td), _ptr(Rd), _ptr(AEd), _ptr(F), _ptr(O),
                                    _ptr(G), _ptr(gt), _ptr(gr), _ptr(ga))
        if st != 0:
            raise RuntimeError(ctx.lib.sbr_last_error(ctx.handle))

    for _ in range(3):
        bwd_call()
    torch.cuda.synchronize()
    pairs = []
    for _ in range(10):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record()
        bwd_call()
        e1.record()
        pairs.append((e0, e1))
    torch.cuda.synchronize()
    times = [e0.elapsed_time(e1) for e0, e1 in pairs]
    bwd_ms = float(np.median(times))
    peaks, src = _peaks()
    bwd_bytes = P * (100 + 32)
    traffic, traffic_rec = recorded_traffic(UNFOLD_TRAFFIC_FILE, UNFOLD_SOURCES)
    print(json.dumps({"metric": "unfolding forward + adjoint paths/s", "value": P / (ms / 1e3), "unit": "paths/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                      "data": "synthetic", "config": {"workload": "1M fixed face-sequence paths of orders 1-6 from the "
                                                                  "urban canyon, Tx/Rx jittered +-1 m", "paths": P},
                      "roofline": {"bound": "hbm", "kernel": "unfold_bwd_staged_kernel", "achieved": bwd_bytes / (bwd_ms / 1e3) / 1e9,
                                   "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                                   "frac": bwd_bytes / (bwd_ms / 1e3) / 1e9 / peaks.get("hbm_gbs", 6800.0),
                                   "traffic": traffic,
                                   "traffic_source": None if traffic is None else traffic_rec.get("capture"),
                                   "peak_source": src, "bwd_ms": bwd_ms}}), flush=True)
    for h in (paths, rxs, scene):
        h.close()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["grad"])
    ap.add_argument("--batch-shape", default="",
                    help="block_threads,lanes_per_path,blocks_per_sm of the batched refinement (default: autotuned)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.steps is None:
        args.steps = 20 if args.workload == "grad" else WORKLOADS[args.workload]["steps"]
    if args.impl == "reference":
        if args.workload == "grad":
            args.workload = DEFAULT_WORKLOAD
        run_reference(args)
    elif args.workload == "grad":
        run_grad(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
