#!/usr/bin/env python3
"""Throughput of the neural in-scattering path: shaded points per second while rendering
1920x1080 frames of a 256^3 FP32 cloud (g 0.85, albedo 0.999) on one GB300.

One step = one pass of the whole path over the frame: density pyramid, transmittance
fields toward the light, phase table, per-pixel first hits, template gathers + SE, 3D-CNN,
backbone MLP and decode.  Inputs are resident in HBM when the timed region starts; L2 is
flushed (256 MB write) between timed steps, outside the timed events.  ``e2e`` times the
same step through the C ABI from page-locked host memory: the density upload and the
image read-back are inside its timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nis|reference]

``--impl reference`` times the FP64 CPU oracle on the host cores (a bounded sample of the
same frame per step).  Under torchrun each rank renders its own copy of the workload (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "shaded points/sec (1080p frame of a 256^3 FP32 cloud)"
UNIT = "points/s"

# Algorithmic work per shading point (one light): FLOPs of the dense layers (backbone 12
# blocks x 3 types, 3 merges, head) and of the 3D-CNN; bytes the gather must write.
MLP_FLOP_PER_POINT = 2 * (24 * (230 * 200 + 200 * 200) + 12 * (85 * 200 + 200 * 200)
                          + 3 * 400 * 200 + 600 * 200 + 200 * 200 + 200 * 3)
CNN_FLOP_PER_POINT = 2 * 12 * (63 * 16 * 27 + 5 * 16 * 16 * 27)
GATHER_BYTES_PER_POINT = 4 * (3 * 12 * 225 + 12 * 8 + 12 * 3 + 5 + 6)
# The gather's algorithmic bytes: the 5400 feature values a point needs (rho, phase and
# transmittance at 12 x 225 template points; FP32) written once, plus the density pyramid
# and the transmittance pyramid read once per frame (levels sum to ~8/7 of the finest).
GATHER_FEATURE_BYTES = 4 * 5400
GATHER_WRITTEN_BYTES_F32 = 12 * (232 * 4 + 3 * 2 * 240 * 2)


def gather_algorithmic_bytes(n_points: int, n: int) -> float:
    return GATHER_FEATURE_BYTES * n_points + 2 * (8.0 / 7.0) * n ** 3 * 4


def mlp_bytes_per_point(op: int, st: int) -> int:
    """Algorithmic HBM bytes per shading point of the dense layers as launched: every layer
    reads its operand and its epilogue inputs once and writes its outputs once.  op: bytes
    per operand element (6 for the FP32 split's three BF16 parts, 2 BF16, 1 e4m3); st:
    bytes per element of e and the running state h (4 FP32 with the split, else 2).  FC-1
    reads the features (+ 24 B of per-row configuration and SE scale) and h_prev, writes e
    and s = h_prev + e; FC-2 reads s and e, writes h (the chain's end: the merge input)."""
    width, total = 200, 0
    for d in (225, 225, 80):                         # rho, f, T feature widths
        for first, last in ((0, 7), (8, 11)):        # diffuse and highlight chains
            for k in range(first, last + 1):
                total += op * d + 24 + (st * width if k != first else 0) + st * width + op * width
                total += op * width + st * width + (op * width if k == last else st * width)
        total += op * 2 * width + op * width         # merge 400 -> 200
    total += op * 3 * width + op * width             # head 600 -> 200
    total += op * width + op * width                 # head 200 -> 200
    total += op * width + 12                         # head 200 -> 3, RGB out
    return total


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("nis", "reference"), default="nis")
    ap.add_argument("--workload", type=int, default=2, choices=(1, 2, 5))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-shear-warp", action="store_true")
    ap.add_argument("--no-paper-model", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=256)
    ap.add_argument("--no-plume-loop", action="store_true")
    ap.add_argument("--no-split-frame", action="store_true")
    ap.add_argument("--plume-march-frames", type=int, default=8)
    ap.add_argument("--oracle-sample", type=int, default=0, help=argparse.SUPPRESS)
    ap.add_argument("--ncu-case", choices=("f32", "bf16", "simt", "sweep", "frame_f32", "frame_bf16",
                                           "frame_fp8"),
                    help="small case for ncu captures: shade 32,768 points of the 64^3 fBm "
                         "volume twice at this precision (sweep: one shear-warp "
                         "transmittance of a 512^3 FP16 plume toward a light along x), print "
                         "nothing else")
    return ap.parse_args()


# ---- distributed plumbing -------------------------------------------------------------
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def dist_init(backend):
    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units: float, seconds: float, world: int):
    """Weak-scaling throughput: the units every rank processed over the slowest rank's
    time.  Returns (units per second, slowest rank's seconds)."""
    slowest = max_over_ranks(seconds, world)
    return sum_over_ranks(units, world) / slowest, slowest


# ---- clocks during the timed region --------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                                   default=None)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


def kernel_source_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2401_14051_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(family: str):
    """DRAM bytes per launch of a kernel family from a committed ncu summary, if the kernel
    source has not changed since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f).get(family)
    if not rec or rec.get("source_hash") != kernel_source_hash(rec["files"]):
        return None
    return rec


# ---- the oracle timed on the host (cpu_baseline and --impl reference) ------------------------
def oracle_sample(cfg, vol, weights, n_pixels: int, seed: int):
    """One bounded sample of the frame on the FP64 oracle: pyramid, lazily marched
    transmittance, phase-table columns, first hits of n_pixels random pixels, shading.
    Returns (shaded points, seconds)."""
    import oracle as O
    t0 = time.perf_counter()
    levels = O.build_pyramid(vol)
    o, d = O.camera_rays(cfg["camera"])
    rng = np.random.default_rng(seed)
    idx = rng.choice(o.shape[0] * o.shape[1], n_pixels, replace=False)
    oo, dd = o.reshape(-1, 3)[idx], d.reshape(-1, 3)[idx]
    hit, pts, _ = O.hit_search(levels[0], float(vol.max()), oo, dd)
    if hit.any():
        om = -dd[hit]
        tl = O.LazyTransmittance(levels, cfg["light"])
        table = O.phase_table(cfg["material"]["g"],
                              columns=O.table_columns(O.view_angle(om, cfg["light"])))
        O.shade_points(pts[hit], om, cfg["light"], levels, tl, table, weights, cfg["material"])
    return int(hit.sum()), time.perf_counter() - t0


def cpu_baseline(cfg, vol, weights, target_s: float = 12.0) -> dict:
    pts_total, secs, rounds, pixels = 0, 0.0, 0, 0
    while secs < target_s and rounds < 20:
        n, s = oracle_sample(cfg, vol, weights, 160, seed=1000 + rounds)
        pts_total += n
        secs += s
        rounds += 1
        pixels += 160
    return {"value": pts_total / secs if secs > 0 else 0.0, "unit": UNIT,
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{rounds} rounds x 160 random pixels of the 1920x1080 frame "
                      f"({pts_total} shading points): full pyramid, transmittance marched "
                      f"only at the voxels the sample's gathers touch, phase-table columns of "
                      f"the sample's angles; numpy float64 (BLAS may use all {os.cpu_count()} "
                      f"cores, elementwise work one)",
            "seconds": round(secs, 2)}


def oracle_single_thread(workload: int, n_pixels: int = 160) -> dict:
    """The oracle on one host thread: a child process with every BLAS / OpenMP pool limited
    to one thread runs one bounded sample of the frame."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", str(n_pixels),
                            "--workload", str(workload)], env=env, capture_output=True, text=True,
                           timeout=900)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError) as e:
        return {"value": None, "threads": 1, "error": str(e)[:200]}
    return {"value": d["points"] / d["seconds"] if d["seconds"] > 0 else None, "unit": UNIT,
            "threads": 1, "points": d["points"], "seconds": round(d["seconds"], 2),
            "sample": f"{n_pixels} random pixels of the same frame"}


def run_oracle_sample(args):
    """Child of oracle_single_thread: one sample, printed as JSON."""
    cfg = synth.config(args.workload)
    vol = cfg["volume"]()
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    n, secs = oracle_sample(cfg, vol, weights, args.oracle_sample, seed=2000)
    print(json.dumps({"points": n, "seconds": secs}), flush=True)


def compact_summary(line: dict) -> dict:
    """The line's figures in a few hundred bytes, placed last in the line (a log that keeps
    only the end of the output still has them)."""
    r = lambda x, n=3: None if x is None else round(float(x), n)
    out = {"f32": {"frame_ms": r(line["frame_ms"]), "mpts_s": r(line["value"] / 1e6),
                   "ms": line["step_breakdown_ms"],
                   "mlp_tensor_frac": r(line["roofline"]["frac"]) if line["roofline"]["bound"] == "tensor" else None,
                   "gather_hbm_frac": r(line["gather_roofline"]["frac"])},
           "e2e_mpts_s": r(line["e2e"]["value"] / 1e6)}
    for k in ("bf16", "fp8"):
        b = line.get(k)
        if b:
            out[k] = {"frame_ms": r(b["frame_ms"]), "mpts_s": r(b["value"] / 1e6),
                      "err_vs_f32": r(b["mean_rel_err_vs_fp32"], 5), "mlp_ms": b["step_breakdown_ms"]["mlp"],
                      "mlp_tensor_frac": r(b["roofline"]["frac"])}
    if line.get("paper_template_model"):
        p = line["paper_template_model"]
        out["paper_model_frame_ms"] = r(p.get("frame_ms"))
    sw = line.get("shear_warp")
    if sw:
        out["shear_warp_frame_ms"] = r(sw.get("frame_ms"))
    for k in ("serving", "serving_shear_warp"):
        sv = line.get(k)
        if sv:
            out[k] = {"req_s": r(sv.get("throughput_req_s")), "p50_ms": r(sv.get("p50_ms"), 1),
                      "p99_ms": r(sv.get("p99_ms"), 1), "batch_reqs": r(sv.get("mean_batch_requests"))}
            if sv.get("load_sweep"):
                out[k]["sweep"] = [[x["load"], x["throughput_req_s"], x["p50_ms"], x["p99_ms"],
                                    x["mean_batch_requests"]] for x in sv["load_sweep"]]
    sp = line.get("split_frame")
    if sp:
        out["split_frame"] = [sp["parts"], r(sp["frame_ms"]), sp.get("equals_whole_frame")]
    pl = line.get("plume1024_60f")
    if pl:
        out["plume_60f"] = {m: [pl[m]["frames"], pl[m]["frame_ms_median"], pl[m]["frame_ms_p99"]]
                            for m in ("shear_warp", "march") if m in pl}
    cb = line.get("cpu_baseline")
    if cb:
        out["oracle_pts_s"] = [r(cb.get("value")), r((cb.get("single_thread") or {}).get("value"))]
    return out


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    cfg = synth.config(args.workload)
    vol = cfg["volume"]()
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    for i in range(args.warmup):
        oracle_sample(cfg, vol, weights, 96, seed=i)
    pts, secs = 0, 0.0
    for i in range(args.steps):
        n, s = oracle_sample(cfg, vol, weights, 96, seed=100 + i)
        pts += n
        secs += s
    value = pts / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": cfg["name"], "sample_per_step": "96 random pixels"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps x 96 random pixels ({pts} shading points)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- the CUDA path ------------------------------------------------------------------------
def _time_builds(ctx, v, light, method, reps, stream):
    import torch
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.build_transmittance(v, light, 0.6, method=method)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def run_shear_warp(args, nis, ctx, v, w, cfg, img, hitmask, flush, stream, n_points) -> dict:
    """The frame of the main measurement with the transmittance from shear-warp rays
    instead of the march: build times of both, frame throughput, and the frame's
    difference from the marched FP32 frame."""
    import torch
    light, mat, cam = cfg["light"], cfg["material"], cfg["camera"]
    march_ms = _time_builds(ctx, v, light, nis.TRANSMITTANCE_MARCH, 3, stream)
    _time_builds(ctx, v, light, nis.TRANSMITTANCE_SHEAR_WARP, 1, stream)
    sw_ms = _time_builds(ctx, v, light, nis.TRANSMITTANCE_SHEAR_WARP, 5, stream)
    img_sw = torch.empty_like(img)

    def step():
        ctx.build_pyramid(v)
        lt = ctx.build_transmittance(v, light, 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
        ctx.build_phase_table(mat["g"])
        ctx.render_frame(v, lt, w, mat, cam, out=img_sw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    a_sw, a_32 = img_sw[hitmask].double(), img[hitmask].double()
    floor = 5e-2 * a_32.abs().amax(dim=0, keepdim=True)
    e = (a_sw - a_32).abs() / torch.maximum(a_32.abs(), floor)
    return {"value": n_points * args.steps / (sum(times) / 1e3), "unit": UNIT,
            "frame_ms": sum(times) / args.steps,
            "transmittance_build_ms": {"march": round(march_ms, 4), "shear_warp": round(sw_ms, 4)},
            "mean_rel_err_vs_marched_frame": float(e.mean()),
            "max_rel_err_vs_marched_frame": float(e.max())}


def run_paper_model(args, nis, ctx, v, cfg, flush, stream, n_points) -> dict:
    """The same frame shaded by the paper-template model (the paper's own template point
    sets and volume-level transmission feature): dense layers FP32-accurate on the tensor
    cores (three-way BF16 split) and, for comparison, on FP32 FFMA."""
    import torch
    W = synth.make_weights_paper(cfg["weights_seed"], cfg["sigma_max"])
    light, mat, cam = cfg["light"], cfg["material"], cfg["camera"]
    img = torch.empty((cam["height"], cam["width"], 3), dtype=torch.float32, device=flush.device)
    out = {"model": "paper templates (194 + 72 points), level-weighted transmission"}
    for name, prec in (("f32", nis.PREC_F32), ("f32_ffma", nis.PREC_F32_SIMT)):
        w = ctx.load_weights(synth.pack_weights_paper(W), prec)

        def step():
            ctx.build_pyramid(v)
            lt = ctx.build_transmittance(v, light, 0.6)
            ctx.render_frame(v, lt, w, mat, cam, out=img)

        step()
        torch.cuda.synchronize()
        ctx.profile(True)
        times = []
        steps = max(2, min(args.steps, 3))
        for _ in range(steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ctx.profile(False)
        fam = {f: ctx.profile_read(f) for f in nis.FAMILIES}
        ctx.release(w)
        res = {"value": n_points * steps / (sum(times) / 1e3), "unit": UNIT,
               "frame_ms": sum(times) / steps, "steps": steps,
               "step_breakdown_ms": {f: round(fam[f][0] / steps, 4) for f in nis.FAMILIES}}
        if name == "f32":
            out.update(res)
        else:
            out["ffma"] = res
    return out


def plume_transmittance(nis, local: int) -> dict:
    """Transmittance of the 1024^3 FP16 plume toward its light (all 11 levels) by the march
    and by shear-warp rays: one build each (timed after a warm-up build of the latter) and
    the level-0 difference."""
    import torch
    cfg = synth.config(5)
    vol = synth.plume_volume_torch(1024, 9, 128.0, device=f"cuda:{local}")
    ctx = nis.Context(local)
    stream = torch.cuda.current_stream()
    v = ctx.upload_volume(vol)
    ctx.build_pyramid(v)
    ctx.sync(timeout_ms=120000)
    march_ms = _time_builds(ctx, v, cfg["light"], nis.TRANSMITTANCE_MARCH, 1, stream)
    _time_builds(ctx, v, cfg["light"], nis.TRANSMITTANCE_SHEAR_WARP, 1, stream)
    sw_ms = _time_builds(ctx, v, cfg["light"], nis.TRANSMITTANCE_SHEAR_WARP, 2, stream)
    a = ctx.build_transmittance(v, cfg["light"], 0.6)
    b = ctx.build_transmittance(v, cfg["light"], 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
    d = (ctx.copy_transmittance(a, v, 0) - ctx.copy_transmittance(b, v, 0)).abs()
    out = {"volume": "1024^3 float16 plume, 11 levels",
           "transmittance_build_ms": {"march": round(march_ms, 3), "shear_warp": round(sw_ms, 3)},
           "level0_max_abs_dT": float(d.max()), "level0_mean_abs_dT": float(d.mean())}
    del d
    ctx.close()
    return out


def run_plume_loop(args, nis, local: int) -> dict:
    """The 1024^3 FP16 plume (11 levels) rendered as an animation at 3840x2160 with the BF16
    network: the light turns 6 degrees a frame and its transmittance is rebuilt every frame,
    by shear-warp rays for 60 frames and by the exact march for the first
    args.plume_march_frames (about 1.1 s per build: O(N^4)).  Each frame's transmittance
    build and its shading (pairs, first hits, gathers, CNN, network, image) are timed with
    CUDA events; the light of the previous frame is released before the next is built."""
    import torch
    cfg = synth.config(5)
    dev = f"cuda:{local}"
    vol = synth.plume_volume_torch(1024, 9, 128.0, device=dev)
    ctx = nis.Context(local)
    stream = torch.cuda.current_stream()
    v = ctx.upload_volume(vol)
    del vol
    ctx.build_pyramid(v)
    w = ctx.load_weights(synth.pack_weights(synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])),
                         nis.PREC_BF16)
    mat, cam = cfg["material"], cfg["camera"]
    ctx.build_phase_table(mat["g"])
    img = torch.empty((cam["height"], cam["width"], 3), dtype=torch.float32, device=dev)
    out = {"volume": "1024^3 float16 plume, 11 levels", "image": "3840x2160 perspective",
           "precision": "bf16", "light": "turns 6 degrees per frame about +y"}
    for name, method, frames in (("shear_warp", nis.TRANSMITTANCE_SHEAR_WARP, 60),
                                 ("march", nis.TRANSMITTANCE_MARCH, args.plume_march_frames)):
        if frames <= 0:
            continue
        lt = ctx.build_transmittance(v, synth.rotating_light(cfg["light"], -1), 0.6, method=method)
        ctx.render_frame(v, lt, w, mat, cam, out=img)               # warm-up frame
        ctx.sync(timeout_ms=600000)
        ctx.release(lt)
        build, shade = [], []
        for f in range(frames):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            lt = ctx.build_transmittance(v, synth.rotating_light(cfg["light"], f), 0.6, method=method)
            ev[1].record(stream)
            ctx.render_frame(v, lt, w, mat, cam, out=img)
            ev[2].record(stream)
            ev[2].synchronize()
            build.append(ev[0].elapsed_time(ev[1]))
            shade.append(ev[1].elapsed_time(ev[2]))
            ctx.release(lt)
        frame = np.array(build) + np.array(shade)
        out[name] = {"frames": frames, "frame_ms_median": round(float(np.median(frame)), 3),
                     "frame_ms_p99": round(float(np.percentile(frame, 99)), 3),
                     "build_ms_median": round(float(np.median(build)), 3),
                     "shade_ms_median": round(float(np.median(shade)), 3)}
    ctx.close()
    return out


def run_split_frame(args, nis, ctx, v, w, cfg, img, flush, stream, world: int) -> dict:
    """Strong scaling of one frame: the whole step (pyramid, transmittance, phase table,
    hits) replicated on every rank, the frame's shading points split into `world` equal
    ranges (one per rank), the ranges gathered to rank 0 and scattered into the image there.
    Per frame: barrier, synchronise, time on the host clock, max over ranks.  Rank 0 also
    checks the assembled image against its own whole-frame render, bit for bit."""
    import torch
    from paper_2401_14051_gb300 import frame_split
    mat, cam, light = cfg["material"], cfg["camera"], cfg["light"]
    dev = img.device
    cap = nis.part_capacity(cam["width"] * cam["height"], world)
    bufs = (torch.empty((cap, 3), dtype=torch.float32, device=dev),
            torch.empty((cap,), dtype=torch.int32, device=dev))
    out = torch.empty_like(img)

    def frame():
        ctx.build_pyramid(v)
        lt = ctx.build_transmittance(v, light, 0.6)
        ctx.build_phase_table(mat["g"])
        return frame_split.render_frame_split(ctx, v, lt, w, mat, cam, out=out, part_bufs=bufs)

    for _ in range(args.warmup):
        frame()
    times, info = [], None
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        _, info = frame()
        torch.cuda.synchronize()
        times.append(max_over_ranks(time.perf_counter() - t0, world))
    res = {"parts": world, "scaling": "strong", "precision": "f32",
           "frame_ms": 1e3 * sum(times) / len(times),
           "points_per_s": info["n_hits"] * len(times) / sum(times),
           "max_part_points": info["rows"], "timer": "host clock around a synchronised frame, "
           "max over ranks", "exchange": "torch.distributed gather of 16 B per point to rank 0"}
    if world == 1 or dist_env()[0] == 0:
        res["equals_whole_frame"] = bool(torch.equal(out, img))
    return res


def serving_volumes(args, local: int):
    import torch
    reqs = synth.serving_requests(args.serving_requests)
    t0 = time.perf_counter()
    # page-locked host volumes: the library reads them in place over NVLink-C2C
    pinned = [torch.from_numpy(synth.serving_volume(r["n"], r["seed"], 32.0,
                                                     device=f"cuda:{local}")).pin_memory()
              for r in reqs]
    torch.cuda.synchronize()
    return reqs, pinned, time.perf_counter() - t0


def run_serving(args, nis, blob, local: int, workload, method: int = 0, sweep=()) -> dict:
    """256 Poisson-arriving render requests (grids 128^3-512^3 FP16, images 256^2 to 1080p,
    g and albedo per request) through the continuous-batching server under a 120 GB HBM
    budget, BF16 network.  The arrival rate targets ~70 % GPU load from a measured
    back-to-back service time.  `method`: the server's transmittance method.  `sweep`: further
    loads (fractions of the service rate) run on the first 128 requests."""
    reqs, pinned, gen_s = workload
    vols = [t.numpy() for t in pinned]
    ctx = nis.Context(local, torch_allocator=False)
    w = ctx.load_weights(blob, nis.PREC_BF16)
    budget = 120 * 2 ** 30
    # service time: 8 requests back to back on their own server
    srv = nis.Server(ctx, w, budget_bytes=budget, max_batch_points=65536, max_inflight=16,
                     transmittance_method=method)
    t0 = time.perf_counter()
    ids = [srv.submit(vols[i], 10 ** 6 + i, reqs[i]["light"], 0.6, reqs[i]["material"],
                      reqs[i]["camera"]) for i in range(8)]
    for rid in ids:
        srv.wait(rid)
    service_s = (time.perf_counter() - t0) / 8
    srv.close()

    def arrivals(load: float, n: int) -> dict:
        rate = load / service_s
        rng = np.random.default_rng(7)
        gaps = rng.exponential(1.0 / rate, size=n)
        srv = nis.Server(ctx, w, budget_bytes=budget, max_batch_points=65536, max_inflight=32,
                         transmittance_method=method)
        ids = []
        due = time.perf_counter()
        for i, r in enumerate(reqs[:n]):
            due += gaps[i]
            delay = due - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            ids.append(srv.submit(vols[i], 1 + i, r["light"], 0.6, r["material"], r["camera"]))
        for rid in ids:
            srv.wait(rid)
        st = srv.stats()
        srv.close()
        st["rate"] = rate
        return st

    st = arrivals(0.7, len(reqs))
    out_sweep = []
    for load in sweep:
        s2 = arrivals(load, min(128, len(reqs)))
        out_sweep.append({"load": load, "requests": s2["completed"] + s2["failed"],
                          "arrival_req_s": round(s2["rate"], 2),
                          "throughput_req_s": round(s2["completed"] / s2["span_seconds"], 2),
                          "p50_ms": round(s2["p50_ms"], 1), "p99_ms": round(s2["p99_ms"], 1),
                          "mean_batch_requests": round(s2["mean_batch_requests"], 3),
                          "failed": s2["failed"]})
    ctx.close()
    pixels = sum(r["camera"]["width"] * r["camera"]["height"] for r in reqs)
    out = {"requests": len(reqs), "precision": "bf16", "hbm_budget_gb": 120,
           "transmittance": "shear-warp" if method else "march",
           "arrival": f"Poisson, {st['rate']:.1f} req/s (0.7 / back-to-back service time "
                      f"{1e3 * service_s:.1f} ms)",
           "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
           "max_ms": st["max_ms"], "throughput_req_s": st["completed"] / st["span_seconds"],
           "points_per_s": st["points_shaded"] / st["span_seconds"],
           "pixels": pixels, "completed": st["completed"], "failed": st["failed"],
           "mean_batch_points": st["mean_batch_points"],
           "mean_batch_requests": st["mean_batch_requests"],
           "cache": {"volume_hits": st["volume_hits"], "volume_misses": st["volume_misses"],
                     "light_hits": st["light_hits"], "light_misses": st["light_misses"],
                     "evictions": st["evictions"]},
           "peak_gb": st["peak_bytes"] / 2 ** 30, "volume_generation_s": round(gen_s, 1)}
    if out_sweep:
        out["load_sweep"] = out_sweep
    return out


def run_nis(args):
    import torch
    rank, local, world = dist_init("nccl")
    torch.cuda.set_device(local)
    from paper_2401_14051_gb300 import nis
    if not os.path.exists(nis.LIB_PATH):
        from paper_2401_14051_gb300 import build
        build.build()
    dev = torch.device(f"cuda:{local}")
    cfg = synth.config(args.workload)
    vol_np = cfg["volume"]()
    weights = synth.make_weights(cfg["weights_seed"], cfg["sigma_max"])
    blob = synth.pack_weights(weights)
    mat, cam, light = cfg["material"], cfg["camera"], cfg["light"]
    ctx = nis.Context(local)
    density = torch.from_numpy(vol_np).to(dev)
    v = ctx.upload_volume(density)
    w = ctx.load_weights(blob)
    w_bf16 = ctx.load_weights(blob, nis.PREC_BF16)
    w_fp8 = ctx.load_weights(blob, nis.PREC_FP8)
    img = torch.empty((cam["height"], cam["width"], 3), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step(weights_handle=w, out=img):
        ctx.build_pyramid(v)
        lt = ctx.build_transmittance(v, light, 0.6)
        ctx.build_phase_table(mat["g"])
        ctx.render_frame(v, lt, weights_handle, mat, cam, out=out)
        return lt

    for _ in range(args.warmup):
        step()
    ctx.sync(timeout_ms=120000)
    hit, _, _ = ctx.find_hits(v, cam)
    n_points = int(hit.sum().item())

    # ---- device-resident timed region
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True)
    launches0 = nis.kernel_launches()
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    launches = nis.kernel_launches() - launches0
    ctx.profile(False)
    barrier(world)
    clk = clocks.stop()
    fam = {f: ctx.profile_read(f) for f in nis.FAMILIES}
    value, total_s = whole_job_rate(n_points * args.steps, sum(times) / 1e3, world)
    total_ms = 1e3 * total_s
    ms_per_step = total_ms / args.steps

    # ---- the same frames with the dense layers in BF16 on the tensor cores
    img_bf = torch.empty_like(img)
    for _ in range(args.warmup):
        step(w_bf16, img_bf)
    torch.cuda.synchronize()
    ctx.profile(True)
    times_bf = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(w_bf16, img_bf)
        e1.record(stream)
        e1.synchronize()
        times_bf.append(e0.elapsed_time(e1))
    ctx.profile(False)
    fam_bf = {f: ctx.profile_read(f) for f in nis.FAMILIES}
    value_bf, total_bf = whole_job_rate(n_points * args.steps, sum(times_bf) / 1e3, world)
    total_bf *= 1e3
    hitmask = hit.bool()
    a_bf, a_32 = img_bf[hitmask].double(), img[hitmask].double()
    floor = 5e-2 * a_32.abs().amax(dim=0, keepdim=True)
    e_bf = ((a_bf - a_32).abs() / torch.maximum(a_32.abs(), floor))
    peaks_bf = measured_peaks()
    mlp_ms, mlp_n = fam_bf["mlp"]
    mlp_tf = MLP_FLOP_PER_POINT * n_points * args.steps / (mlp_ms / 1e3) / 1e12
    bf16 = {"value": value_bf, "unit": UNIT,
            "frame_ms": total_bf / args.steps,
            "mean_rel_err_vs_fp32": float(e_bf.mean()), "max_rel_err_vs_fp32": float(e_bf.max()),
            "step_breakdown_ms": {f: round(fam_bf[f][0] / args.steps, 4) for f in nis.FAMILIES},
            "roofline": {"bound": "tensor", "unit": "TFLOP/s",
                         "kernel": "mlp_fused_kernel<false> (tcgen05, BF16, whole network per 128-point tile)",
                         "achieved": mlp_tf, "peak": peaks_bf["bf16_tflops_sustained"],
                         "frac": mlp_tf / peaks_bf["bf16_tflops_sustained"],
                         "peak_source": f"{peaks_bf['source']} cuBLAS BF16 sustained",
                         "work": "6.30 MFLOP per point", "launches": mlp_n,
                         "avg_launch_ms": mlp_ms / max(mlp_n, 1),
                         "traffic": (recorded_traffic("mlp_bf16") or {}).get("bytes_per_launch")}}

    # ---- the same frames in FP8 e4m3 (dense layers)
    img_f8 = torch.empty_like(img)
    for _ in range(args.warmup):
        step(w_fp8, img_f8)
    torch.cuda.synchronize()
    ctx.profile(True)
    times_f8 = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(w_fp8, img_f8)
        e1.record(stream)
        e1.synchronize()
        times_f8.append(e0.elapsed_time(e1))
    ctx.profile(False)
    fam_f8 = {f: ctx.profile_read(f) for f in nis.FAMILIES}
    value_f8, total_f8 = whole_job_rate(n_points * args.steps, sum(times_f8) / 1e3, world)
    total_f8 *= 1e3
    a_f8 = img_f8[hitmask].double()
    e_f8 = ((a_f8 - a_32).abs() / torch.maximum(a_32.abs(), floor))
    mlp8_ms = fam_f8["mlp"][0]
    mlp8_tf = MLP_FLOP_PER_POINT * n_points * args.steps / (mlp8_ms / 1e3) / 1e12
    fp8 = {"value": value_f8, "unit": UNIT,
           "frame_ms": total_f8 / args.steps,
           "mean_rel_err_vs_fp32": float(e_f8.mean()), "max_rel_err_vs_fp32": float(e_f8.max()),
           "step_breakdown_ms": {f: round(fam_f8[f][0] / args.steps, 4) for f in nis.FAMILIES},
           "roofline": {"bound": "tensor", "unit": "TFLOP/s",
                        "kernel": "mlp_fused_kernel<true> (e4m3 mode: FC-1 of the density and phase "
                                  "chains on kind::f8f6f4, the other layers BF16)",
                        "achieved": mlp8_tf, "peak": peaks_bf["bf16_tflops_sustained"],
                        "frac": mlp8_tf / peaks_bf["bf16_tflops_sustained"],
                        "work": "6.30 MFLOP per point (34 % of it in e4m3)",
                        "peak_source": f"{peaks_bf['source']} cuBLAS BF16 sustained (most of the "
                                       "work is BF16; the e4m3 products would allow 2x)"}}

    # ---- the same frames with the transmittance from shear-warp rays (O(N^3) per level)
    sw = None
    if not args.no_shear_warp:
        sw = run_shear_warp(args, nis, ctx, v, w, cfg, img, hitmask, flush, stream, n_points)

    paper = None if args.no_paper_model else run_paper_model(args, nis, ctx, v, cfg, flush,
                                                             stream, n_points)

    # ---- end to end through the C ABI from page-locked host memory
    host_vol = torch.from_numpy(vol_np).pin_memory()
    host_img = torch.empty(img.shape, dtype=torch.float32).pin_memory()
    e2e_times = []
    barrier(world)
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.update_volume(v, host_vol)
        step()
        host_img.copy_(img, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_times.append(time.perf_counter() - t0)
    e2e_value, e2e_total = whole_job_rate(n_points * args.steps, sum(e2e_times), world)
    ctx.sync(timeout_ms=120000)

    # ---- one frame split across the ranks (strong scaling), beside the replicas above
    split = None if args.no_split_frame else run_split_frame(args, nis, ctx, v, w, cfg, img,
                                                             flush, stream, world)

    if rank != 0:
        ctx.close()
        return

    # ---- roofline of the dominant kernel family
    peaks = measured_peaks()
    dom = max(fam, key=lambda f: fam[f][0])
    dom_ms, dom_n = fam[dom]
    per_launch_s = dom_ms / 1e3 / max(dom_n, 1)
    n_levels = len(range(int(math.log2(cfg["n"])) + 1))
    if dom == "mlp":
        # FP32-accurate dense layers on the tensor pipe: each FP32 product is issued as six
        # BF16 tcgen05 products of the operands' three-way splits, so the work per launch is
        # 6 x the layers' FLOPs and the ceiling the measured BF16 rate (sustained: the kernel
        # runs inside a long step).  The launches' HBM rate on the bytes this launch design
        # moves (activations round-tripping between layers) is kept as a side figure.
        flops = MLP_FLOP_PER_POINT * n_points * args.steps / max(dom_n, 1)
        work = 6 * flops / 1e12
        achieved = work / per_launch_s
        peak = peaks["bf16_tflops_sustained"]
        design = mlp_bytes_per_point(6, 4) * n_points * args.steps / max(dom_n, 1)
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "kernel": "tc_gemm_kernel (tcgen05, FP32 via 3-way BF16 split, 6 products)",
                "peak_source": f"{peaks['source']} cuBLAS BF16 sustained",
                "work": "6 BF16 products x 6.30 MFLOP per point (issued TFLOP per launch)",
                "fp32_tflops": flops / per_launch_s / 1e12,
                "hbm_launch_design": {"gb_s": design / per_launch_s / 1e9,
                                      "frac": design / per_launch_s / 1e9 / peaks["hbm_gbs"],
                                      "bytes_per_point": mlp_bytes_per_point(6, 4),
                                      "note": "bytes of this launch design (activations round-trip "
                                              "between layers), not algorithmic bytes"}}
    elif dom == "cnn":
        work = CNN_FLOP_PER_POINT * n_points * args.steps / max(dom_n, 1)
        achieved = work / per_launch_s / 1e12
        peak = 152 * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s", "kernel": "cnn_f32_kernel",
                "peak_source": "FP32 FFMA derived peak"}
    else:
        if dom == "gather":
            work = GATHER_BYTES_PER_POINT * n_points * args.steps / max(dom_n, 1)
        else:
            vox = sum(((cfg["n"] + (1 << m) - 1) >> m) ** 3 for m in range(n_levels))
            work = 8.0 * vox / max(1, n_levels)
        achieved = work / per_launch_s / 1e9
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "unit": "GB/s", "kernel": dom,
                "peak_source": f"{peaks['source']} STREAM copy"}
    tr = recorded_traffic(dom)
    # the gather against HBM on its algorithmic bytes (feature writes + the pyramid and the
    # transmittance read once)
    g_ms, g_n = fam["gather"]
    g_bytes = gather_algorithmic_bytes(n_points, cfg["n"]) * args.steps / max(g_n, 1)
    g_gbs = g_bytes / (g_ms / 1e3 / max(g_n, 1)) / 1e9
    # what this launch design writes per point (FP32 frame): H_T rows of 232 FP32 and the
    # three BF16 parts of the density and phase rows of 240, per layer
    g_written = GATHER_WRITTEN_BYTES_F32 * n_points * args.steps / max(g_n, 1)
    gather_roof = {"bound": "hbm", "unit": "GB/s",
                   "kernel": "gather_kernel<3> (one lane per shading point; FP32 H_T and "
                             "three-part BF16 density and phase rows)",
                   "achieved": g_gbs, "peak": peaks["hbm_gbs"], "frac": g_gbs / peaks["hbm_gbs"],
                   "work_per_launch": g_bytes, "avg_launch_ms": g_ms / max(g_n, 1),
                   "peak_source": f"{peaks['source']} STREAM copy",
                   "work": "5400 FP32 features per point + density and transmittance pyramids once",
                   "traffic": (recorded_traffic("gather") or {}).get("bytes_per_launch"),
                   "written": {"bytes_per_point": GATHER_WRITTEN_BYTES_F32,
                               "gb_s": g_written / (g_ms / 1e3 / max(g_n, 1)) / 1e9,
                               "note": "bytes this launch design writes (the FP32-accurate "
                                       "split), not algorithmic bytes"}}
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak,
                 "traffic": tr["bytes_per_launch"] if tr else None,
                 "family": dom, "launches": dom_n, "avg_launch_ms": dom_ms / max(dom_n, 1),
                 "work_per_launch": work})

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"], "volume": f"{cfg['n']}^3 float32",
                       "image": f"{cam['width']}x{cam['height']} perspective",
                       "shading_points_per_frame": n_points, "g": mat["g"],
                       "albedo": mat["albedo"][0], "l2": "flushed between steps (256 MB write)",
                       "step": "pyramid + transmittance + phase table + hits + gather/SE + "
                               "3D-CNN + MLP + decode"},
            "frame_ms": ms_per_step,
            "gpu_launches": int(launches),
            "step_breakdown_ms": {f: round(fam[f][0] / args.steps, 4) for f in nis.FAMILIES},
            "roofline": roof,
            "gather_roofline": gather_roof,
            "bf16": bf16,
            "fp8": fp8,
            "shear_warp": sw,
            "paper_template_model": paper,
            "split_frame": split,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(vol_np.nbytes),
                    "d2h_bytes_per_step": int(img.numel() * 4),
                    "ms_per_step": 1e3 * e2e_total / args.steps},
            "clocks": clk}
    ctx.close()
    if not args.no_serving:
        workload = serving_volumes(args, local)
        line["serving"] = run_serving(args, nis, blob, local, workload)
        if not args.no_shear_warp:
            line["serving_shear_warp"] = run_serving(args, nis, blob, local, workload,
                                                     nis.TRANSMITTANCE_SHEAR_WARP, sweep=(1.0, 1.3))
        del workload
    if not args.no_shear_warp:
        line["shear_warp"]["plume1024"] = plume_transmittance(nis, local)
    if not args.no_plume_loop:
        line["plume1024_60f"] = run_plume_loop(args, nis, local)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, vol_np, weights)
        line["cpu_baseline"]["single_thread"] = oracle_single_thread(args.workload)
    line["summary"] = compact_summary(line)
    print(json.dumps(line), flush=True)


def run_ncu_case(args):
    import torch
    from paper_2401_14051_gb300 import nis
    if args.ncu_case == "sweep":
        ctx = nis.Context(0)
        v = ctx.upload_volume(synth.plume_volume_torch(512, 9, 128.0))
        ctx.build_transmittance(v, synth.unit_vector(10), 0.6, method=nis.TRANSMITTANCE_SHEAR_WARP)
        ctx.sync(timeout_ms=60000)
        ctx.close()
        print("ok")
        return
    if args.ncu_case in ("frame_f32", "frame_bf16", "frame_fp8"):
        # the benchmark's volume and view at 800x450 (about 37,000 shading points: the
        # features still exceed L2, the device holds a few GB)
        cfg = synth.config(2)
        cam = dict(cfg["camera"], width=800, height=450)
        ctx = nis.Context(0)
        v = ctx.upload_volume(cfg["volume"]())
        l = ctx.build_transmittance(v, cfg["light"], 0.6)
        prec = {"frame_f32": nis.PREC_F32, "frame_bf16": nis.PREC_BF16, "frame_fp8": nis.PREC_FP8}[args.ncu_case]
        w = ctx.load_weights(synth.pack_weights(synth.make_weights(cfg["weights_seed"],
                                                                   cfg["sigma_max"])), prec)
        for _ in range(2):
            ctx.render_frame(v, l, w, cfg["material"], cam)
        ctx.sync(timeout_ms=60000)
        ctx.close()
        print("ok")
        return
    prec = {"f32": nis.PREC_F32, "bf16": nis.PREC_BF16, "simt": nis.PREC_F32_SIMT}[args.ncu_case]
    cfg = synth.config(1)
    ctx = nis.Context(0)
    v = ctx.upload_volume(cfg["volume"]())
    l = ctx.build_transmittance(v, cfg["light"], 0.6)
    w = ctx.load_weights(synth.pack_weights(synth.make_weights(4, 16.0)), prec)
    p, om = synth.shading_points(32768, 3)
    dev = torch.device("cuda:0")
    pt, ot = torch.from_numpy(p).to(dev), torch.from_numpy(om).to(dev)
    for _ in range(2):
        ctx.shade_points(v, l, w, cfg["material"], pt, ot)
    ctx.sync(timeout_ms=60000)
    ctx.close()
    print("ok")


def main():
    args = parse()
    if args.oracle_sample:
        run_oracle_sample(args)
        return
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_nis(args)


if __name__ == "__main__":
    main()
