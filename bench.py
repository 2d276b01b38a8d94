#!/usr/bin/env python
"""Benchmark of the adaptive event renderer (Alg. 1 of arXiv 2408.07996).

One step = one event frame: every pixel of a 1280x720 frame pair
(t_k, t_k+1) of the procedural terrain workload (2.09M terrain triangles +
200 instanced boxes, HDR sky, depth 6) goes through path tracing of log
luminance in batches (512 first, +64, cap 8192), the Student t-test and the
event rule, carrying the reference state from frame to frame.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle on a bounded crop of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "event frames/s and Mpaths/s at 1280x720 vs uniform-spp on same GPU at matched error"
# Algorithmic work of BVH traversal: 12 FLOP per ray/box slab test (a BVH2
# node fetch tests two child boxes, 24 FLOP) and 25 FLOP per ray/triangle
# test, against the FP32 FMA peak of 128 lanes x 2 FLOP per SM per clock
FLOP_PER_BOX = 12
FLOP_PER_TRI = 25
FP32_LANES_PER_SM = 128
FLOP_PER_LANE_CLOCK = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="terrain720p")
    ap.add_argument("--frames", type=int, default=5, help="video length of --workload ablation")
    ap.add_argument("--scene", default="terrain720p", help="workload that --workload ablation renders")
    ap.add_argument("--dims", type=int, nargs=3, default=None, metavar=("W", "H", "T"),
                    help="video size of --workload quality (default 1280 720 100)")
    ap.add_argument("--no-uniform", action="store_true")
    ap.add_argument("--no-matched", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--crop", type=int, default=24,
                    help="oracle crop side (pixels) of one --impl reference step (the whole run stays within minutes)")
    ap.add_argument("--cpu-crop", type=int, default=64,
                    help="oracle crop side (pixels) of the cpu_baseline sample (one frame pair, ~30 s of CPU work)")
    ap.add_argument("--wavefront", type=int, default=0)
    ap.add_argument("--bvh-width", type=int, default=0, choices=[0, 2, 8],
                    help="BVH node layout (0: the library default)")
    ap.add_argument("--no-tune", action="store_true", help="batch64: skip the autotuner")
    ap.add_argument("--profile-band", type=int, nargs=3, metavar=("ROW0", "ROW1", "SPP"),
                    help="only trace SPP samples of every pixel in image rows [ROW0, ROW1) at keyframe 3 "
                         "(a small, representative case for kernel captures) and exit")
    return ap.parse_args()


def profile_band(args):
    """tracePaths over one band of image rows: the first launches of the
    process are full-size raygen / extend / shade / shadow launches."""
    import torch

    import scenegen as sg
    from paper_2408_07996_gb300.api import Renderer
    w = sg.workload(args.workload)
    r = Renderer(w.width, w.height, 0)
    r.upload(w.scene)
    r.configure(w)
    r.set_params(wavefront=args.wavefront, bvh_width=args.bvh_width)
    r0, r1, spp = args.profile_band
    pix = torch.arange(r0 * w.width, r1 * w.width, dtype=torch.int32, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    L, _ = r.trace_samples(w.times[3], pix, 0, spp, want_sig=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"profile_band": [r0, r1, spp], "paths": int(L.numel()), "ms": ms,
                      "mpaths_per_s": L.numel() / ms / 1e3}), flush=True)
    r.close()


# ------------------------------------------------------------------ multi-rank aggregation
def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / seconds


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_median": statistics.median(power) if power else None, "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------------ oracle (CPU) sample
def oracle_sample(w, crop: int, frame: int):
    """Alg. 1 on a centred crop x crop window for frame pair (t_f, t_f+1),
    reference included: the FP64 oracle as it stands, on all host cores."""
    import numpy as np

    import oracle as O
    osc = O.OracleScene(w.scene)
    cx, cy = w.width // 2, w.height // 2
    ys, xs = np.meshgrid(np.arange(cy - crop // 2, cy - crop // 2 + crop),
                         np.arange(cx - crop // 2, cx - crop // 2 + crop), indexing="ij")
    pix = (ys * w.width + xs).reshape(-1).astype(np.int32)
    p, d = O.params_of(w), O.detect_of(w)
    threads = O.default_threads()

    def run():
        t = time.perf_counter()
        out = O.render_events(osc, p, d, w.times[frame], w.times[frame + 1], pix, threads=threads)
        dt = time.perf_counter() - t
        paths = int(pix.size) * w.spp_max + int(out["n"].sum())
        return dt, paths, out

    return run, pix.size, threads


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import scenegen as sg
    w = sg.workload(args.workload)
    run, npix, threads = oracle_sample(w, args.crop, 0)
    for _ in range(args.warmup):
        run()
    tot_t, tot_paths, per_px = 0.0, 0, []
    for _ in range(args.steps):
        dt, paths, out = run()
        tot_t += dt
        tot_paths += paths
        per_px.append(float(out["n"].mean()))
    mpps = tot_paths / tot_t / 1e6
    # per-path extrapolation: one event frame of this workload at the
    # oracle's path rate, with the adaptive frame's samples per pixel of the crop
    frames_per_s = mpps * 1e6 / (statistics.mean(per_px) * w.width * w.height)
    ms = tot_t / args.steps * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": frames_per_s, "unit": "event frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(w),
        "mpaths_per_s": mpps,
        "cpu_baseline": {"value": frames_per_s, "unit": "event frames/s", "cores": threads, "kind": "oracle",
                         "sample": f"Alg. 1 (reference frame + one event frame) on a {args.crop}x{args.crop} "
                                   f"centred crop per step; {tot_paths} paths in {tot_t:.1f} s; frames/s "
                                   f"extrapolated per path to the full 1280x720 frame"},
        "e2e": {"value": frames_per_s, "unit": "event frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _config(w):
    sc = w.scene
    return {"workload": w.name, "width": w.width, "height": w.height, "triangles": int(sc.n_triangles),
            "instances": int(len(sc.inst_mesh)), "spp_min": w.spp_min, "spp_batch": w.spp_batch,
            "spp_max": w.spp_max, "C": w.C, "alpha": w.alpha, "max_depth": w.max_depth, "eps": w.eps,
            "variant": "one-tailed",
            "l2": "inputs larger than L2: BVH + triangles ~170 MB and the wavefront state (>1 GB) "
                  "are streamed every step"}


# ------------------------------------------------------------------ batched jobs (64 mixed-size frame pairs)
def run_batch(args):
    """64 independent frame pairs (image sizes from 128x128 to 640x480,
    5k-100k triangles each) rendered in shared rounds; one step = one event
    frame of every job.  The BVH node layout and leaf size are picked by the
    autotuner on the first frame pair after warm-up."""
    import torch

    import scenegen as sg
    from paper_2408_07996_gb300.api import Renderer, render_events_batch
    from paper_2408_07996_gb300.autotune import tune_batch

    ws = sg.batch_workloads(64)
    rs = []
    for w in ws:
        r = Renderer(w.width, w.height)
        r.upload(w.scene)
        r.configure(w)
        rs.append(r)
    runner = Renderer(8, 8)
    runner.set_params(profile=1)
    sched = dict(C=ws[0].C, alpha=ws[0].alpha, spp_batch=ws[0].spp_batch, spp_max=ws[0].spp_max)
    times = ws[0].times
    K, Wm = args.steps, max(3, args.warmup)
    assert Wm + K < len(times), "not enough keyframes"

    def frame(k):
        return render_events_batch(runner, [(r, times[k], times[k + 1]) for r in rs], *sched.values())

    for k in range(Wm):
        frame(k)
    # autotune on the next frame pair of all jobs (their references exist,
    # so a trial costs one batched adaptive frame; the wavefront that suits a
    # subset of the jobs does not suit all of them); states are restored
    tune = None
    if not args.no_tune:
        tune = tune_batch(runner, rs, (times[Wm], times[Wm + 1]), sched,
                          wavefronts=(1 << 25,), windows=(16,), leaf_sizes=(2, 4), bvh_widths=(2, 8))
        tune = {"best": tune["best"], "trials": tune["trials"], "jobs": len(rs)}
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    steps = [frame(k)[1] for k in range(Wm, Wm + K)]
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    paths = sum(s["paths"] for s in steps)
    kms = [sum(s["kernel_ms"][i] for s in steps) for i in range(5)]
    total = sum(kms)
    line = {"metric": "event frames/s of 64 batched frame pairs (128x128 to 640x480)", "value": 64 * K / (ms / 1e3),
            "unit": "event frames/s", "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64", "jobs": 64, "pixels": sum(w.width * w.height for w in ws),
                       "triangles": [min(w.scene.n_triangles for w in ws), max(w.scene.n_triangles for w in ws)],
                       "resolutions": sorted({f"{w.width}x{w.height}" for w in ws}), **sched,
                       "spp_min": ws[0].spp_min},
            "mpaths_per_s": paths / (ms / 1e3) / 1e6, "rounds_per_step": sum(s["rounds"] for s in steps) / K,
            "gpu_launches": sum(s["kernel_launches"] for s in steps),
            "kernel_share": {n: round(kms[i] / total, 4) if total else None
                             for i, n in enumerate(["raygen", "traversal", "shade", "shadow", "stats"])},
            "launch_gaps_ms_per_step": (sum(s["gpu_ms"] for s in steps) - total) / K,
            "autotune": tune, "clocks": clk}
    # the same frame rendered job after job (one-job batches through the same
    # runner and wavefront) against all jobs in shared rounds
    if not args.no_uniform:
        k = Wm + K
        states = [r.get_state().clone() for r in rs]
        _, bst = frame(k)
        for r, s0 in zip(rs, states):
            r.set_state(s0)
        seq_ms = 0.0
        for r in rs:
            _, st1 = render_events_batch(runner, [(r, times[k], times[k + 1])], *sched.values())
            seq_ms += st1["gpu_ms"]
        line["batched_vs_one_by_one"] = {"frame": k, "batched_ms": bst["gpu_ms"], "one_by_one_ms": seq_ms,
                                         "speedup": seq_ms / bst["gpu_ms"]}
    for r in rs:
        r.close()
    runner.close()
    print(json.dumps(line), flush=True)


# algorithmic bytes of one mcev_event_quality call: per voxel the frame error
# reads 2, and each of the 4 transforms (2 directions x 2 polarities) reads
# its video (1) and writes 4 in the row pass, reads 4 and writes 4 in each
# column pass, and reads the query video (1) in the match pass; per event,
# the match pass reads its 4-byte distance
QUALITY_BYTES_PER_VOXEL = 2 + 4 * (1 + 4 + 8 + 8 + 1)
# statistics kernel (a7-a10 fused): per pixel visit it reads the queue entry
# (4), the running and reference (n, mean, M2) (24) and writes the running
# state (12) and a re-queue entry or event/spp (4); per path it reads one
# 4-byte radiance
STATS_BYTES_PER_PIXEL_VISIT = 44
STATS_BYTES_PER_PATH = 4
QUALITY_BYTES_PER_EVENT = 4

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per traced ray of
# the traversal launches (k_extend + k_shadow_extend, two-wide BVH), from a
# one-pass ncu capture of every launch of one timed terrain frame (315.2 GB
# over 294 launches that traced 3.852 G closest-hit and shadow rays); set to
# None when the traversal kernels change.
TRAVERSAL_DRAM_BYTES_PER_RAY = 81.82


def traversal_traffic(rays_per_launch: float, bvh_width: int = 2):
    """DRAM bytes of an average traversal launch: the captured bytes per ray
    scaled by the rays an average timed launch traces, or None (no capture
    of this layout's kernels)."""
    if TRAVERSAL_DRAM_BYTES_PER_RAY is None or bvh_width == 8:
        return None
    return TRAVERSAL_DRAM_BYTES_PER_RAY * rays_per_launch


def _hbm_peak():
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        v = pk.get("hbm_gbs")
        if isinstance(v, dict):
            v = v.get("value")
        return float(v), "measured"
    except Exception:
        return 6800.0, "fallback"


def run_quality(args):
    """Event-video quality metrics (Sec. 4.2) of a 1280x720, 100-frame
    synthetic event-video pair (the terrain benchmark's frame size over its
    100 keyframes); one step = one mcev_event_quality call (RMSE, PSNR,
    polarity-aware F1 and chamfer distance over 92M voxels)."""
    import torch

    import scenegen as sg
    from paper_2408_07996_gb300.api import event_quality

    W, H, T = args.dims or (1280, 720, 100)
    a_np, b_np = sg.event_video_pair(W, H, T, seed=20240820)
    a = torch.from_numpy(a_np).cuda()
    b = torch.from_numpy(b_np).cuda()
    K, Wm = args.steps, max(3, args.warmup)
    for _ in range(Wm):
        event_quality(a, b)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    res = [event_quality(a, b) for _ in range(K)]
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    gpu_ms = sum(r["gpu_ms"] for r in res) / K
    n = T * H * W
    peak, basis = _hbm_peak()
    q = res[-1]
    algo_bytes = QUALITY_BYTES_PER_VOXEL * n + QUALITY_BYTES_PER_EVENT * (q["n_a"] + q["n_b"])
    achieved = algo_bytes / (gpu_ms / 1e3) / 1e9
    line = {"metric": "event-video quality metrics (RMSE, PSNR, F1, PSCD) throughput", "value": n * K / (ms / 1e3) / 1e9,
            "unit": "Gvoxels/s", "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"quality_{W}x{H}x{T}", "width": W, "height": H, "frames": T, "tau2": 3,
                       "events_a": q["n_a"], "events_b": q["n_b"],
                       "l2": "two int32 scratch volumes of 369 MB each are streamed every step (> L2)"},
            "gpu_launches": sum(r["kernel_launches"] for r in res),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "basis": basis,
                         "bytes_per_call": algo_bytes, "bytes_per_voxel": QUALITY_BYTES_PER_VOXEL,
                         "bytes_per_event": QUALITY_BYTES_PER_EVENT, "avg_call_ms": gpu_ms},
            "metrics": {k: q[k] for k in ("rmse", "psnr", "precision", "recall", "f1", "pscd")},
            "clocks": clk}
    print(json.dumps(line), flush=True)


def run_ablation(args):
    """The paper's comparison (Sec. 4.2, Table 2) on one workload (--scene,
    default the terrain): a short event video (frames t_3 -> t_{3+F}) rendered from the same
    reference by the uniform-spp baseline and by each detector variant
    (one-tailed t-test = the paper's method, mean-only and two-tailed
    ablations, Welch standard error), each scored against the uniform video
    with the Sec. 4.2 metrics and timed per frame."""
    import torch

    import scenegen as sg
    from paper_2408_07996_gb300 import MEAN_ONLY, ONE_TAILED, SE_WELCH, TWO_TAILED, UNIFORM
    from paper_2408_07996_gb300.api import Renderer, event_quality

    w = sg.workload(args.scene)
    F = args.frames
    k0 = 3
    r = Renderer(w.width, w.height, 0)
    r.upload(w.scene)
    r.configure(w)
    r.render_reference(w.times[k0], w.spp_max)     # Alg. 1 first frame at t_{k0}
    state = r.get_state().clone()

    def video(variant, se_mode=0):
        r.set_params(variant=variant, se_mode=se_mode)
        r.set_state(state)
        ev, ms, spp = [], 0.0, 0
        for k in range(k0, k0 + F):
            out = r.render_events(w.times[k], w.times[k + 1], w.C, w.alpha, w.spp_batch, w.spp_max)
            ev.append(out["events"].clone())
            ms += out["stats"]["gpu_ms"]
            spp += out["stats"]["samples_used"]
        return torch.stack(ev), ms / F, spp / F / (w.width * w.height)

    uni, uni_ms, _ = video(UNIFORM)
    rows = [{"method": "uniform", "ms_per_frame": uni_ms, "mean_spp": float(w.spp_max)}]
    for name, var, se in (("one-tailed t-test (paper)", ONE_TAILED, 0), ("mean only", MEAN_ONLY, 0),
                          ("two-tailed t-test", TWO_TAILED, 0), ("one-tailed, Welch SE", ONE_TAILED, SE_WELCH)):
        v, ms, spp = video(var, se)
        q = event_quality(v, uni)
        rows.append({"method": name, "ms_per_frame": ms, "speedup": uni_ms / ms, "mean_spp": spp,
                     "event_error_pct": 100.0 * float((v != uni).float().mean()),
                     **{k: q[k] for k in ("rmse", "psnr", "f1", "pscd", "precision", "recall")}})
        print(f"[ablation] {name}: {ms:.0f} ms/frame, F1 {q['f1']:.5f}", file=sys.stderr, flush=True)
    r.close()
    print(json.dumps({"metric": "detector ablation against the uniform baseline (Table 2 analogue)",
                      "config": {**_config(w), "frames": F, "first_frame": k0, "tau2": 3}, "rows": rows}),
          flush=True)


def run_diff(args):
    """Differentiable rendering on the 256x256 textured room (49k triangles,
    512x512 RGB texture, 4 emitters, 64 spp, depth 3): one step = the
    per-pixel mean ln(L + eps) at t0 and t1 (forward), the smooth event loss
    against a target event map, and the path-replay adjoint at both times
    (backward: every path traced twice), giving texture and emission
    gradients."""
    import torch

    import scenegen as sg
    from paper_2408_07996_gb300.api import EventFrames, Renderer, event_loss

    w = sg.workload("diff256")
    r = Renderer(w.width, w.height, 0)
    r.upload(w.scene)
    r.configure(w)
    spp = w.spp_max
    t0, t1 = w.times[0], w.times[1]
    other = torch.from_numpy(sg.albedo_texture(w.scene.texture.shape[0], 77)).cuda()
    r.set_texture(other)
    d = r.render_mean(t1, spp) - r.render_mean(t0, spp)
    target = (torch.sign(d) * (d.abs() > w.C)).to(torch.int8)
    T = torch.from_numpy(w.scene.texture).cuda().requires_grad_(True)
    E = torch.from_numpy(w.scene.mat_emit.astype("float32")).cuda().requires_grad_(True)

    def step():
        T.grad = None
        E.grad = None
        m0, m1 = EventFrames.apply(T, E, r, t0, t1, spp)
        loss = event_loss(m0.double(), m1.double(), target, w.C)
        loss.backward()
        return loss

    K, Wm = args.steps, max(3, args.warmup)
    for _ in range(Wm):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(K):
        loss = step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    n_pix = w.width * w.height
    paths = n_pix * spp * (2 + 4)          # forward at t0, t1; backward traces twice at t0, t1
    r.close()
    print(json.dumps({
        "metric": "gradient steps/s (forward + path-replay backward of the event loss)", "value": K / (ms / 1e3),
        "unit": "steps/s", "n_gpus": 1, "steps": K, "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "diff256", "width": w.width, "height": w.height,
                   "triangles": int(w.scene.n_triangles), "texture": list(w.scene.texture.shape), "spp": spp,
                   "max_depth": w.max_depth, "C": w.C},
        "mpaths_per_s": paths * K / (ms / 1e3) / 1e6, "paths_per_step": paths, "loss": float(loss.detach()),
        "grad_norm": {"texture": float(T.grad.norm()), "emission": float(E.grad.norm())}, "clocks": clk}),
        flush=True)


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_band:
        return profile_band(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "quality":
        return run_quality(args)
    if args.workload == "ablation":
        return run_ablation(args)
    if args.workload == "diff256":
        return run_diff(args)
    import numpy as np
    import torch

    import scenegen as sg
    from paper_2408_07996_gb300 import UNIFORM, ONE_TAILED
    from paper_2408_07996_gb300.api import Renderer

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist:
            dist.barrier()

    w = sg.workload(args.workload)
    K, Wm = args.steps, max(3, args.warmup)
    assert Wm + K + 2 < len(w.times), "not enough keyframes for warmup + steps"
    r = Renderer(w.width, w.height, local)
    r.upload(w.scene)
    r.configure(w)
    r.set_params(profile=1, wavefront=args.wavefront, bvh_width=args.bvh_width)
    H, Wd = w.height, w.width
    dev = torch.device("cuda", local)
    out = dict(events=torch.empty((H, Wd), dtype=torch.int8, device=dev),
               spp=torch.empty((H, Wd), dtype=torch.int32, device=dev),
               mean=torch.empty((H, Wd), dtype=torch.float32, device=dev))

    def frame(k, spp_max=None):
        return r.render_events(w.times[k], w.times[k + 1], w.C, w.alpha, w.spp_batch,
                               spp_max or w.spp_max, out=out)

    # warm-up: the first frame renders the reference at t0 (Alg. 1 first frame)
    pre_launches = 0
    for k in range(Wm):
        pre_launches += frame(k)["stats"]["kernel_launches"]
    print(f"[bench] launches before the timed loop: {pre_launches}", file=sys.stderr, flush=True)
    torch.cuda.synchronize()
    state0 = r.get_state().clone()

    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    steps = []
    for k in range(Wm, Wm + K):
        steps.append(dict(frame(k)["stats"]))
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    frames_per_s = job_rate(K, ms / 1e3, world)
    for s_ in steps:
        print(f"[bench] step: {s_['gpu_ms']:.1f} ms, {s_['paths']} paths, {s_['rounds']} rounds, "
              f"events {s_['events_pos']}+{s_['events_neg']}, kernel ms {[round(x, 1) for x in s_['kernel_ms']]}",
              file=sys.stderr, flush=True)
    paths = sum(s["paths"] for s in steps)
    mpaths = job_rate(paths, ms / 1e3, world) / 1e6
    launches = sum(s["kernel_launches"] for s in steps)

    # roofline of the dominant work, BVH traversal (closest-hit and shadow
    # rays; a bounce's shadow rays share a launch with the next bounce's
    # closest hits), from the timed steps: device time of the traversal
    # launches (CUDA events on the library's stream) and the traversal work
    # they did (box and triangle tests counted by the kernels)
    kms = [sum(s["kernel_ms"][i] for s in steps) for i in range(5)]
    kcnt = [sum(s["kernel_count"][i] for s in steps) for i in range(5)]
    boxes = sum(s["boxes_closest"] + s["boxes_shadow"] for s in steps)
    nodes = sum(s["nodes_closest"] + s["nodes_shadow"] for s in steps)
    tris = sum(s["tris_closest"] + s["tris_shadow"] for s in steps)
    rays = sum(s["rays_closest"] + s["rays_shadow"] for s in steps)
    ext_ms = kms[1] + kms[3]
    n_trav = max(1, kcnt[1] + kcnt[3])
    flop = boxes * FLOP_PER_BOX + tris * FLOP_PER_TRI
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max_mhz = clk.get("sm_max_mhz") or 2070.0
    peak_tflops = sm_count * FP32_LANES_PER_SM * FLOP_PER_LANE_CLOCK * sm_max_mhz * 1e6 / 1e12
    achieved = flop / n_trav / (ext_ms / n_trav / 1e3) / 1e12 if ext_ms > 0 else None
    total_kms = sum(kms)
    roofline = {"kernel": "BVH traversal: k_extend, k_shadow_extend (closest-hit + shadow rays)", "bound": "alu",
                "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": (achieved / peak_tflops) if achieved else None,
                "traffic": traversal_traffic(rays / n_trav, args.bvh_width),
                "traffic_basis": "DRAM bytes per traced ray from the ncu capture of a timed frame "
                                 f"({TRAVERSAL_DRAM_BYTES_PER_RAY} B/ray) x rays per average launch",
                "avg_launch_ms": ext_ms / n_trav, "launches": n_trav,
                "flop_per_launch": flop / n_trav,
                "box_tests_per_launch": boxes / n_trav, "tri_tests_per_launch": tris / n_trav,
                "rays_per_launch": rays / n_trav,
                "node_fetches_per_ray": nodes / max(1, rays), "box_tests_per_ray": boxes / max(1, rays),
                "tri_tests_per_ray": tris / max(1, rays),
                "grays_per_s": rays / (ext_ms / 1e3) / 1e9 if ext_ms else None,
                "kernel_share": {n: round(kms[i] / total_kms, 4) if total_kms else None
                                 for i, n in enumerate(["raygen", "traversal", "shade", "shadow", "stats"])},
                "peak_basis": f"nominal FP32 FMA peak: {sm_count} SMs x {FP32_LANES_PER_SM} lanes x "
                              f"{FLOP_PER_LANE_CLOCK} FLOP x {sm_max_mhz:.0f} MHz",
                "work_basis": f"{FLOP_PER_BOX} FLOP per ray/box test, {FLOP_PER_TRI} per ray/triangle test"}

    # statistics kernel against HBM
    hbm_peak, hbm_basis = _hbm_peak()
    stats_bytes = STATS_BYTES_PER_PIXEL_VISIT * sum(s["stats_pixels"] for s in steps) + STATS_BYTES_PER_PATH * paths
    roof_stats = {"kernel": "k_stats (log, batch statistics, t-test, re-queue, events)", "bound": "hbm",
                  "achieved": stats_bytes / (kms[4] / 1e3) / 1e9 if kms[4] else None, "peak": hbm_peak,
                  "unit": "GB/s", "basis": hbm_basis,
                  "frac": stats_bytes / (kms[4] / 1e3) / 1e9 / hbm_peak if kms[4] else None,
                  "bytes_per_frame": stats_bytes / K, "avg_launch_ms": kms[4] / max(1, kcnt[4])}

    # the same K frames from the same reference with the library's default
    # path: per-launch timing off, so the rounds run on the device as one
    # CUDA graph per frame (no host round trip between rounds)
    r.set_state(state0)
    r.set_params(profile=0)
    torch.cuda.synchronize()
    barrier()
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    d0.record()
    dsteps = [dict(frame(k)["stats"]) for k in range(Wm, Wm + K)]
    d1.record()
    torch.cuda.synchronize()
    dms = max_over_ranks(d0.elapsed_time(d1), dist, dev)
    device_loop = {"frames_per_s": job_rate(K, dms / 1e3, world), "ms_per_frame": dms / K,
                   "rounds_per_frame": sum(s["rounds"] for s in dsteps) / K,
                   "gpu_launches": sum(s["kernel_launches"] for s in dsteps),
                   "what": "same frames with per-launch timing off: each frame's rounds run as one CUDA graph "
                           "(conditional loop sized on the device)"}
    line = {"metric": METRIC, "value": frames_per_s, "unit": "event frames/s", "n_gpus": world, "steps": K,
            "warmup": Wm, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(w),
            "mpaths_per_s": mpaths, "paths_per_frame": paths / K,
            "mean_spp": paths / K / (H * Wd),
            "events_per_frame": sum(s["events_pos"] + s["events_neg"] for s in steps) / K,
            "gpu_launches": launches, "roofline": roofline, "roofline_stats": roof_stats, "clocks": clk,
            "device_loop": device_loop}

    # uniform-spp comparator on the same GPU, same frame pair and reference
    r.set_params(profile=1)
    if not args.no_uniform and rank == 0:
        kf = Wm + K
        st = r.get_state().clone()
        ad = frame(kf)
        ev_ad = ad["events"].clone()
        ad_stats = dict(ad["stats"])
        r.set_state(st)
        r.set_params(variant=UNIFORM)
        torch.cuda.synchronize()
        u = frame(kf)
        ev_u = u["events"].clone()
        u_stats = dict(u["stats"])
        err = float((ev_ad != ev_u).float().mean().item())
        print(f"[bench] uniform frame {u_stats['gpu_ms']:.1f} ms, adaptive {ad_stats['gpu_ms']:.1f} ms, "
              f"event error {100 * err:.3f}%", file=sys.stderr, flush=True)
        # the uniform rate over 4 consecutive frames (this one and the next 3)
        u_ms, u_paths = [u_stats["gpu_ms"]], [u_stats["paths"]]
        for k in range(kf + 1, min(kf + 4, len(w.times) - 1)):
            us = frame(k)["stats"]
            u_ms.append(us["gpu_ms"])
            u_paths.append(us["paths"])
        u_mean = sum(u_ms) / len(u_ms)
        uni = {"frames_per_s": 1e3 / u_mean, "mpaths_per_s": sum(u_paths) / sum(u_ms) / 1e3,
               "ms_per_frame": u_mean, "frame_ms": u_ms,
               "measured_on": f"{len(u_ms)} consecutive frame pairs from frame {kf} (every pixel at spp_max)"}
        line["uniform"] = uni
        line["adaptive_check_frame"] = {"ms": ad_stats["gpu_ms"], "paths": ad_stats["paths"]}
        line["event_error_vs_uniform_pct"] = 100.0 * err
        from paper_2408_07996_gb300.api import event_quality
        qv = event_quality(ev_ad, ev_u)
        line["quality_vs_uniform"] = {k: qv[k] for k in ("rmse", "psnr", "precision", "recall", "f1", "pscd")}
        line["quality_vs_uniform"]["tau2"] = 3
        line["speedup_vs_uniform"] = u_mean / (ms / K)
        line["speedup_same_frame"] = u_stats["gpu_ms"] / ad_stats["gpu_ms"]
        if not args.no_matched:
            ladder = []
            spp = w.spp_min
            while spp < w.spp_max:
                r.set_state(st)
                m = frame(kf, spp_max=spp)
                e = float((m["events"] != ev_u).float().mean().item())
                ladder.append({"spp": spp, "event_error_pct": 100 * e, "ms": m["stats"]["gpu_ms"]})
                if e <= err:
                    break
                spp *= 2
            match = next((x for x in ladder if x["event_error_pct"] <= 100 * err), None)
            line["matched_error"] = {"ladder": ladder, "uniform_spp": match["spp"] if match else w.spp_max,
                                     "uniform_frames_per_s": 1e3 / (match["ms"] if match else u_stats["gpu_ms"])}
        r.set_params(variant=ONE_TAILED)

    # end to end through the public API with host buffers: same K frames from
    # the same reference, outputs copied to pinned host memory every step
    if not args.no_e2e:
        r.set_state(state0)
        r.set_params(profile=0)      # the library's default path
        host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in out.items()
                if isinstance(v, torch.Tensor)}
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for k in range(Wm, Wm + K):
            o = frame(k)
            for name in host:
                host[name].copy_(o[name], non_blocking=True)
            torch.cuda.current_stream().synchronize()
            h2d += o["stats"]["h2d_bytes"]
            d2h += o["stats"]["d2h_bytes"] + sum(v.numel() * v.element_size() for v in host.values())
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        line["e2e"] = {"value": job_rate(K, dt, world), "unit": "event frames/s", "h2d_bytes_per_step": h2d / K,
                       "d2h_bytes_per_step": d2h / K}

    r.close()
    if rank == 0 and world == 1 and not args.no_cpu:
        run, npix, threads = oracle_sample(w, args.cpu_crop, Wm)
        dt, cpaths, cout = run()
        mpps = cpaths / dt / 1e6
        per_px = float(cout["n"].mean())
        line["cpu_baseline"] = {
            "value": mpps * 1e6 / (per_px * w.width * w.height), "unit": "event frames/s", "cores": threads,
            "kind": "oracle", "mpaths_per_s": mpps,
            "sample": f"FP64 oracle, Alg. 1 on a {args.cpu_crop}x{args.cpu_crop} centred crop of frame pair "
                      f"{Wm}->{Wm + 1} (reference frame included): {cpaths} paths in {dt:.1f} s; "
                      f"frames/s extrapolated per path to the full frame"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
