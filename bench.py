"""Throughput of the LUDVIG hot path on GB300: uplift views*channels per second.

One step = one pass of the whole path over the paper-scale synthetic
workload: uplift of 150 views (980x546, D=384 float32 features, 1M clustered
Gaussians) -> kNN graph (k=16) with exp(-d^2/0.01) * max(0, cos) weights on
the uplifted features -> 100 row-normalised diffusion steps of a mask.
Inputs (scene and all 123 GB of features) are resident in HBM before the timed
region and larger than L2, so no explicit flush is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on
bounded samples of the same workload instead.
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

METRIC = "uplift views*ch/s"
UNIT = "views*ch/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["paper", "small", "tiny"], default="paper")
    ap.add_argument("--dtype", choices=["f32", "bf16"], default="f32")
    ap.add_argument("--e2e-views", type=int, default=16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="uplift only (not a full step)")
    ap.add_argument("--no-precision", action="store_true", help="skip the bf16 precision-form line")
    ap.add_argument("--no-render", action="store_true", help="skip the render-back (Eq. 4) line")
    ap.add_argument("--no-filter", action="store_true", help="skip the Gaussian-filtering line")
    ap.add_argument("--no-paper-diffusion", action="store_true", help="skip the paper-form diffusion line")
    ap.add_argument("--no-relevancy", action="store_true", help="skip the relevancy / count-normaliser lines")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form line")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-form line")
    ap.add_argument("--profile-case", default=None,
                    choices=["tc2views", "render2views", "render16views", "uplift16views", "batch8", "tinymask"],
                    help="run a small fixed case for an ncu capture and exit (no JSON line)")
    return ap.parse_args()


def workload(name):
    from paper_2410_14462_gb300 import inputs
    if name == "paper":
        return inputs.paper_scale_workload()
    if name == "tiny":
        return inputs.tiny_mask_workload()
    return inputs.paper_scale_workload(n=100_000, views=12, d=64, width=490, height=273)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- CPU oracle timing
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_view_seconds(wl, views, nthreads):
    """Seconds the oracle takes to uplift each of `views` (every Gaussian, all
    D channels); the view's features and the float64 accumulators are made
    outside the timed call."""
    import oracle
    oracle.build()
    out = []
    for v in views:
        F = wl.features(v).numpy()
        num = np.zeros((wl.scene.n, wl.d))
        den = np.zeros(wl.scene.n)
        t0 = time.perf_counter()
        oracle.view_uplift(wl.scene, wl.cams.params[v], wl.cams.width, wl.cams.height, F, num, den,
                           nthreads=nthreads)
        out.append(time.perf_counter() - t0)
    return out


def _cpulist(text):
    cpus = set()
    for part in text.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    return cpus


def gpu_local_cpus(gpu_uuid):
    """(NUMA node, CPU set) of the host memory next to the GPU, read from the
    sysfs entry of its PCI device; (None, None) when unknown."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader", "-i", gpu_uuid],
                             capture_output=True, text=True, timeout=30).stdout.strip()
        dom, rest = bus.split(":", 1)
        dev = f"/sys/bus/pci/devices/{dom[-4:].lower()}:{rest.lower()}"
        node = int(open(dev + "/numa_node").read())
        cpus = _cpulist(open(dev + "/local_cpulist").read())
        return (node if node >= 0 else None), (cpus or None)
    except (OSError, ValueError, subprocess.SubprocessError):
        return None, None


def pinned_near(shape, dtype, cpus):
    """A page-locked host tensor whose pages are placed from `cpus` (the
    calling thread runs there while the pages are allocated and pinned)."""
    import torch
    old = os.sched_getaffinity(0)
    use = (cpus & old) or cpus if cpus else None
    if use:
        os.sched_setaffinity(0, use)
    try:
        t = torch.empty(shape, dtype=dtype, pin_memory=True)
    finally:
        if use:
            os.sched_setaffinity(0, old)
    return t


def copy_rates(host, dev):
    """Measured host->device and device->host GB/s of one copy between a
    pinned host tensor and a device tensor of the same size (CUDA events)."""
    import torch
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    dev.copy_(host, non_blocking=True)        # warm
    torch.cuda.synchronize()
    e[0].record()
    dev.copy_(host, non_blocking=True)
    e[1].record()
    e[2].record()
    host.copy_(dev, non_blocking=True)
    e[3].record()
    torch.cuda.synchronize()
    nbytes = host.numel() * host.element_size()
    return nbytes / (e[0].elapsed_time(e[1]) / 1e3) / 1e9, nbytes / (e[2].elapsed_time(e[3]) / 1e3) / 1e9


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    wl = workload(args.workload)
    nthreads = oracle.default_threads()
    # bounded sample per step: one view, every Gaussian, all D channels; the
    # warm-up steps are views too, untimed
    secs = oracle_view_seconds(wl, [s % wl.cams.v for s in range(args.warmup + args.steps)], nthreads)
    t = float(np.mean(secs[args.warmup:]))
    value = wl.d / t
    sample = (f"views {args.warmup}-{args.warmup + args.steps - 1} of {wl.cams.v}, one per step, after "
              f"{args.warmup} untimed (D={wl.d}, N={wl.scene.n})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "sample": "1 view per step (uplift only), all Gaussians"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "cpu_model": cpu_model(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- our arm
def oracle_child(workload_name, steps=3, warmup=3):
    """`bench.py --impl reference` on a workload, in a child process with no GPU
    visible; its cpu_baseline object, or an error object."""
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", workload_name,
           "--steps", str(steps), "--warmup", str(warmup)]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=900)
    line = next((json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")), None)
    if r.returncode != 0 or line is None:
        return {"value": None, "unit": UNIT, "kind": "oracle", "error": (r.stderr or "no output")[-300:]}
    cb = dict(line["cpu_baseline"])
    cb["sample"] += "; run as a child process, as the reference arm"
    return cb


def tiny_line(with_oracle):
    """The tiny mask workload (20k uniform Gaussians, 8 views of 128x128, D = 1
    float32 sphere masks): latency-bound, so the figure is microseconds per
    call of the whole 8-view uplift (CUDA events over 50 calls after 5 warm-up
    calls, features resident), beside the oracle's views*ch/s on the host."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    wl = workload("tiny")
    V, H, W = wl.cams.v, wl.cams.height, wl.cams.width
    sc = ludvig.Scene.from_inputs(wl.scene)
    feats = torch.stack([wl.features(v, device="cuda") for v in range(V)]).float().contiguous()   # [V,H,W,1]
    out = torch.empty((sc.n, 1), device="cuda")
    beta = torch.empty((sc.n,), device="cuda")
    for _ in range(5):
        ludvig.uplift(sc, wl.cams.params, W, H, feats, out, beta)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    calls = 50
    e0.record()
    for _ in range(calls):
        ludvig.uplift(sc, wl.cams.params, W, H, feats, out, beta)   # ends with ludvig_sync
    e1.record()
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / calls
    # the same calls enqueued back to back (one ludvig_sync at the end), and
    # the host time of one enqueue
    e0.record()
    t0 = time.perf_counter()
    for _ in range(calls):
        ludvig.uplift(sc, wl.cams.params, W, H, feats, out, beta, sync=False)
    host_us = (time.perf_counter() - t0) * 1e6 / calls
    sc.sync()
    e1.record()
    torch.cuda.synchronize()
    us_async = e0.elapsed_time(e1) * 1e3 / calls
    line = {"workload": wl.name, "us_per_call": us, "value": V * 1 / (us / 1e6), "unit": UNIT,
            "us_per_call_back_to_back": us_async, "host_enqueue_us_per_call": host_us,
            "bound": "latency (launches and the D-independent walk; 0.5 MB of features)",
            "timing": "us_per_call: each call ends with ludvig_sync (call to result); back to back: "
                      "50 calls enqueued without a wait, one ludvig_sync after them"}
    if with_oracle:
        line["cpu_baseline"] = oracle_child("tiny")
    return line


def cpu_baseline(args):
    """The oracle on the host cores, timed exactly as the reference arm times
    it: a child process running `bench.py --impl reference` with this run's
    workload, steps and warm-up (at most 8 and 5: one view per step, so the
    same views as the reference arm of the same command), so that the two
    agree; this process's GPU work and its threads stay out of the timing."""
    return oracle_child(args.workload, steps=max(1, min(8, args.steps)), warmup=max(0, min(5, args.warmup)))


# DRAM bytes (read + write) of one k_aggregate_tc launch, from the ncu capture in
# profiles/aggregate_paper_f32_traffic.md (profile case uplift16views: one
# 16-view launch): (workload, dtype, d) -> (bytes, views in the captured
# launch).  Scaled to a launch by its views; re-measure whenever the kernel
# changes.
TRAFFIC = {("paper", "f32", 384): (26.17e9, 15)}


def roofline(tr, steps, alg_bytes_step, traffic_key=None, views_per_launch=None):
    """HBM roofline of the kernel that reads the features: the tensor-core
    aggregation (k_aggregate_tc) when it ran, else the CUDA-core composite.
    Algorithmic bytes per step: the features once, 44 B per Gaussian, and
    num/den once (4 N (D + 1)); per launch, that over the launches of a step
    (one per chunk of up to 16 views).  Time: CUDA events around each launch
    on the stream it runs on."""
    stage = "aggregate" if tr["calls"].get("aggregate", 0) > 0 else "composite"
    kernel = "k_aggregate_tc" if stage == "aggregate" else "k_composite"
    launch_ms = tr["ms"][stage] / max(1, tr["calls"][stage])
    launches = tr["calls"][stage] / steps
    alg_per_launch = alg_bytes_step / max(1.0, launches)
    peak, peak_kind = peaks()
    achieved = alg_per_launch / (launch_ms / 1e3) / 1e9
    traffic = None
    if stage == "aggregate" and traffic_key in TRAFFIC and views_per_launch:
        b, v = TRAFFIC[traffic_key]
        traffic = b * views_per_launch / v
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
            "alg_bytes_per_launch": alg_per_launch, "launch_ms": launch_ms}


def precision_form(sc, wl):
    """bfloat16 features with D=512 on the same scene and cameras (tensor-core
    aggregation), timed over the full uplift; its error is stated against the
    float32 path on the first 8 views."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    V, H, W = wl.cams.v, wl.cams.height, wl.cams.width
    D = 512
    fb = torch.empty((V, H, W, D), dtype=torch.bfloat16, device="cuda")
    for v in range(V):
        fb[v] = wl.features_d(v, D, device="cuda", dtype=torch.bfloat16)
    out = torch.empty((sc.n, D), dtype=torch.float32, device="cuda")
    beta = torch.empty((sc.n,), dtype=torch.float32, device="cuda")
    ludvig.uplift(sc, wl.cams.params, W, H, fb, out, beta)
    torch.cuda.synchronize()
    ludvig.trace_read(reset=True)
    ludvig.trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        ludvig.uplift(sc, wl.cams.params, W, H, fb, out, beta)
    e1.record()
    torch.cuda.synchronize()
    ludvig.trace_enable(False)
    tr = ludvig.trace_read(reset=True)
    ms = e0.elapsed_time(e1) / reps
    # error vs the float32 path on views 0..7 (same D=512 field)
    nv = 8
    f32 = torch.stack([wl.features_d(v, D, device="cuda") for v in range(nv)]).contiguous()
    o32, b32 = ludvig.uplift(sc, wl.cams.params[:nv], W, H, f32)
    obf, bbf = ludvig.uplift(sc, wl.cams.params[:nv], W, H, fb[:nv].contiguous())
    torch.cuda.synchronize()
    pos = b32 > 0
    err = float((obf[pos] - o32[pos]).norm() / o32[pos].norm())
    roof = roofline(tr, reps, V * H * W * D * 2 + sc.n * 44 + sc.n * (D + 1) * 4)
    del fb
    torch.cuda.empty_cache()
    fp8 = fp8_variant(sc, wl, D, o32, b32, nv)
    del f32
    torch.cuda.empty_cache()
    return {"value": V * D / (ms / 1e3), "unit": UNIT, "ms_per_uplift": ms, "dtype": "bf16", "fp8_variant": fp8,
            "config": {"workload": wl.name.replace("-d384", "-d512"), "d": D, "step": "uplift only",
                       "aggregation": "tcgen05 kind::f16, bf16 weights, fp32 accumulation"},
            "rel_l2_vs_f32_path": err, "err_views": nv,
            "roofline": roof,
            "stages_ms_per_uplift": {k: v / reps for k, v in tr["ms"].items() if v > 0}}


def fp8_variant(sc, wl, D, o32, b32, nv):
    """The FP8-E4M3 variant of the precision form: every view of the float32
    field quantised with its absmax scale (ludvig_fp8_quantize), then the
    FP8 uplift (ludvig_uplift_fp8: codes decoded to bfloat16 per 16-view
    group, bfloat16 tensor-core path), timed over the full uplift; its error
    against the float32 path on the first ``nv`` views."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    V, H, W = wl.cams.v, wl.cams.height, wl.cams.width
    try:
        q = torch.empty((V, H, W, D), dtype=torch.uint8, device="cuda")
        s = torch.empty((V,), dtype=torch.float32, device="cuda")
        for v in range(V):
            ludvig.fp8_quantize(wl.features_d(v, D, device="cuda")[None], q[v:v + 1], s[v:v + 1])
        out = torch.empty((sc.n, D), dtype=torch.float32, device="cuda")
        beta = torch.empty((sc.n,), dtype=torch.float32, device="cuda")
        ludvig.uplift_fp8(sc, wl.cams.params, W, H, q, s, out, beta)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ludvig.uplift_fp8(sc, wl.cams.params, W, H, q, s, out, beta)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        o8, _ = ludvig.uplift_fp8(sc, wl.cams.params[:nv], W, H, q[:nv], s[:nv])
        torch.cuda.synchronize()
        pos = b32 > 0
        err = float((o8[pos] - o32[pos]).norm() / o32[pos].norm())
        res = {"value": V * D / (ms / 1e3), "unit": UNIT, "ms_per_uplift": ms, "dtype": "fp8-e4m3",
               "storage_gb": q.numel() / 1e9, "rel_l2_vs_f32_path": err, "err_views": nv,
               "form": "per-view absmax scale; codes decoded to bf16 in the aggregation's shared memory (d % 16 == 0), bf16 tensor-core path"}
        del q, out, beta, o8
        return res
    except Exception as e:   # reported in the line; the other forms stand
        return {"error": str(e)}


# DRAM bytes (read + write) of one k_render_tc launch, from the ncu capture in
# profiles/render_paper_f32.md: d -> (bytes, views in the captured launch).
RENDER_TRAFFIC = {384: (21.758e9, 16)}


def render_back(sc, wl, f):
    """Render-back F_hat = W f (Eq. 4) of the uplifted features f [N, D] into
    every view of the workload, timed over whole ludvig_render calls.  The
    roofline is that of the product kernel (k_render_tc): algorithmic bytes per
    launch = the launch's output maps (views x H x W x D x 4) + f read once
    (N x D x 4)."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    V, H, W = wl.cams.v, wl.cams.height, wl.cams.width
    D = int(f.shape[1])
    out = torch.empty((V, H, W, D), dtype=torch.float32, device="cuda")
    ludvig.render(sc, wl.cams.params, W, H, f, out=out)
    torch.cuda.synchronize()
    ludvig.trace_read(reset=True)
    ludvig.trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        ludvig.render(sc, wl.cams.params, W, H, f, out=out)
    e1.record()
    torch.cuda.synchronize()
    ludvig.trace_enable(False)
    tr = ludvig.trace_read(reset=True)
    ms = e0.elapsed_time(e1) / reps
    launches = tr["calls"]["render_product"] / reps
    launch_ms = tr["ms"]["render_product"] / max(1, tr["calls"]["render_product"])
    views_per_launch = V / launches
    alg = views_per_launch * H * W * D * 4 + sc.n * D * 4
    peak, peak_kind = peaks()
    achieved = alg / (launch_ms / 1e3) / 1e9
    traffic = None
    if D in RENDER_TRAFFIC:
        b, v = RENDER_TRAFFIC[D]
        traffic = b * views_per_launch / v
    del out
    torch.cuda.empty_cache()
    return {"value": V * D / (ms / 1e3), "unit": UNIT, "ms_per_render": ms, "dtype": "f32",
            "config": {"workload": wl.name, "d": D, "views": V,
                       "f": "the step's uplifted features", "out": "[V,H,W,D] float32 in HBM"},
            "roofline": {"bound": "hbm", "kernel": "k_render_tc", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": traffic,
                         "alg_bytes_per_launch": alg, "launch_ms": launch_ms},
            "stages_ms_per_render": {k: v / reps for k, v in tr["ms"].items() if v > 0},
            "gpu_launches_per_render": tr["kernel_launches"] / reps}


def beta_filter(sc, wl, beta, feats):
    """Gaussian filtering (Sec. 3.2): keep the half of the Gaussians with the
    largest beta of the step's uplift (ludvig_beta_select, CUDA events), build
    the filtered scene (ludvig_scene_subset, host clock: it synchronises), and
    uplift the same views on it (the saving that later uplifts see).  Roofline
    of the selection: algorithmic bytes = beta read once (4 N) + the kept
    indices written once (4 keep)."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    V, H, W, D = wl.cams.v, wl.cams.height, wl.cams.width, int(feats.shape[-1])
    n = sc.n
    keep = n - n // 2
    kept = ludvig.beta_select(sc, beta, keep)
    ludvig.beta_select(sc, beta, keep)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record()
    for _ in range(reps):
        kept = ludvig.beta_select(sc, beta, keep)
    e1.record()
    torch.cuda.synchronize()
    sel_ms = e0.elapsed_time(e1) / reps
    t0 = time.perf_counter()
    sub = sc.subset(kept)
    sub_ms = (time.perf_counter() - t0) * 1e3
    out = torch.empty((sub.n, D), dtype=torch.float32, device="cuda")
    b2 = torch.empty((sub.n,), dtype=torch.float32, device="cuda")
    ludvig.uplift(sub, wl.cams.params, W, H, feats, out, b2)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(2):
        ludvig.uplift(sub, wl.cams.params, W, H, feats, out, b2)
    e1.record()
    torch.cuda.synchronize()
    up_ms = e0.elapsed_time(e1) / 2
    sub.close()
    peak, peak_kind = peaks()
    alg = 4.0 * n + 4.0 * keep
    achieved = alg / (sel_ms / 1e3) / 1e9
    return {"kept": keep, "of": n, "select_ms": sel_ms, "subset_ms": sub_ms,
            "uplift_filtered_ms": up_ms, "uplift_filtered_value": V * D / (up_ms / 1e3), "unit": UNIT,
            "roofline": {"bound": "hbm", "kernel": "ludvig_beta_select (sort + mark + compact)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None, "alg_bytes_per_launch": alg,
                         "launch_ms": sel_ms}}


def paper_diffusion(sc, wl, f_all, beta):
    """Paper-form diffusion in the paper's order: the half of the Gaussians
    with the largest beta of the step's uplift is kept (Sec. 5), and their
    uplifted features f are used (Eq. 7 with the appendix's S_f and P, Sec.
    4.1): the scene part (kNN graph, edge feature
    distances, s_f), the segmentation prompt (g_0 from the uplifted view-0
    mask of a sphere around the first cluster centre, P with b_P = 5, A with
    b = 0.5 binarised at 1e-5, reachability weight h after 100 steps) and the
    21-query diffusion of 100 steps on the row-normalised RBF graph (the
    paper's multi-query case).  Roofline of the reachability step kernel:
    algorithmic bytes per step = the CSR streamed once (8 nnz + 8 n) + the bit
    sets read and written once (8 n)."""
    import torch
    from paper_2410_14462_gb300 import inputs, ludvig
    W, H = wl.cams.width, wl.cams.height
    centre = inputs.cluster_centres(wl.seed)[0]
    mask = torch.from_numpy(inputs.sphere_masks(wl.cams.subset([0]), radius=0.3, center=centre)).cuda()
    kept = ludvig.beta_select(sc, beta, sc.n - sc.n // 2)
    full, sc = sc, sc.subset(kept)
    f = f_all[kept.long()].contiguous()
    u, _ = ludvig.uplift(sc, wl.cams.params[:1], W, H, mask.contiguous())
    u = u[:, 0].contiguous()

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3 / reps, r

    scene_ms, G = timed(lambda: ludvig.Graph.rbf(sc, 16, f))
    s_f = G.feature_scale

    def prompt():
        g0 = ludvig.topfrac_positive(sc, u, 10)
        P = G.unary_anchor(f, g0, 5.0)
        G.reweight(0.5, P, binarize=1e-5, row_normalize=False)
        return G.reach_weight(g0, 100, P)

    prompt()
    torch.cuda.synchronize()
    ludvig.trace_read(reset=True)
    ludvig.trace_enable(True)
    prompt_ms, h = timed(prompt, reps=3)
    ludvig.trace_enable(False)
    tr = ludvig.trace_read(reset=True)
    reach_ms = tr["ms"]["diffuse"] / max(1, tr["calls"]["diffuse"]) / 100
    reached = int((h > 0).sum().item())
    anchors = int((ludvig.topfrac_positive(sc, u, 10) > 0).sum().item())
    G.reweight(0.5, None, binarize=0.0, row_normalize=True)
    x0 = torch.zeros((sc.n, 21), device="cuda")
    x0[torch.arange(21, device="cuda") * 997, torch.arange(21, device="cuda")] = 1.0
    q21_ms, _ = timed(lambda: G.diffuse(x0, 100), reps=2)
    nnz = G.nnz
    G.close()
    n_kept = sc.n
    sc.close()
    peak, peak_kind = peaks()
    alg = 8.0 * nnz + 16.0 * n_kept
    achieved = alg / (reach_ms / 1e3) / 1e9
    return {"gaussians": n_kept, "of": full.n, "scene_ms": scene_ms, "prompt_ms": prompt_ms, "q21_diffusion_100_steps_ms": q21_ms, "s_f": s_f,
            "nnz": nnz, "anchors": anchors, "reached_after_100_steps": reached,
            "config": {"k": 16, "b": 0.5, "b_P": 5.0, "binarize": 1e-5, "steps": 100, "g0": "top 10 % of the "
                       "uplifted view-0 mask", "queries_multi": 21},
            "roofline": {"bound": "hbm", "kernel": "k_reach_step", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "alg_bytes_per_launch": alg, "launch_ms": reach_ms}}


def relevancy_line(f):
    """LERF relevancy (appendix) of the step's uplifted features f [N, D] to 21
    seeded query embeddings against 4 canonical-phrase embeddings (T = 10),
    timed with CUDA events.  Roofline: algorithmic bytes = f read once (4 N D)
    + r written once (4 N q)."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    n, d = f.shape
    g = torch.Generator(device="cuda").manual_seed(11)
    pq = torch.randn((21, d), device="cuda", generator=g)
    pc = torch.randn((4, d), device="cuda", generator=g)
    r = ludvig.relevancy(f, pq, pc, 10.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record()
    for _ in range(reps):
        ludvig.relevancy(f, pq, pc, 10.0, out=r)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    alg = 4.0 * n * d + 4.0 * n * 21
    peak, peak_kind = peaks()
    achieved = alg / (ms / 1e3) / 1e9
    return {"ms": ms, "gaussians": n, "d": d, "queries": 21, "phrases": 4,
            "roofline": {"bound": "hbm", "kernel": "k_relevancy", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
                         "alg_bytes_per_launch": alg, "launch_ms": ms}}


def count_normalised_line(sc, wl, feats):
    """The uplift of the step's 150 views with GaussianEditor's normaliser
    (LUDVIG_OPT_COUNT_NORMALISE = 1): same kernels, the weights kernel counts
    instead of summing; CUDA events around one uplift after a warm-up."""
    import torch
    from paper_2410_14462_gb300 import ludvig
    V, H, W, D = wl.cams.v, wl.cams.height, wl.cams.width, int(feats.shape[-1])
    out = torch.empty((sc.n, D), dtype=torch.float32, device="cuda")
    cnt = torch.empty((sc.n,), dtype=torch.float32, device="cuda")
    ludvig.set_option(ludvig.OPT_COUNT_NORMALISE, 1)
    try:
        ludvig.uplift(sc, wl.cams.params, W, H, feats, out, cnt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ludvig.uplift(sc, wl.cams.params, W, H, feats, out, cnt)
        e1.record()
        torch.cuda.synchronize()
    finally:
        ludvig.set_option(ludvig.OPT_COUNT_NORMALISE, 0)
    ms = e0.elapsed_time(e1)
    contrib = float(cnt.double().sum().item())   # sum over views and pixels of the w > 0 contributors
    return {"ms": ms, "value": V * D / (ms / 1e3), "unit": UNIT,
            "max_count": float(cnt.max().item()), "gaussians_counted": int((cnt > 0).sum().item()),
            "contributions": contrib,
            "aggregation_algorithmic_tflop": (2 * D + 1) * contrib / 1e12,
            "note": ("contributions = sum_i count_i = sum over (view, pixel) of the Gaussians with w > 0; "
                     "the aggregation's algorithmic work is 2 D flops per contribution (+1 for den)")}


def batched_form(pools, cams, slots=6):
    """32 uplift jobs of uneven size (N log-uniform in [50k, 1M] clustered
    Gaussians, V uniform in [20, 200] views of 640x480, D uniform over
    {1, 3, 64, 384, 512}) with bfloat16 features from shared device pools,
    run by one ludvig_uplift_batch call: the jobs' views packed into shared
    groups per (dtype, D) class, group sizes picked by the library's tuner
    during the untimed first batch.  Beside it the unpacked forms (every job
    its own ludvig_uplift call) one after another on one stream and on
    ``slots`` concurrent streams, and the plain float32 form (the same values
    widened to float32, views in chunks of 48), each timed with CUDA events.
    The bfloat16 error is stated against the float64 oracle on the same
    bfloat16 values for the two cheapest jobs to check (all their views), and
    against the float32 path on true float32 features (8 views of the first
    job with D >= 64)."""
    import torch
    import oracle
    from paper_2410_14462_gb300 import inputs, ludvig, serve
    W, H = cams.width, cams.height
    specs = inputs.batch_jobs()
    scenes = [ludvig.Scene.from_inputs(inputs.scene_clusters(s.n, seed=s.seed)) for s in specs]
    jobs = [serve.Job(j, scenes[j], s.d, s.v0, s.views) for j, s in enumerate(specs)]
    work = sum(j.views * j.d for j in jobs)
    res = serve.run_batch(jobs, pools, cams.params, W, H, slots=slots)   # warm-up: tuning, workspaces grow
    if res["errors"]:
        raise RuntimeError(f"batched form: {res['errors']}")
    plan = ludvig.batch_last_plan()
    ludvig.trace_read(reset=True)
    reps = 2
    runs = [serve.run_batch(jobs, pools, cams.params, W, H, slots=slots, keep_outputs=(r == reps - 1))
            for r in range(reps)]
    batched = [r["device_ms"] for r in runs]
    launches = ludvig.trace_read(reset=True)["kernel_launches"] / reps
    kept = runs[-1]["outputs"]
    ludvig.batch_release_workspaces()     # the packed contexts; the unpacked form lends slot workspaces
    ludvig.set_option(ludvig.OPT_BATCH_PACK, 0)
    unpacked_slots = 3   # each slot lends a workspace grown to its largest job: bounded beside the pools

    def unpacked(n_slots):
        r = serve.run_batch(jobs, pools, cams.params, W, H, slots=n_slots)
        if r["errors"]:
            raise RuntimeError(f"unpacked batched form: {r['errors']}")
        return r["device_ms"]

    try:
        unpacked(unpacked_slots)     # the lent workspaces grow
        ludvig.trace_read(reset=True)
        ludvig.trace_enable(True)    # stage split of the one-stream run (stages do not overlap there)
        serial = unpacked(1)
        ludvig.trace_enable(False)
        tr = ludvig.trace_read(reset=True)
        stages = {k: v for k, v in tr["ms"].items() if v > 0}
        launches_unpacked = tr["kernel_launches"]
        concurrent = unpacked(unpacked_slots)
    finally:
        ludvig.set_option(ludvig.OPT_BATCH_PACK, 1)
        ludvig.batch_release_workspaces()
        torch.cuda.empty_cache()
    # bfloat16 vs float64 on sampled jobs: the two cheapest for the oracle
    checks = []
    for j in sorted(jobs, key=lambda j: j.scene.n * j.views * (j.d + 32))[:2]:
        s = specs[j.jid]
        host = inputs.scene_clusters(s.n, seed=s.seed)
        sub = inputs.Cameras(cams.params[j.v0:j.v0 + j.views], W, H)
        X = pools[j.d][j.v0:j.v0 + j.views].float().cpu().numpy()
        t0 = time.perf_counter()
        f_ref, b_ref = oracle.uplift(host, sub, lambda v: X[v])
        out, beta = kept[j.jid]
        pos = b_ref > 0
        got = out.cpu().numpy().astype(np.float64)
        e = float(np.linalg.norm(got[pos] - f_ref[pos]) / max(np.linalg.norm(f_ref[pos]), 1e-300))
        checks.append({"job": j.jid, "n": s.n, "views": j.views, "d": j.d, "rel_l2_vs_fp64": e,
                       "beta_support_equal": bool(np.array_equal(beta.cpu().numpy() > 0, pos)),
                       "oracle_s": time.perf_counter() - t0})
        del X, f_ref, b_ref
    del kept, runs
    # plain float32 form, one job after another; each job's scene is made
    # afresh (the resident scenes' workspaces are freed first) and its float32
    # pass runs once untimed so that the workspace has grown before timing
    je = next(j for j in jobs if j.d >= 64)
    nv = 8
    fe = torch.stack([inputs.feature_field(5, je.v0 + v, je.d, H, W, device="cuda") for v in range(nv)]).contiguous()
    o32, b32 = ludvig.uplift(je.scene, cams.params[je.v0:je.v0 + nv], W, H, fe)
    obf, _ = ludvig.uplift(je.scene, cams.params[je.v0:je.v0 + nv], W, H, pools[je.d][je.v0:je.v0 + nv])
    torch.cuda.synchronize()
    pos = b32 > 0
    err = float((obf[pos] - o32[pos]).norm() / o32[pos].norm())
    err_case = f"job with N={je.scene.n}, D={je.d}, {nv} views"
    del fe, o32, b32, obf, pos
    for sc in scenes:
        sc.close()
    ludvig.batch_release_workspaces()
    torch.cuda.empty_cache()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plain_ms = 0.0
    for j in jobs:
        sc = ludvig.Scene.from_inputs(inputs.scene_clusters(specs[j.jid].n, seed=specs[j.jid].seed))
        num = torch.zeros((sc.n, j.d), dtype=torch.float32, device="cuda")
        den = torch.zeros((sc.n,), dtype=torch.float32, device="cuda")
        for rep in range(2):
            num.zero_()
            den.zero_()
            for c0 in range(0, j.views, 48):
                c1 = min(j.views, c0 + 48)
                f32 = pools[j.d][j.v0 + c0:j.v0 + c1].float()
                torch.cuda.synchronize()
                e0.record()
                ludvig.uplift_accumulate(sc, cams.params[j.v0 + c0:j.v0 + c1], W, H, f32, num, den)
                e1.record()
                torch.cuda.synchronize()
                plain_ms += e0.elapsed_time(e1) if rep == 1 else 0.0
                del f32
            e0.record()
            ludvig.uplift_finalize(num, den)
            e1.record()
            torch.cuda.synchronize()
            plain_ms += e0.elapsed_time(e1) if rep == 1 else 0.0
        del num, den
        sc.close()
        torch.cuda.empty_cache()
    ms = float(np.median(batched))
    out = {"value": work / (ms / 1e3), "unit": UNIT, "dtype": "bf16", "ms_per_batch": ms,
           "ms_per_batch_runs": batched, "serial_bf16_ms": serial, "unpacked_concurrent_bf16_ms": concurrent,
           "plain_f32_serial_ms": plain_ms,
           "unpacked_concurrent_slots": unpacked_slots,
           "speedup_vs_serial_bf16": serial / ms, "speedup_vs_unpacked_concurrent": concurrent / ms,
           "speedup_vs_plain_f32": plain_ms / ms,
           "plain_f32_value": work / (plain_ms / 1e3), "gpu_launches_per_batch": launches,
           "gpu_launches_unpacked": launches_unpacked, "plan": plan,
           "bf16_vs_fp64_sampled_jobs": checks,
           "rel_l2_bf16_vs_f32": err, "err_case": err_case, "serial_stages_ms": stages,
           "config": {"workload": "32 jobs: N log-uniform [50k, 1M], V U[20, 200] of 640x480, "
                                  "D U{1, 3, 64, 384, 512}, bf16 pools, seed 3",
                      "jobs": len(jobs), "views_ch": work, "gaussians": sum(s.n for s in specs),
                      "slots": slots,
                      "form": "ludvig_uplift_batch: views packed into shared groups per (dtype, D) class, "
                              "group size tuned per class, classes on concurrent contexts"}}
    return out


def serving_form(pools, cams, slots=2, n_requests=900, rate=200.0):
    """Requests against 4 resident scenes (N = 250k, 500k, 750k, 1M clustered
    Gaussians, seeds 40-43): Poisson arrivals at ``rate`` req/s; each request
    uplifts V U[10, 150] views of 640x480 bfloat16 features with D uniform
    over {1, 64, 384, 512}, and half of them then run U[20, 100] diffusion
    steps (k = 16 graph from an uplift of 20 views at D = 384) on the uplifted
    first channel.  A 150 GB budget covers the replicas, every replica's and
    graph's workspace and the outputs in flight; the replicas' groups are
    bounded at 512 MiB of scratch (LUDVIG_OPT_GROUP_MB) so that eight
    workspaces leave room for the outputs.  The first run offers more
    work than the GPU serves for 4.5 s (the queue grows), so its throughput
    is the service capacity; the second replays 100 requests at 70% of that
    capacity.  Both report latency percentiles and the queue depth at
    arrival."""
    import torch
    from paper_2410_14462_gb300 import inputs, ludvig, serve
    W, H = cams.width, cams.height
    scenes = [ludvig.Scene.from_inputs(inputs.scene_clusters(n, seed=s)) for n, s in inputs.SERVING_SCENES]
    graphs = []
    for sc in scenes:
        f, _ = ludvig.uplift(sc, cams.params[:20], W, H, pools[384][:20])
        graphs.append(ludvig.Graph(sc, 16, f, spatial_h=0.01))
        del f
    pools = {d: pools[d] for d in (1, 64, 384, 512)}
    group_mb = ludvig.get_option(ludvig.OPT_GROUP_MB)
    ludvig.set_option(ludvig.OPT_GROUP_MB, 512)
    server = serve.Server(scenes, graphs, pools, cams.params, W, H, 150e9, slots=slots)
    # warm-up: every replica's workspace grows to the largest request
    warm = [serve.Request(i, 0.0, i % len(scenes), 512, 0, 150, 100) for i in range(len(scenes) * slots)]
    server.run(warm)
    resident = server.resident_bytes()

    def served_work(reqs, res):
        return sum(q.views * q.d for q, r in zip(reqs, res) if r.ok)

    reqs = serve.poisson_requests(n_requests, rate, len(scenes), cams.v, (1, 64, 384, 512), seed=4)
    ludvig.trace_read(reset=True)
    res = server.run(reqs)
    launches = ludvig.trace_read(reset=True)["kernel_launches"]
    over = serve.latency_summary(res)
    cap = over["throughput_req_s"] or 1.0
    span = max(r.done for r in res) - min(r.arrival for r in res)
    reqs2 = serve.poisson_requests(100, 0.7 * cap, len(scenes), cams.v, (1, 64, 384, 512), seed=45)
    res2 = server.run(reqs2)
    under = serve.latency_summary(res2)
    span2 = max(r.done for r in res2) - min(r.arrival for r in res2)
    server.close()
    ludvig.set_option(ludvig.OPT_GROUP_MB, group_mb)
    for g in graphs:
        g.close()
    for sc in scenes:
        sc.close()
    torch.cuda.synchronize()
    over.update({"rate_req_s": rate, "views_ch_per_s": served_work(reqs, res) / span, "gpu_launches": launches})
    under.update({"rate_req_s": 0.7 * cap, "views_ch_per_s": served_work(reqs2, res2) / span2})
    return {"p50_ms": over["p50_ms"], "p99_ms": over["p99_ms"], "throughput_req_s": over["throughput_req_s"],
            "unit": "ms (latency = completion - arrival, queueing included)",
            "offered_200_req_s": over, "at_70pct_capacity": under,
            "config": {"workload": "4 resident scenes N 250k/500k/750k/1M (seeds 40-43); Poisson arrivals; "
                                   "V U[10, 150] of 640x480, D U{1, 64, 384, 512} bf16; 50% + U[20, 100] "
                                   "diffusion steps", "slots_per_scene": slots, "budget_bytes": 150e9,
                       "group_mb": 512,
                       "resident_bytes_after_warmup": resident,
                       "requests": [n_requests, 100], "seeds": [4, 45]}}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2410_14462_gb300 import build, inputs, ludvig, shard

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    L = ludvig.load()

    wl = workload(args.workload)
    W, H, V, D = wl.cams.width, wl.cams.height, wl.cams.v, wl.d
    fdt = torch.float32 if args.dtype == "f32" else torch.bfloat16
    esize = 4 if args.dtype == "f32" else 2
    sc = ludvig.Scene.from_inputs(wl.scene)
    feats = torch.empty((V, H, W, D), dtype=fdt, device="cuda")
    for v in range(V):
        feats[v] = wl.features(v, device="cuda", dtype=fdt)
    out = torch.empty((sc.n, D), dtype=torch.float32, device="cuda")
    beta = torch.empty((sc.n,), dtype=torch.float32, device="cuda")
    centre = inputs.cluster_centres(wl.seed)[0]
    x0 = torch.from_numpy((np.linalg.norm(wl.scene.means - centre, axis=1) < 0.15).astype(np.float32)).cuda()
    g_out = torch.empty_like(x0)
    torch.cuda.synchronize()

    def step():
        ludvig.uplift(sc, wl.cams.params, W, H, feats, out, beta)
        if not args.no_graph:
            g = ludvig.Graph(sc, 16, out, spatial_h=0.01)
            g.diffuse(x0, 100, out=g_out)
            g.close()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    ludvig.trace_read(reset=True)
    ludvig.trace_enable(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ludvig.trace_enable(False)
    tr = ludvig.trace_read(reset=True)
    clk = clocks.stop()
    ms = shard.max_over_ranks(ms, device="cuda")
    value = world * V * D / (ms / 1e3)

    launches = max(1.0, tr["calls"].get("aggregate", 0) / args.steps)
    roof = roofline(tr, args.steps, V * H * W * D * esize + sc.n * 44 + sc.n * (D + 1) * 4,
                    (args.workload, args.dtype, D), V / launches)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": wl.name, "n_gaussians": sc.n, "views": V, "width": W, "height": H,
                       "d": D, "step": ("uplift" if args.no_graph else
                                        "uplift + kNN(k=16) graph + 100 diffusion steps"),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs (features) larger than L2; no flush"},
            "stages_ms_per_step": {k: v / args.steps for k, v in tr["ms"].items()},
            "stages_note": ("device-event intervals on the stream that runs each stage; a group's front end "
                            "(project, depth sort) is enqueued while the previous group's aggregation holds "
                            "every SM, so those intervals include the wait for SMs; the kernel times are in "
                            "the ncu launch list"),
            "gpu_launches": tr["kernel_launches"],
            "roofline": roof, "clocks": clk}

    if rank == 0 and not args.no_e2e:
        nv = min(args.e2e_views, V)
        node, cpus = gpu_local_cpus(gpu_id)
        hf = pinned_near(tuple(feats[:nv].shape), fdt, cpus)   # pages next to the GPU
        hf.copy_(feats[:nv])
        scratch = torch.empty_like(feats[:nv])
        h2d_gbs, d2h_gbs = copy_rates(hf, scratch)
        del scratch
        torch.cuda.empty_cache()
        ho = pinned_near((sc.n, D), torch.float32, cpus)   # the caller's result buffers, made once
        hb = pinned_near((sc.n,), torch.float32, cpus)
        for _ in range(2):   # warm-up: the first call grows the upload buffers
            ludvig.uplift_host(sc, wl.cams.params[:nv], W, H, hf, out=ho, beta=hb)
        ts = []
        for _ in range(max(3, min(5, args.steps))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ludvig.uplift_host(sc, wl.cams.params[:nv], W, H, hf, out=ho, beta=hb)
            ts.append(time.perf_counter() - t0)
        te = float(np.median(ts))
        bi, bo = int(hf.numel() * esize), int(sc.n * (D + 1) * 4)
        line["e2e"] = {"value": nv * D / te, "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                       "seconds_per_step": te, "seconds_samples": [round(x, 4) for x in ts],
                       "h2d_gbs_measured": h2d_gbs, "d2h_gbs_measured": d2h_gbs,
                       "copy_floor_s": bi / (h2d_gbs * 1e9) + bo / (d2h_gbs * 1e9),
                       "pinned_numa_node": node, "pinned_near_cpus": len(cpus) if cpus else None,
                       "sample": (f"views 0-{nv - 1} of {V} through ludvig_uplift_host (uplift only) into "
                                  "pinned result buffers the caller made once; "
                                  "the host->device rate is one plain copy of the same pinned buffer")}
        del hf, ho, hb
    if rank == 0 and not args.no_relevancy and args.workload == "paper" and args.dtype == "f32":
        line["count_normalised_uplift"] = count_normalised_line(sc, wl, feats)
        line["relevancy"] = relevancy_line(out)
    if rank == 0 and not args.no_filter and args.workload == "paper" and args.dtype == "f32":
        line["beta_filter"] = beta_filter(sc, wl, beta, feats)
    if rank == 0 and not args.no_precision and args.workload == "paper":
        del feats
        feats = None
        torch.cuda.empty_cache()
        line["precision_form"] = precision_form(sc, wl)
        torch.cuda.empty_cache()
    if rank == 0 and not args.no_paper_diffusion and args.workload == "paper" and args.dtype == "f32":
        line["paper_diffusion"] = paper_diffusion(sc, wl, out, beta)
    if rank == 0 and not args.no_render and args.dtype == "f32":
        feats = None
        torch.cuda.empty_cache()
        line["render_back"] = render_back(sc, wl, out)
    if rank == 0 and args.workload == "paper" and not (args.no_batched and args.no_serving):
        feats = None
        torch.cuda.empty_cache()
        fcams = inputs.form_cameras(200)
        dims = (1, 64, 384, 512) if args.no_batched else (1, 3, 64, 384, 512)
        pools = {d: inputs.form_pool(d, fcams) for d in dims}
        if not args.no_batched:
            line["batched_form"] = batched_form(pools, fcams)
        if not args.no_serving:
            line["serving"] = serving_form(pools, fcams)
        pools = None
        torch.cuda.empty_cache()
    if rank == 0 and args.workload == "paper":
        line["tiny_config"] = tiny_line(world == 1 and not args.no_cpu_baseline)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        del feats
        torch.cuda.empty_cache()
        line["cpu_baseline"] = cpu_baseline(args)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def profile_case(name):
    """ncu captures on views 0-1 of the paper-scale workload, D=384.
    tc2views: uplift twice with float32 features and twice with the same field
    in bfloat16.  render2views: render of seeded unit-norm features, three
    times.  render16views: the same render of views 0-15 (one full launch of
    the render kernels), three times.  uplift16views: float32 uplift of
    views 0-15 (one full launch of the aggregation, 13 GB of features), three
    times.  batch8: the first 8 jobs of the
    32-job batched mix through one ludvig_uplift_batch call (6 slots).
    tinymask: the tiny mask workload (20k Gaussians, 8 views of 128x128,
    D = 1 float32), uplifted four times."""
    import torch
    from paper_2410_14462_gb300 import build, inputs, ludvig
    build.build()
    ludvig.load()
    if name == "batch8":
        from paper_2410_14462_gb300 import serve
        cams = inputs.form_cameras(200)
        specs = inputs.batch_jobs()[:8]
        pools = {d: inputs.form_pool(d, cams) for d in sorted({s.d for s in specs})}
        scenes = [ludvig.Scene.from_inputs(inputs.scene_clusters(s.n, seed=s.seed)) for s in specs]
        jobs = [serve.Job(j, scenes[j], s.d, s.v0, s.views) for j, s in enumerate(specs)]
        res = serve.run_batch(jobs, pools, cams.params, cams.width, cams.height, slots=6)
        torch.cuda.synchronize()
        return 1 if res["errors"] else 0
    if name == "tinymask":
        wl = inputs.tiny_mask_workload()
        sc = ludvig.Scene.from_inputs(wl.scene)
        F = torch.stack([wl.features(v, device="cuda") for v in range(wl.cams.v)]).float().contiguous()
        for _ in range(4):
            ludvig.uplift(sc, wl.cams.params, wl.cams.width, wl.cams.height, F)
        torch.cuda.synchronize()
        return 0
    wl = inputs.paper_scale_workload(views=16 if name in ("render16views", "uplift16views") else 2, d=384)
    sc = ludvig.Scene.from_inputs(wl.scene)
    W, H = wl.cams.width, wl.cams.height
    if name in ("render2views", "render16views"):
        f = torch.from_numpy(inputs.gaussian_features(sc.n, 384, seed=21)).cuda()
        for _ in range(3):
            ludvig.render(sc, wl.cams.params, W, H, f)
        torch.cuda.synchronize()
        return 0
    if name == "uplift16views":
        F = torch.empty((16, H, W, 384), dtype=torch.float32, device="cuda")
        for v in range(16):
            F[v] = wl.features(v, device="cuda")
        for _ in range(3):
            ludvig.uplift(sc, wl.cams.params, W, H, F)
        torch.cuda.synchronize()
        return 0
    F = torch.stack([wl.features(v, device="cuda") for v in range(2)]).contiguous()
    Fb = F.to(torch.bfloat16)
    for _ in range(2):
        ludvig.uplift(sc, wl.cams.params, W, H, F)
        ludvig.uplift(sc, wl.cams.params, W, H, Fb)
    torch.cuda.synchronize()
    return 0


def main():
    args = parse()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
