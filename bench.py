#!/usr/bin/env python
"""Benchmark of the GES rasterizer hot path: fwd+bwd Mpixel/s at 1.5M splats.

Workload (default "drt8-1.5M"): the 1.5M-splat heightfield scene rendered into 8
views whose sizes follow the cosine dynamic-resolution schedule of Eq. 15
(400x260 ... 1600x1040, 6,252,862 pixels), SH degree 3, random upstream
gradients N(0,1) on colour, depth, alpha and normal. One step is the whole hot
path for all views: preprocess + binning, render forward, render backward,
preprocess backward, run as captured CUDA graphs (persistent render over a
longest-first tile queue). The same views are also timed through the plain
one-view-per-launch path for comparison ("per_view").

Beside the headline: per-kernel rooflines of the render kernels against FP32-FMA and
ex2 peaks measured on the GPU by the library's microbenchmarks ("rooflines",
"peaks_measured"), HBM fractions of preprocess, binning and preprocess backward
("hbm_stages"), the end-to-end step from pinned host buffers with the host link's
own bandwidth ("e2e"), the training step with the Eq. 8 loss, binary16 colour
storage, the GSR and level-set legs, and the other workloads ("other_workloads":
the 1k-splat, 100k-splat and 1.5M-splat single views, and the 3M-splat 16-view
batch against 16 sequential one-view steps).

Prints one JSON line (rank 0). With --impl reference it times the FP64 CPU
oracle instead (the reference arm of this benchmark), on a bounded pixel sample.
Under torchrun each rank renders its own independent batch of views (weak
scaling, no collective on the data path); the reported time is the max over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Mpixel/s at 1.5M splats, batched vs per-view, and % of HBM roofline"
F_TEST = 10          # FP32 flops per evaluated (pixel, list entry) pair: dx, dy, Q
F_BLEND_FWD = 26     # per blended pair in the forward (falloff, alpha, transmittance, 7 accumulations)
F_BLEND_BWD = 104    # per blended pair in the backward replay (forward blend + 78 gradient flops)
MUFU_FWD = 3         # special-function operations per blended pair: log2 Q, exp2 for Q^(beta/2), exp2 for G
MUFU_BWD = 6         # the replay's three, rcp(1 - alpha), rcp(Q) and log2 Q of the beta gradient
F_LOSS = 1188        # per pixel of the Eq. 8 loss and its gradient (3 channels x 396: 5 window maps x 2
                     # separable passes x 11 taps x 2, 3 derivative maps likewise, products, SSIM terms)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="drt8-1.5M")
    p.add_argument("--no-per-view", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--tile", default=None, help="fix the tile shape, WxH (skips the autotuner)")
    p.add_argument("--batch", type=int, default=None, help="fix the prefetch distance (skips the autotuner)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-persistent", action="store_true",
                   help="render with one CTA per tile in tile order instead of the persistent longest-first queue")
    p.add_argument("--no-train-step", action="store_true", help="skip the step with the Eq. 8 loss")
    p.add_argument("--no-color16", action="store_true", help="skip the step with binary16 colour storage")
    p.add_argument("--no-gsr", action="store_true", help="skip the KNN build, the GSR point evaluation and the level-set extraction")
    p.add_argument("--no-other-workloads", action="store_true",
                   help="skip the other workloads (tiny, object, one-view scene, 3M-splat 16-view batch)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target length of the oracle sample")
    p.add_argument("--splats", type=int, default=None,
                   help="override the workload's splat count (smaller cases for profiling; not a bench line)")
    return p.parse_args()


# --------------------------------------------------------------------------- distributed
def dist_setup(backend: str = "nccl"):
    """One process per GPU from the torchrun environment; ranks run independent replicas and
    meet only in barriers and the max-over-ranks timing (gloo serves the CPU tests)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend, init_method="env://")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
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
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- workload
def make_workload(name: str, rank: int = 0, n_override=None):
    from paper_2411_09156_gb300.drt import drt_sizes
    from paper_2411_09156_gb300.scenes import random_sphere_cameras, workload
    if name == "drt8-1.5M":
        sizes = drt_sizes(1600, 1040, 8)
    elif name == "drt16-3M":
        sizes = drt_sizes(1920, 1080, 16)
    else:
        sizes = None
    sc, cams = workload(name, sizes=sizes, n_override=n_override)
    if rank > 0 and sizes is not None:  # independent batch of views per rank
        cams = random_sphere_cameras(np.random.default_rng(1000 + rank), len(sizes), 5.0, sizes)
    return sc, cams


def upstream_grads(P: int, seed: int):
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    return [torch.randn(n, generator=g, device="cuda") for n in (3 * P, P, P, 3 * P)]


def kernel_source_sha256() -> str:
    """sha256 of the render kernels' sources (render.cu followed by ges_internal.cuh)."""
    h = hashlib.sha256()
    for f in ("render.cu", "ges_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2411_09156_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def timed_call(fn, warmup: int, steps: int, flush, world: int) -> float:
    """Mean CUDA-event time (ms) of fn over `steps` calls after `warmup`, L2 flushed before
    each call, max over ranks."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return max_over_ranks(statistics.mean(ts), world)


def render_roofline(kname: str, t_ms: float, blended: int, f_blend: int, mufu_blend: int, dense_flops: int,
                    events: int, pk: dict) -> dict:
    """Roofline of a render kernel against the measured FP32-FMA and ex2 peaks of this GPU.
    achieved: the method's arithmetic, f_blend FP32 flops per blended pair (the pairs the
    compositing needs); beside it the dense equivalent that also charges every (pixel, list entry)
    pair walked a support test, and the (pixel, splat) lane pairs the warps actually evaluate
    (32 per pair of an 8x4 block and a splat that passed the warp cull)."""
    t = t_ms / 1e3
    fl = f_blend * blended
    traffic, _ = profile_traffic(kname)
    mu = mufu_blend * blended
    return {"bound": "alu", "kernel": kname, "achieved": fl / t / 1e12, "peak": pk["fp32_tflops"], "unit": "TFLOP/s",
            "frac": fl / t / 1e12 / pk["fp32_tflops"], "traffic": traffic,
            "peak_source": f"measured: FP32 FMA microbenchmark (ges_peak_run) on this GPU, {pk['sm_count']} SMs",
            "flops_per_launch": fl, "flops_per_blended_pair": f_blend, "time_ms": t_ms,
            "dense_equivalent": {"flops_per_launch": dense_flops + fl,
                                 "frac": (dense_flops + fl) / t / 1e12 / pk["fp32_tflops"]},
            "lane_pairs_evaluated": 32 * events,
            "mufu": {"ops_per_launch": mu, "achieved_gops": mu / t / 1e9, "peak_gops": pk["mufu_ex2_gops"],
                     "frac": mu / t / 1e9 / pk["mufu_ex2_gops"], "ops_per_blended_pair": mufu_blend}}


def hbm_stage_fractions(plan, sc, cams, n_inst: int, flush, hbm: float, warmup: int, steps: int, world: int) -> dict:
    """Preprocess (K1), binning (K2-K5) and preprocess backward (K8) timed alone (eager calls,
    L2 flushed) against the measured HBM copy bandwidth, with the algorithmic bytes per unit of
    the method: K1 reads each splat's attributes once (48 B + the colour) and writes a 64 B render
    and a 32 B binning record per (splat, view); binning moves 28 B per (splat, view) and 44 B per
    instance; K8 reads the 64 B screen gradient per (splat, view) and each splat's attributes and
    writes its gradients once."""
    r, x = plan.rast, plan.inputs
    n, nv = sc.n, sc.n * len(cams)
    col = x[3].numel() * x[3].element_size() // max(n, 1)
    b_k1 = n * (48 + col) + nv * 96
    b_bin = 28 * nv + 44 * n_inst
    b_k8 = nv * 64 + n * (48 + col) + n * (48 + 4 * (col // x[3].element_size()))
    t_k1 = timed_call(lambda: r.preprocess(*x), warmup, steps, flush, world)
    t_bin = timed_call(lambda: r.bin(), warmup, steps, flush, world)
    t_k8 = timed_call(lambda: r.preprocess_bwd(*x, plan.grads), warmup, steps, flush, world)
    out = {}
    for k, b, t in (("k_preprocess", b_k1, t_k1), ("binning", b_bin, t_bin), ("k_preprocess_bwd", b_k8, t_k8)):
        gbs = b / (t / 1e3) / 1e9
        out[k] = {"bytes": b, "time_ms": t, "achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm}
    return out


def host_link_gbs(nbytes: int = 1 << 29) -> dict:
    """Pinned host <-> device bandwidth of one large cudaMemcpyAsync per direction (best of 5)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    res = {}
    for name, fn in (("h2d", lambda: d.copy_(h, non_blocking=True)), ("d2h", lambda: h.copy_(d, non_blocking=True))):
        best = 0.0
        fn()
        torch.cuda.synchronize()
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = max(best, nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9)
        res[name] = best
    return res


def other_workloads(cfg, args, flush, rank: int, world: int) -> dict:
    """fwd+bwd Mpixel/s of the other workloads, timed like the main line (graphed steps, L2
    flushed, random upstream gradients): the 1k-splat 128x128 view, the 100k-splat 800x800 view,
    the 1.5M-splat 1600x1040 view, and the 3M-splat 16-view batch both batched and as 16
    sequential one-view steps. Each workload gets its own autotuned tile shape and prefetch
    distance, as the main line does (the main line's with --no-autotune, --tile or --batch)."""
    import torch
    from paper_2411_09156_gb300 import api
    from paper_2411_09156_gb300.batch import BatchPlan, autotune
    out = {}
    for name in ("tiny-1k-128", "object-100k-800", "scene-1.5M-1600x1040", "drt16-3M"):
        sc, cams = make_workload(name, rank)
        inputs = api.scene_tensors(sc)
        P = sum(c.width * c.height for c in cams)
        ups = upstream_grads(P, 4000 + rank)
        c = dataclasses.replace(cfg, sh_degree=sc.sh_degree)
        if not (args.no_autotune or args.tile or args.batch):
            c = autotune(sc.n, cams, c, inputs, ups, key=name)
        plan = BatchPlan(sc.n, cams, c, inputs, ups)
        ms = timed_call(plan.step, args.warmup, args.steps, flush, world)
        plan.check()
        rec = {"value": world * P / (ms / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": ms, "splats": sc.n,
               "views": len(cams), "pixels": P, "tile": [c.tile_w, c.tile_h], "batch": c.batch,
               "gpu_launches": plan.launches_per_step() * args.steps}
        del plan
        if len(cams) > 1:
            pv_cfg = c.replace(persistent=0)
            plans, base = [], 0
            for cam in cams:
                w, h = cam.width, cam.height
                u = [ups[0][3 * base:3 * base + 3 * w * h], ups[1][base:base + w * h], ups[2][base:base + w * h],
                     ups[3][3 * base:3 * base + 3 * w * h]]
                plans.append(BatchPlan(sc.n, [cam], pv_cfg, inputs, u))
                base += w * h

            def seq():
                for p_ in plans:
                    p_.step()

            pv = timed_call(seq, args.warmup, args.steps, flush, world)
            for p_ in plans:
                p_.check()
            rec["per_view"] = {"value": world * P / (pv / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": pv,
                               "launches": f"{len(cams)} sequential one-view steps, each as CUDA graphs"}
            del plans
        out[name] = rec
        del inputs, ups
        torch.cuda.empty_cache()
    return out


def levelset_launches(n: int) -> int:
    """Kernels one ges_levelset call launches: start points, splat records, the grid build
    (bounding box, grid, cell keys, ranges, 5 per 8-bit radix pass), the query keys and their
    radix sort, the point queries and the march."""
    p_n = ((2 * n - 1).bit_length() + 7) // 8
    p_q = ((2 * n).bit_length() + 7) // 8
    return 8 + 5 * p_n + 5 * p_q


def profile_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_drt8-1.5M.md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    cur = kernel_source_sha256()
    if not m or not b or m.group(1) != cur:
        return None, cur
    return float(b.group(1)), cur


# --------------------------------------------------------------------------- CPU oracle leg
def _oracle_cfg(cfg):
    return dict(phi_mode=cfg.phi_mode, rho=cfg.rho, lowpass=cfg.lowpass, alpha_min=cfg.alpha_min,
                alpha_max=cfg.alpha_max, t_min=cfg.t_min, jac_clamp=cfg.jac_clamp, bg=tuple(cfg.bg), flag_eps=1e-4)


def run_oracle(sc, cams, cfg, n_pix: int, seed: int, views=None):
    """Oracle forward + backward on n_pix seeded pixels spread over the views (all, or the listed
    ones; pixel counts proportional to view size). Returns elapsed seconds."""
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    sel = list(range(len(cams))) if views is None else list(views)
    sizes = [(cams[v].width, cams[v].height) for v in sel]
    total = sum(w * h for w, h in sizes)
    t0 = time.perf_counter()
    for cam, (w, h) in zip([cams[v] for v in sel], sizes):
        k = max(1, int(round(n_pix * w * h / total)))
        px = np.stack([rng.integers(0, w, k), rng.integers(0, h, k)], 1).astype(np.int32)
        d = cam.as_dict()
        O.render(sc, d, _oracle_cfg(cfg), pixels=px)
        g = rng.standard_normal((k, 8))
        O.backward(sc, d, _oracle_cfg(cfg), g[:, 0:3], g[:, 3], g[:, 4], g[:, 5:8], pixels=px)
    return time.perf_counter() - t0


def sample_size(sc, cams, cfg, seconds: float, views=None) -> int:
    """Pixels whose oracle fwd+bwd takes about `seconds` (fit of a fixed per-view cost plus a per-pixel cost)."""
    t_a = run_oracle(sc, cams, cfg, 16, 11, views)
    t_b = run_oracle(sc, cams, cfg, 16 + 256, 12, views)
    slope = max((t_b - t_a) / 256.0, 1e-7)
    fixed = max(t_a - 16 * slope, 0.0)
    return int(min(max(16, (seconds - fixed) / slope), 1 << 20))


def cpu_baseline(sc, cams, cfg, seconds: float):
    from oracle import oracle as O
    O.build_oracle()
    n_final = sample_size(sc, cams, cfg, seconds)
    t = run_oracle(sc, cams, cfg, n_final, 125)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_final / t, n_final, t, cores


# --------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    if rank != 0:
        return
    from paper_2411_09156_gb300.api import GESConfig
    sc, cams = make_workload(args.workload, 0, args.splats)
    cfg = GESConfig(sh_degree=sc.sh_degree, persistent=1)
    from oracle import oracle as O
    O.build_oracle()
    # one step = seeded pixels of one view (the views in turn), sized for about 3 s of host work:
    # the oracle projects every splat once per view and call, so a step over all eight views
    # would spend most of its time there and sample few pixels
    n_step = sample_size(sc, cams, cfg, 3.0, views=[len(cams) - 1])
    for w in range(args.warmup):
        run_oracle(sc, cams, cfg, max(16, n_step // 8), 100 + w, views=[w % len(cams)])
    times = [run_oracle(sc, cams, cfg, n_step, 200 + s, views=[s % len(cams)]) for s in range(args.steps)]
    total = sum(times)
    value = n_step * args.steps / total / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"metric": METRIC, "value": value, "unit": "Mpixel/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "sample_pixels_per_step": n_step, "views": len(cams),
                       "splats": sc.n},
            "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n_step} seeded pixels per step from one of the {len(cams)} views, "
                                       f"the views in turn (fwd + analytic bwd, brute force over all "
                                       f"{sc.n} splats)"},
            "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    from paper_2411_09156_gb300 import api
    from paper_2411_09156_gb300.batch import BatchPlan, autotune

    torch.cuda.set_device(local)
    dev_name = torch.cuda.get_device_name()
    sc, cams = make_workload(args.workload, rank, args.splats)
    inputs = api.scene_tensors(sc)
    P = sum(c.width * c.height for c in cams)
    ups = upstream_grads(P, 1000 + rank)
    base = api.GESConfig(sh_degree=sc.sh_degree, persistent=0 if args.no_persistent else 1)
    if args.tile or args.batch:
        tw, th = (int(x) for x in (args.tile or f"{base.tile_w}x{base.tile_h}").split("x"))
        cfg = dataclasses.replace(base, tile_w=tw, tile_h=th, batch=args.batch or base.batch)
    else:
        cfg = base if args.no_autotune else autotune(sc.n, cams, base, inputs, ups, key=args.workload)
    plan = BatchPlan(sc.n, cams, cfg, inputs, ups)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2

    # warm-up (untimed), then check the device status once
    for _ in range(args.warmup):
        plan.step()
    torch.cuda.synchronize()
    plan.check()

    # algorithmic work counts of the render kernels (outside the timed region)
    n_eval = torch.empty(P, dtype=torch.int32, device="cuda")
    plan.rast.render_fwd(n_eval=n_eval)
    torch.cuda.synchronize()
    o = plan.rast.out
    evals_fwd = int(n_eval.double().sum().item())
    blended = int(o["n_contrib"].double().sum().item())
    lay = plan.rast.layout()
    ranges = plan.rast.bins[lay.bins_ranges:lay.bins_ranges + 8 * lay.n_tiles].view(torch.int32).view(-1, 2)
    starts = torch.empty(P, dtype=torch.int64, device="cuda")
    tw, th = cfg.tile_w, cfg.tile_h
    for v, (w, h) in enumerate(plan.rast.sizes):
        ys, xs = torch.meshgrid(torch.arange(h, device="cuda"), torch.arange(w, device="cuda"), indexing="ij")
        tiles = lay.tile_base[v] + (ys // th) * ((w + tw - 1) // tw) + xs // tw
        starts[plan.rast.pix_base[v]:plan.rast.pix_base[v + 1]] = ranges[tiles.reshape(-1), 0].long()
    evals_bwd = int((o["last"].long() - starts).double().sum().item())
    events = plan.rast.cull_events()
    n_inst = plan.rast.instance_count()
    plan.step()  # restore the step's own state
    torch.cuda.synchronize()
    from paper_2411_09156_gb300 import peaks as PK
    pk = PK.measure()

    # timed region
    sampler = ClockSampler(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between steps, outside the step's events
        plan.step(evs[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier(world)
    clocks = sampler.stop()
    stage_ms = [[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(4)] for k in range(args.steps)]
    step_ms = [evs[k][0].elapsed_time(evs[k][4]) for k in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = world * P / (ms_per_step / 1e3) / 1e6
    st = plan.rast.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {st} after the timed steps")
    launches_main = plan.launches_per_step() * args.steps
    stage_avg = [statistics.mean(s[i] for s in stage_ms) for i in range(4)]
    names = ["preprocess_bin", "render_fwd", "render_bwd", "preprocess_bwd"]

    # roofline of the dominant kernel
    dom = int(np.argmax(stage_avg))
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    fp32_peak = pk["fp32_tflops"]
    kernels = {"render_fwd": ("k_render_fwd", F_BLEND_FWD, MUFU_FWD, F_TEST * evals_fwd),
               "render_bwd": ("k_render_bwd", F_BLEND_BWD, MUFU_BWD, F_TEST * evals_bwd)}
    rooflines = {k: render_roofline(kn, stage_avg[names.index(k)], blended, fb, mb, dense, events, pk)
                 for k, (kn, fb, mb, dense) in kernels.items()}
    if names[dom] in kernels:
        roofline = rooflines[names[dom]]
    else:
        roofline = {"bound": "hbm", "kernel": names[dom], "achieved": None, "peak": hbm, "unit": "GB/s",
                    "frac": None, "traffic": None}
    hbm_stages = hbm_stage_fractions(plan, sc, cams, n_inst, flush, hbm, args.warmup, args.steps, world)

    # per-view path (one launch sequence per view, each captured as graphs)
    per_view = None
    if not args.no_per_view:
        pv_cfg = cfg.replace(persistent=0)
        plans = []
        for v, cam in enumerate(cams):
            w, h = cam.width, cam.height
            b = plan.rast.pix_base[v]
            u = [ups[0][3 * b:3 * b + 3 * w * h], ups[1][b:b + w * h], ups[2][b:b + w * h],
                 ups[3][3 * b:3 * b + 3 * w * h]]
            plans.append(BatchPlan(sc.n, [cam], pv_cfg, inputs, u))
        for _ in range(args.warmup):
            for p_ in plans:
                p_.step()
        torch.cuda.synchronize()
        pv_ms = []
        for k in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for p_ in plans:
                p_.step()
            e1.record()
            torch.cuda.synchronize()
            pv_ms.append(e0.elapsed_time(e1))
        for p_ in plans:
            p_.check()
        pv = statistics.mean(pv_ms)
        per_view = {"value": world * P / (pv / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": pv,
                    "launches": f"{len(cams)} sequential one-view steps, each as CUDA graphs, one CTA per tile"}
        del plans
        torch.cuda.empty_cache()

    # end to end through the public API with host buffers (H2D inputs + upstream, D2H gradients)
    e2e = None
    if not args.no_e2e:
        host_in = [t.cpu().pin_memory() for t in inputs]
        host_up = [t.cpu().pin_memory() for t in ups]
        host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in plan.grads.items()}
        h2d = sum(t.numel() * 4 for t in host_in + host_up)
        d2h = sum(t.numel() * 4 for t in host_out.values())

        def e2e_step():
            plan.step_host(host_in, host_up, host_out)

        for _ in range(max(1, args.warmup // 2)):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = []
        for k in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            e2e_step()
            e1.record()
            torch.cuda.synchronize()
            e_ms.append(e0.elapsed_time(e1))
        em = max_over_ranks(statistics.mean(e_ms), world)
        e2e = {"value": world * P / (em / 1e3) / 1e6, "unit": "Mpixel/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": em, "host_link_gbs": host_link_gbs(),
               "copy_bound_ms": None}
        lk = e2e["host_link_gbs"]
        e2e["copy_bound_ms"] = 1e3 * (h2d / (lk["h2d"] * 1e9) + d2h / (lk["d2h"] * 1e9))

    # precision variant: the colour input (SH coefficients) stored as IEEE binary16 and widened
    # to float32 on load; the same batched step otherwise
    color16 = None
    if not args.no_color16 and sc.sh_degree >= 0:
        c16 = inputs[3].half().contiguous()
        plan16 = BatchPlan(sc.n, cams, dataclasses.replace(cfg, color_storage=1),
                           [inputs[0], inputs[1], inputs[2], c16], ups, capacity=plan.capacity)
        for _ in range(args.warmup):
            plan16.step()
        torch.cuda.synchronize()
        plan16.check()
        evs16 = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            plan16.step(evs16[k])
        torch.cuda.synchronize()
        if plan16.rast.sync_status() != 0:
            raise RuntimeError("device status after the binary16-colour steps")
        t16 = max_over_ranks(statistics.mean(evs16[k][0].elapsed_time(evs16[k][4]) for k in range(args.steps)),
                             world)
        st16 = [statistics.mean(evs16[k][i].elapsed_time(evs16[k][i + 1]) for k in range(args.steps))
                for i in range(4)]
        kc = (sc.sh_degree + 1) ** 2
        color16 = {"value": world * P / (t16 / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": t16,
                   "stages_ms": dict(zip(names, st16)), "color_storage": "binary16",
                   "color_bytes_per_splat": {"float32": 12 * kc, "binary16": 6 * kc},
                   "gpu_launches": plan16.launches_per_step() * args.steps}
        del plan16, c16
        torch.cuda.empty_cache()

    # training step: the same views with the Eq. 8 loss against target images between the render
    # passes (colour gradient from the loss instead of random upstream gradients)
    train = None
    if not args.no_train_step:
        tgt_in = list(inputs)
        gen = torch.Generator(device="cuda").manual_seed(2000 + rank)
        tgt_in[3] = inputs[3] + 0.05 * torch.randn(inputs[3].shape, generator=gen, device="cuda")
        tr = api.Rasterizer(sc.n, cams, cfg, capacity=plan.capacity)
        tr.preprocess(*tgt_in)
        tr.bin()
        target = tr.render_fwd()["color"].clone()
        del tr
        tplan = BatchPlan(sc.n, cams, cfg, inputs, target=target, capacity=plan.capacity)
        for _ in range(args.warmup):
            tplan.step()
        torch.cuda.synchronize()
        tplan.check()
        ns = len(tplan.stages)
        tevs = [[torch.cuda.Event(enable_timing=True) for _ in range(ns + 1)] for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            tplan.step(tevs[k])
        torch.cuda.synchronize()
        if tplan.rast.sync_status() != 0:
            raise RuntimeError("device status after the training steps")
        t_stage = [statistics.mean(tevs[k][i].elapsed_time(tevs[k][i + 1]) for k in range(args.steps))
                   for i in range(ns)]
        t_ms = max_over_ranks(statistics.mean(tevs[k][0].elapsed_time(tevs[k][ns]) for k in range(args.steps)),
                              world)
        loss_ms = t_stage[tplan.stages.index("loss")]
        loss_fl = F_LOSS * P
        train = {"value": world * P / (t_ms / 1e3) / 1e6, "unit": "Mpixel/s", "ms_per_step": t_ms,
                 "stages_ms": dict(zip(tplan.stages, t_stage)),
                 "loss_per_view": [round(float(x), 6) for x in tplan.loss.cpu().tolist()],
                 "target": "the same views rendered with SH coefficients perturbed by N(0, 0.05^2)",
                 "loss_roofline": {"bound": "alu", "kernel": "k_loss", "achieved": loss_fl / (loss_ms / 1e3) / 1e12,
                                   "peak": fp32_peak, "unit": "TFLOP/s",
                                   "frac": loss_fl / (loss_ms / 1e3) / 1e12 / fp32_peak,
                                   "flops_per_launch": loss_fl},
                 "gpu_launches": tplan.launches_per_step() * args.steps}
        del tplan
        torch.cuda.empty_cache()

    # GSR point evaluation (Eq. 9-13): one sample per splat, KNN-16 lists built on the device
    gsr = None
    if not args.no_gsr:
        n = sc.n
        kws = torch.empty(api.ges_knn_workspace_bytes(n), dtype=torch.uint8, device="cuda")
        knn = torch.empty((n, 16), dtype=torch.int32, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(3000 + rank)
        js = torch.arange(n, dtype=torch.int32, device="cuda")
        zs = torch.randn((n, 3), generator=gen, device="cuda")
        gws = torch.empty(api.ges_gsr_workspace_bytes(n, n), dtype=torch.uint8, device="cuda")
        losses = torch.empty(3, device="cuda")
        gg = [torch.empty_like(t) for t in inputs[:3]]
        cfg_c = cfg.to_c()

        knn_ms = timed_call(lambda: api.ges_knn(n, inputs[0], kws, knn), args.warmup, args.steps, flush, world)
        fwd_ms = timed_call(lambda: api.ges_gsr(n, inputs[0], inputs[1], inputs[2], cfg_c, knn, n, js, zs, 1.0, 1.0,
                                                gws, losses), args.warmup, args.steps, flush, world)
        fb_ms = timed_call(lambda: api.ges_gsr(n, inputs[0], inputs[1], inputs[2], cfg_c, knn, n, js, zs, 1.0, 1.0,
                                               gws, losses, None, *gg), args.warmup, args.steps, flush, world)
        gsr = {"value": world * n / (fb_ms / 1e3) / 1e6, "unit": "Msample/s", "samples": n,
               "gsr_fwd_bwd_ms": fb_ms, "gsr_fwd_ms": fwd_ms, "knn_ms": knn_ms,
               "losses": [round(float(x), 6) for x in losses.cpu().tolist()],
               "sampling": "one sample per splat, z ~ N(0, I), neighbours = the splat's 16 nearest centres",
               "gpu_launches": args.steps * ((6 + 5 * (((2 * n - 1).bit_length() + 7) // 8)) + 3 + 4)}
        del kws, knn, gws, gg
        torch.cuda.empty_cache()

    # level-set points (Sec. 3.3, level 0.3) from the rendered depth / alpha of every pixel of the
    # batch's views: start points, KNN point queries, the density march and the normals
    levelset = None
    if not args.no_gsr:
        n = sc.n
        o = plan.rast.out
        pix = torch.cat([torch.stack([torch.full((c.width * c.height,), v, dtype=torch.int32, device="cuda"),
                                      torch.arange(c.width * c.height, dtype=torch.int32, device="cuda")], 1)
                         for v, c in enumerate(cams)]).contiguous()
        lws = torch.empty(api.ges_levelset_workspace_bytes(n, P), dtype=torch.uint8, device="cuda")
        pts = torch.empty((P, 8), dtype=torch.float32, device="cuda")
        cams_c = api.cameras_to_c(cams)
        cfg_c = cfg.to_c()
        ls_ms = timed_call(lambda: api.ges_levelset(n, inputs[0], inputs[1], inputs[2], cfg_c, len(cams), cams_c,
                                                    o["depth"], o["alpha"], P, pix, 32, 0.3, lws, pts),
                           args.warmup, args.steps, flush, world)
        n_pts = int(pts[:, 7].sum().item())
        levelset = {"value": world * P / (ls_ms / 1e3) / 1e6, "unit": "Mpixel/s", "pixels": P, "points": n_pts,
                    "levelset_ms": ls_ms, "n_steps": 32, "level": 0.3,
                    "sampling": "every pixel of the batch's views, depth / alpha from the rendered step",
                    "gpu_launches": args.steps * levelset_launches(n)}
        del lws, pts, pix
        torch.cuda.empty_cache()

    others = None
    if not args.no_other_workloads and args.splats is None:
        del plan
        torch.cuda.empty_cache()
        others = other_workloads(cfg, args, flush, rank, world)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, npx, secs, cores = cpu_baseline(sc, cams, cfg, args.cpu_seconds)
        cpu = {"value": rate / 1e6, "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
               "sample": f"{npx} seeded pixels over the {len(cams)} views, fwd + analytic bwd, "
                         f"brute force over all {sc.n} splats, {secs:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded heightfield scene, random upstream grads)",
            "config": {"workload": args.workload if args.splats is None else f"{args.workload} (splats={sc.n})",
                       "splats": sc.n, "views": len(cams),
                       "sizes": [[c.width, c.height] for c in cams], "pixels": P, "sh_degree": sc.sh_degree,
                       "tile": [cfg.tile_w, cfg.tile_h], "batch": cfg.batch, "persistent": cfg.persistent,
                       "instances": n_inst, "l2": "flushed between steps (256 MB write)", "gpu": dev_name,
                       "parallelism": "replicas" if world > 1 else "single-gpu"},
            "stages_ms": dict(zip(names, stage_avg)),
            "roofline": roofline,
            "rooflines": rooflines,
            "hbm_stages": hbm_stages,
            "peaks_measured": pk,
            "per_view": per_view,
            "e2e": e2e,
            "train_step": train,
            "color_binary16": color16,
            "gsr": gsr,
            "levelset": levelset,
            "other_workloads": others,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": launches_main,
            "work": {"evaluated_pairs_fwd": evals_fwd, "evaluated_pairs_bwd": evals_bwd, "blended_pairs": blended,
                     "warp_cull_passes_fwd": events, "lane_pairs_evaluated_fwd": 32 * events},
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
