"""Batched dynamic-resolution steps as CUDA graphs, and the tile/batch autotuner.

A DRT step (Eq. 15, Sec. 3.4) renders several views of uneven size forward and
backward. BatchPlan runs it as captured CUDA graphs -- (preprocess + bin),
render forward, render backward (screen space), preprocess backward -- over
buffers sized for a fixed tile-instance capacity, so a step is a few graph
launches with no host synchronisation. With target images the step also runs
the Eq. 8 loss between the render passes, and the render backward takes its
colour gradient from it (a training step); otherwise it takes the given
upstream gradients. After a replay, `check()` reads the device error word; a
capacity overflow re-sizes the buffers and re-captures.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, List, Optional, Sequence

import torch

from . import build as _build
from .api import GESConfig, Rasterizer, ges_loss_rgb, ges_loss_workspace_bytes
from ._lib import GES_ERR_CAPACITY, GES_OK, GESError

STAGES = ("preprocess_bin", "render_fwd", "render_bwd", "preprocess_bwd")
STAGES_WITH_LOSS = ("preprocess_bin", "render_fwd", "loss", "render_bwd", "preprocess_bwd")


class BatchPlan:
    def __init__(self, n: int, cams: Sequence, cfg: GESConfig, inputs: Sequence[torch.Tensor],
                 upstream: Optional[Sequence[Optional[torch.Tensor]]] = None, capacity: Optional[int] = None,
                 headroom: float = 1.15, use_graphs: bool = True, target: Optional[torch.Tensor] = None,
                 lam: float = 0.2):
        """upstream: (g_color, g_depth, g_alpha, g_normal) for the render backward; or target: the
        views' target images (colour layout), whose Eq. 8 loss (weight lam on D-SSIM) supplies g_color."""
        self.n, self.cams, self.cfg = n, list(cams), cfg
        self.inputs = list(inputs)
        if (upstream is None) == (target is None):
            raise ValueError("give either upstream gradients or target images")
        self.target, self.lam = target, float(lam)
        self.upstream = list(upstream) if upstream is not None else None
        self.stages = STAGES if target is None else STAGES_WITH_LOSS
        self.headroom = headroom
        self.use_graphs = use_graphs
        if capacity is None:
            probe = Rasterizer(n, cams, cfg)
            probe.preprocess(*self.inputs)
            capacity = max(1024, int(math.ceil(probe.instance_count() * headroom)))
            del probe
        self._setup(capacity)

    def _setup(self, capacity: int) -> None:
        self.rast = Rasterizer(self.n, self.cams, self.cfg, capacity=capacity)
        self.capacity = capacity
        # gradients are float32 whatever the colour storage
        self.grads = {k: torch.empty(t.shape, dtype=torch.float32, device=t.device) for k, t in
                      zip(("g_pos_op", "g_lscale_beta", "g_quat", "g_color"), self.inputs)}
        if self.target is not None:
            r = self.rast
            if self.target.numel() != 3 * r.P:
                raise ValueError("target must hold 3 * sum(W * H) values")
            self.loss = torch.empty(r.n_views, dtype=torch.float32, device=r.device)
            self.g_color_loss = torch.empty(3 * r.P, dtype=torch.float32, device=r.device)
            self.loss_ws = torch.empty(ges_loss_workspace_bytes(r.n_views, r.cams_c), dtype=torch.uint8,
                                       device=r.device)
            self.upstream = [self.g_color_loss, None, None, None]
        self.graphs: List[Optional[torch.cuda.CUDAGraph]] = [None] * len(self.stages)
        self.bin_graph: Optional[torch.cuda.CUDAGraph] = None
        if self.use_graphs:
            self._capture()

    def _run_stage(self, k: int) -> None:
        r, x = self.rast, self.inputs
        name = self.stages[k]
        if name == "preprocess_bin":
            r.preprocess(*x)
            r.bin()
        elif name == "render_fwd":
            # a training step's loss reads the colour only: depth and normal are not rendered
            r.render_fwd(depth_normal=self.target is None)
        elif name == "loss":
            ges_loss_rgb(r.n_views, r.cams_c, r.out["color"], self.target, self.lam, self.loss_ws, self.loss,
                         self.g_color_loss)
        elif name == "render_bwd":
            r.backward_screen(*self.upstream)
        else:
            r.preprocess_bwd(*x, self.grads)

    def _capture(self) -> None:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for k in range(len(self.stages)):  # one eager pass before capture
                self._run_stage(k)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        for k in range(len(self.stages)):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._run_stage(k)
            self.graphs[k] = g
        # binning alone, for steps whose preprocess runs in splat ranges (step_host)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.rast.bin()
        self.bin_graph = g
        torch.cuda.synchronize()

    def run_stage(self, k: int) -> None:
        if self.graphs[k] is not None:
            self.graphs[k].replay()
        else:
            self._run_stage(k)

    def step(self, events: Optional[List[torch.cuda.Event]] = None) -> Dict[str, torch.Tensor]:
        """One fwd+bwd step; events (len(stages) + 1, optional) bracket the stages on the current stream."""
        n = len(self.stages)
        for k in range(n):
            if events is not None:
                events[k].record()
            self.run_stage(k)
        if events is not None:
            events[n].record()
        return self.grads

    def step_host(self, host_inputs: Sequence[torch.Tensor],
                  host_upstream: Optional[Sequence[Optional[torch.Tensor]]] = None,
                  host_grads: Optional[Dict[str, torch.Tensor]] = None, chunks: int = 8) -> Dict[str, torch.Tensor]:
        """One step whose inputs come from (pinned) host tensors and whose gradients go back to
        host_grads. The splat parameters are copied in `chunks` splat ranges on a copy stream,
        and the preprocess of each range starts as soon as its rows have arrived; the upstream
        gradients, which only the render backward reads, follow on the same stream while the
        forward runs; the preprocess backward runs in the same ranges and each range's gradient
        rows are copied back on a second stream while the next range is computed."""
        cur = torch.cuda.current_stream()
        r, x = self.rast, self.inputs
        n = self.n
        chunks = max(1, min(int(chunks), n)) if n > 0 else 1
        bounds = [(n * c // chunks, n * (c + 1) // chunks) for c in range(chunks)]
        if not hasattr(self, "_h2d"):
            self._h2d, self._d2h = torch.cuda.Stream(), torch.cuda.Stream()
            self._up_ready = torch.cuda.Event()
        ev_in = [torch.cuda.Event() for _ in bounds]
        # the copies wait for the previous step, which still reads the device inputs
        self._h2d.wait_stream(cur)
        with torch.cuda.stream(self._h2d):
            for c, (a, b) in enumerate(bounds):
                for d, h in zip(x, host_inputs):
                    d[a:b].copy_(h[a:b], non_blocking=True)
                ev_in[c].record()
            overlap = host_upstream is not None and self.target is None
            if overlap:
                for d, h in zip(self.upstream, host_upstream):
                    if d is not None and h is not None:
                        d.copy_(h, non_blocking=True)
                self._up_ready.record()
        for c, (a, b) in enumerate(bounds):
            cur.wait_event(ev_in[c])
            r.preprocess_range(a, b - a, *x)
        if self.bin_graph is not None:
            self.bin_graph.replay()
        else:
            r.bin()
        for k, name in enumerate(self.stages):
            if name in ("preprocess_bin", "preprocess_bwd"):
                continue
            if name == "render_bwd" and overlap:
                cur.wait_event(self._up_ready)
            self.run_stage(k)
        for c, (a, b) in enumerate(bounds):
            r.preprocess_bwd_range(a, b - a, *x, self.grads)
            if host_grads is not None:
                done = torch.cuda.Event()
                done.record(cur)
                self._d2h.wait_event(done)
                with torch.cuda.stream(self._d2h):
                    for k, h in host_grads.items():
                        h[a:b].copy_(self.grads[k][a:b], non_blocking=True)
        cur.wait_stream(self._d2h)
        return self.grads

    def check(self) -> int:
        """Reads the device error word; on a capacity overflow grows the buffers and re-captures."""
        st = self.rast.sync_status()
        if st == GES_ERR_CAPACITY:
            needed = self.rast.instance_count()
            self._setup(max(int(needed * self.headroom), 2 * self.capacity))
        elif st != GES_OK:
            raise GESError(st, "batched step")
        return st

    def launches_per_step(self) -> int:
        """Kernels of this library launched by one step (cudaMemsetAsync nodes not counted)."""
        lay = self.rast.layout()
        n_tiles = int(lay.n_tiles)
        tile_bits = max(0, (n_tiles - 1).bit_length())
        tile_passes = (tile_bits + 7) // 8
        n_entries = self.n * len(self.cams)
        if n_entries == 0:
            binning = 1 if self.cfg.persistent else 0
        else:
            binning = 1 + 4 * 5 + 1 + 3 + 1 + 1 + tile_passes * 5 + 1 + (1 if self.cfg.persistent else 0)
        return 1 + binning + 1 + 1 + 1 + (2 if self.target is not None else 0)


# --------------------------------------------------------------------------- autotune
TILE_SHAPES = ((16, 16), (16, 8), (8, 16), (8, 8), (32, 8), (8, 32))
BATCHES = (128, 256)
AUTOTUNE_FILE = os.path.join(_build.BUILD, "autotune.json")


def autotune(n, cams, base_cfg: GESConfig, inputs, upstream, key: str, reps: int = 3,
             persist: bool = True, candidates=None) -> GESConfig:
    """Times one full step for each tile shape x batch size and returns the fastest config.
    Results persist in AUTOTUNE_FILE keyed by GPU name and `key`."""
    gpu = torch.cuda.get_device_name()
    db = {}
    if persist and os.path.exists(AUTOTUNE_FILE):
        try:
            with open(AUTOTUNE_FILE) as fh:
                db = json.load(fh)
        except (OSError, ValueError):
            db = {}
    k = f"{gpu}|{key}"
    if k in db:
        tw, th, b = db[k]["tile_w"], db[k]["tile_h"], db[k]["batch"]
        return base_cfg.replace(tile_w=tw, tile_h=th, batch=b)
    results = []
    cand = candidates or [(tw, th, b) for (tw, th) in TILE_SHAPES for b in BATCHES]
    for (tw, th, b) in cand:
        cfg = base_cfg.replace(tile_w=tw, tile_h=th, batch=b)
        plan = BatchPlan(n, cams, cfg, inputs, upstream)
        plan.step()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            plan.step()
        ev[1].record()
        torch.cuda.synchronize()
        results.append((ev[0].elapsed_time(ev[1]) / reps, tw, th, b))
        del plan
        torch.cuda.empty_cache()
    results.sort()
    _, tw, th, b = results[0]
    db[k] = dict(tile_w=tw, tile_h=th, batch=b, ms=results[0][0],
                 all=[dict(ms=r[0], tile_w=r[1], tile_h=r[2], batch=r[3]) for r in results],
                 when=time.strftime("%Y-%m-%dT%H:%M:%S"))
    if persist:
        os.makedirs(os.path.dirname(AUTOTUNE_FILE), exist_ok=True)
        with open(AUTOTUNE_FILE, "w") as fh:
            json.dump(db, fh, indent=1)
    return base_cfg.replace(tile_w=tw, tile_h=th, batch=b)
