"""Python binding of the GES rasterizer C ABI (include/ges.h).

The functions named like the C calls only marshal arguments (tensor data
pointers, the current CUDA stream, the config and camera structs); every step
of the computation runs in libges.so. `Rasterizer` owns the device buffers of
one (scene size, views, config) and sequences the calls for the common
forward / backward use.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import torch

from . import _lib
from ._lib import GESError, check


# --------------------------------------------------------------------------- config / cameras
@dataclasses.dataclass
class GESConfig:
    """Rasterizer settings (mirrors ges_config); defaults are the readings documented in ges.h."""
    tile_w: int = 16
    tile_h: int = 16
    batch: int = 256
    sh_degree: int = -1
    phi_mode: int = 1
    rho: float = 0.1
    lowpass: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    jac_clamp: float = 1.3
    bg: tuple = (0.0, 0.0, 0.0)
    persistent: int = 0
    color_storage: int = 0  # colour input: 0 float32, 1 float16, 2 bfloat16

    def to_c(self) -> _lib.Config:
        c = _lib.Config()
        for f in ("tile_w", "tile_h", "batch", "sh_degree", "phi_mode", "persistent", "color_storage"):
            setattr(c, f, int(getattr(self, f)))
        for f in ("rho", "lowpass", "alpha_min", "alpha_max", "t_min", "jac_clamp"):
            setattr(c, f, float(getattr(self, f)))
        for i in range(3):
            c.bg[i] = float(self.bg[i])
        return c

    def replace(self, **kw) -> "GESConfig":
        return dataclasses.replace(self, **kw)


# torch element type of the colour input for each ges_config.color_storage
COLOR_DTYPES = {0: torch.float32, 1: torch.float16, 2: torch.bfloat16}


def _cam_dict(cam) -> dict:
    return cam.as_dict() if hasattr(cam, "as_dict") else dict(cam)


def cameras_to_c(cams: Sequence) -> ctypes.Array:
    """Array of ges_camera from Camera objects or dicts (width, height, fx, fy, cx, cy, viewmat, znear)."""
    arr = (_lib.Camera * len(cams))()
    for i, cam in enumerate(cams):
        d = _cam_dict(cam)
        c = arr[i]
        c.width, c.height = int(d["width"]), int(d["height"])
        c.fx, c.fy, c.cx, c.cy = float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"])
        vm = [float(x) for x in torch.as_tensor(d["viewmat"], dtype=torch.float32).reshape(12).tolist()]
        for k in range(12):
            c.viewmat[k] = vm[k]
        c.znear = float(d.get("znear", 0.2))
    return arr


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("GES tensors must live on the GPU")
    if not t.is_contiguous():
        raise ValueError("GES tensors must be contiguous")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# --------------------------------------------------------------------------- raw C-ABI calls
def ges_abi_version() -> int:
    return int(_lib.lib().ges_abi_version())


def ges_proj_bytes(n: int, n_views: int) -> int:
    return int(_lib.lib().ges_proj_bytes(n, n_views))


def ges_bins_bytes(n: int, n_views: int, cams_c, cfg_c, capacity: int) -> int:
    return int(_lib.lib().ges_bins_bytes(n, n_views, cams_c, ctypes.byref(cfg_c), capacity))


def ges_get_layout(n: int, n_views: int, cams_c, cfg_c, capacity: int) -> _lib.Layout:
    lay = _lib.Layout()
    check(_lib.lib().ges_get_layout(n, n_views, cams_c, ctypes.byref(cfg_c), capacity, ctypes.byref(lay)),
          "ges_get_layout")
    return lay


def ges_preprocess(n, pos_op, lscale_beta, quat, color, n_views, cams_c, cfg_c, proj, stream=None) -> None:
    check(_lib.lib().ges_preprocess(n, _ptr(pos_op), _ptr(lscale_beta), _ptr(quat), _ptr(color), n_views, cams_c,
                                    ctypes.byref(cfg_c), _ptr(proj), proj.numel(), _stream(stream)),
          "ges_preprocess")


def ges_preprocess_range(n, first, count, pos_op, lscale_beta, quat, color, n_views, cams_c, cfg_c, proj,
                         stream=None) -> None:
    check(_lib.lib().ges_preprocess_range(n, first, count, _ptr(pos_op), _ptr(lscale_beta), _ptr(quat), _ptr(color),
                                          n_views, cams_c, ctypes.byref(cfg_c), _ptr(proj), proj.numel(),
                                          _stream(stream)), "ges_preprocess_range")


def ges_instance_count(proj, stream=None) -> int:
    v = ctypes.c_uint64()
    check(_lib.lib().ges_instance_count(_ptr(proj), proj.numel(), ctypes.byref(v), _stream(stream)),
          "ges_instance_count")
    return int(v.value)


def ges_bin(n, n_views, cams_c, cfg_c, proj, bins, stream=None) -> None:
    check(_lib.lib().ges_bin(n, n_views, cams_c, ctypes.byref(cfg_c), _ptr(proj), proj.numel(), _ptr(bins),
                             bins.numel(), _stream(stream)), "ges_bin")


def ges_render_fwd(n, n_views, cams_c, cfg_c, proj, bins, color, depth, alpha, normal, t_final, last, n_contrib,
                   n_eval=None, stream=None) -> None:
    check(_lib.lib().ges_render_fwd(n, n_views, cams_c, ctypes.byref(cfg_c), _ptr(proj), proj.numel(), _ptr(bins),
                                    bins.numel(), _ptr(color), _ptr(depth), _ptr(alpha), _ptr(normal),
                                    _ptr(t_final), _ptr(last), _ptr(n_contrib), _ptr(n_eval), _stream(stream)),
          "ges_render_fwd")


def ges_render_bwd_screen(n, n_views, cams_c, cfg_c, proj, bins, color, depth, normal, t_final, last, g_color,
                          g_depth, g_alpha, g_normal, g2d=None, stream=None) -> None:
    check(_lib.lib().ges_render_bwd_screen(n, n_views, cams_c, ctypes.byref(cfg_c), _ptr(proj), proj.numel(),
                                           _ptr(bins), bins.numel(), _ptr(color), _ptr(depth), _ptr(normal),
                                           _ptr(t_final), _ptr(last), _ptr(g_color), _ptr(g_depth), _ptr(g_alpha),
                                           _ptr(g_normal), _ptr(g2d), _stream(stream)), "ges_render_bwd_screen")


def ges_preprocess_bwd(n, n_views, cams_c, cfg_c, pos_op, lscale_beta, quat, color_in, proj, g2d, g_pos_op,
                       g_lscale_beta, g_quat, g_color_in, stream=None) -> None:
    check(_lib.lib().ges_preprocess_bwd(n, n_views, cams_c, ctypes.byref(cfg_c), _ptr(pos_op), _ptr(lscale_beta),
                                        _ptr(quat), _ptr(color_in), _ptr(proj), proj.numel(), _ptr(g2d),
                                        _ptr(g_pos_op), _ptr(g_lscale_beta), _ptr(g_quat), _ptr(g_color_in),
                                        _stream(stream)), "ges_preprocess_bwd")


def ges_preprocess_bwd_range(n, first, count, n_views, cams_c, cfg_c, pos_op, lscale_beta, quat, color_in, proj, g2d,
                             g_pos_op, g_lscale_beta, g_quat, g_color_in, stream=None) -> None:
    check(_lib.lib().ges_preprocess_bwd_range(n, first, count, n_views, cams_c, ctypes.byref(cfg_c), _ptr(pos_op),
                                              _ptr(lscale_beta), _ptr(quat), _ptr(color_in), _ptr(proj), proj.numel(),
                                              _ptr(g2d), _ptr(g_pos_op), _ptr(g_lscale_beta), _ptr(g_quat),
                                              _ptr(g_color_in), _stream(stream)), "ges_preprocess_bwd_range")


def ges_render_bwd(n, n_views, cams_c, cfg_c, pos_op, lscale_beta, quat, color_in, proj, bins, color, depth, normal,
                   t_final, last, g_color, g_depth, g_alpha, g_normal, g_pos_op, g_lscale_beta, g_quat, g_color_in,
                   g2d=None, stream=None) -> None:
    check(_lib.lib().ges_render_bwd(n, n_views, cams_c, ctypes.byref(cfg_c), _ptr(pos_op), _ptr(lscale_beta),
                                    _ptr(quat), _ptr(color_in), _ptr(proj), proj.numel(), _ptr(bins), bins.numel(),
                                    _ptr(color), _ptr(depth), _ptr(normal), _ptr(t_final), _ptr(last),
                                    _ptr(g_color), _ptr(g_depth), _ptr(g_alpha), _ptr(g_normal), _ptr(g_pos_op),
                                    _ptr(g_lscale_beta), _ptr(g_quat), _ptr(g_color_in), _ptr(g2d),
                                    _stream(stream)), "ges_render_bwd")


def ges_render_bwd_noalloc(n, n_views, cams_c, cfg_c, pos_op, lscale_beta, quat, color_in, proj, bins, color, depth,
                           normal, t_final, last, g_color, g_depth, g_alpha, g_normal, g_pos_op, g_lscale_beta,
                           g_quat, g_color_in, stream=None) -> None:
    """ges_render_bwd with its accumulator in the library's fixed array (no caller scratch;
    n * n_views <= 524,288; calls overlapping on the GPU race)."""
    check(_lib.lib().ges_render_bwd_noalloc(n, n_views, cams_c, ctypes.byref(cfg_c), _ptr(pos_op), _ptr(lscale_beta),
                                            _ptr(quat), _ptr(color_in), _ptr(proj), proj.numel(), _ptr(bins),
                                            bins.numel(), _ptr(color), _ptr(depth), _ptr(normal), _ptr(t_final),
                                            _ptr(last), _ptr(g_color), _ptr(g_depth), _ptr(g_alpha),
                                            _ptr(g_normal), _ptr(g_pos_op), _ptr(g_lscale_beta), _ptr(g_quat),
                                            _ptr(g_color_in), _stream(stream)), "ges_render_bwd_noalloc")


def ges_loss_workspace_bytes(n_views, cams_c) -> int:
    """Device bytes of the workspace ges_loss_rgb needs for these view sizes."""
    nb = int(_lib.lib().ges_loss_workspace_bytes(n_views, cams_c))
    if nb == 0:
        raise ValueError("invalid views for ges_loss_rgb")
    return nb


def ges_loss_rgb(n_views, cams_c, color, target, lam, workspace, loss, g_color=None, stream=None) -> None:
    """L_rgb = (1 - lam) L1 + lam (1 - SSIM) per view (Eq. 8) into loss[n_views], and its gradient
    with respect to color into g_color (same layout as color; None: loss only)."""
    check(_lib.lib().ges_loss_rgb(n_views, cams_c, _ptr(color), _ptr(target), float(lam), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _ptr(loss), _ptr(g_color),
                                  _stream(stream)), "ges_loss_rgb")


def loss_rgb(color: torch.Tensor, target: torch.Tensor, sizes: Sequence, lam: float = 0.2, stream=None):
    """Eq. 8 loss of rendered views against targets (planar colour layout, views concatenated).
    sizes: [(W, H)] per view. Returns (loss [n_views] float32, g_color like color)."""
    cams = [dict(width=int(w), height=int(h), fx=1.0, fy=1.0, cx=0.0, cy=0.0,
                 viewmat=[1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0]) for (w, h) in sizes]
    cams_c = cameras_to_c(cams)
    n_px = sum(int(w) * int(h) for (w, h) in sizes)
    if color.numel() != 3 * n_px or target.numel() != 3 * n_px:
        raise ValueError("color and target must hold 3 * sum(W * H) values")
    ws = torch.empty(ges_loss_workspace_bytes(len(sizes), cams_c), dtype=torch.uint8, device=color.device)
    loss = torch.empty(len(sizes), dtype=torch.float32, device=color.device)
    g = torch.empty_like(color)
    ges_loss_rgb(len(sizes), cams_c, color, target, lam, ws, loss, g, stream)
    return loss, g


def ges_knn_workspace_bytes(n: int) -> int:
    nb = int(_lib.lib().ges_knn_workspace_bytes(n))
    if nb == 0:
        raise ValueError("ges_knn needs 16 <= n <= 2^26 splats")
    return nb


def ges_knn(n, pos_op, workspace, knn, stream=None) -> None:
    """The 16 nearest splat centres of every splat (self included) into knn [n, 16] int32."""
    check(_lib.lib().ges_knn(n, _ptr(pos_op), _ptr(workspace), workspace.numel() * workspace.element_size(),
                             _ptr(knn), _stream(stream)), "ges_knn")


def ges_gsr_workspace_bytes(n: int, m: int) -> int:
    nb = int(_lib.lib().ges_gsr_workspace_bytes(n, m))
    if nb == 0:
        raise ValueError("invalid sizes for ges_gsr")
    return nb


def ges_gsr(n, pos_op, lscale_beta, quat, cfg_c, knn, m, sample_splat, sample_z, lambda_sdf, lambda_nor, workspace,
            losses, sample_out=None, g_pos_op=None, g_lscale_beta=None, g_quat=None, stream=None) -> None:
    """GSR losses (Eq. 9-13) at m sample points into losses[3]; their gradient into g_* (or None)."""
    check(_lib.lib().ges_gsr(n, _ptr(pos_op), _ptr(lscale_beta), _ptr(quat), ctypes.byref(cfg_c), _ptr(knn), m,
                             _ptr(sample_splat), _ptr(sample_z), float(lambda_sdf), float(lambda_nor),
                             _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(losses),
                             _ptr(sample_out), _ptr(g_pos_op), _ptr(g_lscale_beta), _ptr(g_quat), _stream(stream)),
          "ges_gsr")


def knn(pos_op: torch.Tensor, stream=None) -> torch.Tensor:
    """[n, 16] int32 nearest-centre lists of the splats in pos_op [n, 4]."""
    n = pos_op.shape[0]
    ws = torch.empty(ges_knn_workspace_bytes(n), dtype=torch.uint8, device=pos_op.device)
    out = torch.empty((n, 16), dtype=torch.int32, device=pos_op.device)
    ges_knn(n, pos_op, ws, out, stream)
    return out


def gsr(pos_op, lscale_beta, quat, knn_idx, sample_splat, sample_z, cfg: Optional["GESConfig"] = None,
        lambda_sdf: float = 1.0, lambda_nor: float = 1.0, grads: bool = True, per_sample: bool = False,
        stream=None) -> Dict[str, Optional[torch.Tensor]]:
    """GSR losses at the samples and (optionally) their gradient. Returns dict(losses [3]: L_sdf, L_nor,
    weighted sum; g_pos_op, g_lscale_beta, g_quat or None; sample_out [m, 8] or None)."""
    cfg = cfg or GESConfig()
    n, m = pos_op.shape[0], sample_splat.shape[0]
    dev = pos_op.device
    ws = torch.empty(ges_gsr_workspace_bytes(n, m), dtype=torch.uint8, device=dev)
    losses = torch.empty(3, dtype=torch.float32, device=dev)
    so = torch.empty((m, 8), dtype=torch.float32, device=dev) if per_sample else None
    g = [torch.empty_like(pos_op), torch.empty_like(lscale_beta), torch.empty_like(quat)] if grads else [None] * 3
    ges_gsr(n, pos_op, lscale_beta, quat, cfg.to_c(), knn_idx, m, sample_splat, sample_z, lambda_sdf, lambda_nor,
            ws, losses, so, *g, stream=stream)
    return dict(losses=losses, g_pos_op=g[0], g_lscale_beta=g[1], g_quat=g[2], sample_out=so)


def ges_knn_points_workspace_bytes(n: int, m: int) -> int:
    nb = int(_lib.lib().ges_knn_points_workspace_bytes(n, m))
    if nb == 0:
        raise ValueError("invalid sizes for ges_knn_points")
    return nb


def ges_knn_points(n, pos_op, m, points, workspace, knn, stream=None) -> None:
    check(_lib.lib().ges_knn_points(n, _ptr(pos_op), m, _ptr(points), _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _ptr(knn), _stream(stream)),
          "ges_knn_points")


def knn_points(pos_op: torch.Tensor, points: torch.Tensor, stream=None) -> torch.Tensor:
    """[m, 16] int32: the 16 splat centres nearest to each of the points [m, 4] (w = 0: none, -1)."""
    n, m = pos_op.shape[0], points.shape[0]
    ws = torch.empty(ges_knn_points_workspace_bytes(n, m), dtype=torch.uint8, device=pos_op.device)
    out = torch.empty((m, 16), dtype=torch.int32, device=pos_op.device)
    ges_knn_points(n, pos_op, m, points, ws, out, stream)
    return out


def ges_levelset_workspace_bytes(n: int, m: int) -> int:
    nb = int(_lib.lib().ges_levelset_workspace_bytes(n, m))
    if nb == 0:
        raise ValueError("invalid sizes for ges_levelset")
    return nb


def ges_levelset(n, pos_op, lscale_beta, quat, cfg_c, n_views, cams_c, depth, alpha, m, pixels, n_steps, level,
                 workspace, points, stream=None) -> None:
    """Isosurface points and normals (Sec. 3.3) for m sampled pixels into points [m, 8]."""
    check(_lib.lib().ges_levelset(n, _ptr(pos_op), _ptr(lscale_beta), _ptr(quat), ctypes.byref(cfg_c), n_views,
                                  cams_c, _ptr(depth), _ptr(alpha), m, _ptr(pixels), int(n_steps), float(level),
                                  _ptr(workspace), workspace.numel() * workspace.element_size(), _ptr(points),
                                  _stream(stream)), "ges_levelset")


def levelset(pos_op, lscale_beta, quat, cams, depth, alpha, pixels, n_steps: int = 32, level: float = 0.3,
             cfg: Optional["GESConfig"] = None, stream=None) -> torch.Tensor:
    """[m, 8] isosurface points (x, y, z, normal, t, valid) of the sampled pixels ([m, 2] int32:
    view, y * W + x) of rendered views (depth, alpha: ges_render_fwd's outputs)."""
    cfg = cfg or GESConfig()
    n, m = pos_op.shape[0], pixels.shape[0]
    cams_c = cameras_to_c(cams)
    ws = torch.empty(ges_levelset_workspace_bytes(n, m), dtype=torch.uint8, device=pos_op.device)
    out = torch.empty((m, 8), dtype=torch.float32, device=pos_op.device)
    ges_levelset(n, pos_op, lscale_beta, quat, cfg.to_c(), len(cams), cams_c, depth, alpha, m, pixels, n_steps,
                 level, ws, out, stream)
    return out


def ges_sync_status(proj, stream=None) -> int:
    """Synchronises the stream; returns (and clears) the device-recorded status code."""
    return int(_lib.lib().ges_sync_status(_ptr(proj), proj.numel(), _stream(stream)))


# --------------------------------------------------------------------------- buffers + sequencing
class Rasterizer:
    """Device buffers and call sequence for n splats rendered into a fixed set of views.

    Per-pixel outputs are concatenated over views; colour and normal are planar
    per view ([3, H_v, W_v] blocks), depth / alpha / t_final / last / n_contrib
    are [sum_v H_v W_v]. `capacity` fixes the tile-instance capacity (needed
    for CUDA-graph capture); by default it grows to fit each frame.
    """

    def __init__(self, n: int, cams: Sequence, cfg: GESConfig, capacity: Optional[int] = None,
                 device: str = "cuda", headroom: float = 1.25):
        self.n = int(n)
        self.cams = [_cam_dict(c) for c in cams]
        self.n_views = len(self.cams)
        self.cfg = cfg
        self.cams_c = cameras_to_c(self.cams)
        self.cfg_c = cfg.to_c()
        self.device = torch.device(device)
        self.headroom = headroom
        self.sizes = [(c["width"], c["height"]) for c in self.cams]
        self.pix = [w * h for (w, h) in self.sizes]
        self.pix_base = [0]
        for p in self.pix:
            self.pix_base.append(self.pix_base[-1] + p)
        self.P = self.pix_base[-1]
        pb = ges_proj_bytes(self.n, self.n_views)
        if pb == 0:
            raise GESError(_lib.GES_ERR_INVALID_ARG, "ges_proj_bytes")
        self.proj = torch.empty(pb, dtype=torch.uint8, device=self.device)
        self.fixed_capacity = capacity is not None
        self.capacity = 0
        self.bins = None
        if capacity is not None:
            self._alloc_bins(int(capacity))
        P = self.P
        f32 = dict(dtype=torch.float32, device=self.device)
        self.out = dict(color=torch.empty(3 * P, **f32), depth=torch.empty(P, **f32), alpha=torch.empty(P, **f32),
                        normal=torch.empty(3 * P, **f32), t_final=torch.empty(P, **f32),
                        last=torch.empty(P, dtype=torch.int32, device=self.device),
                        n_contrib=torch.empty(P, dtype=torch.int32, device=self.device))
        self.last_instance_count = None

    # -- buffers
    def _alloc_bins(self, cap: int) -> None:
        nb = ges_bins_bytes(self.n, self.n_views, self.cams_c, self.cfg_c, cap)
        if nb == 0:
            raise GESError(_lib.GES_ERR_INVALID_ARG, f"ges_bins_bytes(capacity={cap})")
        self.bins = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.capacity = cap

    def layout(self) -> _lib.Layout:
        return ges_get_layout(self.n, self.n_views, self.cams_c, self.cfg_c, self.capacity)

    # -- calls
    def check_inputs(self, pos_op, lscale_beta, quat, color) -> None:
        """Shapes and element types the C ABI cannot see behind its pointers."""
        n, k = self.n, (1 if self.cfg.sh_degree < 0 else (self.cfg.sh_degree + 1) ** 2)
        cdt = COLOR_DTYPES[self.cfg.color_storage]
        for name, t, numel, dt in (("pos_op", pos_op, 4 * n, torch.float32),
                                   ("lscale_beta", lscale_beta, 4 * n, torch.float32),
                                   ("quat", quat, 4 * n, torch.float32), ("color", color, 3 * k * n, cdt)):
            if t.dtype != dt or t.numel() != numel:
                raise ValueError(f"{name}: expected {numel} {dt} values, got {t.numel()} {t.dtype}")

    def preprocess(self, pos_op, lscale_beta, quat, color, stream=None) -> None:
        self.check_inputs(pos_op, lscale_beta, quat, color)
        ges_preprocess(self.n, pos_op, lscale_beta, quat, color, self.n_views, self.cams_c, self.cfg_c, self.proj,
                       stream)

    def preprocess_range(self, first: int, count: int, pos_op, lscale_beta, quat, color, stream=None) -> None:
        """S1-S4 for the splats [first, first + count) (the range from 0 goes first)."""
        self.check_inputs(pos_op, lscale_beta, quat, color)
        ges_preprocess_range(self.n, first, count, pos_op, lscale_beta, quat, color, self.n_views, self.cams_c,
                             self.cfg_c, self.proj, stream)

    def bin(self, stream=None) -> None:
        if not self.fixed_capacity:
            m = ges_instance_count(self.proj, stream)
            self.last_instance_count = m
            if self.bins is None or m > self.capacity:
                self._alloc_bins(max(1024, int(math.ceil(m * self.headroom))))
        ges_bin(self.n, self.n_views, self.cams_c, self.cfg_c, self.proj, self.bins, stream)

    def render_fwd(self, stream=None, n_eval: Optional[torch.Tensor] = None,
                   depth_normal: bool = True) -> Dict[str, torch.Tensor]:
        """S6. depth_normal=False leaves the depth and normal outputs unwritten (and their
        accumulation out), for renders that only feed a loss on the colour."""
        o = self.out
        ges_render_fwd(self.n, self.n_views, self.cams_c, self.cfg_c, self.proj, self.bins, o["color"],
                       o["depth"] if depth_normal else None, o["alpha"], o["normal"] if depth_normal else None,
                       o["t_final"], o["last"], o["n_contrib"], n_eval, stream)
        return o

    def forward(self, pos_op, lscale_beta, quat, color, stream=None) -> Dict[str, torch.Tensor]:
        self.preprocess(pos_op, lscale_beta, quat, color, stream)
        self.bin(stream)
        return self.render_fwd(stream)

    def backward(self, pos_op, lscale_beta, quat, color, g_color=None, g_depth=None, g_alpha=None, g_normal=None,
                 grads: Optional[Dict[str, torch.Tensor]] = None, g2d: Optional[torch.Tensor] = None,
                 stream=None) -> Dict[str, torch.Tensor]:
        if grads is None:
            grads = dict(g_pos_op=torch.empty_like(pos_op), g_lscale_beta=torch.empty_like(lscale_beta),
                         g_quat=torch.empty_like(quat),
                         g_color=torch.empty(color.shape, dtype=torch.float32, device=color.device))
        o = self.out
        ges_render_bwd(self.n, self.n_views, self.cams_c, self.cfg_c, pos_op, lscale_beta, quat, color, self.proj,
                       self.bins, o["color"], o["depth"], o["normal"], o["t_final"], o["last"], g_color, g_depth,
                       g_alpha, g_normal, grads["g_pos_op"], grads["g_lscale_beta"], grads["g_quat"],
                       grads["g_color"], g2d, stream)
        return grads

    def backward_screen(self, g_color=None, g_depth=None, g_alpha=None, g_normal=None,
                        g2d: Optional[torch.Tensor] = None, stream=None) -> None:
        o = self.out
        ges_render_bwd_screen(self.n, self.n_views, self.cams_c, self.cfg_c, self.proj, self.bins, o["color"],
                              o["depth"], o["normal"], o["t_final"], o["last"], g_color, g_depth, g_alpha, g_normal,
                              g2d, stream)

    def preprocess_bwd(self, pos_op, lscale_beta, quat, color, grads: Dict[str, torch.Tensor],
                       g2d: Optional[torch.Tensor] = None, stream=None) -> Dict[str, torch.Tensor]:
        ges_preprocess_bwd(self.n, self.n_views, self.cams_c, self.cfg_c, pos_op, lscale_beta, quat, color, self.proj,
                           g2d, grads["g_pos_op"], grads["g_lscale_beta"], grads["g_quat"], grads["g_color"], stream)
        return grads

    def preprocess_bwd_range(self, first: int, count: int, pos_op, lscale_beta, quat, color,
                             grads: Dict[str, torch.Tensor], g2d: Optional[torch.Tensor] = None,
                             stream=None) -> Dict[str, torch.Tensor]:
        """S8 for the splats [first, first + count): only their gradient rows are written."""
        ges_preprocess_bwd_range(self.n, first, count, self.n_views, self.cams_c, self.cfg_c, pos_op, lscale_beta,
                                 quat, color, self.proj, g2d, grads["g_pos_op"], grads["g_lscale_beta"],
                                 grads["g_quat"], grads["g_color"], stream)
        return grads

    def sync_status(self, stream=None) -> int:
        return ges_sync_status(self.proj, stream)

    def cull_events(self) -> int:
        """(8x4 pixel block, splat) pairs that passed the forward's warp cull in the last
        render_fwd call given n_eval (read from the bins header; synchronises)."""
        torch.cuda.synchronize()
        return int(self.bins[16:24].view(torch.int64).item())

    def instance_count(self, stream=None) -> int:
        """Tile instances produced by the last preprocess (synchronises the stream)."""
        return ges_instance_count(self.proj, stream)

    # -- views of the outputs
    def image(self, name: str, v: int) -> torch.Tensor:
        w, h = self.sizes[v]
        if name in ("color", "normal"):
            b = 3 * self.pix_base[v]
            return self.out[name][b:b + 3 * w * h].view(3, h, w)
        b = self.pix_base[v]
        return self.out[name][b:b + w * h].view(h, w)

    def proj_views(self) -> Dict[str, torch.Tensor]:
        """Intermediate per-entry arrays inside `proj` (records, binning records, g2d)."""
        lay = self.layout()
        nv = self.n * self.n_views
        rec = self.proj[lay.proj_records:lay.proj_records + nv * 64].view(torch.float32).view(nv, 16)
        binrec = self.proj[lay.proj_binrec:lay.proj_binrec + nv * 32].view(torch.int32).view(nv, 8)
        g2d = self.proj[lay.proj_g2d:lay.proj_g2d + nv * 64].view(torch.float32).view(nv, 16)
        return dict(rec=rec, binrec=binrec, g2d=g2d)

    def bins_views(self, n_inst: int) -> Dict[str, torch.Tensor]:
        lay = self.layout()
        b = self.bins
        n_inst = min(n_inst, self.capacity)
        return dict(tile=b[lay.bins_inst_tile:lay.bins_inst_tile + 4 * n_inst].view(torch.int32),
                    entry=b[lay.bins_inst_entry:lay.bins_inst_entry + 4 * n_inst].view(torch.int32),
                    ranges=b[lay.bins_ranges:lay.bins_ranges + 8 * lay.n_tiles].view(torch.int32).view(-1, 2),
                    queue=b[lay.bins_queue:lay.bins_queue + 4 * lay.n_tiles].view(torch.int32),
                    tile_base=list(lay.tile_base[:self.n_views]), n_tiles=int(lay.n_tiles))


def scene_tensors(scene, device="cuda") -> List[torch.Tensor]:
    """(pos_op, lscale_beta, quat, color) of a scenes.Scene as contiguous float32 device tensors."""
    return [torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
            for a in (scene.pos_op, scene.lscale_beta, scene.quat, scene.color)]
