"""Seeded synthetic scenes and cameras for the GES rasterizer.

This module produces inputs only: splat parameter arrays and pinhole cameras.
It holds none of the rasterizer's arithmetic (no projection, falloff,
compositing or gradients), so both the CUDA path and the FP64 oracle can be fed
from it without sharing method code.

Layouts (all float32, C-contiguous):
  pos_op      [N, 4]  world position x, y, z and activated opacity o in (0, 1)
  lscale_beta [N, 4]  log-scales l1, l2, l3 and the GES shape parameter beta
                      (the paper's epsilon, Eq. 1 and Eq. 3)
  quat        [N, 4]  rotation quaternion (w, x, y, z), not necessarily unit
  color       [N, 3]  linear RGB when sh_degree == -1, else [N, K, 3]
                      spherical-harmonic coefficients with K = (deg + 1)^2

Cameras follow the usual computer-vision convention: camera x right, y down,
z forward; viewmat is the row-major 3x4 world-to-camera matrix [R | t].

The five workloads mirror the paper's scene scales (object scale, and the
1.72M-2.78M splat counts of Table 2) with seeded distributions, standing in
for the Mip-NeRF360 / Deep Blending captures the paper trains on (Sec. 4.1),
which are not used here.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    viewmat: np.ndarray  # (3, 4) float32, world -> camera
    znear: float = 0.2

    def as_dict(self) -> dict:
        return dict(width=int(self.width), height=int(self.height), fx=float(self.fx),
                    fy=float(self.fy), cx=float(self.cx), cy=float(self.cy),
                    viewmat=np.asarray(self.viewmat, np.float32).reshape(3, 4),
                    znear=float(self.znear))


@dataclasses.dataclass
class Scene:
    pos_op: np.ndarray
    lscale_beta: np.ndarray
    quat: np.ndarray
    color: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.pos_op.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.pos_op[idx].copy(), self.lscale_beta[idx].copy(), self.quat[idx].copy(),
                     self.color[idx].copy(), self.sh_degree)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def look_at(eye, target, width, height, fov_x_deg=60.0, up=(0.0, 0.0, 1.0), znear=0.2) -> Camera:
    """Pinhole camera at `eye` looking at `target`; horizontal field of view fov_x."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    if abs(np.dot(fwd, up)) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    rot = np.stack([right, down, fwd], 0)  # rows: camera axes in world coordinates
    t = -rot @ eye
    vm = np.concatenate([rot, t[:, None]], 1).astype(np.float32)
    f = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(int(width), int(height), f, f, 0.5 * width, 0.5 * height, vm, znear)


def random_sphere_cameras(rng, n, radius, sizes, fov_x_deg=60.0) -> List[Camera]:
    cams = []
    for k in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        w, h = sizes[k]
        cams.append(look_at(radius * d, (0.0, 0.0, 0.0), w, h, fov_x_deg))
    return cams


def _random_quats(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _rotmat_to_quat(m):
    """Unit quaternions (w, x, y, z) for a batch of proper rotation matrices (Shepperd)."""
    n = m.shape[0]
    q = np.empty((n, 4))
    tr = m[:, 0, 0] + m[:, 1, 1] + m[:, 2, 2]
    cand = np.stack([tr, m[:, 0, 0], m[:, 1, 1], m[:, 2, 2]], 1)
    k = np.argmax(cand, 1)
    for case in range(4):
        s = k == case
        if not np.any(s):
            continue
        r = m[s]
        if case == 0:
            w = np.sqrt(1.0 + tr[s]) * 0.5
            q[s] = np.stack([w, (r[:, 2, 1] - r[:, 1, 2]) / (4 * w), (r[:, 0, 2] - r[:, 2, 0]) / (4 * w),
                             (r[:, 1, 0] - r[:, 0, 1]) / (4 * w)], 1)
        elif case == 1:
            x = np.sqrt(1.0 + r[:, 0, 0] - r[:, 1, 1] - r[:, 2, 2]) * 0.5
            q[s] = np.stack([(r[:, 2, 1] - r[:, 1, 2]) / (4 * x), x, (r[:, 0, 1] + r[:, 1, 0]) / (4 * x),
                             (r[:, 0, 2] + r[:, 2, 0]) / (4 * x)], 1)
        elif case == 2:
            y = np.sqrt(1.0 - r[:, 0, 0] + r[:, 1, 1] - r[:, 2, 2]) * 0.5
            q[s] = np.stack([(r[:, 0, 2] - r[:, 2, 0]) / (4 * y), (r[:, 0, 1] + r[:, 1, 0]) / (4 * y), y,
                             (r[:, 1, 2] + r[:, 2, 1]) / (4 * y)], 1)
        else:
            z = np.sqrt(1.0 - r[:, 0, 0] - r[:, 1, 1] + r[:, 2, 2]) * 0.5
            q[s] = np.stack([(r[:, 1, 0] - r[:, 0, 1]) / (4 * z), (r[:, 0, 2] + r[:, 2, 0]) / (4 * z),
                             (r[:, 1, 2] + r[:, 2, 1]) / (4 * z), z], 1)
    return q


def make_scene(n, seed, kind="uniform", sh_degree=-1) -> Scene:
    """Seeded splat cloud.

    kind = "uniform"     centres U[-1,1]^3, log-scales N(-3, 0.5), beta U[1,4],
                         opacity sigmoid(N(0,1)), RGB U[0,1] (sh_degree -1) or SH.
    kind = "object"      centres N(0, 0.5^2 I), log-scales N(-4.5, 0.7),
                         opacity sigmoid(N(0,1.5)), beta U[1,6], SH coeffs N(0, 0.2).
    kind = "heightfield" centres on z = h(x, y) over [-2,2]^2 (four seeded sinusoids,
                         total amplitude <= 0.3) plus N(0, 0.02^2) noise; smallest
                         log-scale N(-9, 0.3) on the axis aligned with the surface
                         normal, the other two N(-5, 0.8); opacity sigmoid(N(0,1));
                         beta U[1,6]; SH coeffs N(0, 0.2).
    """
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        mu = rng.uniform(-1.0, 1.0, size=(n, 3))
        ls = rng.normal(-3.0, 0.5, size=(n, 3))
        q = _random_quats(rng, n)
        op = _sigmoid(rng.normal(0.0, 1.0, size=n))
        beta = rng.uniform(1.0, 4.0, size=n)
    elif kind == "object":
        mu = rng.normal(0.0, 0.5, size=(n, 3))
        ls = rng.normal(-4.5, 0.7, size=(n, 3))
        q = _random_quats(rng, n)
        op = _sigmoid(rng.normal(0.0, 1.5, size=n))
        beta = rng.uniform(1.0, 6.0, size=n)
    elif kind == "heightfield":
        amps = rng.uniform(0.02, 0.075, size=4)
        freqs = rng.uniform(0.5, 3.0, size=4)
        angs = rng.uniform(0.0, 2 * np.pi, size=4)
        phases = rng.uniform(0.0, 2 * np.pi, size=4)
        kx, ky = freqs * np.cos(angs), freqs * np.sin(angs)
        xy = rng.uniform(-2.0, 2.0, size=(n, 2))
        arg = xy[:, :1] * kx[None] + xy[:, 1:] * ky[None] + phases[None]
        h = (amps[None] * np.sin(arg)).sum(1)
        hx = (amps[None] * kx[None] * np.cos(arg)).sum(1)
        hy = (amps[None] * ky[None] * np.cos(arg)).sum(1)
        mu = np.stack([xy[:, 0], xy[:, 1], h], 1) + rng.normal(0.0, 0.02, size=(n, 3))
        nrm = np.stack([-hx, -hy, np.ones(n)], 1)
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        # tangent frame with a random in-plane angle; third column = surface normal
        ref = np.zeros((n, 3))
        ref[:, 0] = 1.0
        t1 = ref - nrm * nrm[:, :1]
        t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
        t2 = np.cross(nrm, t1)
        th = rng.uniform(0.0, 2 * np.pi, size=n)[:, None]
        a1 = np.cos(th) * t1 + np.sin(th) * t2
        a2 = np.cross(nrm, a1)
        rot = np.stack([a1, a2, nrm], 2)  # columns are the splat's local axes
        q = _rotmat_to_quat(rot)
        ls = np.stack([rng.normal(-5.0, 0.8, size=n), rng.normal(-5.0, 0.8, size=n),
                       rng.normal(-9.0, 0.3, size=n)], 1)
        op = _sigmoid(rng.normal(0.0, 1.0, size=n))
        beta = rng.uniform(1.0, 6.0, size=n)
    else:
        raise ValueError(kind)
    # scale the quaternion norm randomly: inputs need not be unit length
    q = q * rng.uniform(0.5, 2.0, size=(n, 1))
    if sh_degree < 0:
        color = rng.uniform(0.0, 1.0, size=(n, 3))
    else:
        k = (sh_degree + 1) ** 2
        color = rng.normal(0.0, 0.2, size=(n, k, 3))
    pos_op = np.concatenate([mu, op[:, None]], 1)
    lsb = np.concatenate([ls, beta[:, None]], 1)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f32(pos_op), f32(lsb), f32(q), f32(color), int(sh_degree))


# --------------------------------------------------------------------------- workloads
WORKLOADS = {
    "tiny-1k-128": "1,000 uniform splats, RGB, one 128x128 camera at distance 4",
    "object-100k-800": "100k object-scale splats, SH3, one 800x800 camera on a sphere of radius 4",
    "scene-1.5M-1600x1040": "1.5M heightfield splats, SH3, one 1600x1040 camera above the surface at 45 deg",
    "drt8-1.5M": "the 1.5M heightfield scene, 8 views on a radius-5 sphere, cosine-schedule sizes 400x260..1600x1040",
    "drt16-3M": "3M heightfield splats, 16 views, cosine-schedule sizes 480x270..1920x1080",
}


def workload(name: str, sizes: Optional[List[tuple]] = None, n_override: Optional[int] = None):
    """(scene, cameras) for a named workload.

    Batched workloads need their view sizes from the caller (the cosine
    dynamic-resolution schedule lives with the rasterizer, not here).
    """
    if name == "tiny-1k-128":
        sc = make_scene(n_override or 1000, 0, "uniform", -1)
        cams = [look_at((0.0, -4.0, 0.0), (0, 0, 0), 128, 128)]
    elif name == "object-100k-800":
        sc = make_scene(n_override or 100_000, 1, "object", 3)
        rng = np.random.default_rng(101)
        cams = random_sphere_cameras(rng, 1, 4.0, [(800, 800)])
    elif name == "scene-1.5M-1600x1040":
        sc = make_scene(n_override or 1_500_000, 2, "heightfield", 3)
        r = 4.0
        cams = [look_at((0.0, -r * math.cos(math.pi / 4), r * math.sin(math.pi / 4)), (0, 0, 0), 1600, 1040)]
    elif name == "drt8-1.5M":
        sc = make_scene(n_override or 1_500_000, 2, "heightfield", 3)
        if sizes is None:
            raise ValueError("batched workloads need view sizes")
        rng = np.random.default_rng(103)
        cams = random_sphere_cameras(rng, len(sizes), 5.0, sizes)
    elif name == "drt16-3M":
        sc = make_scene(n_override or 3_000_000, 4, "heightfield", 3)
        if sizes is None:
            raise ValueError("batched workloads need view sizes")
        rng = np.random.default_rng(104)
        cams = random_sphere_cameras(rng, len(sizes), 5.0, sizes)
    else:
        raise KeyError(name)
    return sc, cams


def upstream_grads(seed, n_pix_total, with_alpha=True):
    """Random upstream gradients N(0,1) per pixel and channel (colour 3, depth 1, alpha 1, normal 3)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal(size=(8, n_pix_total)).astype(np.float32)
    if not with_alpha:
        g[4] = 0.0
    return g
