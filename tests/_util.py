"""Shared helpers for the tests (no rasterizer arithmetic here)."""
import math

import numpy as np

from paper_2411_09156_gb300.scenes import Camera, Scene


def oracle_cfg(**kw):
    """The readings' default thresholds (alpha_min = 1/255, alpha_max = 0.99, t_min = 1e-4,
    low-pass 0.3, Jacobian clamp 1.3, rho = 0.1 with the centred phi) as an oracle config dict."""
    c = dict(phi_mode=1, rho=0.1, lowpass=0.3, alpha_min=float(np.float32(1.0 / 255.0)), alpha_max=0.99,
             t_min=1e-4, jac_clamp=1.3, bg=(0.0, 0.0, 0.0), flag_eps=1e-4)
    c.update(kw)
    return c


def axis_camera(width, height, f, znear=0.2):
    """Camera at the origin looking down +z (viewmat = [I | 0])."""
    vm = np.zeros((3, 4), np.float32)
    vm[:, :3] = np.eye(3)
    return Camera(width, height, f, f, 0.5 * width, 0.5 * height, vm, znear).as_dict()


def make_splats(mu, lscale, beta, opacity, quat=None, rgb=None):
    mu = np.atleast_2d(np.asarray(mu, np.float64))
    n = mu.shape[0]
    lscale = np.broadcast_to(np.asarray(lscale, np.float64), (n, 3))
    beta = np.broadcast_to(np.asarray(beta, np.float64), (n,))
    opacity = np.broadcast_to(np.asarray(opacity, np.float64), (n,))
    if quat is None:
        quat = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    if rgb is None:
        rgb = np.ones((n, 3))
    pos_op = np.concatenate([mu, opacity[:, None]], 1).astype(np.float32)
    lsb = np.concatenate([lscale, beta[:, None]], 1).astype(np.float32)
    return Scene(pos_op, lsb, np.asarray(quat, np.float32), np.asarray(rgb, np.float32).reshape(n, -1)
                 if np.asarray(rgb).ndim <= 2 else np.asarray(rgb, np.float32), -1)


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = max(np.linalg.norm(b), 1e-30)
    return float(np.linalg.norm(a - b) / den)


def fov_f(width, fov_deg=60.0):
    return 0.5 * width / math.tan(math.radians(fov_deg) / 2)
