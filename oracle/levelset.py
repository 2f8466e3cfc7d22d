"""Level-set point extraction from rendered depth (Sec. 3.3, "Mesh Extraction"; the level
alpha = 0.3 of Sec. 4.2) -- oracle side, FP64.

TEST INFRASTRUCTURE ONLY: imported by tests; the CUDA path never imports it and it imports
nothing of the CUDA path.

The paper describes the steps; the readings (R) fill in what it leaves open:
  * R: a sampled pixel (view, x, y) gives the point x0 on the ray through the pixel centre
    at camera depth z = D / A (D, A the rendered depth and alpha: the depth output is the
    alpha-weighted sum of the splats' depths, so D / A is their weighted mean); pixels with
    A below 1e-4 give no point. The ray direction v is the unit vector from the camera
    centre through the pixel centre.
  * R: the density d of Eq. 9 along the ray is summed over the 16 splats whose centres are
    nearest to x0 (the neighbourhood of the GSR, Sec. 4.2), the same 16 for the whole ray.
  * R: g, whose spread along v sets the search range, is the one of those 16 with the
    largest falloff exp(-1/2 Q^(beta/2)) at x0 (the smallest exponent, ties to the nearer
    centre); sigma_g(v) = sqrt(v^T Sigma_g v) with Sigma_g = R diag(s'^2) R^T.
  * The range t in [-3 sigma, 3 sigma] is sampled at n_steps evenly spaced t_k (first and
    last included); d_k = d(x0 + t_k v).
  * R: the isosurface point is the first crossing from the camera side, the smallest k with
    d_k < level <= d_{k+1}, at t* = t_k + (level - d_k) / (d_{k+1} - d_k) (t_{k+1} - t_k)
    (linear interpolation); none if no interval crosses upward.
  * The normal is grad f / |grad f| at the point, the direction of -grad d (as in the GSR
    oracle: the neighbour sum taken relative to its largest term).

Returns per pixel: point (3), normal (3), t*, valid, plus conditioning flags for the tests.
"""
from __future__ import annotations

import numpy as np

from oracle import gsr as OG


def _phi(beta, rho, mode):
    if mode == 0:
        return np.ones_like(beta)
    if mode == 1:
        return 2.0 / (1.0 + np.exp(-rho * (beta - 2.0)))
    return 2.0 / (1.0 + np.exp(-(rho * beta - 2.0 * beta)))


def _rot(q):
    import torch
    return OG.rotation(torch.as_tensor(np.asarray(q, np.float64))).numpy()


def ray(cam: dict, px: int, py: int):
    """Camera centre, unit world direction through the pixel centre, and the camera-frame ray
    (X/Z, Y/Z, 1)."""
    vm = np.asarray(cam["viewmat"], np.float64).reshape(3, 4)
    Rw, tw = vm[:, :3], vm[:, 3]
    c = -Rw.T @ tw
    rc = np.array([(px + 0.5 - cam["cx"]) / cam["fx"], (py + 0.5 - cam["cy"]) / cam["fy"], 1.0])
    v = Rw.T @ rc
    return c, v / np.linalg.norm(v), rc


def extract(pos_op, lscale_beta, quat, cam: dict, depth: float, alpha: float, px: int, py: int, n_steps=32,
            level=0.3, rho=0.1, phi_mode=1, flag_eps=1e-4):
    """One pixel. Returns dict(valid, point, normal, t, x0, neighbours, sigma, flag)."""
    pos = np.asarray(pos_op, np.float64)
    ls = np.asarray(lscale_beta, np.float64)
    out = dict(valid=False, point=np.zeros(3), normal=np.zeros(3), t=0.0, x0=np.zeros(3), neighbours=None, flag=False,
               sigma=0.0)
    if not alpha >= 1e-4:
        return out
    c, v, rc = ray(cam, px, py)
    vm = np.asarray(cam["viewmat"], np.float64).reshape(3, 4)
    x0 = c + vm[:, :3].T @ (rc * (float(depth) / float(alpha)))
    out["x0"] = x0
    d2 = ((pos[:, :3] - x0) ** 2).sum(1)
    order = np.argsort(d2, kind="stable")
    nb = order[:16]
    flag = bool(d2[order[16]] - d2[order[15]] <= flag_eps * d2[order[15]]) if len(order) > 16 else False
    out["neighbours"] = nb
    mu, op = pos[nb, :3], pos[nb, 3]
    beta = ls[nb, 3]
    sp = _phi(beta, rho, phi_mode)[:, None] * np.exp(ls[nb, :3])
    R = _rot(np.asarray(quat, np.float64)[nb])

    def terms(x):
        delta = x - mu
        loc = np.einsum("kab,ka->kb", R, delta) / sp
        Q = (loc ** 2).sum(1)
        P = Q ** (beta / 2.0)
        return delta, loc, Q, P

    _, _, Q0, P0 = terms(x0)
    g = int(np.argmin(P0))
    srt = np.sort(P0)
    flag = flag or bool(srt[1] - srt[0] <= flag_eps * (1.0 + srt[0]))
    sigma = np.sqrt((((R[g].T @ v) * sp[g]) ** 2).sum())
    out["sigma"] = sigma
    ts = np.linspace(-3.0 * sigma, 3.0 * sigma, n_steps)
    dk = np.empty(n_steps)
    for k, t in enumerate(ts):
        _, _, _, P = terms(x0 + t * v)
        dk[k] = (op * np.exp(-0.5 * P)).sum()
    hit = None
    for k in range(n_steps - 1):
        if dk[k] < level <= dk[k + 1]:
            hit = k
            break
    # decisions float32 may take the other way: a sample within rounding of the level
    flag = flag or bool(np.any(np.abs(dk - level) <= flag_eps * level))
    out["flag"] = flag
    if hit is None:
        return out
    k = hit
    t = ts[k] + (level - dk[k]) / (dk[k + 1] - dk[k]) * (ts[k + 1] - ts[k])
    x = x0 + t * v
    delta, loc, Q, P = terms(x)
    pmin = P.min()
    rel = op * np.exp(-0.5 * (P - pmin)) * (beta / 2.0) * P / Q
    ainv = np.einsum("kab,kb->ka", R, loc / sp)  # Sigma^-1 (x - mu)
    w = (rel[:, None] * ainv).sum(0)
    out.update(valid=True, point=x, normal=w / np.linalg.norm(w), t=t)
    return out
