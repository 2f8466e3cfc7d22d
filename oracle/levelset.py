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

extract() does one pixel; start_point() and march() are its two halves (the tests move x0
by the rounding of a float32 start point to see which decisions that can flip), and
normal_at() / density_at() evaluate the normal and d at any point for a given neighbour set.
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


def start_point(cam: dict, depth: float, alpha: float, px: int, py: int):
    """(x0, v) of a pixel, or None when its alpha is below 1e-4."""
    if not alpha >= 1e-4:
        return None
    c, v, rc = ray(cam, px, py)
    vm = np.asarray(cam["viewmat"], np.float64).reshape(3, 4)
    return c + vm[:, :3].T @ (rc * (float(depth) / float(alpha))), v


class _Neighbours:
    """The falloff terms of a fixed set of splats."""

    def __init__(self, pos, ls, quat, nb, rho, phi_mode):
        self.mu, self.op = pos[nb, :3], pos[nb, 3]
        self.beta = ls[nb, 3]
        self.sp = _phi(self.beta, rho, phi_mode)[:, None] * np.exp(ls[nb, :3])
        self.R = _rot(np.asarray(quat, np.float64)[nb])

    def terms(self, x):
        delta = x - self.mu
        loc = np.einsum("kab,ka->kb", self.R, delta) / self.sp  # axis coordinates over s'
        Q = (loc ** 2).sum(1)
        P = Q ** (self.beta / 2.0)
        return loc, Q, P

    def density(self, x):
        _, _, P = self.terms(x)
        return (self.op * np.exp(-0.5 * P)).sum()

    def normal(self, x):
        """grad f / |grad f| (= -grad d / |grad d|) and the cancellation of the sum,
        sum |term| / |sum term|."""
        loc, Q, P = self.terms(x)
        pmin = P.min()
        rel = self.op * np.exp(-0.5 * (P - pmin)) * (self.beta / 2.0) * P / Q
        ainv = np.einsum("kab,kb->ka", self.R, loc / self.sp)  # Sigma^-1 (x - mu)
        terms = rel[:, None] * ainv
        w = terms.sum(0)
        nw = np.linalg.norm(w)
        return w / nw, np.linalg.norm(terms, axis=1).sum() / nw


def nearest(pos, x0, flag_eps=1e-4, cand=None):
    """Indices of the 16 centres nearest to x0 (by distance, ties to the lower index) and
    whether the 16th and 17th are within flag_eps (relative, squared distance) of each other.
    cand: indices known to hold the 17 nearest (searched instead of all centres)."""
    idx = np.arange(len(pos)) if cand is None else np.sort(np.asarray(cand))
    d2 = ((np.asarray(pos, np.float64)[idx, :3] - x0) ** 2).sum(1)
    order = np.argsort(d2, kind="stable")
    flag = bool(d2[order[16]] - d2[order[15]] <= flag_eps * d2[order[15]]) if len(order) > 16 else False
    return idx[order[:16]], flag


def march(pos_op, lscale_beta, quat, x0, v, n_steps=32, level=0.3, rho=0.1, phi_mode=1, flag_eps=1e-4, cand=None):
    """The density march from x0 along v. Returns dict(valid, point, normal, t, neighbours, g,
    sigma, flag, hit, ts, dk, dmag, cond): hit = k of the crossing interval (-1 if none), dk the
    sampled densities, dmag the sums of |o exp(-P/2)| (1 + P (1 + |ln Q|)) per sample (the
    scale of float32's rounding of d_k), cond the cancellation of the normal's sum. cand as in
    nearest()."""
    pos = np.asarray(pos_op, np.float64)
    ls = np.asarray(lscale_beta, np.float64)
    x0 = np.asarray(x0, np.float64)
    v = np.asarray(v, np.float64)
    nb, flag = nearest(pos, x0, flag_eps, cand)
    N = _Neighbours(pos, ls, quat, nb, rho, phi_mode)
    _, _, P0 = N.terms(x0)
    g = int(np.argmin(P0))
    srt = np.sort(P0)
    flag = flag or bool(srt[1] - srt[0] <= flag_eps * (1.0 + srt[0]))
    sigma = np.sqrt((((N.R[g].T @ v) * N.sp[g]) ** 2).sum())
    ts = np.linspace(-3.0 * sigma, 3.0 * sigma, n_steps)
    dk = np.empty(n_steps)
    dmag = np.empty(n_steps)
    for k, t in enumerate(ts):
        _, Q, P = N.terms(x0 + t * v)
        e = N.op * np.exp(-0.5 * P)
        dk[k] = e.sum()
        with np.errstate(divide="ignore"):
            dmag[k] = (e * (1.0 + P * (1.0 + np.abs(np.log(np.maximum(Q, 1e-300)))))).sum()
    hit = -1
    for k in range(n_steps - 1):
        if dk[k] < level <= dk[k + 1]:
            hit = k
            break
    # decisions float32 may take the other way: a sample within rounding of the level
    flag = flag or bool(np.any(np.abs(dk - level) <= flag_eps * level))
    out = dict(valid=False, point=np.zeros(3), normal=np.zeros(3), t=0.0, neighbours=nb, g=g, sigma=sigma,
               flag=flag, hit=hit, ts=ts, dk=dk, dmag=dmag, cond=0.0)
    if hit < 0:
        return out
    k = hit
    t = ts[k] + (level - dk[k]) / (dk[k + 1] - dk[k]) * (ts[k + 1] - ts[k])
    x = x0 + t * v
    n, cond = N.normal(x)
    out.update(valid=True, point=x, normal=n, t=t, cond=cond)
    return out


def normal_at(pos_op, lscale_beta, quat, nb, x, rho=0.1, phi_mode=1):
    """(normal, cancellation) at x summed over the splats nb."""
    N = _Neighbours(np.asarray(pos_op, np.float64), np.asarray(lscale_beta, np.float64), quat, np.asarray(nb), rho,
                    phi_mode)
    return N.normal(np.asarray(x, np.float64))


def density_at(pos_op, lscale_beta, quat, nb, x, rho=0.1, phi_mode=1):
    """d(x) of Eq. 9 summed over the splats nb."""
    N = _Neighbours(np.asarray(pos_op, np.float64), np.asarray(lscale_beta, np.float64), quat, np.asarray(nb), rho,
                    phi_mode)
    return N.density(np.asarray(x, np.float64))


def extract(pos_op, lscale_beta, quat, cam: dict, depth: float, alpha: float, px: int, py: int, n_steps=32,
            level=0.3, rho=0.1, phi_mode=1, flag_eps=1e-4):
    """One pixel. Returns march()'s dict plus x0 (valid False and x0 = 0 when alpha < 1e-4)."""
    sp = start_point(cam, depth, alpha, px, py)
    if sp is None:
        return dict(valid=False, point=np.zeros(3), normal=np.zeros(3), t=0.0, x0=np.zeros(3), neighbours=None,
                    g=-1, sigma=0.0, flag=False, hit=-1, ts=None, dk=None, dmag=None, cond=0.0)
    x0, v = sp
    out = march(pos_op, lscale_beta, quat, x0, v, n_steps, level, rho, phi_mode, flag_eps)
    out["x0"] = x0
    return out
