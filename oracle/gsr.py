"""Generalized surface regularization (GSR) point evaluation, Eq. 9-13 (Sec. 3.3),
and the 16-nearest-neighbour lists it uses (Sec. 4.2) -- oracle side, FP64.

TEST INFRASTRUCTURE ONLY: imported by tests and by the benchmark's CPU leg; the
CUDA path never imports it and it imports nothing of the CUDA path.

Written with plain PyTorch CPU float64 operations; the gradient is PyTorch's
autograd of this forward (a library step, independent of the analytic backward of
the CUDA path).

Per sample point k (readings marked R; the paper gives the equations only):
  * R: the point is drawn from splat j_k's own distribution, x = mu_j + R_j (s'_j * z_k)
    with z_k ~ N(0, I) passed in (reparameterised, so gradients reach splat j), s' the
    phi(beta)-modulated scales of Eq. 6-7 and R the rotation of the normalised
    quaternion.
  * R: its neighbours are the 16 splats nearest to splat j by centre distance,
    j included (Sec. 4.2: density "from the 16 closest points").
  * Eq. 9: d(x) = sum_i o_i exp(-1/2 Q_i^(beta_i/2)), Q_i = (x - mu_i)^T Sigma_i^-1 (x - mu_i),
    Sigma_i = R_i diag(s'_i^2) R_i^T.
  * R: g* = the neighbour with the largest falloff exp(-1/2 Q_i^(beta_i/2)) (the ideal
    scene has opacity 1), i.e. the smallest exponent Q_i^(beta_i/2); ties to the earlier
    neighbour.
  * R: n* = the axis of g*'s smallest scale, turned so that e = <x - mu*, n*> >= 0;
    s_min = g*'s smallest phi-modulated scale.
  * Eq. 10 (exponent placement garbled in the paper), R: the ideal density is a flat
    GES of opacity 1 evaluated with Eq. 9's falloff, dbar = exp(-1/2 (e^2 / s_min^2)^(beta*/2)).
  * Eq. 11, R: f = s_min sqrt(-2 ln d), fbar = s_min sqrt(-2 ln dbar) (the "+" branch),
    with d clamped to [1e-30, 1] (a sum of overlapping splats can exceed 1).
  * Eq. 12: L_sdf = mean_k |fbar - f|.
  * Eq. 13: L_nor = mean_k || grad f / |grad f| - n* ||^2, grad f taken in x (its
    direction, that of -grad d, from the sum of the neighbours' terms scaled by the
    largest one, so it stays defined where d underflows).
  * The value returned for the step is lambda_sdf L_sdf + lambda_nor L_nor (the
    weights of Eq. 14 are not given in the paper and are the caller's).

KNN: exact 16 nearest centres per splat in Euclidean distance, self included
(distance 0), ordered by distance, ties by index (brute force).
"""
from __future__ import annotations

import numpy as np
import torch

K = 16
D_MIN = 1e-30


def phi(beta: torch.Tensor, rho: float, mode: int) -> torch.Tensor:
    """phi(beta) of Eq. 7 under the reading of the rasterizer (mode 1 centred, 2 as printed, 0 off)."""
    if mode == 0:
        return torch.ones_like(beta)
    if mode == 1:
        return 2.0 / (1.0 + torch.exp(-rho * (beta - 2.0)))
    return 2.0 / (1.0 + torch.exp(-(rho * beta - 2.0 * beta)))


def rotation(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrices (N, 3, 3) of quaternions (w, x, y, z), normalised first."""
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def knn(pos: np.ndarray, k: int = K) -> np.ndarray:
    """(N, k) indices of the k nearest centres, self first, by distance then index (brute force, FP64)."""
    p = torch.as_tensor(np.asarray(pos, np.float64)[:, :3])
    out = np.empty((p.shape[0], k), np.int64)
    for s in range(0, p.shape[0], 2048):
        d2 = ((p[s:s + 2048, None, :] - p[None, :, :]) ** 2).sum(-1)
        # stable order by (distance, index): sort by index is the identity, so a stable sort on distance
        order = torch.sort(d2, dim=1, stable=True).indices[:, :k]
        out[s:s + 2048] = order.numpy()
    return out


def knn_distances(pos: np.ndarray, idx: np.ndarray) -> np.ndarray:
    """FP64 distances from each splat to the listed neighbours (for checking another KNN's lists)."""
    p = np.asarray(pos, np.float64)[:, :3]
    return np.sqrt(((p[:, None, :] - p[idx]) ** 2).sum(-1))


def evaluate(pos_op, lscale_beta, quat, knn_idx, sample_splat, sample_z, rho=0.1, phi_mode=1,
             lambda_sdf=1.0, lambda_nor=1.0, with_grad=True, flag_eps=1e-4):
    """GSR losses at the sample points and their gradient with respect to the splat parameters.

    Returns dict(l_sdf, l_nor, loss, x (M,3), d, f, fbar, cos (u . n*), e, smin, beta_star,
    wcond (the direction terms' total length over the length of their sum), pscale (the largest
    (beta/2) Q^(beta/2) among the direction's terms above 1e-3 of the largest), gstar (M,)
    neighbour slot of g*, flags (M,) bool: g* decided by an exponent gap below flag_eps (1 + P),
    e within flag_eps s_min of 0, |fbar - f| within flag_eps (fbar + f), |ln d| within flag_eps,
    d within 5 % of the lower clamp, or pscale above 60; grads dict g_pos_op, g_lscale_beta,
    g_quat (N,4) or None)."""
    po = torch.tensor(np.asarray(pos_op, np.float64), requires_grad=with_grad)
    lsb = torch.tensor(np.asarray(lscale_beta, np.float64), requires_grad=with_grad)
    qt = torch.tensor(np.asarray(quat, np.float64), requires_grad=with_grad)
    nb = torch.as_tensor(np.asarray(knn_idx, np.int64))
    js = torch.as_tensor(np.asarray(sample_splat, np.int64))
    z = torch.as_tensor(np.asarray(sample_z, np.float64))
    mu, op = po[:, :3], po[:, 3]
    beta = lsb[:, 3]
    sp = phi(beta, rho, phi_mode)[:, None] * torch.exp(lsb[:, :3])  # s' (N, 3)
    R = rotation(qt)  # (N, 3, 3), columns = axes
    # sample points
    x = mu[js] + torch.einsum("mab,mb->ma", R[js], sp[js] * z)
    # neighbours
    ni = nb[js]  # (M, 16)
    delta = x[:, None, :] - mu[ni]  # (M, 16, 3)
    loc = torch.einsum("mkab,mka->mkb", R[ni], delta) / sp[ni]  # coordinates in the splat's axes / s'
    Q = (loc * loc).sum(-1)  # Mahalanobis^2
    hb = beta[ni] / 2.0
    G = torch.exp(-0.5 * Q ** hb)
    t = op[ni] * G
    d = t.sum(-1)
    # g*: largest falloff, first on ties -- the smallest exponent P = Q^(beta/2), since
    # G = exp(-P/2) decreases in P; P does not underflow where G does
    P = Q ** hb
    Pd = P.detach()
    gslot = torch.argmin(Pd, dim=1)  # torch returns the first minimal index
    # a near tie: float32 evaluates P with an error relative to P, so exponents within
    # flag_eps (1 + P) of each other may swap order
    low2 = torch.topk(Pd, 2, dim=1, largest=False).values
    flags = (low2[:, 1] - low2[:, 0]) <= flag_eps * (1.0 + low2[:, 0])
    gs = ni[torch.arange(ni.shape[0]), gslot]
    kmin = torch.argmin(lsb.detach()[:, :3], dim=1)  # smallest scale axis (ties: lowest index)
    n_raw = R[gs, :, kmin[gs]]  # (M, 3) column kmin of R*
    e_raw = ((x - mu[gs]) * n_raw).sum(-1)
    sg = torch.where(e_raw.detach() < 0, -1.0, 1.0)
    nstar = sg[:, None] * n_raw
    e = sg * e_raw
    flags = flags | (e.detach().abs() <= flag_eps * sp.detach()[gs].min(-1).values)
    smin = sp[gs, kmin[gs]]
    hs = beta[gs] / 2.0
    fbar = smin * (e / smin) ** hs  # s_min sqrt(-2 ln dbar), -2 ln dbar = (e^2 / s_min^2)^(beta*/2)
    dc = torch.clamp(d, D_MIN, 1.0)
    pl = -2.0 * torch.log(dc)
    pos = pl > 0
    f = torch.where(pos, smin * torch.sqrt(torch.where(pos, pl, torch.ones_like(pl))), torch.zeros_like(pl))
    # grad f in x is -s_min^2 grad d / (d f): its direction is that of
    # -grad d = sum_i t_i (beta_i/2) Q_i^(beta_i/2 - 1) Sigma_i^-1 (x - mu_i). A positive
    # common factor does not change the direction, so the sum is taken relative to the
    # largest term, exp(-P_min/2), which keeps it representable when every t_i underflows
    # (samples far out in the tail of all 16 neighbours).
    pmin = Pd.min(dim=1, keepdim=True).values
    rel = op[ni] * torch.exp(-0.5 * (P - pmin)) * hb * P / Q  # t_i (beta_i/2) Q^(beta_i/2-1) / exp(-P_min/2)
    ainv = torch.einsum("mkab,mkb->mka", R[ni], loc / sp[ni])  # Sigma_i^-1 (x - mu_i) = R diag(1/s') loc
    w = (rel[..., None] * ainv).sum(1)
    u = w / torch.linalg.norm(w, dim=-1, keepdim=True)
    cosv = (u * nstar).sum(-1)
    # conditioning of the direction: the sum of the terms' lengths over the length of their
    # sum, and the largest (beta/2) P among the terms that matter (float32 rounds P to about
    # 2.5e-6 (beta/2) P, so the terms' relative weights exp(-P/2) carry half that)
    wcond = ((rel[..., None] * ainv).norm(dim=-1).sum(1) / torch.linalg.norm(w, dim=-1)).detach()
    live = torch.exp(-0.5 * (Pd - pmin)) >= 1e-3
    pscale = torch.where(live, (hb * P).detach(), torch.zeros_like(Pd)).max(dim=1).values
    # decisions float32 may take the other way: the kink of |fbar - f|, d at the clamp at 1
    # (where f's derivative in d diverges), and samples so far in the tails that a term that
    # matters has (beta/2) P above 60: float32 rounds P to about 2.5e-6 (beta/2) P, and the
    # weights' derivatives carry a further factor of about P / 2, so their gradient terms are
    # uncertain to 2.5e-6 P^2 / 2, about 5e-3 at 60
    fd_, fbd = f.detach(), fbar.detach()
    flags = flags | ((fbd - fd_).abs() <= flag_eps * (fbd + fd_)) | (torch.log(d.detach()).abs() <= flag_eps)
    flags = flags | (pscale > 60.0)
    # d at the lower clamp (1e-30), whose side decides whether the density path carries gradient
    flags = flags | ((torch.log(d.detach().clamp(min=1e-300)) - np.log(D_MIN)).abs() <= 0.05)
    l_sdf = (fbar - f).abs().mean()
    l_nor = ((u - nstar) ** 2).sum(-1).mean()
    loss = lambda_sdf * l_sdf + lambda_nor * l_nor
    out = dict(l_sdf=float(l_sdf.detach()), l_nor=float(l_nor.detach()), loss=float(loss.detach()), x=x.detach().numpy(),
               d=d.detach().numpy(), f=f.detach().numpy(), fbar=fbar.detach().numpy(), cos=cosv.detach().numpy(),
               e=e.detach().numpy(), smin=smin.detach().numpy(), beta_star=(2.0 * hs).detach().numpy(),
               wcond=wcond.numpy(), pscale=pscale.numpy(), gstar=gslot.numpy(), flags=flags.numpy(), grads=None)
    if with_grad:
        g = torch.autograd.grad(loss, [po, lsb, qt], allow_unused=True)
        out["grads"] = dict(g_pos_op=g[0].numpy(), g_lscale_beta=g[1].numpy(), g_quat=g[2].numpy())
    return out
