"""Reconstruction loss of Eq. 8 (Sec. 3.2) and its gradient -- oracle side, FP64.

TEST INFRASTRUCTURE ONLY: imported by tests and by the benchmark's CPU leg; the
CUDA path never imports it and it imports nothing of the CUDA path.

    L_rgb = (1 - lambda) L_1 + lambda L_SSIM,   lambda = 0.2          (Eq. 8)

The paper names the two terms and lambda only. The readings taken here (the
usual ones for Gaussian-splatting training) are:

  * L_1 = mean over the pixels and the 3 channels of |C - C_target|.
  * L_SSIM = 1 - mean over the pixels and channels of the SSIM map (Wang et al.
    2004): per channel,
        SSIM(p) = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2))
    with mu, s^2, s_xy the local means, variances and covariance under an 11 x 11
    Gaussian window of standard deviation 1.5 (normalised to sum 1), C1 = 0.01^2,
    C2 = 0.03^2 (data range 1). Outside the image both images are 0 (zero padding),
    and the map is taken at every pixel of the image.
  * A batch of views has one loss per view; the gradient of each view is that of
    its own loss.

Images are planar float arrays (3, H, W). Everything here is float64, written as
the definitions above: the window filter is a direct 2-D correlation (a sum over
the 121 offsets), and the gradient is the chain rule through the local
statistics, with d mu_x(p)/d x(q) = g(p - q), d s_x^2(p)/d x(q) = 2 g(p - q)(x(q) -
mu_x(p)), d s_xy(p)/d x(q) = g(p - q)(y(q) - mu_y(p)).
"""
from __future__ import annotations

import numpy as np

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def window() -> np.ndarray:
    """The 11 x 11 Gaussian window (sum 1), as the outer product of the 1-D one."""
    k = np.arange(WIN, dtype=np.float64) - WIN // 2
    g = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    g /= g.sum()
    return np.outer(g, g)


def filt(img: np.ndarray) -> np.ndarray:
    """Zero-padded 2-D correlation of one (H, W) plane with the window, same size."""
    w = window()
    h, wd = img.shape
    r = WIN // 2
    pad = np.zeros((h + 2 * r, wd + 2 * r))
    pad[r:r + h, r:r + wd] = img
    out = np.zeros((h, wd))
    for dy in range(WIN):
        for dx in range(WIN):
            out += w[dy, dx] * pad[dy:dy + h, dx:dx + wd]
    return out


def ssim_map(x: np.ndarray, y: np.ndarray):
    """SSIM map of one plane pair and the local statistics it came from."""
    mx, my = filt(x), filt(y)
    sxx = filt(x * x) - mx * mx
    syy = filt(y * y) - my * my
    sxy = filt(x * y) - mx * my
    num1, num2 = 2.0 * mx * my + C1, 2.0 * sxy + C2
    den1, den2 = mx * mx + my * my + C1, sxx + syy + C2
    return (num1 * num2) / (den1 * den2), (mx, my, sxx, syy, sxy, num1, num2, den1, den2)


def loss(color: np.ndarray, target: np.ndarray, lam: float = LAMBDA, with_grad: bool = True):
    """L_rgb of one view and dL_rgb/dcolor. color, target: (3, H, W).

    Returns dict(loss, l1, dssim, grad (3, H, W) or None, ssim (3, H, W))."""
    x = np.asarray(color, np.float64)
    y = np.asarray(target, np.float64)
    c, h, w = x.shape
    n = c * h * w
    d = x - y
    l1 = np.abs(d).sum() / n
    maps, grad = [], np.zeros_like(x) if with_grad else None
    for ch in range(c):
        s, (mx, my, sxx, syy, sxy, num1, num2, den1, den2) = ssim_map(x[ch], y[ch])
        maps.append(s)
        if with_grad:
            # dSSIM(p) / d(mu_x, s_x^2, s_xy) at each output pixel p
            den = den1 * den2
            d_mx = (2.0 * my * num2) / den - (2.0 * mx * num1 * num2) / (den1 * den1 * den2)
            d_sxx = -(num1 * num2) / (den1 * den2 * den2)
            d_sxy = (2.0 * num1) / den
            # chain rule to x(q): sum over p of g(p - q) [d_mx + 2 d_sxx (x(q) - mx) + d_sxy (y(q) - my)]
            a = d_mx - 2.0 * d_sxx * mx - d_sxy * my
            gs = filt(a) + 2.0 * x[ch] * filt(d_sxx) + y[ch] * filt(d_sxy)
            grad[ch] = (1.0 - lam) * np.sign(d[ch]) / n - lam * gs / n
    ssim = np.stack(maps)
    dssim = 1.0 - ssim.mean()
    return dict(loss=(1.0 - lam) * l1 + lam * dssim, l1=l1, dssim=dssim, grad=grad, ssim=ssim)
