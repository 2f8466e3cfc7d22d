"""Pins of the Eq. 8 loss oracle (oracle/loss.py) to facts other than its own formulas:
window properties, closed forms of SSIM on constant and offset images, identities
(SSIM(x, x) = 1, symmetry), a separable re-implementation of the window filter,
and central finite differences of the loss for its gradient."""
import numpy as np
import pytest

from oracle import loss as OL


def test_window_is_a_normalised_symmetric_gaussian():
    w = OL.window()
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w, w.T, rtol=0, atol=1e-18)
    np.testing.assert_allclose(w, w[::-1, ::-1], rtol=0, atol=1e-18)
    g = w.sum(1)  # the 1-D marginal
    # ratio of neighbouring taps of exp(-k^2 / (2 sigma^2)) is exp(-(2k+1) / (2 sigma^2))
    k = np.arange(5, 10)
    np.testing.assert_allclose(g[k + 1] / g[k], np.exp(-(2 * (k - 5) + 1) / (2 * 1.5 ** 2)), rtol=1e-12)


def test_filter_equals_separable_convolution_and_keeps_constants_inside():
    rng = np.random.default_rng(0)
    img = rng.random((23, 31))
    g = OL.window().sum(1)
    # rows then columns with numpy's 1-D convolution (zero padding, same size)
    rows = np.stack([np.convolve(r, g, mode="same") for r in img])
    sep = np.stack([np.convolve(c, g, mode="same") for c in rows.T]).T
    np.testing.assert_allclose(OL.filt(img), sep, rtol=0, atol=1e-14)
    const = np.full((30, 30), 0.7)
    np.testing.assert_allclose(OL.filt(const)[5:-5, 5:-5], 0.7, rtol=0, atol=1e-14)


def test_ssim_of_an_image_with_itself_is_one_everywhere():
    x = np.random.default_rng(1).random((3, 17, 26))
    out = OL.loss(x, x)
    np.testing.assert_allclose(out["ssim"], 1.0, rtol=0, atol=1e-12)
    assert abs(out["loss"]) < 1e-12
    np.testing.assert_allclose(out["grad"], 0.0, atol=1e-12)


def test_ssim_of_constant_images_is_the_luminance_term():
    a, b = 0.3, 0.8
    x = np.full((3, 40, 40), a)
    y = np.full((3, 40, 40), b)
    s = OL.loss(x, y)["ssim"][:, 5:-5, 5:-5]  # away from the zero padding
    np.testing.assert_allclose(s, (2 * a * b + OL.C1) / (a * a + b * b + OL.C1), rtol=1e-12)


def test_ssim_of_an_offset_texture_is_its_luminance_term():
    # y = x + k: equal variances and covariance = variance, so the structure term is 1
    rng = np.random.default_rng(2)
    x = rng.random((1, 36, 36)) * 0.5
    k = 0.25
    _, (mx, my, *_rest) = OL.ssim_map(x[0], x[0] + k)
    s = OL.ssim_map(x[0], x[0] + k)[0]
    inner = (slice(10, -10), slice(10, -10))
    lum = (2 * mx * my + OL.C1) / (mx * mx + my * my + OL.C1)
    np.testing.assert_allclose(s[inner], lum[inner], rtol=1e-10)


def test_ssim_is_symmetric():
    rng = np.random.default_rng(3)
    x, y = rng.random((3, 19, 21)), rng.random((3, 19, 21))
    np.testing.assert_allclose(OL.loss(x, y)["ssim"], OL.loss(y, x)["ssim"], rtol=0, atol=1e-13)


def test_l1_part_with_lambda_zero():
    rng = np.random.default_rng(4)
    x, y = rng.random((3, 9, 13)), rng.random((3, 9, 13))
    out = OL.loss(x, y, lam=0.0)
    assert abs(out["loss"] - np.abs(x - y).mean()) < 1e-15
    np.testing.assert_allclose(out["grad"], np.sign(x - y) / x.size, rtol=0, atol=1e-18)


@pytest.mark.parametrize("lam", [0.2, 1.0])
def test_gradient_matches_central_differences(lam):
    rng = np.random.default_rng(5)
    x = rng.random((3, 14, 17))
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1)
    out = OL.loss(x, y, lam=lam)
    h = 1e-6
    picks = [(c, i, j) for c in range(3) for (i, j) in [(0, 0), (0, 16), (13, 0), (7, 8), (3, 12), (11, 2)]]
    for (c, i, j) in picks:
        if abs(x[c, i, j] - y[c, i, j]) < 1e-3 and lam < 1.0:
            continue  # |d| is not differentiable at 0
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (OL.loss(xp, y, lam=lam, with_grad=False)["loss"] - OL.loss(xm, y, lam=lam, with_grad=False)["loss"]) / (2 * h)
        assert abs(fd - out["grad"][c, i, j]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (c, i, j, fd, out["grad"][c, i, j])
