"""The oracle's analytic gradient (S7 + S8) against central finite differences of
its own FP64 forward, on tiny scenes with no threshold near a decision (CPU only).

The loss is L = sum over pixels of <g, (colour, depth, alpha, normal)> with
random upstream gradients g, so every output channel and every parameter
(position, opacity, log-scales, beta, quaternion, RGB or SH) is exercised,
including the clamped branch of the Jacobian.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_09156_gb300.scenes import Scene, look_at
from tests._util import oracle_cfg

W, H = 40, 32


def _scene(seed, sh_degree):
    rng = np.random.default_rng(seed)
    n = 9
    mu = rng.uniform(-0.35, 0.35, size=(n, 3))
    mu[:, 1] = np.linspace(-0.5, 0.5, n) + rng.uniform(-0.02, 0.02, n)  # distinct depths along the view axis
    ls = rng.normal(-2.3, 0.35, size=(n, 3))
    q = rng.normal(size=(n, 4))
    op = rng.uniform(0.25, 0.85, size=n)
    beta = rng.uniform(1.2, 5.5, size=n)
    # one large splat beyond the right frustum edge: exercises the clamped Jacobian
    mu[0] = [2.6, 0.0, 0.0]
    ls[0] = [-0.6, -0.8, -0.7]
    op[0] = 0.7
    beta[0] = 2.5
    if sh_degree < 0:
        col = rng.uniform(0.0, 1.0, size=(n, 3))
    else:
        col = rng.normal(0.0, 0.3, size=(n, (sh_degree + 1) ** 2, 3))
        col[:, 0, :] += 1.0
    return Scene(np.concatenate([mu, op[:, None]], 1), np.concatenate([ls, beta[:, None]], 1), q, col, sh_degree)


def _loss(sc, cam, cfg, g):
    out = O.render(sc, cam, cfg)
    return (np.sum(out["color"] * g["c"]) + np.sum(out["depth"] * g["d"]) + np.sum(out["alpha"] * g["a"])
            + np.sum(out["normal"] * g["n"])), out


@pytest.mark.parametrize("seed,sh_degree", [(0, -1), (1, 0), (2, 3), (3, 1)])
def test_analytic_gradient_matches_central_differences(seed, sh_degree):
    cam = look_at((0.0, -3.0, 0.25), (0, 0, 0), W, H).as_dict()
    cfg = oracle_cfg(bg=(0.2, 0.4, 0.1), flag_eps=2e-5)
    sc = _scene(seed, sh_degree)
    rng = np.random.default_rng(100 + seed)
    npx = W * H
    g = dict(c=rng.normal(size=(npx, 3)), d=rng.normal(size=npx), a=rng.normal(size=npx), n=rng.normal(size=(npx, 3)))
    L0, out = _loss(sc, cam, cfg, g)
    assert (out["flags"] & O.DECISION_FLAGS).max() == 0, "scene has a pixel near a decision threshold"
    assert out["n_contrib"].max() >= 3
    # the clamped splat must reach into the image and be clamped
    pre = O.preprocess(sc, cam, cfg)
    vm = np.asarray(cam["viewmat"], np.float64)
    t = vm[:, :3] @ sc.pos_op[0, :3] + vm[:, 3]
    tx_over_tz = t[0] / t[2]
    assert abs(tx_over_tz) > 1.3 * 0.5 * W / cam["fx"] and pre["visible"][0]
    an = O.backward(sc, cam, cfg, g["c"], g["d"], g["a"], g["n"])
    fields = [("pos_op", "g_pos_op"), ("lscale_beta", "g_lscale_beta"), ("quat", "g_quat"), ("color", "g_color")]
    worst = 0.0
    for fname, gname in fields:
        arr = getattr(sc, fname)
        ga = an[gname]
        scale = np.abs(ga).max() + 1e-12
        flat = arr.reshape(-1)
        for j in range(flat.size):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            flat[j] = x0 + h
            lp, op = _loss(sc, cam, cfg, g)
            flat[j] = x0 - h
            lm, om = _loss(sc, cam, cfg, g)
            flat[j] = x0
            assert np.array_equal(op["n_contrib"], out["n_contrib"]) and np.array_equal(om["n_contrib"], out["n_contrib"])
            fd = (lp - lm) / (2 * h)
            err = abs(fd - ga.reshape(-1)[j])
            worst = max(worst, err / scale)
            assert err <= 2e-6 * max(abs(fd), 1e-2 * scale), (fname, j, fd, ga.reshape(-1)[j])
    assert worst < 1e-5


def test_rgb_gradient_is_the_blend_weight():
    """dC/d rgb_i = w_i: a one-hot colour upstream gradient at one pixel returns the weights,
    and they sum to that pixel's alpha."""
    cam = look_at((0.0, -3.0, 0.25), (0, 0, 0), W, H).as_dict()
    cfg = oracle_cfg()
    sc = _scene(5, -1)
    px = [[20, 15]]
    out = O.render(sc, cam, cfg, pixels=px)
    gc = np.array([[1.0, 0.0, 0.0]])
    z = np.zeros(1)
    an = O.backward(sc, cam, cfg, gc, z, z, np.zeros((1, 3)), pixels=px)
    w = an["g_color"][:, 0]
    assert np.all(an["g_color"][:, 1:] == 0)
    assert np.count_nonzero(w) == out["n_contrib"][0]
    np.testing.assert_allclose(w.sum(), out["alpha"][0], rtol=1e-12)


def test_chain_alone_reproduces_backward():
    """The S8 entry applied to backward's own screen-space gradient gives backward's 3-D gradient."""
    cam = look_at((0.0, -3.0, 0.25), (0, 0, 0), W, H).as_dict()
    cfg = oracle_cfg()
    sc = _scene(7, 2)
    rng = np.random.default_rng(9)
    npx = W * H
    an = O.backward(sc, cam, cfg, rng.normal(size=(npx, 3)), rng.normal(size=npx), rng.normal(size=npx),
                    rng.normal(size=(npx, 3)))
    ch = O.chain(sc, cam, cfg, an["g2d"])
    for k in ("g_pos_op", "g_lscale_beta", "g_quat", "g_color"):
        np.testing.assert_allclose(ch[k], an[k], rtol=1e-12, atol=1e-14)
