"""Parity of the Eq. 8 loss kernel (ges_loss_rgb through the C ABI) with the FP64 oracle.

Tolerances: per-view loss within 2e-6 absolute (float32 statistics, double sums);
gradient elementwise within 1e-4 of the view's largest oracle gradient plus 1e-3
relative (the SSIM derivatives are ratios with denominators as small as C1 = 1e-4
in dark regions, so float32 rounding of the local statistics moves them by about
1e-6 relative to their largest values)."""
import numpy as np
import pytest
import torch

from oracle import loss as OL
from paper_2411_09156_gb300 import api
from paper_2411_09156_gb300.drt import drt_sizes

pytestmark = pytest.mark.gpu


def _images(sizes, seed, noise=0.1):
    """Smooth seeded textures in [0, 1] and perturbed targets, planar per view, concatenated."""
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for (w, h) in sizes:
        yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
        img = np.zeros((3, h, w))
        for c in range(3):
            for _ in range(3):
                f = rng.uniform(0.02, 0.3, 2)
                img[c] += rng.uniform(0.1, 0.3) * np.sin(f[0] * xx + f[1] * yy + rng.uniform(0, 6.3))
        img = np.clip(0.5 + img + rng.normal(0, 0.05, img.shape), 0, 1)
        tgt = np.clip(img + rng.normal(0, noise, img.shape), 0, 1)
        xs.append(img.astype(np.float32).reshape(-1))
        ys.append(tgt.astype(np.float32).reshape(-1))
    return np.concatenate(xs), np.concatenate(ys)


def _run(sizes, x, y, lam, grad=True):
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    if grad:
        loss, g = api.loss_rgb(xt, yt, sizes, lam)
        torch.cuda.synchronize()
        return loss.cpu().numpy(), g.cpu().numpy()
    cams_c = api.cameras_to_c([dict(width=w, height=h, fx=1.0, fy=1.0, cx=0.0, cy=0.0,
                                    viewmat=[1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0]) for (w, h) in sizes])
    ws = torch.empty(api.ges_loss_workspace_bytes(len(sizes), cams_c), dtype=torch.uint8, device="cuda")
    loss = torch.empty(len(sizes), device="cuda")
    api.ges_loss_rgb(len(sizes), cams_c, xt, yt, lam, ws, loss, None)
    torch.cuda.synchronize()
    return loss.cpu().numpy(), None


def _views(arr, sizes):
    out, o = [], 0
    for (w, h) in sizes:
        out.append(arr[o:o + 3 * w * h].reshape(3, h, w))
        o += 3 * w * h
    return out


def _check_grad(g, ref):
    scale = np.abs(ref).max()
    bad = np.abs(g - ref) > 1e-4 * scale + 1e-3 * np.abs(ref)
    assert bad.sum() == 0, (int(bad.sum()), float(np.abs(g - ref).max()), float(scale))


@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_loss_and_gradient_match_oracle_on_ragged_views(lam):
    sizes = [(37, 29), (64, 32), (100, 71), (1, 1), (5, 3)]
    x, y = _images(sizes, 10)
    loss, g = _run(sizes, x, y, lam)
    for v, (xv, yv, gv) in enumerate(zip(_views(x, sizes), _views(y, sizes), _views(g, sizes))):
        ref = OL.loss(xv, yv, lam=lam)
        assert abs(loss[v] - ref["loss"]) <= 2e-6, (v, loss[v], ref["loss"])
        _check_grad(gv, ref["grad"])


def test_identical_images_have_zero_loss_and_gradient():
    sizes = [(48, 40), (33, 17)]
    x, _ = _images(sizes, 11)
    loss, g = _run(sizes, x, x.copy(), 0.2)
    _, gp = _run(sizes, x, np.clip(x + 0.05, 0, 1).astype(np.float32), 0.2)
    assert np.abs(loss).max() < 1e-6
    assert np.abs(g).max() < 1e-4 * np.abs(gp).max()


def test_loss_only_call_gives_the_same_loss():
    sizes = [(70, 50), (31, 64)]
    x, y = _images(sizes, 12)
    l1, _ = _run(sizes, x, y, 0.2)
    l2, _ = _run(sizes, x, y, 0.2, grad=False)
    np.testing.assert_array_equal(l1, l2)


def test_full_size_drt8_views_loss_and_sampled_gradient():
    """The eight DRT view sizes of the 1.5M benchmark (400x260 .. 1600x1040) in one call: the loss of
    the smallest and largest views against the oracle on the whole frame, and the gradient at 64
    interior pixels of the largest view against the oracle on the 21 x 21 neighbourhood that
    determines it (window radius 5 for the statistics, 5 more for the derivatives' window)."""
    sizes = drt_sizes(1600, 1040, 8)
    x, y = _images(sizes, 13)
    loss, g = _run(sizes, x, y, 0.2)
    xs, ys, gs = _views(x, sizes), _views(y, sizes), _views(g, sizes)
    for v in (0, 7):
        ref = OL.loss(xs[v], ys[v], lam=0.2, with_grad=False)
        assert abs(loss[v] - ref["loss"]) <= 2e-6, (v, loss[v], ref["loss"])
    w, h = sizes[7]
    n = 3 * w * h
    rng = np.random.default_rng(14)
    for _ in range(64):
        qx, qy = int(rng.integers(10, w - 10)), int(rng.integers(10, h - 10))
        cx, cy = xs[7][:, qy - 10:qy + 11, qx - 10:qx + 11], ys[7][:, qy - 10:qy + 11, qx - 10:qx + 11]
        crop = OL.loss(cx, cy, lam=0.2)
        # the crop's own normalisation is 3 * 21 * 21; rescale to the full view's
        ref = crop["grad"][:, 10, 10] * (3 * 21 * 21) / n
        got = gs[7][:, qy, qx]
        scale = 1.0 / n
        assert np.all(np.abs(got - ref) <= 1e-4 * scale * 10 + 1e-3 * np.abs(ref)), (qx, qy, got, ref)


def test_invalid_arguments_are_rejected():
    cams_c = api.cameras_to_c([dict(width=8, height=8, fx=1.0, fy=1.0, cx=0.0, cy=0.0,
                                    viewmat=[1.0, 0, 0, 0, 0, 1.0, 0, 0, 0, 0, 1.0, 0])])
    x = torch.rand(3 * 64, device="cuda")
    ws = torch.empty(api.ges_loss_workspace_bytes(1, cams_c), dtype=torch.uint8, device="cuda")
    loss = torch.empty(1, device="cuda")
    with pytest.raises(api.GESError):
        api.ges_loss_rgb(1, cams_c, x, x, 1.5, ws, loss, None)  # lambda outside [0, 1]
    with pytest.raises(api.GESError):
        api.ges_loss_rgb(1, cams_c, x, x, 0.2, ws[:8], loss, None)  # workspace too small


def test_training_step_with_loss_matches_direct_calls():
    """BatchPlan with target images (graphs: preprocess + bin, render, loss, render backward,
    preprocess backward) gives the loss and gradients of the same calls made one by one."""
    from paper_2411_09156_gb300.batch import BatchPlan
    from paper_2411_09156_gb300.scenes import look_at, make_scene
    sc = make_scene(3000, 21, "heightfield", 1)
    sizes = drt_sizes(160, 104, 3)
    rng = np.random.default_rng(22)
    cams = [look_at(5.0 * d / np.linalg.norm(d), (0, 0, 0), w, h) for d, (w, h) in zip(rng.normal(size=(3, 3)), sizes)]
    cfg = api.GESConfig(sh_degree=1, persistent=1)
    inputs = api.scene_tensors(sc)
    pert = list(inputs)
    pert[3] = inputs[3] + 0.1
    tr = api.Rasterizer(sc.n, cams, cfg)
    target = tr.forward(*pert)["color"].clone()
    plan = BatchPlan(sc.n, cams, cfg, inputs, target=target)
    g_plan = {k: v.clone() for k, v in plan.step().items()}
    torch.cuda.synchronize()
    assert plan.check() == 0
    r = api.Rasterizer(sc.n, cams, cfg)
    out = r.forward(*inputs)
    loss, gc = api.loss_rgb(out["color"], target, sizes, 0.2)
    g_direct = r.backward(*inputs, gc)
    torch.cuda.synchronize()
    assert torch.equal(loss, plan.loss)
    assert torch.equal(gc, plan.g_color_loss)
    for k in g_plan:
        rel = float((g_plan[k] - g_direct[k]).norm() / g_direct[k].norm())
        assert rel < 1e-5, (k, rel)
