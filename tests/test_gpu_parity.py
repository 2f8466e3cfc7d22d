"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: keys, order and contributor counts bit-exact; colour, depth,
alpha and normal within 2e-4 absolute; gradients within 1e-3 relative L2 per
tensor, with an elementwise guard of 3e-3 * max(|g|, 0.25 rms(g)) (see
gpu_helpers.compare_grads for its float32 error model). Pixels where FP32 and FP64 may
take a threshold decision differently are flagged by the oracle, excluded from
the image comparison (their count is asserted small) and given zero upstream
gradient on both sides.
"""
import numpy as np
import pytest
import torch

from oracle import binning as OB
from oracle import oracle as O
from paper_2411_09156_gb300 import _lib, api
from paper_2411_09156_gb300.drt import drt_sizes
from paper_2411_09156_gb300.scenes import Scene, look_at, make_scene, workload
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _tiny():
    return workload("tiny-1k-128")


# ----------------------------------------------------------------- S1-S4
def test_preprocess_matches_oracle():
    sc, cams = workload("object-100k-800", n_override=20000)
    cfg = api.GESConfig(sh_degree=3)
    rast, _ = H.gpu_forward(sc, cams, cfg)
    pv = rast.proj_views()
    rec = pv["rec"].double().cpu().numpy()
    binrec = pv["binrec"].cpu().numpy()
    ref = O.preprocess(sc, cams[0].as_dict(), H.oracle_cfg(cfg))
    vis_g = binrec[:, 3].astype(np.uint32) != 0xFFFFFFFF
    vis_o = (ref["visible"] == 1)
    # the GPU lists a splat only if it touches a tile; the oracle's visibility has no tiles
    assert np.all(~vis_g | vis_o)
    v = vis_g
    np.testing.assert_array_equal(binrec[v, 3].astype(np.uint32), ref["z32"][v].view(np.uint32))
    np.testing.assert_allclose(rec[v, 0], ref["uvz"][v, 0], rtol=1e-5, atol=2e-3)
    np.testing.assert_allclose(rec[v, 1], ref["uvz"][v, 1], rtol=1e-5, atol=2e-3)
    con = ref["conic"][v]
    scale = np.abs(con).max(1, keepdims=True)
    assert np.max(np.abs(rec[v][:, [2, 3, 4]] - con) / scale) < 2e-4
    np.testing.assert_allclose(rec[v, 5], ref["qcut"][v], rtol=2e-5)
    np.testing.assert_allclose(rec[v, 8:11], ref["rgb"][v], atol=2e-5)
    np.testing.assert_allclose(rec[v, 11], ref["uvz"][v, 2], rtol=1e-6)
    nrm_ok = v.copy()
    np.testing.assert_allclose(rec[nrm_ok, 12:15], ref["normal"][nrm_ok], atol=2e-5)


@pytest.mark.parametrize("name", ["object-100k-800", "scene-1.5M-1600x1040"])
def test_screen_centres_within_the_oracles_rounding_bound(name):
    """The oracle flags a decision as borderline within the change that the float32 rounding of the
    splat's screen centre can make, using an a-priori bound (du, dv) on that rounding. Every
    listed splat's float32 centre lies within that bound of the FP64 centre."""
    sc, cams = workload(name)
    cfg = api.GESConfig(sh_degree=3)
    rast, _ = H.gpu_forward(sc, cams, cfg)
    pv = rast.proj_views()
    rec = pv["rec"].double().cpu().numpy()
    listed = pv["binrec"][:, 3].cpu().numpy().astype(np.uint32) != 0xFFFFFFFF
    ref = O.preprocess(sc, cams[0].as_dict(), H.oracle_cfg(cfg))
    assert listed.sum() > 0.3 * sc.n
    du, dv = ref["duv"][listed, 0], ref["duv"][listed, 1]
    eu = np.abs(rec[listed, 0] - ref["uvz"][listed, 0])
    ev = np.abs(rec[listed, 1] - ref["uvz"][listed, 1])
    assert (eu <= du).all() and (ev <= dv).all(), (float((eu / du).max()), float((ev / dv).max()))


# ----------------------------------------------------------------- S5: bit-exact keys and order
def _check_binning(sc, cams, tile):
    """Bit-exact tile counts, (tile, entry) instances in order, and tile ranges against the oracle's
    float32 integer stage; returns the per-entry tile-box sizes."""
    cfg = api.GESConfig(tile_w=tile[0], tile_h=tile[1])
    rast, _ = H.gpu_forward(sc, cams, cfg)
    pv = rast.proj_views()
    rec = pv["rec"].cpu().numpy()
    binrec = pv["binrec"].cpu().numpy()
    ext = binrec[:, :2].copy().view(np.float32)
    vis = binrec[:, 3].astype(np.uint32) != 0xFFFFFFFF
    recd = dict(u=rec[:, 0], v=rec[:, 1], a=rec[:, 2], b=rec[:, 3], c=rec[:, 4], qcut=rec[:, 5],
                ext_x=ext[:, 0], ext_y=ext[:, 1])
    z32 = binrec[:, 3].astype(np.uint32).view(np.float32)
    views = [(c.width, c.height) for c in cams]
    keys, ents, touched, ranges = OB.instances(recd, vis, z32, views, tile[0], tile[1], sc.n)
    np.testing.assert_array_equal(binrec[:, 2], touched)
    m = len(keys)
    assert m > 1000 and rast.last_instance_count == m
    bv = rast.bins_views(m)
    np.testing.assert_array_equal(bv["tile"].cpu().numpy(), keys)
    np.testing.assert_array_equal(bv["entry"].cpu().numpy(), ents)
    np.testing.assert_array_equal(bv["ranges"].cpu().numpy(), ranges)
    assert rast.sync_status() == 0
    rdim = binrec[:, 6].astype(np.int64)
    return np.where(vis, (rdim & 0xFFFF) * (rdim >> 16), 0)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8), (8, 32), (16, 8), (8, 16)])
def test_binning_is_bit_exact(tile):
    sc, _ = _tiny()
    cams = [look_at((0.3, -3.6, 0.8), (0, 0, 0), 131, 97), look_at((-1.0, -3.0, 0.5), (0, 0, 0), 64, 80)]
    _check_binning(sc, cams, tile)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_binning_bit_exact_with_boxes_over_32_tiles(tile):
    """One splat in twenty scaled up 7.4x: boxes of hundreds of tiles next to boxes of one, so the
    warps' tile tests and emission run many rounds and the no-mask emission path is exercised."""
    sc = make_scene(1000, 11, "uniform")
    big = np.random.default_rng(12).random(sc.n) < 0.05
    sc.lscale_beta = sc.lscale_beta.copy()
    sc.lscale_beta[big, :3] += 2.0
    cams = [look_at((0.3, -3.6, 0.8), (0, 0, 0), 320, 240), look_at((-1.0, -3.0, 0.5), (0, 0, 0), 160, 120)]
    box = _check_binning(sc, cams, tile)
    assert (box > 32).sum() >= 10 and box.max() > 256


# ----------------------------------------------------------------- S6
@pytest.mark.parametrize("tile,batch", [((16, 16), 256), ((8, 8), 64), ((32, 8), 128), ((8, 32), 96),
                                        ((16, 8), 128), ((8, 16), 64)])
def test_forward_tiny_scene_full_image(tile, batch):
    sc, cams = _tiny()
    cfg = api.GESConfig(tile_w=tile[0], tile_h=tile[1], batch=batch)
    rast, _ = H.gpu_forward(sc, cams, cfg)
    rep, ref, mask = H.compare_forward(rast, sc, cams, cfg)
    assert rep["flagged"] <= 0.01 * rep["pixels"]
    assert ref["n_contrib"].max() > 5


def test_forward_ragged_sizes_sh3_and_background():
    sc = make_scene(3000, 21, "object", 3)
    cfg = api.GESConfig(sh_degree=3, bg=(0.2, 0.5, 0.8))
    for (w, h) in ((131, 97), (17, 250), (1, 1), (300, 3)):
        cams = [look_at((0.4, -2.5, 0.9), (0, 0, 0), w, h)]
        rast, _ = H.gpu_forward(sc, cams, cfg)
        rep, _, _ = H.compare_forward(rast, sc, cams, cfg)
        assert rep["flagged"] <= max(2, 0.01 * rep["pixels"])


def test_zero_splats_and_zero_opacity_give_background():
    cams = [look_at((0, -4, 0), (0, 0, 0), 40, 24)]
    cfg = api.GESConfig(bg=(0.25, 0.5, 0.75))
    for sc in (make_scene(0, 1, "uniform", -1), make_scene(50, 1, "uniform", -1)):
        sc.pos_op[:, 3] = 0.001
        rast, t = H.gpu_forward(sc, cams, cfg)
        img = rast.image("color", 0)
        for c in range(3):
            assert torch.all(img[c] == np.float32(cfg.bg[c]))
        assert int(rast.out["n_contrib"].max()) == 0
        grads = rast.backward(*t, *H.upstream(rast, 0))
        torch.cuda.synchronize()
        for k, g in grads.items():
            assert torch.all(g == 0), k


# ----------------------------------------------------------------- S7 + S8
@pytest.mark.parametrize("sh_degree", [-1, 3])
def test_backward_matches_oracle_gradient(sh_degree):
    if sh_degree < 0:
        sc, cams = _tiny()
    else:
        sc = make_scene(2000, 31, "object", 3)
        cams = [look_at((0.5, -2.2, 0.7), (0, 0, 0), 96, 80)]
    cfg = api.GESConfig(sh_degree=sh_degree, bg=(0.1, 0.2, 0.3))
    rast, t = H.gpu_forward(sc, cams, cfg)
    rep, ref, _ = H.compare_forward(rast, sc, cams, cfg)
    ups = H.mask_upstream(rast, H.upstream(rast, 1000), [H.grad_mask(ref)])
    g2d = torch.empty(sc.n * 16, dtype=torch.float32, device="cuda")
    grads = rast.backward(*t, *ups, g2d=g2d)
    torch.cuda.synchronize()
    got = {k: v.double().cpu().numpy() for k, v in grads.items()}
    oc, od, oa, on = H.oracle_upstream(rast, ups, 0)
    refg = O.backward(sc, cams[0].as_dict(), H.oracle_cfg(cfg), oc, od, oa, on)
    H.compare_grads(got, refg)
    # screen-space accumulators too (u, v, Sigma', opacity, beta, z, rgb, normal), column by column
    g2 = g2d.view(-1, 16).double().cpu().numpy()
    ref2 = H.oracle_g2d_sigma(refg["g2d"], O.preprocess(sc, cams[0].as_dict(), H.oracle_cfg(cfg))["conic"])
    for c in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 13, 14):
        a, b = g2[:, c], ref2[:, c]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-3, c


@pytest.mark.parametrize("with_alpha", [False, True])
def test_backward_colour_only_upstream_matches_oracle(with_alpha):
    """Upstream gradients on the colour (and the alpha) only, as in the training step: the
    backward's replay without the depth and normal channels."""
    sc = make_scene(2000, 32, "object", 3)
    cams = [look_at((0.5, -2.2, 0.7), (0, 0, 0), 96, 80), look_at((-1.9, 1.2, 0.4), (0, 0, 0), 70, 52)]
    cfg = api.GESConfig(sh_degree=3, bg=(0.1, 0.2, 0.3))
    rast, t = H.gpu_forward(sc, cams, cfg)
    keep = []
    for v in range(len(cams)):
        _, ref, _ = H.compare_forward(rast, sc, cams, cfg, v=v)
        keep.append(H.grad_mask(ref))
    gc, gd, ga, gn = H.mask_upstream(rast, H.upstream(rast, 2000), keep)
    ups = (gc, None, ga if with_alpha else None, None)
    grads = rast.backward(*t, *ups)
    torch.cuda.synchronize()
    got = {k: v.double().cpu().numpy() for k, v in grads.items()}
    refg = None
    for v in range(len(cams)):
        oc, _, oa, _ = H.oracle_upstream(rast, (gc, gd, ga, gn), v)
        z1, z3 = np.zeros_like(oa), np.zeros_like(oc)
        r = O.backward(sc, cams[v].as_dict(), H.oracle_cfg(cfg), oc, z1, oa if with_alpha else z1, z3)
        refg = r if refg is None else {k: refg[k] + r[k] for k in refg}
    H.compare_grads(got, refg)


def test_autograd_function_matches_direct_calls():
    from paper_2411_09156_gb300.autograd import rasterize
    sc, cams = _tiny()
    cfg = api.GESConfig()
    t = [x.clone().requires_grad_(True) for x in api.scene_tensors(sc)]
    rast = api.Rasterizer(sc.n, cams, cfg)
    c, d, a, n = rasterize(*t, rast)
    ups = H.upstream(rast, 3)
    loss = (c * ups[0]).sum() + (d * ups[1]).sum() + (a * ups[2]).sum() + (n * ups[3]).sum()
    loss.backward()
    rast2, t2 = H.gpu_forward(sc, cams, cfg)
    direct = rast2.backward(*t2, *ups)
    torch.cuda.synchronize()
    for x, k in zip(t, ("g_pos_op", "g_lscale_beta", "g_quat", "g_color")):
        r = (x.grad - direct[k]).norm() / direct[k].norm()
        assert r < 1e-5, k


# ----------------------------------------------------------------- forms agree bit for bit
def test_tile_shapes_batches_and_persistent_are_bit_identical():
    sc = make_scene(4000, 41, "object", 3)
    cams = [look_at((0.3, -2.4, 0.6), (0, 0, 0), 150, 110)]
    base = None
    for cfg in (api.GESConfig(sh_degree=3), api.GESConfig(sh_degree=3, tile_w=8, tile_h=8, batch=64),
                api.GESConfig(sh_degree=3, tile_w=32, tile_h=8, batch=96),
                api.GESConfig(sh_degree=3, tile_w=8, tile_h=32, batch=64, persistent=1),
                api.GESConfig(sh_degree=3, tile_w=16, tile_h=8, batch=128, persistent=1),
                api.GESConfig(sh_degree=3, tile_w=8, tile_h=16, batch=64),
                api.GESConfig(sh_degree=3, persistent=1), api.GESConfig(sh_degree=3, batch=32, persistent=1)):
        rast, _ = H.gpu_forward(sc, cams, cfg)
        out = {k: rast.out[k].clone() for k in ("color", "depth", "alpha", "normal", "t_final", "n_contrib")}
        if base is None:
            base = out
            continue
        for k in out:
            assert torch.equal(out[k], base[k]), (cfg, k)


def test_colour_only_forward_equals_the_full_forward():
    """Without depth and normal outputs (a render for a loss on the colour) the forward leaves
    their accumulations out; everything it does write is bit-identical to the full render."""
    sc = make_scene(4000, 41, "object", 3)
    cams = [look_at((0.3, -2.4, 0.6), (0, 0, 0), 150, 110), look_at((-1.5, 1.9, 0.8), (0, 0, 0), 97, 131)]
    for persistent in (0, 1):
        cfg = api.GESConfig(sh_degree=3, persistent=persistent)
        rast, _ = H.gpu_forward(sc, cams, cfg)
        full = {k: rast.out[k].clone() for k in ("color", "alpha", "t_final", "last", "n_contrib")}
        depth = rast.out["depth"].clone()
        rast.out["depth"].fill_(-7.0)
        rast.render_fwd(depth_normal=False)
        torch.cuda.synchronize()
        for k, v in full.items():
            assert torch.equal(rast.out[k], v), k
        assert (rast.out["depth"] == -7.0).all()  # not written
        assert not torch.equal(depth, rast.out["depth"])


@pytest.mark.parametrize("n_views,sh_degree", [(4, 2), (5, 3), (20, 3)])
def test_batched_views_equal_per_view_calls(n_views, sh_degree):
    """The batched launch gives each view the image of a one-view call, and the sum of the one-view
    gradients; 5 views leave idle lanes in the backward's 8-lane view segments, 20 views use
    32-lane segments."""
    sc = make_scene(5000, 51, "heightfield", sh_degree)
    sizes = drt_sizes(160, 104, n_views)
    rng = np.random.default_rng(7)
    cams = [look_at(5.0 * d / np.linalg.norm(d), (0, 0, 0), w, h)
            for d, (w, h) in zip(rng.normal(size=(n_views, 3)), sizes)]
    for persistent in (0, 1):
        cfg = api.GESConfig(sh_degree=sh_degree, persistent=persistent)
        rast, t = H.gpu_forward(sc, cams, cfg)
        ups = H.upstream(rast, 5)
        gb = rast.backward(*t, *ups)
        torch.cuda.synchronize()
        gsum = {k: torch.zeros_like(v) for k, v in gb.items()}
        for v, cam in enumerate(cams):
            r1, t1 = H.gpu_forward(sc, [cam], cfg)
            for k in ("color", "depth", "alpha", "normal", "t_final", "n_contrib"):
                assert torch.equal(r1.image(k, 0), rast.image(k, v)), (v, k)
            w, h = sizes[v]
            b = rast.pix_base[v]
            u1 = [ups[0][3 * b:3 * b + 3 * w * h], ups[1][b:b + w * h], ups[2][b:b + w * h],
                  ups[3][3 * b:3 * b + 3 * w * h]]
            g1 = r1.backward(*t1, *[x.contiguous() for x in u1])
            torch.cuda.synchronize()
            for k in gsum:
                gsum[k] += g1[k]
        for k in gsum:
            r = float((gsum[k] - gb[k]).norm() / gb[k].norm())
            assert r < 1e-5, (k, r)


# ----------------------------------------------------------------- device-detected conditions
def test_capacity_overflow_is_reported_and_recoverable():
    sc, cams = _tiny()
    cfg = api.GESConfig()
    t = api.scene_tensors(sc)
    rast = api.Rasterizer(sc.n, cams, cfg, capacity=100)
    rast.forward(*t)
    assert rast.sync_status() == 2  # GES_ERR_CAPACITY
    assert rast.sync_status() == 0  # cleared
    big = api.Rasterizer(sc.n, cams, cfg)
    big.forward(*t)
    assert big.sync_status() == 0


# ----------------------------------------------------------------- full-size workloads, sampled
# Largest share of borderline pixels allowed in a full-size view: pixels where some threshold
# decision (support edge, alpha_min, t_min, normal facing) lies within the change that the float32
# rounding of the splat's screen centre, or the 1e-4 relative band, can make. With the hundreds of
# list entries a pixel walks at 1.5M splats, 3 to 4.5 % of the pixels are flagged.
FLAG_FRAC = 0.06


def _sample_pixels(rng, w, h, k):
    """k distinct seeded pixels (x, y) of a w x h view: a pixel drawn twice would count twice in
    the oracle's gradient but once in the masked upstream gradient of the CUDA path."""
    idx = rng.choice(w * h, size=min(k, w * h), replace=False)
    return np.stack([idx % w, idx // w], 1).astype(np.int32)


def _batch_parity(sc, cams, cfg, rast, t, views, k, seed, full_views=()):
    """Forward parity on k seeded pixels of each listed view (every pixel of full_views), then the
    batched backward with upstream gradients on the unflagged sampled pixels of all those views
    (zero elsewhere) against the sum of the oracle's per-view gradients, the elementwise guard
    allowing for the gradient's sensitivity to the float32 rounding of the screen centres."""
    rng = np.random.default_rng(seed)
    keep = [np.zeros(w * h, bool) for (w, h) in rast.sizes]
    px_by_view = {}
    for v in views:
        w, h = rast.sizes[v]
        if v in full_views:
            ys, xs = np.divmod(np.arange(w * h), w)
            px = np.stack([xs, ys], 1).astype(np.int32)
        else:
            px = _sample_pixels(rng, w, h, k)
        rep, ref, _ = H.compare_forward(rast, sc, cams, cfg, v=v, pixels=px)
        assert rep["flagged"] <= max(3, FLAG_FRAC * len(px)), (v, rep)
        keep[v][(px[:, 1] * w + px[:, 0])[H.grad_mask(ref)]] = True
        px_by_view[v] = px
    ups = H.mask_upstream(rast, H.upstream(rast, seed + 1000), keep)
    grads = rast.backward(*t, *ups)
    torch.cuda.synchronize()
    got = {key: x.double().cpu().numpy() for key, x in grads.items()}
    refg, per_view = None, {}
    for v, px in px_by_view.items():
        up = H.oracle_upstream(rast, ups, v, pixels=px)
        r = O.backward(sc, cams[v].as_dict(), H.oracle_cfg(cfg), *up, pixels=px)
        per_view[v] = (px, up, r)
        refg = r if refg is None else {key: refg[key] + r[key] for key in refg}
    rows = np.nonzero(np.abs(refg["g_pos_op"]).sum(1) + np.abs(got["g_pos_op"]).sum(1) > 0)[0]
    assert len(rows) > 100
    H.compare_grads(got, refg, rows=rows, sens=H.sensitivity(sc, cams, cfg, per_view))


def test_full_size_scene_1p5m_sampled_fwd_bwd():
    """The 1.5M-splat 1600x1040 view: 8,192 seeded pixels, forward and gradient."""
    sc, cams = workload("scene-1.5M-1600x1040")
    cfg = api.GESConfig(sh_degree=3)
    rast, t = H.gpu_forward(sc, cams, cfg)
    _batch_parity(sc, cams, cfg, rast, t, [0], 8192, 0)


def test_object_100k_800_full_frame_fwd_bwd():
    """The 100k-splat 800x800 object view, every pixel: forward and the gradient of all of them."""
    sc, cams = workload("object-100k-800")
    cfg = api.GESConfig(sh_degree=3)
    rast, t = H.gpu_forward(sc, cams, cfg)
    _batch_parity(sc, cams, cfg, rast, t, [0], 0, 5, full_views=(0,))


def test_full_size_drt8_batch_every_view_fwd_bwd():
    """The bench's batch (1.5M splats, 8 views 400x260 .. 1600x1040, one persistent launch): every
    pixel of the smallest view and 4,096 seeded pixels of each other view, forward, and the
    batched gradient from all of them against the oracle's per-view gradients summed."""
    sizes = drt_sizes(1600, 1040, 8)
    sc, cams = workload("drt8-1.5M", sizes=sizes)
    cfg = api.GESConfig(sh_degree=3, persistent=1)
    rast, t = H.gpu_forward(sc, cams, cfg)
    _batch_parity(sc, cams, cfg, rast, t, list(range(8)), 4096, 1, full_views=(0,))


def test_full_size_drt16_3m_batch_sampled_fwd_bwd():
    """3M splats, 16 views (480x270 .. 1920x1080 by the cosine schedule), one batched persistent
    launch: 4,096 seeded pixels of each of the four largest views and 512 of views 0 and 8,
    forward, and the batched gradient from all of them."""
    sizes = drt_sizes(1920, 1080, 16)
    sc, cams = workload("drt16-3M", sizes=sizes)
    cfg = api.GESConfig(sh_degree=3, persistent=1)
    rast, t = H.gpu_forward(sc, cams, cfg)
    rng = np.random.default_rng(2)
    for v in (0, 8):
        w, h = sizes[v]
        rep, _, _ = H.compare_forward(rast, sc, cams, cfg, v=v, pixels=_sample_pixels(rng, w, h, 512))
        assert rep["flagged"] <= FLAG_FRAC * 512, (v, rep)
    _batch_parity(sc, cams, cfg, rast, t, [12, 13, 14, 15], 4096, 2)


def test_non_finite_inputs_are_culled_and_reported():
    """Splats with a NaN centre, an infinite log-scale, a NaN quaternion, a NaN opacity or a
    negative beta (made on the host) are culled and reported as GES_ERR_NUMERIC by the status
    read, which clears it: the images equal those of the same scene with those splats at zero
    opacity bit for bit, and their gradients are zero while the others stay finite."""
    sc = make_scene(3000, 91, "object", 3)
    cams = [look_at((0.3, -2.4, 0.7), (0, 0, 0), 140, 100), look_at((-1.9, 1.2, 0.6), (0, 0, 0), 72, 96)]
    cfg = api.GESConfig(sh_degree=3)
    bad = [5, 17, 33, 41, 50]
    pos, lsb, quat = sc.pos_op.copy(), sc.lscale_beta.copy(), sc.quat.copy()
    pos[5, 0] = np.nan
    lsb[17, 1] = np.inf
    quat[33, 2] = np.nan
    pos[50, 3] = np.nan
    lsb[41, 3] = -1.0
    clean_pos = sc.pos_op.copy()
    clean_pos[bad, 3] = 0.0
    dirty = Scene(pos, lsb, quat, sc.color, sc.sh_degree)
    clean = Scene(clean_pos, sc.lscale_beta, sc.quat, sc.color, sc.sh_degree)
    rd, td = H.gpu_forward(dirty, cams, cfg)
    assert rd.sync_status() == _lib.GES_ERR_NUMERIC
    assert rd.sync_status() == _lib.GES_OK
    rc, tc = H.gpu_forward(clean, cams, cfg)
    assert rc.sync_status() == _lib.GES_OK
    for k in ("color", "depth", "alpha", "normal", "t_final", "n_contrib"):
        assert torch.equal(rd.out[k], rc.out[k]), k
    ups = H.upstream(rd, 9)
    g = rd.backward(*td, *ups)
    torch.cuda.synchronize()
    for k, x in g.items():
        x = x.reshape(sc.n, -1)
        assert torch.isfinite(x[[i for i in range(sc.n) if i not in bad]]).all(), k
        assert (x[bad] == 0).all(), k


def test_step_from_host_buffers_equals_the_device_step():
    """BatchPlan.step_host (parameters copied from pinned host memory in splat ranges, each
    range's preprocess started on arrival, the upstream copy overlapped with the forward, the
    preprocess backward in ranges with their gradient rows copied back as they finish) gives
    the images of the device-resident step bit for bit and its gradients up to the order of
    the float32 atomics, for 1, 3 and 4 ranges."""
    from paper_2411_09156_gb300.batch import BatchPlan
    sc = make_scene(5000, 71, "heightfield", 3)
    sizes = drt_sizes(160, 104, 4)
    rng = np.random.default_rng(72)
    cams = [look_at(5.0 * d / np.linalg.norm(d), (0, 0, 0), w, h) for d, (w, h) in zip(rng.normal(size=(4, 3)), sizes)]
    cfg = api.GESConfig(sh_degree=3, persistent=1)
    t = api.scene_tensors(sc)
    P = sum(w * h for w, h in sizes)
    g = torch.Generator().manual_seed(5)
    ups_h = [torch.randn(3 * P, generator=g), torch.randn(P, generator=g), torch.randn(P, generator=g),
             torch.randn(3 * P, generator=g)]
    ref_plan = BatchPlan(sc.n, cams, cfg, t, [u.cuda() for u in ups_h])
    ref = {k: v.clone() for k, v in ref_plan.step().items()}
    ref_img = ref_plan.rast.out["color"].clone()
    torch.cuda.synchronize()
    dev_in = [torch.zeros_like(x) for x in t]
    plan = BatchPlan(sc.n, cams, cfg, dev_in, [torch.zeros_like(u).cuda() for u in ups_h], capacity=ref_plan.capacity)
    host_in = [x.cpu().pin_memory() for x in t]
    host_up = [u.pin_memory() for u in ups_h]
    host_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in ref.items()}
    for chunks in (1, 3, 4):  # later steps overwrite buffers the earlier ones read
        plan.step_host(host_in, host_up, host_out, chunks=chunks)
        torch.cuda.synchronize()
        assert plan.check() == 0
        assert torch.equal(plan.rast.out["color"], ref_img)
        for k, v in ref.items():
            a, b = host_out[k].double(), v.cpu().double()
            assert float((a - b).norm() / b.norm()) <= 1e-4, k


def test_preprocess_ranges_equal_the_whole_call():
    """S1-S4 over splat ranges (empty ones included) write the records of the single call and the
    same instance total."""
    sc = make_scene(3001, 81, "object", 3)
    cams = [look_at((0.4, -2.3, 0.8), (0, 0, 0), 120, 90), look_at((-1.8, 1.1, 0.6), (0, 0, 0), 64, 80)]
    cfg = api.GESConfig(sh_degree=3)
    t = api.scene_tensors(sc)
    whole = api.Rasterizer(sc.n, cams, cfg)
    whole.preprocess(*t)
    parts = api.Rasterizer(sc.n, cams, cfg)
    for first, count in ((0, 1000), (1000, 0), (1000, 1), (1001, 2000), (3001, 0)):
        parts.preprocess_range(first, count, *t)
    torch.cuda.synchronize()
    assert parts.instance_count() == whole.instance_count()
    a, b = whole.proj_views(), parts.proj_views()
    assert torch.equal(a["rec"], b["rec"]) and torch.equal(a["binrec"], b["binrec"])

