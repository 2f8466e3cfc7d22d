"""Parity of the level-set point extraction (ges_levelset) with the FP64 oracle
(oracle/levelset.py), through the C ABI.

Both sides take the same float32 inputs: the splats, the cameras as the C ABI stores them,
and depth / alpha values at the sampled pixels, written by the oracle's renderer
(oracle/oracle.py) or placed at the projection of a splat centre (depth = alpha times the
centre's camera depth, perturbed), plus pixels whose alpha is 0 or below 1e-4.

The kernel's start point x0 carries the rounding of its float32 arithmetic, eps_x (a few
units in the last place of the coordinates and of the camera depth). The oracle therefore
also marches from x0 moved by +-eps_x along each axis; a sample is left out where that, or
the oracle's own flags (near-ties between the 16th and 17th neighbour, or between the two
smallest exponents that choose g, a sampled density within 1e-4 of the level), changes a
decision: the neighbour set, g, whether there is a crossing, or its interval. Elsewhere:
validity equal; t* within the spread of those moved marches plus the float32 rounding of
the two densities that interpolate it (dt (e_k + e_k+1) / |d_k+1 - d_k|, e_k = 4e-6 sum
|o exp(-P/2)| (1 + P (1 + |ln Q|)), as the oracle reports); the point within that plus
3 eps_x; the normal against the oracle's normal at the kernel's point, within its spread
over +-3 eps_x moves plus 1e-5 times the cancellation of its sum. Invalid outputs are all
zeros."""
import numpy as np
import pytest
import torch

from oracle import levelset as OLS
from oracle import oracle as O
from paper_2411_09156_gb300 import api
from paper_2411_09156_gb300.scenes import Scene, look_at, make_scene, random_sphere_cameras, workload
from tests.gpu_helpers import oracle_cfg

pytestmark = pytest.mark.gpu

LEVEL = 0.3


def _cam32(cam) -> dict:
    """A camera with the float32 values the C ABI holds."""
    d = api._cam_dict(cam)
    for k in ("fx", "fy", "cx", "cy"):
        d[k] = float(np.float32(d[k]))
    d["viewmat"] = np.asarray(d["viewmat"], np.float32).astype(np.float64).reshape(-1)
    return d


def _lifted_heightfield(n, seed):
    """The heightfield scene at n splats with the log-scales lifted so that the surface is
    covered as densely as at 1.5M splats (scales times sqrt(1.5M / n))."""
    sc = make_scene(n, seed, "heightfield", -1)
    ls = sc.lscale_beta.copy()
    ls[:, :3] += np.float32(0.5 * np.log(1.5e6 / n))
    return Scene(sc.pos_op, np.ascontiguousarray(ls, np.float32), sc.quat, sc.color, sc.sh_degree)


def _centre_samples(sc, cams, count, rng):
    """(view, x, y, depth, alpha) at the projections of random splat centres."""
    out = []
    for j in rng.choice(sc.pos_op.shape[0], 4 * count, replace=False):
        v = int(rng.integers(len(cams)))
        c = cams[v]
        vm = np.asarray(c["viewmat"], np.float64).reshape(3, 4)
        pc = vm[:, :3] @ sc.pos_op[j, :3].astype(np.float64) + vm[:, 3]
        if pc[2] < 0.3:
            continue
        x, y = int(np.floor(c["fx"] * pc[0] / pc[2] + c["cx"])), int(np.floor(c["fy"] * pc[1] / pc[2] + c["cy"]))
        if not (0 <= x < c["width"] and 0 <= y < c["height"]):
            continue
        a = rng.uniform(0.2, 1.0)
        out.append((v, x, y, a * pc[2] * (1.0 + rng.uniform(-2e-3, 2e-3)), a))
        if len(out) == count:
            break
    return out


def _render_samples(sc, cams, count, rng, cfg):
    """(view, x, y, depth, alpha) from the oracle's renderer at random pixels."""
    out = []
    for v, c in enumerate(cams):
        k = count // len(cams)
        px = np.stack([rng.integers(c["width"], size=k), rng.integers(c["height"], size=k)], 1)
        r = O.render(sc, c, oracle_cfg(cfg), pixels=px)
        out += [(v, int(x), int(y), float(d), float(a)) for (x, y), d, a in zip(px, r["depth"], r["alpha"])]
    return out


def _edge_samples(cams, rng):
    """Pixels with alpha 0 and alpha 5e-5 (no point)."""
    c = cams[0]
    return [(0, int(rng.integers(c["width"])), int(rng.integers(c["height"])), 1.0, a) for a in (0.0, 5e-5, 0.0)]


def _images(cams, samples, base=None):
    """depth / alpha buffers (all views) holding the samples' float32 values; pixels [m, 2].
    Later duplicates of a pixel are dropped."""
    sizes = [c["width"] * c["height"] for c in cams]
    off = np.concatenate([[0], np.cumsum(sizes)])
    if base is None:
        depth, alpha = np.zeros(off[-1], np.float32), np.zeros(off[-1], np.float32)
    else:
        depth, alpha = base
    seen, kept = set(), []
    for (v, x, y, d, a) in samples:
        pix = y * cams[v]["width"] + x
        if (v, pix) in seen:
            continue
        seen.add((v, pix))
        depth[off[v] + pix], alpha[off[v] + pix] = np.float32(d), np.float32(a)
        kept.append((v, x, y, float(np.float32(d)), float(np.float32(a))))
    pixels = np.array([(v, y * cams[v]["width"] + x) for (v, x, y, _, _) in kept], np.int32)
    return depth, alpha, pixels, kept


def _decisions(r):
    return (r["valid"], r["hit"], r["g"], tuple(np.sort(r["neighbours"])))


def _check(sc, cams, kept, got, phi_mode, n_steps, cand_fn=None, min_valid=0.2):
    pos, lsb, q = sc.pos_op, sc.lscale_beta, sc.quat
    kw = dict(n_steps=n_steps, level=LEVEL, rho=0.1, phi_mode=phi_mode)
    n_flag = n_valid = 0
    worst = dict(t=0.0, x=0.0, n=0.0)
    for i, (v, x, y, d, a) in enumerate(kept):
        g = got[i]
        sp = OLS.start_point(cams[v], d, a, x, y)
        if sp is None:
            np.testing.assert_array_equal(g, np.zeros(8, np.float32))
            continue
        x0, ray_v = sp
        c, _, rc = OLS.ray(cams[v], x, y)
        eps_x = 1.2e-6 * (np.abs(c).max() + np.abs(x0).max() + d / a * np.linalg.norm(rc))
        cand = cand_fn(x0) if cand_fn else None
        ref = OLS.march(pos, lsb, q, x0, ray_v, cand=cand, **kw)
        moved = [OLS.march(pos, lsb, q, x0 + s * eps_x * e, ray_v, cand=cand, **kw)
                 for e in np.eye(3) for s in (-1.0, 1.0)]
        if ref["flag"] or any(m["flag"] or _decisions(m) != _decisions(ref) for m in moved):
            n_flag += 1
            continue
        assert bool(g[7]) == ref["valid"], (i, g, ref["valid"])
        if not ref["valid"]:
            np.testing.assert_array_equal(g, np.zeros(8, np.float32))
            continue
        n_valid += 1
        k = ref["hit"]
        dt = ref["ts"][k + 1] - ref["ts"][k]
        e_d = 4e-6 * (ref["dmag"][k] + ref["dmag"][k + 1])
        tol_t = (1.5 * max(abs(m["t"] - ref["t"]) for m in moved) + 2e-5 * ref["sigma"]
                 + dt * e_d / abs(ref["dk"][k + 1] - ref["dk"][k]))
        assert abs(g[6] - ref["t"]) <= tol_t, (i, g[6], ref["t"], tol_t)
        err_x = np.abs(g[:3].astype(np.float64) - ref["point"]).max()
        assert err_x <= tol_t + 3 * eps_x, (i, err_x, tol_t, eps_x)
        xg = g[:3].astype(np.float64)
        nref, cond = OLS.normal_at(pos, lsb, q, ref["neighbours"], xg, 0.1, phi_mode)
        spread = max(np.abs(OLS.normal_at(pos, lsb, q, ref["neighbours"], xg + s * 3 * eps_x * e, 0.1, phi_mode)[0]
                            - nref).max() for e in np.eye(3) for s in (-1.0, 1.0))
        err_n = np.abs(g[3:6].astype(np.float64) - nref).max()
        assert err_n <= 1.5 * spread + 1e-5 * cond + 1e-6, (i, err_n, spread, cond)
        worst["t"] = max(worst["t"], abs(g[6] - ref["t"]) / tol_t)
        worst["x"] = max(worst["x"], err_x)
        worst["n"] = max(worst["n"], err_n)
    m = len(kept)
    assert n_flag <= 0.2 * m, (n_flag, m)
    assert n_valid >= min_valid * (m - n_flag), (n_valid, m, n_flag)
    return dict(flagged=n_flag, valid=n_valid, **worst)


def _run(sc, cams, depth, alpha, pixels, n_steps, phi_mode):
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (sc.pos_op, sc.lscale_beta, sc.quat)]
    out = api.levelset(*t, cams, torch.from_numpy(depth).cuda(), torch.from_numpy(alpha).cuda(),
                       torch.from_numpy(pixels).cuda(), n_steps=n_steps, level=LEVEL,
                       cfg=api.GESConfig(phi_mode=phi_mode))
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("phi_mode,n_steps", [(1, 32), (0, 7), (1, 200)])
def test_levelset_matches_oracle(phi_mode, n_steps):
    sc = _lifted_heightfield(30000, 7)
    cams = [_cam32(look_at((0.0, -2.5, 2.5), (0, 0, 0), 192, 144)),
            _cam32(random_sphere_cameras(np.random.default_rng(11), 1, 3.5, [(160, 120)])[0])]
    rng = np.random.default_rng(100 + n_steps)
    cfg = api.GESConfig(phi_mode=phi_mode)
    samples = _centre_samples(sc, cams, 150, rng) + _render_samples(sc, cams, 120, rng, cfg) + _edge_samples(cams, rng)
    depth, alpha, pixels, kept = _images(cams, samples)
    got = _run(sc, cams, depth, alpha, pixels, n_steps, phi_mode)
    rep = _check(sc, cams, kept, got, phi_mode, n_steps)
    print(rep)


def test_levelset_single_pixel_and_no_points():
    sc = _lifted_heightfield(2000, 8)
    cams = [_cam32(look_at((0.0, -2.5, 2.5), (0, 0, 0), 64, 48))]
    rng = np.random.default_rng(3)
    samples = _centre_samples(sc, cams, 1, rng)
    depth, alpha, pixels, kept = _images(cams, samples)
    got = _run(sc, cams, depth, alpha, pixels, 32, 1)
    _check(sc, cams, kept, got, 1, 32, min_valid=0.0)
    # every pixel of an empty image: no points, all zeros
    depth, alpha = np.zeros(64 * 48, np.float32), np.zeros(64 * 48, np.float32)
    pixels = np.stack([np.zeros(64 * 48, np.int32), np.arange(64 * 48, dtype=np.int32)], 1)
    got = _run(sc, cams, depth, alpha, np.ascontiguousarray(pixels), 32, 1)
    assert not got.any()
    # pixels naming a view that does not exist or an index outside the view give no point,
    # whatever the depth and alpha buffers hold
    depth, alpha = np.full(64 * 48, 4.0, np.float32), np.ones(64 * 48, np.float32)
    bad = np.array([[-1, 10], [1, 10], [5, 0], [0, -3], [0, 64 * 48], [0, 1 << 30]], np.int32)
    got = _run(sc, cams, depth, alpha, bad, 32, 1)
    assert not got.any()


def test_levelset_invalid_arguments():
    sc = _lifted_heightfield(2000, 8)
    cams = [_cam32(look_at((0.0, -2.5, 2.5), (0, 0, 0), 64, 48))]
    t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (sc.pos_op, sc.lscale_beta, sc.quat)]
    img = torch.zeros(64 * 48, device="cuda")
    px = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    for kw in (dict(n_steps=1), dict(n_steps=1025), dict(level=0.0)):
        with pytest.raises(api.GESError):
            api.levelset(*t, cams, img, img, px, **kw)
    with pytest.raises(ValueError):
        api.ges_levelset_workspace_bytes(15, 4)


def test_levelset_full_size_sampled():
    """The 1.5M-splat heightfield scene and its eight batched views at their full sizes, every
    pixel of all views extracted in one launch (depth and alpha from the CUDA renderer), with
    the oracle's rendered depth and alpha planted at 48 sampled pixels and those compared. (The
synthetic heightfield scatters its flat splats by 0.02 across the surface, far more than
their thickness, so most rays find no crossing among the 16 centres nearest x0.)"""
    from paper_2411_09156_gb300.drt import drt_sizes
    sc, cams0 = workload("drt8-1.5M", sizes=drt_sizes(1600, 1040, 8))
    cams = [_cam32(c) for c in cams0]
    cfg = api.GESConfig(sh_degree=sc.sh_degree)
    rast = api.Rasterizer(sc.n, cams, cfg)
    rast.forward(*api.scene_tensors(sc))
    torch.cuda.synchronize()
    base = (rast.out["depth"].cpu().numpy().copy(), rast.out["alpha"].cpu().numpy().copy())
    rng = np.random.default_rng(21)
    samples = []
    for v in rng.choice(len(cams), 4, replace=False):
        c = cams[v]
        px = np.stack([rng.integers(c["width"] // 4, 3 * c["width"] // 4, size=12),
                       rng.integers(c["height"] // 4, 3 * c["height"] // 4, size=12)], 1)
        r = O.render(sc, c, oracle_cfg(cfg), pixels=px)
        samples += [(int(v), int(x), int(y), float(d), float(a)) for (x, y), d, a in zip(px, r["depth"], r["alpha"])]
    depth, alpha, sampled, kept = _images(cams, samples, base)
    P = depth.shape[0]
    all_px = np.concatenate([np.stack([np.full(c["width"] * c["height"], v, np.int32),
                                       np.arange(c["width"] * c["height"], dtype=np.int32)], 1)
                             for v, c in enumerate(cams)])
    assert all_px.shape[0] == P
    got = _run(sc, cams, depth, alpha, np.ascontiguousarray(all_px), 32, 1)
    off = np.concatenate([[0], np.cumsum([c["width"] * c["height"] for c in cams])])
    rows = np.array([off[v] + pix for v, pix in sampled])
    pos64 = sc.pos_op[:, :3].astype(np.float64)

    def cand(x0):  # a superset of the 17 nearest centres of any x0 moved by rounding
        d2 = ((pos64 - x0) ** 2).sum(1)
        return np.argpartition(d2, 64)[:64]

    rep = _check(sc, cams, kept, got[rows], 1, 32, cand_fn=cand, min_valid=0.05)
    # every output row is either all zeros or a unit normal with valid = 1
    v = got[:, 7]
    assert set(np.unique(v)) <= {0.0, 1.0}
    assert not got[v == 0].any()
    nn = np.linalg.norm(got[v == 1][:, 3:6], axis=1)
    assert np.abs(nn - 1).max() < 1e-5
    print(rep, int(v.sum()), P)
