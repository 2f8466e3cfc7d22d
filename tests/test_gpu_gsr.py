"""Parity of the KNN build (ges_knn) and of the GSR point evaluation (ges_gsr) with the FP64
oracle (oracle/gsr.py), through the C ABI.

KNN: where several lists are correct (centres at nearly equal distances) the test checks
validity instead of identity: every listed neighbour is at most the oracle's 16th distance
away (plus float32 rounding), the list is ordered and duplicate-free and starts with the
splat itself; the index sets are equal wherever the oracle's 16th and 17th distances are
apart by more than the rounding.

GSR: samples whose g* is decided by a near tie, that lie within rounding of g*'s plane, at
the kink of |fbar - f|, at d = 1, or so far in the tails that a contributing term's exponent
(beta/2) Q^(beta/2) exceeds 60, or with d at its lower clamp (flagged by the oracle: float32
cannot resolve them) are left
out of both sides. Per-sample values within 1e-4 relative (d, f, fbar), f and fbar also
within the float32 error of ln d near d = 1 and of e near g*'s plane (_check_f, _check_fbar),
and u.n* within the rounding of the direction sum (_check_cos); losses within 1e-4 relative;
gradients within 2e-3 relative L2 per tensor with an elementwise guard of
1e-2 max(|g|, 0.25 rms), float32 against float64 through Q^(beta/2 - 1) and 1/|grad d| terms."""
import numpy as np
import pytest
import torch

from oracle import gsr as OG
from paper_2411_09156_gb300 import api
from paper_2411_09156_gb300.scenes import make_scene, workload

pytestmark = pytest.mark.gpu


def _check_knn(pos, got, rows=None, ref=None):
    """got: (n, 16) GPU lists. rows: which splats to check (all if None); ref: the oracle's lists for them."""
    rows = np.arange(pos.shape[0]) if rows is None else np.asarray(rows)
    p = pos[:, :3].astype(np.float64)
    g = got[rows]
    assert (g >= 0).all() and (g < pos.shape[0]).all()
    assert all(len(set(r)) == 16 for r in g)
    dg = np.sqrt(((p[rows][:, None, :] - p[g]) ** 2).sum(-1))
    if ref is None:
        ref = np.stack([np.argsort(((p - p[i]) ** 2).sum(-1), kind="stable")[:17] for i in rows])
    dr = np.sqrt(((p[rows][:, None, :] - p[ref]) ** 2).sum(-1))
    tol = 1e-6 * np.maximum(dr[:, 15:16], 1e-6) + 1e-9
    assert (np.diff(dg, axis=1) >= -tol).all(), "lists not ordered"
    assert (dg[:, 15] <= dr[:, 15] + tol[:, 0]).all(), "a listed neighbour is farther than the 16th nearest"
    assert (g[:, 0] == rows).mean() > 0.999
    if ref.shape[1] > 16:
        sep = dr[:, 16] - dr[:, 15] > 10 * tol[:, 0]
        same = np.array([set(a) == set(b[:16]) for a, b in zip(g, ref)])
        assert same[sep].all()


def _pos(n, seed, kind):
    sc = make_scene(n, seed, kind)
    return np.ascontiguousarray(sc.pos_op, np.float32)


@pytest.mark.parametrize("kind,n", [("uniform", 20000), ("heightfield", 50000), ("object", 30000)])
def test_knn_matches_brute_force(kind, n):
    pos = _pos(n, 3, kind)
    got = api.knn(torch.from_numpy(pos).cuda()).cpu().numpy()
    rows = np.random.default_rng(0).choice(n, 2000, replace=False)
    _check_knn(pos, got, rows)


def test_knn_degenerate_layouts():
    rng = np.random.default_rng(5)
    line = np.zeros((3000, 4), np.float32)
    line[:, 0] = rng.uniform(-1, 1, 3000)  # all on the x axis: zero extent in y and z
    plane = np.zeros((3000, 4), np.float32)
    plane[:, :2] = rng.uniform(-1, 1, (3000, 2))
    dup = np.repeat(rng.uniform(-1, 1, (300, 4)).astype(np.float32), 10, axis=0)  # each centre 10 times
    for pos in (line, plane, dup):
        got = api.knn(torch.from_numpy(np.ascontiguousarray(pos)).cuda()).cpu().numpy()
        p = pos[:, :3].astype(np.float64)
        rows = np.arange(0, pos.shape[0], 7)
        dg = np.sqrt(((p[rows][:, None, :] - p[got[rows]]) ** 2).sum(-1))
        d16 = np.stack([np.sort(np.sqrt(((p - p[i]) ** 2).sum(-1)))[15] for i in rows])
        assert (dg[:, 15] <= d16 * (1 + 1e-6) + 1e-9).all()
        assert all(len(set(r)) == 16 for r in got[rows])


def test_knn_full_size_sampled():
    """The 1.5M-splat heightfield scene of the benchmark; 256 sampled splats against brute force."""
    sc, _ = workload("scene-1.5M-1600x1040")
    pos = np.ascontiguousarray(sc.pos_op, np.float32)
    got = api.knn(torch.from_numpy(pos).cuda()).cpu().numpy()
    rows = np.random.default_rng(1).choice(pos.shape[0], 256, replace=False)
    pt = torch.from_numpy(pos[:, :3].astype(np.float64))
    ref = []
    for i in rows:
        d2 = ((pt - pt[i]) ** 2).sum(-1)
        ref.append(torch.sort(d2, stable=True).indices[:17].numpy())
    _check_knn(pos, got, rows, np.stack(ref))


def _gsr_case(n, m, seed, phi_mode=1):
    """A dense slab of flat splats (spacing ~0.01 below the in-plane scales ~0.03), so that the 16
    neighbours of a sample overlap it and g* is not always the sample's own splat."""
    rng = np.random.default_rng(seed)
    pos = np.concatenate([rng.uniform(-0.3, 0.3, (n, 2)), rng.normal(0, 0.01, (n, 1)),
                          1 / (1 + np.exp(-rng.normal(0, 1, (n, 1))))], 1).astype(np.float32)
    ls = np.stack([rng.normal(-3.5, 0.3, n), rng.normal(-3.5, 0.3, n), rng.normal(-6.0, 0.3, n)], 1)
    lsb = np.concatenate([ls, rng.uniform(1.0, 6.0, (n, 1))], 1).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    q[:, 0] += 3.0  # mostly near the identity: the flat axes near z
    if phi_mode == 2:
        # Eq. 7 as printed shrinks the scales by phi(beta) = 2 / (1 + e^(1.9 beta)) (down to 2e-5);
        # lift the log-scales by -ln phi so the splats keep the sizes above and only the phi
        # chain differs (collapsed splats are below float32's resolution at these coordinates)
        b = lsb[:, 3].astype(np.float64)
        lsb[:, :3] -= np.log(2.0 / (1.0 + np.exp(-(0.1 * b - 2.0 * b))))[:, None].astype(np.float32)
    knn = OG.knn(pos).astype(np.int32)
    rng = np.random.default_rng(seed + 1)
    js = rng.integers(0, n, m).astype(np.int32)
    z = rng.normal(size=(m, 3)).astype(np.float32)
    return pos, lsb, q, knn, js, z


def _run_gsr(pos, lsb, q, knn, js, z, phi_mode, lam=(1.0, 0.5)):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    cfg = api.GESConfig(phi_mode=phi_mode)
    out = api.gsr(t(pos), t(lsb), t(q), t(knn), t(js), t(z), cfg, lam[0], lam[1], grads=True, per_sample=True)
    torch.cuda.synchronize()
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def _check_f(f, ref):
    """f = s_min sqrt(pl), pl = -2 ln d: a float32 sum of 16 terms, each an exponential with its
    own rounding, carries a relative error of up to about 4e-6 in d, which moves f by
    4e-6 f / pl (large where d nears 1, the SDF's zero)."""
    fr = ref["f"]
    pl = -2.0 * np.log(np.clip(ref["d"], 1e-30, 1.0))
    tol = 1e-4 * np.abs(fr) + 4e-6 * np.abs(fr) / np.maximum(pl, 1e-30) + 1e-9
    assert (np.abs(f - fr) <= tol).all(), float(np.max(np.abs(f - fr) / tol))


def _check_fbar(fb, ref):
    """fbar = s_min (e / s_min)^(beta*/2) with e = <x - mu*, n*>: x and mu* are float32 coordinates
    (rounding 6e-8 of their magnitude, here below 2), so e carries an absolute error of about
    2e-7, which moves fbar by (beta*/2) fbar 2e-7 / e (large for samples near g*'s plane)."""
    fr, e = ref["fbar"], np.maximum(ref["e"], 1e-30)
    tol = 1e-4 * np.abs(fr) + 0.5 * ref["beta_star"] * np.abs(fr) * 2e-7 / e + 1e-9
    assert (np.abs(fb - fr) <= tol).all(), float(np.max(np.abs(fb - fr) / tol))


def _check_cos(c, ref, dist):
    """u . n*, u the direction of a sum of up to 16 terms. A term's weight exp(-P/2) (beta/2) P / Q
    carries the rounding of its exponent P = Q^(beta/2): Q is good to about 2e-6 relative, so P to
    2e-6 (beta/2) P and the weight to half that absolute, plus a few 1e-6 of other rounding. The
    direction then moves by that relative error times wcond (the terms' total length over the
    sum's length, large where neighbours pull in opposite directions). Close to g*'s plane the
    normal component of a term is the projection e of an offset of length dist = |x - mu*|, a dot
    product rounded to about 1e-7 dist, a relative error of 1e-7 dist / e."""
    tol = 2e-5 + ref["wcond"] * (1e-5 + 2e-6 * ref["pscale"]) + 1e-7 * dist / np.maximum(ref["e"], 1e-30)
    assert (np.abs(c - ref["cos"]) <= tol).all(), float(np.max(np.abs(c - ref["cos"]) / tol))


def _dist_gstar(pos, knn, js, ref):
    """|x - mu*| per sample, g* the oracle's."""
    gs = knn[js, ref["gstar"]]
    return np.linalg.norm(ref["x"] - pos[gs, :3].astype(np.float64), axis=1)


def _compare_grads(got, ref):
    for k in ("g_pos_op", "g_lscale_beta", "g_quat"):
        a, b = got[k].astype(np.float64), ref[k]
        rms = np.sqrt((b ** 2).mean())
        r = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert r <= 2e-3, (k, r)
        bad = np.abs(a - b) > 1e-2 * np.maximum(np.abs(b), 0.25 * rms)
        assert bad.sum() == 0, (k, int(bad.sum()), float(np.abs(a - b).max()), float(rms))


@pytest.mark.parametrize("phi_mode", [1, 0, 2])
def test_gsr_matches_oracle(phi_mode):
    pos, lsb, q, knn, js, z = _gsr_case(3000, 1500, 7, phi_mode)
    ref = OG.evaluate(pos, lsb, q, knn, js, z, phi_mode=phi_mode, lambda_sdf=1.0, lambda_nor=0.5, with_grad=False)
    assert (ref["gstar"] > 0).mean() > 0.05
    keep = ~ref["flags"]
    assert keep.mean() > 0.9
    js, z = js[keep], z[keep]
    ref = OG.evaluate(pos, lsb, q, knn, js, z, phi_mode=phi_mode, lambda_sdf=1.0, lambda_nor=0.5)
    got = _run_gsr(pos, lsb, q, knn, js, z, phi_mode)
    so = got["sample_out"]
    np.testing.assert_allclose(so[:, :3], ref["x"], rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(so[:, 7].astype(np.int64), ref["gstar"])
    np.testing.assert_allclose(so[:, 3], ref["d"], rtol=1e-4, atol=1e-7 * np.abs(ref["d"]).max())
    _check_f(so[:, 4], ref)
    _check_fbar(so[:, 5], ref)
    _check_cos(so[:, 6], ref, _dist_gstar(pos, knn, js, ref))
    np.testing.assert_allclose(got["losses"][:2], [ref["l_sdf"], ref["l_nor"]], rtol=1e-4)
    assert abs(got["losses"][2] - ref["loss"]) <= 1e-4 * abs(ref["loss"])
    _compare_grads(got, ref["grads"])


def test_gsr_forward_only_and_out_of_range_indices():
    pos, lsb, q, knn, js, z = _gsr_case(500, 200, 9)
    full = _run_gsr(pos, lsb, q, knn, js, z, 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    fwd = api.gsr(t(pos), t(lsb), t(q), t(knn), t(js), t(z), api.GESConfig(), 1.0, 0.5, grads=False)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(fwd["losses"].cpu().numpy(), full["losses"])
    # a sample whose splat index is out of range contributes nothing (but still counts in m)
    js2 = js.copy()
    js2[0] = 10 ** 6
    out = api.gsr(t(pos), t(lsb), t(q), t(knn), t(js2), t(z), api.GESConfig(), 1.0, 0.5, grads=False,
                  per_sample=True)
    torch.cuda.synchronize()
    assert np.isfinite(out["losses"].cpu().numpy()).all()


def test_gsr_full_size_scene_subset():
    """The benchmark's 1.5M-splat scene with its GPU-built KNN lists; 1000 samples against the oracle."""
    sc, _ = workload("scene-1.5M-1600x1040")
    pos = np.ascontiguousarray(sc.pos_op, np.float32)
    lsb = np.ascontiguousarray(sc.lscale_beta, np.float32)
    q = np.ascontiguousarray(sc.quat, np.float32)
    knn = api.knn(torch.from_numpy(pos).cuda()).cpu().numpy()
    rng = np.random.default_rng(11)
    js = rng.integers(0, pos.shape[0], 1000).astype(np.int32)
    z = rng.normal(size=(1000, 3)).astype(np.float32)
    ref = OG.evaluate(pos, lsb, q, knn, js, z, lambda_sdf=1.0, lambda_nor=0.5, with_grad=False)
    keep = ~ref["flags"]
    js, z = js[keep], z[keep]
    ref = OG.evaluate(pos, lsb, q, knn, js, z, lambda_sdf=1.0, lambda_nor=0.5)
    got = _run_gsr(pos, lsb, q, knn, js, z, 1)
    so = got["sample_out"]
    np.testing.assert_array_equal(so[:, 7].astype(np.int64), ref["gstar"])
    np.testing.assert_allclose(so[:, 3], ref["d"], rtol=1e-4, atol=1e-7)
    _check_cos(so[:, 6], ref, _dist_gstar(pos, knn, js, ref))
    np.testing.assert_allclose(got["losses"][:2], [ref["l_sdf"], ref["l_nor"]], rtol=1e-4)
    _compare_grads(got, ref["grads"])
