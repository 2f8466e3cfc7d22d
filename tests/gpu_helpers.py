"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI,
run the oracle on the same seeded inputs, and compare."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2411_09156_gb300 import api

# tolerances stated by the method's parity contract
IMG_ATOL = 2e-4
GRAD_REL_L2 = 1e-3


def oracle_cfg(cfg: api.GESConfig, flag_eps=1e-4, cell=16) -> dict:
    """The oracle's config for a GESConfig; cell: the oracle's pixel-cell index (bit-identical to
    its brute-force loop, pinned in tests/test_oracle_pins.py), 0 for the brute-force loop."""
    return dict(phi_mode=cfg.phi_mode, rho=cfg.rho, lowpass=cfg.lowpass, alpha_min=cfg.alpha_min,
                alpha_max=cfg.alpha_max, t_min=cfg.t_min, jac_clamp=cfg.jac_clamp, bg=tuple(cfg.bg),
                flag_eps=flag_eps, cell=cell)


def gpu_forward(scene, cams, cfg: api.GESConfig, **kw):
    t = api.scene_tensors(scene)
    rast = api.Rasterizer(scene.n, cams, cfg, **kw)
    rast.forward(*t)
    torch.cuda.synchronize()
    return rast, t


def view_outputs(rast, v):
    """One view's outputs in the oracle's per-pixel layout (row-major pixels, channels last)."""
    w, h = rast.sizes[v]
    o = {}
    o["color"] = rast.image("color", v).permute(1, 2, 0).reshape(-1, 3).double().cpu().numpy()
    o["normal"] = rast.image("normal", v).permute(1, 2, 0).reshape(-1, 3).double().cpu().numpy()
    for k in ("depth", "alpha", "t_final"):
        o[k] = rast.image(k, v).reshape(-1).double().cpu().numpy()
    for k in ("last", "n_contrib"):
        o[k] = rast.image(k, v).reshape(-1).cpu().numpy().astype(np.int64)
    return o


def compare_forward(rast, scene, cams, cfg, v=0, pixels=None, atol=IMG_ATOL):
    """Forward parity of one view against the oracle. Returns (report dict, oracle output, mask)."""
    cam = cams[v].as_dict() if hasattr(cams[v], "as_dict") else cams[v]
    ref = O.render(scene, cam, oracle_cfg(cfg), pixels=pixels)
    got = view_outputs(rast, v)
    w = cam["width"]
    if pixels is not None:
        idx = np.asarray(pixels)[:, 1] * w + np.asarray(pixels)[:, 0]
        got = {k: a[idx] for k, a in got.items()}
    # image values are compared wherever no threshold decision is borderline; gradients
    # (see grad_mask) also skip the centre-cusp pixels of beta < 2 splats
    mask = (ref["flags"] & O.DECISION_FLAGS) == 0
    rep = {"flagged": int((~mask).sum()), "pixels": int(mask.size), "cusp": int(((ref["flags"] & O.FLAG_CUSP) != 0).sum())}
    for k in ("color", "depth", "alpha", "normal"):
        err = np.abs(got[k][mask] - ref[k][mask])
        rep[k] = float(err.max()) if err.size else 0.0
        if err.size and rep[k] > atol:  # the worst pixel, for the report
            j = np.nonzero(mask)[0][np.argmax(err.reshape(err.shape[0], -1).max(1))]
            rep["worst"] = dict(index=int(j), got=np.asarray(got[k][j]).tolist(), ref=np.asarray(ref[k][j]).tolist(),
                                n_contrib=int(ref["n_contrib"][j]), T=float(ref["T"][j]), flags=int(ref["flags"][j]))
        assert rep[k] <= atol, (k, rep[k], rep.get("worst"))
    np.testing.assert_array_equal(got["n_contrib"][mask], ref["n_contrib"][mask])
    # last contributor: splat id of the instance before `last`
    n_inst = rast.capacity
    ent = rast.bins_views(n_inst)["entry"].cpu().numpy().astype(np.int64)
    has = got["n_contrib"] > 0
    ids = np.full(got["last"].shape, -1, np.int64)
    ids[has] = ent[got["last"][has] - 1] % scene.n
    np.testing.assert_array_equal(ids[mask], ref["last_id"][mask])
    return rep, ref, mask


def grad_mask(ref):
    """Pixels whose upstream gradient is kept on both sides: no borderline decision, no cusp."""
    return ref["flags"] == 0


def upstream(rast, seed):
    """Random N(0,1) upstream gradients in the rasterizer's output layouts (device tensors)."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    P = rast.P
    gc = torch.randn(3 * P, generator=g)
    gd = torch.randn(P, generator=g)
    ga = torch.randn(P, generator=g)
    gn = torch.randn(3 * P, generator=g)
    return [x.cuda() for x in (gc, gd, ga, gn)]


def mask_upstream(rast, grads, keep_by_view):
    """Zero the upstream gradients outside keep_by_view[v] (bool per pixel of view v)."""
    gc, gd, ga, gn = [x.clone() for x in grads]
    for v, keep in enumerate(keep_by_view):
        w, h = rast.sizes[v]
        k = torch.as_tensor(keep, device="cuda").reshape(-1)
        b = rast.pix_base[v]
        gd[b:b + w * h] *= k
        ga[b:b + w * h] *= k
        for c in range(3):
            gc[3 * b + c * w * h:3 * b + (c + 1) * w * h] *= k
            gn[3 * b + c * w * h:3 * b + (c + 1) * w * h] *= k
    return gc, gd, ga, gn


def oracle_upstream(rast, grads, v, pixels=None):
    """One view's upstream gradients in the oracle layout ((P,3), (P,), (P,), (P,3))."""
    w, h = rast.sizes[v]
    b = rast.pix_base[v]
    gc, gd, ga, gn = [x.double().cpu().numpy() for x in grads]
    c = gc[3 * b:3 * b + 3 * w * h].reshape(3, -1).T
    n = gn[3 * b:3 * b + 3 * w * h].reshape(3, -1).T
    d = gd[b:b + w * h]
    a = ga[b:b + w * h]
    if pixels is not None:
        idx = np.asarray(pixels)[:, 1] * w + np.asarray(pixels)[:, 0]
        return c[idx], d[idx], a[idx], n[idx]
    return c, d, a, n


# Per-tensor gradient errors of every compare_grads call in this run, printed by
# tests/conftest.py at the end of the session: the tensor-level relative L2, and the largest
# elementwise error in the form |d| / max(|g|, 1e-2 rms(g)) (bound 1e-3 in the method's
# parity contract) with the number of elements above 1e-3 in that form.
GRAD_REPORT = []


def compare_grads(got: dict, ref: dict, rel_l2=GRAD_REL_L2, elem=3e-3, floor=0.25, rows=None, sens=None):
    """Tensor-level relative L2 <= 1e-3 (the gradient tolerance) and, as a guard against a wrong
    formula for a single parameter, elementwise |d| <= elem * max(|g|, floor * rms(g)).

    The elementwise bound allows for the float32 error model of the front-to-back
    replay: the colour/depth/normal behind a splat is the final value minus the
    prefix sum, so a splat deep in a pixel's list (T_i ~ 1e-4) carries an absolute
    error of a few ulp of the final value, i.e. a relative error up to ~1e-3 of its
    own small gradient. Each call also records the error in the tighter form
    |d| / max(|g|, 1e-2 rms(g)) in GRAD_REPORT.

    sens (optional, per tensor, the shape of the gradient): how far the oracle's gradient moves when
    its sample points move by the float32 rounding of the splats' screen centres (see
    sensitivity()); the elementwise bounds then allow 2 sens more. A position gradient is a sum
    over pixels whose terms largely cancel, so that rounding, tiny per pixel, can move it by
    more than 3e-3 of itself."""
    import os
    rep = {}
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    for k in ("g_pos_op", "g_lscale_beta", "g_quat", "g_color"):
        a = np.asarray(got[k], np.float64).reshape(len(got[k]), -1)
        b = np.asarray(ref[k], np.float64).reshape(len(ref[k]), -1)
        if rows is not None:
            a, b = a[rows], b[rows]
        den = np.linalg.norm(b)
        r = float(np.linalg.norm(a - b) / max(den, 1e-30))
        rms = float(np.sqrt(np.mean(b * b))) if b.size else 0.0
        d = np.abs(a - b)
        sv = 0.0
        if sens is not None:
            sv = np.asarray(sens[k], np.float64).reshape(len(sens[k]), -1)
            sv = sv[rows] if rows is not None else sv
        bad = d > elem * np.maximum(np.abs(b), floor * rms) + 2.0 * sv
        tight = d / np.maximum(np.maximum(np.abs(b), 1e-2 * rms), 1e-30)
        tight_s = d / np.maximum(1e-3 * np.maximum(np.abs(b), 1e-2 * rms) + 2.0 * sv, 1e-30)
        rep[k] = dict(rel_l2=r, max_abs=float(d.max()) if a.size else 0.0, n_bad=int(bad.sum()),
                      tight_max=float(tight.max()) if a.size else 0.0, tight_over=int((tight > 1e-3).sum()),
                      tight_sens_max=float(tight_s.max()) if a.size else 0.0, sens=sens is not None,
                      guard_max=float((d / np.maximum(np.maximum(np.abs(b), floor * rms), 1e-30)).max())
                      if a.size else 0.0, n=int(a.size))
        if a.size:
            w = np.unravel_index(np.argmax(d / np.maximum(np.maximum(np.abs(b), floor * rms), 1e-30)), d.shape)
            rep[k]["worst"] = dict(row=int(w[0]) if rows is None else int(np.asarray(rows)[w[0]]), col=int(w[1]),
                                   got=float(a[w]), ref=float(b[w]), rms=rms)
        GRAD_REPORT.append(dict(test=test, tensor=k, **rep[k]))
        assert r <= rel_l2, (k, rep[k])
        assert bad.sum() == 0, (k, rep[k])
    return rep


def sensitivity(sc, cams, cfg, per_view):
    """Per-element sensitivity of the oracle's gradient to the float32 rounding of the screen
    centres: |g(shift (d, 0)) - g| + |g(shift (0, d)) - g|, summed over the views, with d the
    largest bound (du, dv) of the view's visible splats. per_view: {v: (pixels, (oc, od, oa, on),
    g)}, g the unshifted oracle gradient of view v."""
    from oracle import oracle as O
    out = None
    for v, (px, up, g0) in per_view.items():
        cam = cams[v].as_dict()
        pre = O.preprocess(sc, cam, oracle_cfg(cfg))
        d = float(pre["duv"][pre["visible"] == 1].max()) if (pre["visible"] == 1).any() else 0.0
        acc = {k: np.zeros_like(g0[k]) for k in ("g_pos_op", "g_lscale_beta", "g_quat", "g_color")}
        for shift in ((d, 0.0), (0.0, d)):
            gs = O.backward(sc, cam, dict(oracle_cfg(cfg), shift=shift), *up, pixels=px)
            for k in acc:
                acc[k] += np.abs(gs[k] - g0[k])
        out = acc if out is None else {k: out[k] + acc[k] for k in out}
    return out


def oracle_g2d_sigma(g2d, conic):
    """The oracle's screen-space gradient with its conic columns (a, b, c) mapped to the
    gradient w.r.t. Sigma' (G = -C G_C C, symmetric entries 00, 01, 11), in FP64, the
    layout the CUDA path accumulates."""
    out = np.array(g2d, np.float64, copy=True)
    a, b, c = conic[:, 0], conic[:, 1], conic[:, 2]
    ga, gb, gc = g2d[:, 2], 0.5 * g2d[:, 3], g2d[:, 4]
    # C G_C C for symmetric 2x2 C = [[a, b], [b, c]], G_C = [[ga, gb], [gb, gc]]
    t00, t01 = ga * a + gb * b, ga * b + gb * c
    t10, t11 = gb * a + gc * b, gb * b + gc * c
    out[:, 2] = -(a * t00 + b * t10)
    out[:, 3] = -(a * t01 + b * t11)
    out[:, 4] = -(b * t01 + c * t11)
    return out
