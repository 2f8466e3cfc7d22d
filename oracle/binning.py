"""Integer stage of the rasterizer (tile overlap, keys, order) -- oracle side.

TEST INFRASTRUCTURE ONLY.

The paper does not describe binning (it only names "rasterization", Sec. 3.2);
this is the reading the library documents in its header. A splat's screen
support is the ellipse Q(p - m) <= q_cut (Eq. 3 at alpha = alpha_min). For
binning the support is widened by the factor QM = 1 + 2^-10 (qm = q_cut * QM),
so that rounding can never drop a pixel that is inside the exact support. Then:

  pixel box:  x in [ceil(u - ext_x - 1/2), floor(u + ext_x - 1/2)] clipped to the
              image, ext_x = sqrt(Sigma'_00 qm), and likewise in y
  tile t is listed for the splat iff the minimum of Q over the rectangle of pixel
  centres of t (clipped to the pixel box) is <= qm.

These are integer decisions, so they are taken in the kernel's precision:
float32, every operation rounded, in the operation order written below. The
inputs are the CUDA path's own float32 values (u, v, conic, q_cut, ext_x,
ext_y, z32), so the comparison of keys and order is bit for bit.

Order within a tile: ascending float32 camera depth bits, ties by entry index
(entry = view * N + splat), i.e. a stable sort by (global tile, z32 bits).
"""
from __future__ import annotations

import numpy as np

F = np.float32
QM = F(1.0 + 2.0 ** -10)


def _qf(a, b2, c, X, Y):
    t1 = F(F(a * X) * X)
    t2 = F(F(b2 * X) * Y)
    t3 = F(F(c * Y) * Y)
    return F(F(t1 + t2) + t3)


def rect_min_q(a, b, c, X0, X1, Y0, Y1):
    """Minimum of Q(X, Y) = a X^2 + 2 b X Y + c Y^2 over [X0, X1] x [Y0, Y1] (float32 steps).

    Q is convex; if the rectangle holds the origin the minimum is 0, otherwise it
    lies on an edge, where it is the clamped 1-D minimiser of a quadratic, found
    with the float32 reciprocals 1/a and 1/c.
    """
    a, b, c, X0, X1, Y0, Y1 = map(F, (a, b, c, X0, X1, Y0, Y1))
    if X0 <= 0 <= X1 and Y0 <= 0 <= Y1:
        return F(0.0)
    b2 = F(b + b)
    ia, ic = F(F(1.0) / a), F(F(1.0) / c)  # correctly rounded reciprocals
    best = F(np.inf)
    for X in (X0, X1):
        ys = F(F(-F(b * X)) * ic)
        ys = min(max(ys, Y0), Y1)
        best = min(best, _qf(a, b2, c, X, ys))
    for Y in (Y0, Y1):
        xs = F(F(-F(b * Y)) * ia)
        xs = min(max(xs, X0), X1)
        best = min(best, _qf(a, b2, c, xs, Y))
    return best


def tile_hit(u, v, a, b, c, qm, px0, px1, py0, py1):
    """True iff min over pixel-centre rectangle [px0..px1] x [py0..py1] of Q <= qm (float32)."""
    X0 = F(F(F(px0) + F(0.5)) - u)
    X1 = F(F(F(px1) + F(0.5)) - u)
    Y0 = F(F(F(py0) + F(0.5)) - v)
    Y1 = F(F(F(py1) + F(0.5)) - v)
    return bool(rect_min_q(a, b, c, X0, X1, Y0, Y1) <= qm)


def pixel_box(u, v, ext_x, ext_y, width, height):
    x0 = int(np.ceil(F(F(u - ext_x) - F(0.5))))
    x1 = int(np.floor(F(F(u + ext_x) - F(0.5))))
    y0 = int(np.ceil(F(F(v - ext_y) - F(0.5))))
    y1 = int(np.floor(F(F(v + ext_y) - F(0.5))))
    x0, y0 = max(x0, 0), max(y0, 0)
    x1, y1 = min(x1, width - 1), min(y1, height - 1)
    return x0, x1, y0, y1


def splat_tiles(u, v, a, b, c, qcut, ext_x, ext_y, width, height, tw, th):
    """Local tile ids (ty * tiles_x + tx) listed for one splat, in row-major tile order."""
    u, v, a, b, c, qcut, ext_x, ext_y = map(F, (u, v, a, b, c, qcut, ext_x, ext_y))
    qm = F(qcut * QM)
    x0, x1, y0, y1 = pixel_box(u, v, ext_x, ext_y, width, height)
    if x0 > x1 or y0 > y1:
        return []
    tiles_x = (width + tw - 1) // tw
    out = []
    for ty in range(y0 // th, y1 // th + 1):
        for tx in range(x0 // tw, x1 // tw + 1):
            px0, px1 = max(tx * tw, x0), min(tx * tw + tw - 1, x1)
            py0, py1 = max(ty * th, y0), min(ty * th + th - 1, y1)
            if tile_hit(u, v, a, b, c, qm, px0, px1, py0, py1):
                out.append(ty * tiles_x + tx)
    return out


def instances(rec, visible, z32, views, tw, th, n):
    """All (global tile, entry) instances in the rasterizer's order, plus tile ranges.

    rec: per-entry float32 arrays dict with u, v, a, b, c, qcut, ext_x, ext_y (length V*N);
    visible: bool per entry; z32: float32 per entry; views: list of (width, height).
    Returns (keys, entries, tiles_touched, ranges) with ranges (T_total, 2); empty tiles are (0, 0).
    """
    tile_base, tb = [], 0
    for (w, h) in views:
        tile_base.append(tb)
        tb += ((w + tw - 1) // tw) * ((h + th - 1) // th)
    total_tiles = tb
    touched = np.zeros(len(visible), np.int64)
    items = []
    zbits = np.asarray(z32, np.float32).view(np.uint32)
    for e in np.nonzero(visible)[0]:
        vw = int(e) // n
        w, h = views[vw]
        ts = splat_tiles(rec["u"][e], rec["v"][e], rec["a"][e], rec["b"][e], rec["c"][e], rec["qcut"][e],
                         rec["ext_x"][e], rec["ext_y"][e], w, h, tw, th)
        touched[e] = len(ts)
        for t in ts:
            items.append((tile_base[vw] + t, int(zbits[e]), int(e)))
    items.sort()
    keys = np.array([it[0] for it in items], np.int64)
    ents = np.array([it[2] for it in items], np.int64)
    ranges = np.zeros((total_tiles, 2), np.int64)
    if len(keys):
        starts = np.searchsorted(keys, np.arange(total_tiles), "left")
        ends = np.searchsorted(keys, np.arange(total_tiles), "right")
        ranges[:, 0], ranges[:, 1] = starts, ends
        ranges[ends == starts] = 0
    return keys, ents, touched, ranges
