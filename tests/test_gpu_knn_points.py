"""KNN point queries (ges_knn_points, the search ges_levelset runs) against brute force.

Queries near and far from the centres, outside their bounding box, in empty space between
sheets, on degenerate clouds (a line, a plane, coincident centres) and rows marked w = 0.
Where several lists are correct (the 16th and 17th distances within float32 rounding) the
check is validity: every listed neighbour at most the brute-force 16th distance away, the
list ordered and duplicate-free; elsewhere the sets are identical. (On the line, the plane
and the duplicates nearly every query has such near-ties, so there only validity is asserted
in bulk.)"""
import numpy as np
import pytest
import torch

from paper_2411_09156_gb300 import api
from paper_2411_09156_gb300.scenes import make_scene

pytestmark = pytest.mark.gpu


def _brute(pos, q, k=17):
    p = pos[:, :3].astype(np.float64)
    out = []
    for lo in range(0, len(q), 256):
        d2 = ((q[lo:lo + 256, None, :3].astype(np.float64) - p[None]) ** 2).sum(-1)
        idx = np.argsort(d2, axis=1, kind="stable")[:, :k]
        out.append(idx)
    return np.concatenate(out)


def _check(pos, q, got, min_sep=0.9):
    valid = q[:, 3] != 0
    assert (got[~valid] == -1).all()
    g = got[valid]
    qv = q[valid, :3].astype(np.float64)
    p = pos[:, :3].astype(np.float64)
    assert (g >= 0).all() and (g < len(pos)).all()
    assert all(len(set(r)) == 16 for r in g)
    ref = _brute(pos, q[valid])
    dg = np.sqrt(((qv[:, None] - p[g]) ** 2).sum(-1))
    dr = np.sqrt(((qv[:, None] - p[ref]) ** 2).sum(-1))
    tol = 1e-6 * np.maximum(dr[:, 15:16], 1e-6) + 1e-6 * (np.abs(qv).max(1, keepdims=True) + 1.0)
    assert (np.diff(dg, axis=1) >= -tol).all(), "lists not ordered"
    assert (dg[:, 15] <= dr[:, 15] + tol[:, 0]).all(), "a listed neighbour is farther than the 16th nearest"
    if ref.shape[1] < 17:  # sixteen centres in all: every list is all of them
        assert all(set(a) == set(b) for a, b in zip(g, ref))
        return
    sep = dr[:, 16] - dr[:, 15] > 10 * tol[:, 0]
    same = np.array([set(a) == set(b[:16]) for a, b in zip(g, ref)])
    assert same[sep].all()
    assert sep.mean() >= min_sep


def _run(pos, q):
    return api.knn_points(torch.from_numpy(np.ascontiguousarray(pos, np.float32)).cuda(),
                          torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda()).cpu().numpy()


def test_points_near_far_and_outside_a_surface():
    sc = make_scene(50000, 9, "heightfield", -1)
    pos = sc.pos_op
    rng = np.random.default_rng(1)
    base = pos[rng.choice(len(pos), 2400), :3].astype(np.float64)
    parts = [base[:600] + rng.normal(0, 0.01, (600, 3)),                       # on the surface
             base[600:1200] + np.array([0, 0, 1.0]) * rng.uniform(0.05, 0.6, (600, 1)),  # above it
             base[1200:1600] * np.array([1.3, 1.3, 1.0]),                      # past its edge
             rng.uniform(-3, 3, (400, 3)),                                     # anywhere in and around
             base[1600:1800] + rng.normal(0, 10.0, (200, 3))]                  # far away
    pts = np.concatenate(parts)
    q = np.concatenate([pts, np.ones((len(pts), 1))], 1)
    q = np.concatenate([q, np.zeros((300, 4))])  # rows without a query
    q[-300:, :3] = base[:300]
    q = q[rng.permutation(len(q))]
    _check(pos, q, _run(pos, q))


@pytest.mark.parametrize("kind", ["line", "plane", "duplicates", "uniform"])
def test_points_on_degenerate_clouds(kind):
    rng = np.random.default_rng(5)
    if kind == "line":
        pos = np.zeros((3000, 4)); pos[:, 0] = rng.uniform(-1, 1, 3000)
    elif kind == "plane":
        pos = np.zeros((3000, 4)); pos[:, :2] = rng.uniform(-1, 1, (3000, 2))
    elif kind == "duplicates":
        pos = np.repeat(rng.uniform(-1, 1, (300, 4)), 10, axis=0)
    else:
        pos = make_scene(20000, 3, "uniform", -1).pos_op.astype(np.float64)
    q = np.concatenate([rng.uniform(-1.5, 1.5, (700, 3)), np.ones((700, 1))], 1)
    _check(pos, q, _run(pos.astype(np.float32), q), min_sep=0.9 if kind == "uniform" else 0.0)


def test_points_host_checks():
    pos = torch.zeros((100, 4), device="cuda")
    with pytest.raises(ValueError):
        api.ges_knn_points_workspace_bytes(15, 4)
    with pytest.raises(ValueError):
        api.ges_knn_points_workspace_bytes(100, 0)
    ws = torch.empty(api.ges_knn_points_workspace_bytes(100, 4), dtype=torch.uint8, device="cuda")
    pts = torch.zeros((5, 4), device="cuda")
    out = torch.empty((5, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(api.GESError):  # points off the 16-byte grid
        api.ges_knn_points(100, pos, 4, pts.view(-1)[1:17], ws, out)


def test_single_point_query():
    pos = make_scene(2000, 13, "uniform", -1).pos_op.astype(np.float64)
    q = np.array([[0.1, -0.2, 0.3, 1.0]])
    got = _run(pos.astype(np.float32), q)
    assert got.shape == (1, 16)
    _check(pos, q, got, min_sep=0.0)


def test_smallest_cloud_of_sixteen_centres():
    """n = 16, the smallest size: every list holds all sixteen centres, ordered by distance."""
    rng = np.random.default_rng(17)
    pos = np.concatenate([rng.uniform(-1, 1, (16, 3)), np.ones((16, 1))], 1)
    q = np.concatenate([rng.uniform(-2, 2, (40, 3)), np.ones((40, 1))], 1)
    got = _run(pos.astype(np.float32), q)
    assert all(set(r) == set(range(16)) for r in got)
    _check(pos, q, got, min_sep=0.0)
    lists = api.knn(torch.from_numpy(pos.astype(np.float32)).cuda()).cpu().numpy()
    assert all(set(r) == set(range(16)) for r in lists) and (lists[:, 0] == np.arange(16)).all()

