"""The no-allocation backward entry point (ges_render_bwd_noalloc).

It exists for callers that cannot allocate device memory while they run: it
keeps its accumulator in a fixed array inside the library instead of memory the
caller hands in. Here it is called twice in a row through the C ABI and each
result is compared with the standard ges_render_bwd on the same inputs, within
the gradient tolerance the other tests use. The second call checks that what the
first call left in the shared array does not leak into the next result. This
file is collected last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2411_09156_gb300 import _lib, api
from paper_2411_09156_gb300.scenes import look_at, make_scene

pytestmark = pytest.mark.gpu

REL_L2 = 1e-3  # the gradient tolerance of the parity tests


def _upstream(P, seed):
    g = torch.Generator().manual_seed(seed)
    return [torch.randn(k, generator=g).cuda() for k in (3 * P, P, P, 3 * P)]


def _noalloc(rast, t, ups):
    out = {k: torch.full_like(x, float("nan")) for k, x in
           zip(("g_pos_op", "g_lscale_beta", "g_quat", "g_color"), t)}
    o = rast.out
    api.ges_render_bwd_noalloc(rast.n, rast.n_views, rast.cams_c, rast.cfg_c, *t, rast.proj, rast.bins, o["color"],
                               o["depth"], o["normal"], o["t_final"], o["last"], *ups, out["g_pos_op"],
                               out["g_lscale_beta"], out["g_quat"], out["g_color"])
    torch.cuda.synchronize()
    return out


def test_no_alloc_backward_matches_the_standard_entry_point_on_two_calls():
    sc = make_scene(20000, 61, "object", 3)
    cams = [look_at((0.5, -2.4, 0.8), (0, 0, 0), 160, 120), look_at((-1.8, -1.5, 0.6), (0, 0, 0), 96, 128)]
    cfg = api.GESConfig(sh_degree=3)
    t = api.scene_tensors(sc)
    rast = api.Rasterizer(sc.n, cams, cfg)
    rast.forward(*t)
    for call, seed in enumerate((11, 12)):
        ups = _upstream(rast.P, seed)
        ref = {k: v.clone() for k, v in rast.backward(*t, *ups).items()}
        got = _noalloc(rast, t, ups)
        for k in ref:
            assert torch.isfinite(got[k]).all(), (call, k)
            r = float((got[k] - ref[k]).norm() / ref[k].norm())
            assert r <= REL_L2, (call, k, r)
    assert rast.sync_status() == 0


def test_no_alloc_rejects_problems_beyond_its_array():
    lib = _lib.lib()
    cams = api.cameras_to_c([look_at((0, -4, 0), (0, 0, 0), 32, 32)])
    cfg = api.GESConfig().to_c()
    n = _lib.NOALLOC_MAX_ENTRIES + 1
    st = lib.ges_render_bwd_noalloc(n, 1, cams, ctypes.byref(cfg), *([None] * 4), None, 0, None, 0,
                                    *([None] * 5), *([None] * 4), *([None] * 4), None)
    assert st == _lib.GES_ERR_TOO_LARGE
