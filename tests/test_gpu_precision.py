"""16-bit storage of the colour input (SH coefficients or RGB) in IEEE binary16 or bfloat16,
through the C ABI (ges_config.color_storage).

The kernels widen each stored value to float32 on load, which is exact, and compute as
before, so a render from 16-bit colours equals bit for bit the float32 render of the same
values widened, and its gradients (float32) agree up to the order of the float32 atomics
(1e-4 relative L2). The oracle is given the widened values: forward and gradient parity against it hold with
the tolerances of the float32 path. The full-size case renders the eight batched views of
the 1.5M-splat scene (SH degree 3) from binary16 coefficients, the launch configuration the
bench times for this variant, and compares every pixel."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2411_09156_gb300 import api
from paper_2411_09156_gb300.drt import drt_sizes
from paper_2411_09156_gb300.scenes import Scene, look_at, make_scene, random_sphere_cameras, workload
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

OUTS = ("color", "depth", "alpha", "normal", "t_final", "last", "n_contrib")


def _widened(sc, dtype):
    """(16-bit colour on the device, the scene with those values widened to float32)."""
    c16 = torch.as_tensor(sc.color).to(dtype).contiguous().cuda()
    wide = Scene(sc.pos_op, sc.lscale_beta, sc.quat, np.ascontiguousarray(c16.float().cpu().numpy()), sc.sh_degree)
    return c16, wide


def _grads_close(a, b, rel=1e-4):
    """Two backward runs on the same inputs differ by the order of their float32 atomics; at
    the full size that reaches 2e-5 relative L2 in the log-scale gradient (thin splats sum
    terms of both signs), so the bound is 1e-4, ten times below the parity tolerance."""
    for k in ("g_pos_op", "g_lscale_beta", "g_quat", "g_color"):
        x, y = a[k].double(), b[k].double()
        assert a[k].dtype == torch.float32, k
        d = float((x - y).norm() / y.norm().clamp_min(1e-30))
        assert d <= rel, (k, d)


@pytest.mark.parametrize("storage,dtype", [(1, torch.float16), (2, torch.bfloat16)])
@pytest.mark.parametrize("sh_degree", [3, 2, 1, 0, -1])
def test_16bit_colour_equals_the_widened_float32_render(storage, dtype, sh_degree):
    sc = make_scene(6000, 61, "object", sh_degree)
    cams = [look_at((0.4, -2.3, 0.8), (0, 0, 0), 131, 97)] + \
        random_sphere_cameras(np.random.default_rng(62), 2, 3.0, [(77, 120), (64, 64)])
    c16, wide = _widened(sc, dtype)
    t = api.scene_tensors(wide)
    cfg = api.GESConfig(sh_degree=sh_degree)
    r32 = api.Rasterizer(sc.n, cams, cfg)
    r32.forward(*t)
    r16 = api.Rasterizer(sc.n, cams, cfg.replace(color_storage=storage))
    r16.forward(t[0], t[1], t[2], c16)
    torch.cuda.synchronize()
    for k in OUTS:
        assert torch.equal(r16.out[k], r32.out[k]), k
    ups = H.upstream(r32, 7)
    g32 = r32.backward(*t, *ups)
    g16 = r16.backward(t[0], t[1], t[2], c16, *ups)
    torch.cuda.synchronize()
    _grads_close(g16, g32)


@pytest.mark.parametrize("storage,dtype", [(1, torch.float16), (2, torch.bfloat16)])
def test_16bit_colour_matches_oracle(storage, dtype):
    sc = make_scene(2000, 31, "object", 3)
    cams = [look_at((0.5, -2.2, 0.7), (0, 0, 0), 96, 80)]
    c16, wide = _widened(sc, dtype)
    t = api.scene_tensors(wide)
    cfg = api.GESConfig(sh_degree=3, bg=(0.1, 0.2, 0.3), color_storage=storage)
    rast = api.Rasterizer(sc.n, cams, cfg)
    rast.forward(t[0], t[1], t[2], c16)
    torch.cuda.synchronize()
    rep, ref, _ = H.compare_forward(rast, wide, cams, cfg)
    ups = H.mask_upstream(rast, H.upstream(rast, 1000), [H.grad_mask(ref)])
    grads = rast.backward(t[0], t[1], t[2], c16, *ups)
    torch.cuda.synchronize()
    got = {k: v.double().cpu().numpy() for k, v in grads.items()}
    oc, od, oa, on = H.oracle_upstream(rast, ups, 0)
    refg = O.backward(wide, cams[0].as_dict(), H.oracle_cfg(cfg), oc, od, oa, on)
    H.compare_grads(got, refg)


def test_16bit_colour_full_size_drt8():
    sizes = drt_sizes(1600, 1040, 8)
    sc, cams = workload("drt8-1.5M", sizes=sizes)
    c16, wide = _widened(sc, torch.float16)
    t = api.scene_tensors(wide)
    cfg = api.GESConfig(sh_degree=3, persistent=1)
    r32 = api.Rasterizer(sc.n, cams, cfg)
    r32.forward(*t)
    r16 = api.Rasterizer(sc.n, cams, cfg.replace(color_storage=1))
    r16.forward(t[0], t[1], t[2], c16)
    torch.cuda.synchronize()
    for k in OUTS:
        assert torch.equal(r16.out[k], r32.out[k]), k
    ups = H.upstream(r32, 11)
    g32 = r32.backward(*t, *ups)
    g16 = r16.backward(t[0], t[1], t[2], c16, *ups)
    torch.cuda.synchronize()
    _grads_close(g16, g32)


def test_colour_storage_host_checks():
    sc = make_scene(500, 3, "uniform", 3)
    cams = [look_at((0.0, -3.0, 0.0), (0, 0, 0), 32, 32)]
    t = api.scene_tensors(sc)
    with pytest.raises(ValueError):  # float32 colours under binary16 storage
        api.Rasterizer(sc.n, cams, api.GESConfig(sh_degree=3, color_storage=1)).forward(*t)
    bad = api.GESConfig(sh_degree=3, color_storage=3)
    with pytest.raises(api.GESError):
        api.ges_preprocess(sc.n, t[0], t[1], t[2], t[3].half(), 1, api.cameras_to_c(cams), bad.to_c(),
                           torch.empty(api.ges_proj_bytes(sc.n, 1), dtype=torch.uint8, device="cuda"))
    # a colour pointer off the 16-byte grid is rejected before any launch
    c = torch.empty(sc.n * 48 + 8, dtype=torch.float16, device="cuda")
    with pytest.raises(api.GESError):
        api.ges_preprocess(sc.n, t[0], t[1], t[2], c[1:], 1, api.cameras_to_c(cams),
                           api.GESConfig(sh_degree=3, color_storage=1).to_c(),
                           torch.empty(api.ges_proj_bytes(sc.n, 1), dtype=torch.uint8, device="cuda"))
