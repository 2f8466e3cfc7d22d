"""The debug build (compiled with GES_DEBUG, selected by GES_LIB_VARIANT=debug): its render kernels
check every tile-list entry they read against the number of (view, splat) entries, and every
pixel's replay end against its tile's list, and record GES_ERR_BOUNDS instead of faulting.

Each case runs in a child process, since a process loads one build. A child that corrupts a
tile list or a replay end first asserts that the loaded library reports the debug build; the
release build has no such checks and is never given corrupted lists."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch

from paper_2411_09156_gb300 import api
from paper_2411_09156_gb300.scenes import look_at, make_scene

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCENE = '''
import numpy as np, torch
from paper_2411_09156_gb300 import _lib, api
from paper_2411_09156_gb300.scenes import look_at, make_scene
sc = make_scene(20000, 31, "object", 3)
cams = [look_at((0.5, -2.4, 0.8), (0, 0, 0), 160, 120), look_at((-1.8, -1.5, 0.6), (0, 0, 0), 96, 128)]
cfg = api.GESConfig(sh_degree=3, persistent=1)
t = api.scene_tensors(sc)
rast = api.Rasterizer(sc.n, cams, cfg)
rast.forward(*t)
g = torch.Generator().manual_seed(3)
ups = [torch.randn(k, generator=g).cuda() for k in (3 * rast.P, rast.P, rast.P, 3 * rast.P)]
'''


def _child(code: str) -> str:
    env = dict(os.environ, GES_LIB_VARIANT="debug")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return r.stdout


def test_debug_build_gives_the_release_results():
    """The checks change no arithmetic: the debug build's images equal the release build's bit for
    bit, and its gradients agree up to the order of the float32 atomics."""
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "dbg.npz")
        _child(_SCENE + f'''
assert _lib.lib().ges_build_flags() & _lib.GES_BUILD_DEBUG
grads = rast.backward(*t, *ups)
assert rast.sync_status() == 0
np.savez({out!r}, **{{k: v.cpu().numpy() for k, v in rast.out.items()}},
         **{{k: v.cpu().numpy() for k, v in grads.items()}})
''')
        dbg = np.load(out)
        sc = make_scene(20000, 31, "object", 3)
        cams = [look_at((0.5, -2.4, 0.8), (0, 0, 0), 160, 120), look_at((-1.8, -1.5, 0.6), (0, 0, 0), 96, 128)]
        t = api.scene_tensors(sc)
        rast = api.Rasterizer(sc.n, cams, api.GESConfig(sh_degree=3, persistent=1))
        rast.forward(*t)
        g = torch.Generator().manual_seed(3)
        ups = [torch.randn(k, generator=g).cuda() for k in (3 * rast.P, rast.P, rast.P, 3 * rast.P)]
        grads = rast.backward(*t, *ups)
        torch.cuda.synchronize()
        for k in ("color", "depth", "alpha", "normal", "t_final", "last", "n_contrib"):
            np.testing.assert_array_equal(dbg[k], rast.out[k].cpu().numpy(), err_msg=k)
        for k, v in grads.items():
            ref = v.double().cpu().numpy()
            assert np.linalg.norm(dbg[k] - ref) <= 1e-5 * np.linalg.norm(ref), k


def test_corrupted_list_entry_and_replay_end_are_reported_not_faulted():
    """A tile-list entry beyond the (view, splat) records, written on the host into the longest
    tile's list, makes the debug forward report GES_ERR_BOUNDS; a pixel whose stored replay end
    lies past its tile's list makes the debug backward report it too. Both calls complete, and
    the status read clears the word."""
    out = _child(_SCENE + '''
assert _lib.lib().ges_build_flags() & _lib.GES_BUILD_DEBUG  # the checks are compiled in
assert rast.sync_status() == 0
lay = rast.layout()
n_inst = rast.instance_count()
ranges = rast.bins[lay.bins_ranges:lay.bins_ranges + 8 * lay.n_tiles].view(torch.int32).view(-1, 2).cpu()
tile = int(torch.argmax(ranges[:, 1] - ranges[:, 0]))
first = int(ranges[tile, 0])
ent = rast.bins[lay.bins_inst_entry:lay.bins_inst_entry + 4 * n_inst].view(torch.int32)
saved = int(ent[first])
ent[first] = 0x7FFFFF00
rast.render_fwd()
assert rast.sync_status() == _lib.GES_ERR_BOUNDS
assert rast.sync_status() == 0
ent[first] = saved
rast.render_fwd()
assert rast.sync_status() == 0
last = rast.out["last"]
last[0] = int(last[0]) + 100000000
rast.backward_screen(*ups)
assert rast.sync_status() == _lib.GES_ERR_BOUNDS
print("REPORTED")
''')
    assert "REPORTED" in out
