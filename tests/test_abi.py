"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/ges.h declares; host-only calls behave as documented (CPU only: no
compute is launched)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2411_09156_gb300 import _lib, api, build
from paper_2411_09156_gb300.drt import drt_sizes
from paper_2411_09156_gb300.scenes import look_at
from oracle import drt as ODRT

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "ges.h")


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^GES_API\s+[\w\s\*]+?\b(ges_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_function():
    lib = _lib.lib()
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert set(_lib.SIGNATURES) == set(names)
    assert lib.ges_abi_version() == 3
    assert lib.ges_build_flags() == 0  # the release build (no device-side bounds checks)


def test_built_for_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors agree with a C compiler's view of include/ges.h (size and offsets)."""
    src = tmp_path / "probe.c"
    fields = {"ges_camera": [f for f, _ in _lib.Camera._fields_], "ges_config": [f for f, _ in _lib.Config._fields_],
              "ges_layout": [f for f, _ in _lib.Layout._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ges.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n") if l)
    for st, cls in (("ges_camera", _lib.Camera), ("ges_config", _lib.Config), ("ges_layout", _lib.Layout)):
        assert int(out[st]) == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert int(out[f"{st}.{f}"]) == getattr(cls, f).offset, (st, f)


def test_status_strings():
    lib = _lib.lib()
    for s in range(5):
        assert lib.ges_status_string(s).decode()
    assert lib.ges_status_string(99).decode() == "unknown status"


def _cams(sizes):
    return api.cameras_to_c([look_at((0, -4, 0), (0, 0, 0), w, h) for w, h in sizes])


def test_sizes_and_layout_are_consistent():
    cfg = api.GESConfig().to_c()
    cams = _cams([(128, 96), (33, 17)])
    n, nv = 1000, 2
    pb = api.ges_proj_bytes(n, nv)
    assert pb >= 256 + n * nv * (64 + 32 + 64)
    lay = api.ges_get_layout(n, nv, cams, cfg, 5000)
    assert lay.proj_bytes == pb
    assert lay.n_tiles == 8 * 6 + 3 * 2
    assert list(lay.tile_base[:2]) == [0, 48]
    bb = api.ges_bins_bytes(n, nv, cams, cfg, 5000)
    assert bb == lay.bins_bytes
    for off in (lay.proj_records, lay.proj_binrec, lay.proj_g2d, lay.bins_inst_tile, lay.bins_inst_entry,
                lay.bins_ranges, lay.bins_queue):
        assert off % 256 == 0
    # capacity grows the bins buffer by at least 16 bytes per instance (double-buffered keys and values)
    assert api.ges_bins_bytes(n, nv, cams, cfg, 10000) - bb >= 16 * 5000


def test_invalid_arguments_are_rejected_on_the_host():
    lib = _lib.lib()
    cams = _cams([(64, 64)])
    bad = [api.GESConfig(tile_w=12), api.GESConfig(batch=100), api.GESConfig(sh_degree=4),
           api.GESConfig(alpha_min=0.0), api.GESConfig(alpha_max=1.0), api.GESConfig(phi_mode=3),
           api.GESConfig(color_storage=3), api.GESConfig(tile_w=32, tile_h=32)]
    for cfg in bad:
        assert api.ges_bins_bytes(10, 1, cams, cfg.to_c(), 100) == 0
        st = lib.ges_preprocess(10, 16, 16, 16, 16, 1, cams, ctypes.byref(cfg.to_c()), 256, 1 << 20, None)
        assert st == _lib.GES_ERR_INVALID_ARG
    ok = api.GESConfig().to_c()
    # too many views, misaligned pointers, short buffers, null pointers
    assert lib.ges_preprocess(10, 16, 16, 16, 16, 33, cams, ctypes.byref(ok), 256, 1 << 20, None) == 1
    assert lib.ges_preprocess(10, 8, 16, 16, 16, 1, cams, ctypes.byref(ok), 256, 1 << 20, None) == 1
    assert lib.ges_preprocess(10, 16, 16, 16, 16, 1, cams, ctypes.byref(ok), 256, 100, None) == 1
    assert lib.ges_preprocess(10, None, 16, 16, 16, 1, cams, ctypes.byref(ok), 256, 1 << 20, None) == 1
    assert lib.ges_bin(10, 1, cams, ctypes.byref(ok), 256, 1 << 20, 256, 10, None) == 1
    # a colour pointer off the 16-byte grid; splat ranges outside [0, n)
    assert lib.ges_preprocess(10, 16, 16, 16, 24, 1, cams, ctypes.byref(ok), 256, 1 << 20, None) == 1
    for first, count in ((-1, 5), (6, 5), (0, 11), (3, -1)):
        assert lib.ges_preprocess_range(10, first, count, 16, 16, 16, 16, 1, cams, ctypes.byref(ok), 256, 1 << 20,
                                        None) == 1
        assert lib.ges_preprocess_bwd_range(10, first, count, 1, cams, ctypes.byref(ok), 16, 16, 16, 16, 256,
                                            1 << 20, None, 16, 16, 16, 16, None) == 1
    badcam = _cams([(0, 64)])
    assert api.ges_bins_bytes(10, 1, badcam, ok, 100) == 0
    assert api.ges_proj_bytes(-1, 1) == 0 and api.ges_proj_bytes(10, 0) == 0


def test_drt_sizes_agree_with_oracle_schedule():
    for (w, h, v) in ((1600, 1040, 8), (1920, 1080, 16), (800, 600, 3), (64, 48, 1)):
        assert drt_sizes(w, h, v) == (ODRT.batch_sizes(w, h, v) if v > 1 else [(w, h)])


def test_loss_sizes_and_arguments_on_the_host():
    lib = _lib.lib()
    cams = _cams([(64, 64), (33, 31)])
    # one CTA per 32 x 32 tile, two doubles each: 4 + 2 tiles
    assert lib.ges_loss_workspace_bytes(2, cams) == 16 * (4 + 2)
    assert lib.ges_loss_workspace_bytes(0, cams) == 0
    assert lib.ges_loss_workspace_bytes(2, _cams([(64, 64), (0, 5)])) == 0
    ws = lib.ges_loss_workspace_bytes(2, cams)
    # null images, lambda outside [0, 1], short or misaligned workspace: rejected before any launch
    assert lib.ges_loss_rgb(2, cams, None, 256, 0.2, 512, ws, 1024, None, None) == _lib.GES_ERR_INVALID_ARG
    assert lib.ges_loss_rgb(2, cams, 256, 256, -0.1, 512, ws, 1024, None, None) == _lib.GES_ERR_INVALID_ARG
    assert lib.ges_loss_rgb(2, cams, 256, 256, 0.2, 512, ws - 1, 1024, None, None) == _lib.GES_ERR_INVALID_ARG
    assert lib.ges_loss_rgb(2, cams, 256, 256, 0.2, 516, ws, 1024, None, None) == _lib.GES_ERR_INVALID_ARG
    assert lib.ges_loss_rgb(2, cams, 256, 256, 0.2, 512, ws, None, None, None) == _lib.GES_ERR_INVALID_ARG
