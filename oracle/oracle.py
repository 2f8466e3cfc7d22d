"""Python front end of the FP64 CPU oracle (ges_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and by the
CPU-baseline leg of the benchmark. The CUDA path never imports it and it never
imports the CUDA path.

Every function takes plain numpy arrays (any float dtype; converted to float64),
a camera dict (width, height, fx, fy, cx, cy, viewmat (3, 4), znear) and a
config dict (sh_degree, phi_mode, rho, lowpass, alpha_min, alpha_max, t_min,
jac_clamp, bg, flag_eps, and optionally cell: walk a cell index of cell x cell pixels
instead of every visible splat, bit-identical and far faster on large images; shift: (dx, dy)
offset of the sample points from the pixel centres, (0, 0) for the method). The arithmetic itself lives in the C file, which
cites the paper's equations step by step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ges_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libges_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_SUPPORT, FLAG_ALPHA_MIN, FLAG_T_MIN, FLAG_FACING, FLAG_CUSP = 1, 2, 4, 8, 16
DECISION_FLAGS = FLAG_SUPPORT | FLAG_ALPHA_MIN | FLAG_T_MIN | FLAG_FACING


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP over pixels, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Cam(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("viewmat", ctypes.c_float * 12), ("znear", ctypes.c_float)]


class _Cfg(ctypes.Structure):
    _fields_ = [("sh_degree", ctypes.c_int32), ("phi_mode", ctypes.c_int32), ("rho", ctypes.c_float),
                ("lowpass", ctypes.c_float), ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("t_min", ctypes.c_float), ("jac_clamp", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("flag_eps", ctypes.c_float), ("cell", ctypes.c_int32), ("shift", ctypes.c_float * 2)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_oracle())
            P = ctypes.c_void_p
            lib.orc_preprocess.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_render.argtypes = [ctypes.c_int, P, P, P, P, P, P, ctypes.c_int, P, P, P, P, P, P, P, P, P]
            lib.orc_backward.argtypes = [ctypes.c_int, P, P, P, P, P, P, ctypes.c_int, P, P, P, P, P, P, P, P,
                                         P, P]
            lib.orc_chain.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, P, P, P, P]
            lib.orc_sh_basis.argtypes = [ctypes.c_int, P, P, P]
            lib.orc_phi.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, P, P]
            _lib = lib
    return _lib


def _cam(c: dict) -> _Cam:
    cam = _Cam()
    cam.width, cam.height = int(c["width"]), int(c["height"])
    cam.fx, cam.fy, cam.cx, cam.cy = float(c["fx"]), float(c["fy"]), float(c["cx"]), float(c["cy"])
    vm = np.asarray(c["viewmat"], np.float32).reshape(12)
    for i in range(12):
        cam.viewmat[i] = float(vm[i])
    cam.znear = float(c.get("znear", 0.2))
    return cam


def _cfg(c: dict, sh_degree: int) -> _Cfg:
    cfg = _Cfg()
    cfg.sh_degree = int(sh_degree)
    cfg.phi_mode = int(c["phi_mode"])
    for k in ("rho", "lowpass", "alpha_min", "alpha_max", "t_min", "jac_clamp"):
        setattr(cfg, k, float(c[k]))
    for i in range(3):
        cfg.bg[i] = float(c["bg"][i])
    cfg.flag_eps = float(c.get("flag_eps", 1e-4))
    cfg.cell = int(c.get("cell", 0))
    sh = c.get("shift", (0.0, 0.0))
    cfg.shift[0], cfg.shift[1] = float(sh[0]), float(sh[1])
    return cfg


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _arrays(scene):
    return (_d(scene.pos_op), _d(scene.lscale_beta), _d(scene.quat), _d(scene.color))


def preprocess(scene, cam: dict, cfg: dict) -> dict:
    """Per-splat projection of S1-S4 (FP64; z32 is the float32 sort depth), and duv: the bound on
    the float32 rounding of (u, v) that the borderline flags use."""
    lib = _load()
    pos, lsb, q, col = _arrays(scene)
    n = pos.shape[0]
    out = dict(visible=np.zeros(n, np.int32), z32=np.zeros(n, np.float32), uvz=np.zeros((n, 3)),
               cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)), qcut=np.zeros(n), rgb=np.zeros((n, 3)),
               normal=np.zeros((n, 3)), duv=np.zeros((n, 2)))
    c, g = _cam(cam), _cfg(cfg, scene.sh_degree)
    lib.orc_preprocess(n, _p(pos), _p(lsb), _p(q), _p(col), ctypes.byref(c), ctypes.byref(g),
                       _p(out["visible"]), _p(out["z32"]), _p(out["uvz"]), _p(out["cov2d"]), _p(out["conic"]),
                       _p(out["qcut"]), _p(out["rgb"]), _p(out["normal"]), _p(out["duv"]))
    return out


def _pix(pixels, cam):
    if pixels is None:
        return None, int(cam["width"]) * int(cam["height"])
    px = np.ascontiguousarray(np.asarray(pixels, np.int32).reshape(-1, 2))
    return px, px.shape[0]


def render(scene, cam: dict, cfg: dict, pixels=None) -> dict:
    """Forward S6 by brute force per pixel. pixels: (P, 2) int (x, y), or None = whole image row-major."""
    lib = _load()
    pos, lsb, q, col = _arrays(scene)
    n = pos.shape[0]
    px, npix = _pix(pixels, cam)
    out = dict(color=np.zeros((npix, 3)), depth=np.zeros(npix), alpha=np.zeros(npix), normal=np.zeros((npix, 3)),
               T=np.zeros(npix), n_contrib=np.zeros(npix, np.int32), last_id=np.zeros(npix, np.int32),
               flags=np.zeros(npix, np.int32))
    c, g = _cam(cam), _cfg(cfg, scene.sh_degree)
    lib.orc_render(n, _p(pos), _p(lsb), _p(q), _p(col), ctypes.byref(c), ctypes.byref(g), npix,
                   _p(px) if px is not None else None, _p(out["color"]), _p(out["depth"]), _p(out["alpha"]),
                   _p(out["normal"]), _p(out["T"]), _p(out["n_contrib"]), _p(out["last_id"]), _p(out["flags"]))
    return out


def backward(scene, cam: dict, cfg: dict, g_color, g_depth, g_alpha, g_normal, pixels=None) -> dict:
    """Analytic gradient (S7 + S8) of sum over listed pixels of <upstream, outputs>.

    g_color, g_normal: (P, 3); g_depth, g_alpha: (P,). Returns g2d (N, 16) in the
    screen-space layout (u, v, a, b, c, opacity, beta, z, r, g, b, -, nx, ny, nz, -)
    and the 3-D gradients in the input layouts.
    """
    lib = _load()
    pos, lsb, q, col = _arrays(scene)
    n = pos.shape[0]
    px, npix = _pix(pixels, cam)
    gc, gd, ga, gn = _d(g_color).reshape(npix, 3), _d(g_depth).reshape(npix), _d(g_alpha).reshape(npix), \
        _d(g_normal).reshape(npix, 3)
    out = dict(g2d=np.zeros((n, 16)), g_pos_op=np.zeros((n, 4)), g_lscale_beta=np.zeros((n, 4)),
               g_quat=np.zeros((n, 4)), g_color=np.zeros_like(col))
    c, g = _cam(cam), _cfg(cfg, scene.sh_degree)
    lib.orc_backward(n, _p(pos), _p(lsb), _p(q), _p(col), ctypes.byref(c), ctypes.byref(g), npix,
                     _p(px) if px is not None else None, _p(gc), _p(gd), _p(ga), _p(gn), _p(out["g2d"]),
                     _p(out["g_pos_op"]), _p(out["g_lscale_beta"]), _p(out["g_quat"]), _p(out["g_color"]))
    return out


def chain(scene, cam: dict, cfg: dict, g2d) -> dict:
    """S8 alone: the 3-D gradients implied by a per-splat screen-space gradient g2d (N, 16)
    in the layout `backward` returns (conic columns a, b, c)."""
    lib = _load()
    pos, lsb, q, col = _arrays(scene)
    n = pos.shape[0]
    g2 = _d(g2d).reshape(n, 16)
    out = dict(g_pos_op=np.zeros((n, 4)), g_lscale_beta=np.zeros((n, 4)), g_quat=np.zeros((n, 4)),
               g_color=np.zeros_like(col))
    c, g = _cam(cam), _cfg(cfg, scene.sh_degree)
    lib.orc_chain(n, _p(pos), _p(lsb), _p(q), _p(col), ctypes.byref(c), ctypes.byref(g), _p(g2),
                  _p(out["g_pos_op"]), _p(out["g_lscale_beta"]), _p(out["g_quat"]), _p(out["g_color"]))
    return out


def sh_basis(deg: int, d):
    """Real SH basis Y_k(d) (K = (deg+1)^2) and its gradient (K, 3) at unit direction d."""
    lib = _load()
    d = _d(d).reshape(3)
    k = (deg + 1) ** 2
    Y = np.zeros(k)
    dY = np.zeros((k, 3))
    lib.orc_sh_basis(deg, _p(d), _p(Y), _p(dY))
    return Y, dY


def phi(beta: float, rho: float, mode: int):
    """phi(beta) of Eq. 7 (by reading mode) and its derivative."""
    lib = _load()
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib.orc_phi(float(beta), float(rho), int(mode), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value
