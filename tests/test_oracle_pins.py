"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks the oracle against a closed form, an invariant, a textbook or
library routine, or brute force, chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.special as sps
from scipy.spatial.transform import Rotation
from scipy.stats import gennorm, multivariate_normal

from oracle import binning as OB
from oracle import drt as ODRT
from oracle import oracle as O
from paper_2411_09156_gb300.scenes import Scene, look_at, make_scene
from tests._util import axis_camera, make_splats, oracle_cfg

AMIN = float(np.float32(1.0 / 255.0))


# ----------------------------------------------------------------- independent routes
def indep_cov2d(mu, lscale, quat, cam, lowpass=0.3, phi=1.0):
    """Sigma' by an independent route: scipy's rotation for R, a finite-difference
    Jacobian of the actual perspective map for J W (valid off the clamp), plus h I."""
    vm = np.asarray(cam["viewmat"], np.float64)
    Rw, tw = vm[:, :3], vm[:, 3]
    q = np.asarray(quat, np.float64)
    rot = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    sig = rot @ np.diag((phi * np.exp(np.asarray(lscale, np.float64))) ** 2) @ rot.T

    fx, fy, cx, cy = (float(np.float32(cam[k])) for k in ("fx", "fy", "cx", "cy"))

    def proj(p):
        t = Rw @ p + tw
        return np.array([fx * t[0] / t[2] + cx, fy * t[1] / t[2] + cy])

    mu = np.asarray(mu, np.float64)
    hh = 1e-5
    jac = np.stack([(proj(mu + e * hh) - proj(mu - e * hh)) / (2 * hh) for e in np.eye(3)], 1)
    return jac @ sig @ jac.T + float(np.float32(lowpass)) * np.eye(2), proj(mu)


def gef_falloff(r, beta):
    """exp(-1/2 r^beta) written through scipy's generalized normal density
    (gennorm.pdf(x, b) = b / (2 Gamma(1/b)) exp(-|x|^b)) at x = r / 2^(1/beta)."""
    x = r / 2.0 ** (1.0 / beta)
    return gennorm.pdf(x, beta) * 2.0 * sps.gamma(1.0 / beta) / beta


def pixel_grid(w, h):
    xs, ys = np.meshgrid(np.arange(w) + 0.5, np.arange(h) + 0.5)
    return xs.ravel(), ys.ravel()


# ----------------------------------------------------------------- S1-S3 + falloff
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_projection_matches_fd_jacobian_and_scipy_rotation(seed):
    rng = np.random.default_rng(seed)
    cam = look_at(rng.normal(size=3) * 0.3 + np.array([0.3, -4.0, 1.0]), (0, 0, 0), 96, 80).as_dict()
    n = 6
    mu = rng.uniform(-0.4, 0.4, size=(n, 3))
    ls = rng.normal(-2.5, 0.4, size=(n, 3))
    q = rng.normal(size=(n, 4))
    sc = make_splats(mu, ls, rng.uniform(1, 5, n), 0.7, quat=q)
    pre = O.preprocess(sc, cam, oracle_cfg(phi_mode=0))
    for i in range(n):
        cov, uv = indep_cov2d(sc.pos_op[i, :3], sc.lscale_beta[i, :3], sc.quat[i], cam)
        got = pre["cov2d"][i]
        np.testing.assert_allclose([got[0], got[1], got[2]], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7)
        np.testing.assert_allclose(pre["uvz"][i, :2], uv, rtol=1e-9)
        inv = np.linalg.inv(cov)
        np.testing.assert_allclose(pre["conic"][i], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-7)


@pytest.mark.parametrize("beta", [1.0, 1.7, 2.0, 3.3, 6.0])
def test_single_splat_alpha_is_generalized_normal_of_mahalanobis_radius(beta):
    """One rotated splat: alpha(p) = min(alpha_max, o exp(-1/2 Q^(beta/2))) inside the
    support, 0 outside, with Q the Mahalanobis distance under the independent Sigma'."""
    cam = look_at((0.5, -3.5, 1.2), (0, 0, 0), 72, 56).as_dict()
    o = 0.93
    sc = make_splats([[0.05, 0.1, -0.05]], [-1.8, -2.3, -3.4], beta, o, quat=[[0.8, 0.3, -0.4, 0.2]])
    out = O.render(sc, cam, oracle_cfg(phi_mode=0))
    beta, o = float(sc.lscale_beta[0, 3]), float(sc.pos_op[0, 3])  # the float32 inputs
    cov, uv = indep_cov2d(sc.pos_op[0, :3], sc.lscale_beta[0, :3], sc.quat[0], cam)
    xs, ys = pixel_grid(72, 56)
    d = np.stack([xs - uv[0], ys - uv[1]], 1)
    Qm = np.einsum("pi,ij,pj->p", d, np.linalg.inv(cov), d)
    alpha = np.minimum(0.99, o * gef_falloff(np.sqrt(Qm), beta))
    alpha[alpha < AMIN] = 0.0
    assert (alpha > 0).sum() > 20
    np.testing.assert_allclose(out["alpha"], alpha, atol=1e-9)
    np.testing.assert_array_equal(out["n_contrib"], (alpha > 0).astype(np.int32))


def test_beta2_is_the_ewa_gaussian():
    """beta = 2: the falloff is the 3DGS EWA Gaussian, exp(-Q/2) = 2 pi sqrt(det) N(p; m, Sigma')."""
    cam = look_at((-0.7, -3.8, 0.9), (0, 0, 0), 64, 64).as_dict()
    o = 0.6
    sc = make_splats([[0.1, -0.05, 0.0]], [-2.0, -2.6, -3.0], 2.0, o, quat=[[0.3, -0.2, 0.9, 0.1]])
    out = O.render(sc, cam, oracle_cfg(phi_mode=1))  # phi(2) = 1 in the centred reading
    cov, uv = indep_cov2d(sc.pos_op[0, :3], sc.lscale_beta[0, :3], sc.quat[0], cam)
    xs, ys = pixel_grid(64, 64)
    g = multivariate_normal(mean=uv, cov=cov).pdf(np.stack([xs, ys], 1)) * 2 * np.pi * np.sqrt(np.linalg.det(cov))
    alpha = o * g
    alpha[alpha < AMIN] = 0.0
    np.testing.assert_allclose(out["alpha"], alpha, atol=1e-10)


def test_axis_aligned_on_optical_axis_by_hand():
    """Camera [I | 0], splat on the axis at depth z0, identity rotation:
    Sigma' = diag((f s1 / z0)^2 + h, (f s2 / z0)^2 + h); off-axis at x0 the
    Jacobian's third column adds (f x0 / z0^2)^2 s3^2 to Sigma'_00."""
    f, z0, h = 40.0, 2.5, 0.3
    cam = axis_camera(48, 48, f)
    s = np.array([0.08, 0.05, 0.03])
    for x0 in (0.0, 0.4):
        sc = make_splats([[x0, 0.0, z0]], np.log(s), 3.0, 0.5)
        pre = O.preprocess(sc, cam, oracle_cfg(phi_mode=0))
        s00 = (f * s[0] / z0) ** 2 + (f * x0 / z0 ** 2) ** 2 * s[2] ** 2 + h
        s11 = (f * s[1] / z0) ** 2 + h
        np.testing.assert_allclose(pre["cov2d"][0], [s00, 0.0, s11], rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(pre["uvz"][0], [f * x0 / z0 + 24.0, 24.0, z0], rtol=1e-6)
        # normal: smallest scale is axis 3 = world +z, flipped to face the camera at the origin
        np.testing.assert_allclose(pre["normal"][0], [0, 0, -1], atol=1e-12)


def test_gef_along_axis_is_eq1():
    """Along the pixel row through the centre of an axis-aligned splat the falloff is
    the 1-D generalized exponential of Eq. 1, g(x | delta = u, gamma, epsilon = beta,
    A = o) with gamma = 2^(1/beta) sqrt(Sigma'_00), evaluated here through scipy's
    generalized normal density."""
    f, z0 = 40.0, 2.0
    cam = axis_camera(63, 63, f)  # c = 31.5: pixel (31, 31) is the splat centre
    beta, o = 1.3, 0.9
    s = np.array([0.1, 0.05, 0.02])
    sc = make_splats([[0.0, 0.0, z0]], np.log(s), beta, o)
    out = O.render(sc, cam, oracle_cfg(phi_mode=0))
    s00 = (f * s[0] / z0) ** 2 + 0.3
    gamma = 2.0 ** (1.0 / beta) * math.sqrt(s00)
    dx = np.arange(63) + 0.5 - 31.5
    b32, o32 = float(np.float32(beta)), float(np.float32(o))
    g = gennorm.pdf(dx / gamma, b32) * 2.0 * sps.gamma(1.0 / b32) / b32
    a = o32 * g
    a[a < AMIN] = 0
    np.testing.assert_allclose(out["alpha"].reshape(63, 63)[31], a, atol=1e-9)


def test_qcut_is_the_alpha_min_level_set():
    rng = np.random.default_rng(5)
    cam = axis_camera(32, 32, 30.0)
    for _ in range(20):
        beta, o = rng.uniform(0.8, 6.0), rng.uniform(0.01, 0.99)
        sc = make_splats([[0, 0, 2.0]], [-3, -3, -3], beta, o)
        pre = O.preprocess(sc, cam, oracle_cfg(phi_mode=0))
        q = pre["qcut"][0]
        assert abs(float(np.float32(o)) * math.exp(-0.5 * q ** (float(np.float32(beta)) / 2)) - AMIN) < 1e-12


def test_support_brute_force_no_pixel_outside_box_has_alpha():
    """Every pixel with alpha >= alpha_min lies inside the pixel box of the binning reading."""
    sc = make_scene(60, 11, "uniform", -1)
    cam = look_at((0.3, -3.0, 0.4), (0, 0, 0), 80, 72).as_dict()
    cfg = oracle_cfg()
    pre = O.preprocess(sc, cam, cfg)
    xs, ys = pixel_grid(80, 72)
    for i in np.nonzero(pre["visible"])[0]:
        one = sc.subset([i])
        out = O.render(one, cam, cfg)
        hit = out["n_contrib"] > 0
        qm = pre["qcut"][i] * float(OB.QM)
        ex = math.sqrt(pre["cov2d"][i, 0] * qm)
        ey = math.sqrt(pre["cov2d"][i, 2] * qm)
        u, v = pre["uvz"][i, :2]
        inside = (np.abs(xs - u) <= ex) & (np.abs(ys - v) <= ey)
        assert not np.any(hit & ~inside)


# ----------------------------------------------------------------- compositing
def test_two_splats_on_axis_hand_composite():
    """Centre pixel of two on-axis splats: Q = 0, alpha_i = o_i, so
    C = o1 c1 + (1 - o1) o2 c2 + (1 - o1)(1 - o2) bg, D = o1 z1 + (1 - o1) o2 z2."""
    cam = axis_camera(33, 33, 30.0)  # c = 16.5: pixel (16, 16) is centred on the axis
    o1, o2 = 0.6, 0.45
    c1, c2, bg = np.array([0.9, 0.1, 0.3]), np.array([0.2, 0.8, 0.5]), np.array([0.05, 0.1, 0.2])
    sc = make_splats([[0, 0, 3.0], [0, 0, 2.0]], [-2.5, -2.5, -3.0], [1.5, 4.0], [o2, o1], rgb=[c2, c1])
    out = O.render(sc, cam, oracle_cfg(bg=tuple(bg)), pixels=[[16, 16]])
    o1f, o2f = float(np.float32(o1)), float(np.float32(o2))
    expect_c = o1f * c1.astype(np.float32) + (1 - o1f) * o2f * c2.astype(np.float32) + (1 - o1f) * (1 - o2f) * bg.astype(np.float32)
    np.testing.assert_allclose(out["color"][0], expect_c, rtol=1e-6)
    np.testing.assert_allclose(out["depth"][0], o1f * 2.0 + (1 - o1f) * o2f * 3.0, rtol=1e-6)
    np.testing.assert_allclose(out["alpha"][0], 1 - (1 - o1f) * (1 - o2f), rtol=1e-12)
    assert out["n_contrib"][0] == 2 and out["last_id"][0] == 0


def test_transmittance_cutoff_ends_the_pixel():
    """On-axis centre pixel (Q = 0, alpha_i = o_i): after o = 0.99 and 0.985, T = 1.5e-4;
    the next splat (o = 0.5) would take T below t_min = 1e-4, so the pixel ends there and
    the later o = 0.1 splat, which alone would keep T above t_min, is not blended."""
    cam = axis_camera(33, 33, 30.0)
    ops = [0.99, 0.985, 0.5, 0.1]
    zs = [2.0, 2.2, 2.4, 2.6]
    sc = make_splats([[0, 0, z] for z in zs], [-2.5, -2.5, -3.0], 2.0, ops)
    out = O.render(sc, cam, oracle_cfg(), pixels=[[16, 16]])
    o = [float(np.float32(x)) for x in ops]
    T = (1 - o[0]) * (1 - o[1])
    assert out["n_contrib"][0] == 2 and out["last_id"][0] == 1
    np.testing.assert_allclose(out["T"][0], T, rtol=1e-12)
    np.testing.assert_allclose(out["depth"][0], o[0] * 2.0 + (1 - o[0]) * o[1] * 2.2, rtol=1e-6)


def test_zero_opacity_gives_background_and_zero_gradient():
    sc = make_scene(40, 3, "uniform", -1)
    sc.pos_op[:, 3] = 0.5 * AMIN
    cam = look_at((0, -4, 0), (0, 0, 0), 40, 40).as_dict()
    bg = (0.3, 0.6, 0.9)
    out = O.render(sc, cam, oracle_cfg(bg=bg))
    np.testing.assert_array_equal(out["color"], np.tile(np.float32(bg), (1600, 1)))
    assert out["n_contrib"].max() == 0 and np.all(out["depth"] == 0) and np.all(out["alpha"] == 0)
    rng = np.random.default_rng(0)
    g = O.backward(sc, cam, oracle_cfg(bg=bg), rng.normal(size=(1600, 3)), rng.normal(size=1600),
                   rng.normal(size=1600), rng.normal(size=(1600, 3)))
    for k in ("g_pos_op", "g_lscale_beta", "g_quat", "g_color"):
        assert np.all(g[k] == 0)


def test_constant_colour_invariant():
    sc = make_scene(80, 4, "uniform", -1)
    k = np.float32(0.37)
    sc.color[:] = k
    cam = look_at((0.2, -3.5, 0.5), (0, 0, 0), 48, 40).as_dict()
    out = O.render(sc, cam, oracle_cfg(bg=(float(k),) * 3))
    assert out["n_contrib"].max() > 3
    np.testing.assert_allclose(out["color"], float(k), atol=1e-14)


def test_weights_sum_to_alpha():
    """rgb = 1, bg = 0: C = sum_i w_i, which must equal A = 1 - T_final."""
    sc = make_scene(80, 6, "uniform", -1)
    sc.color[:] = 1.0
    cam = look_at((0.2, -3.5, 0.5), (0, 0, 0), 48, 40).as_dict()
    out = O.render(sc, cam, oracle_cfg())
    for c in range(3):
        np.testing.assert_allclose(out["color"][:, c], out["alpha"], atol=1e-13)
    np.testing.assert_allclose(out["alpha"], 1 - out["T"], atol=1e-15)


def test_equal_depth_plane_depth_is_z0_alpha():
    """All centres on one fronto-parallel plane z = z0: D = z0 * A exactly."""
    rng = np.random.default_rng(7)
    n, z0 = 30, 2.75
    mu = np.concatenate([rng.uniform(-0.6, 0.6, size=(n, 2)), np.full((n, 1), z0)], 1)
    sc = make_splats(mu, rng.normal(-2.5, 0.3, size=(n, 3)), rng.uniform(1, 5, n), rng.uniform(0.2, 0.9, n),
                     quat=rng.normal(size=(n, 4)))
    cam = axis_camera(40, 40, 35.0)
    out = O.render(sc, cam, oracle_cfg())
    assert out["n_contrib"].max() >= 3
    np.testing.assert_allclose(out["depth"], z0 * out["alpha"], atol=1e-12)


def test_permutation_invariance():
    sc = make_scene(120, 8, "uniform", -1)
    cam = look_at((0.2, -3.5, 0.5), (0, 0, 0), 56, 48).as_dict()
    out = O.render(sc, cam, oracle_cfg())
    perm = np.random.default_rng(1).permutation(sc.n)
    out2 = O.render(sc.subset(perm), cam, oracle_cfg())
    for k in ("color", "depth", "alpha", "normal", "T"):
        np.testing.assert_array_equal(out[k], out2[k])
    np.testing.assert_array_equal(out["n_contrib"], out2["n_contrib"])
    has = out["last_id"] >= 0
    np.testing.assert_array_equal(perm[out2["last_id"][has]], out["last_id"][has])


def test_scale_invariance():
    """Scaling positions, scales, camera translation and z_near by k leaves the image
    unchanged (J scales by 1/k, Sigma by k^2) and scales the depth by k."""
    sc = make_scene(100, 9, "uniform", -1)
    cam = look_at((0.2, -3.5, 0.5), (0, 0, 0), 48, 40).as_dict()
    k = 2.0
    sc2 = Scene(sc.pos_op.copy(), sc.lscale_beta.copy(), sc.quat, sc.color, -1)
    sc2.pos_op[:, :3] *= k
    sc2.lscale_beta[:, :3] += np.float32(math.log(k))
    cam2 = dict(cam)
    cam2["viewmat"] = cam["viewmat"].copy()
    cam2["viewmat"][:, 3] *= k
    cam2["znear"] = cam["znear"] * k
    a = O.render(sc, cam, oracle_cfg())
    b = O.render(sc2, cam2, oracle_cfg())
    mask = (a["flags"] == 0) & (b["flags"] == 0)
    np.testing.assert_allclose(b["color"][mask], a["color"][mask], atol=2e-6)
    np.testing.assert_allclose(b["depth"][mask], k * a["depth"][mask], atol=5e-6)


# ----------------------------------------------------------------- colour, phi
def _real_sh_scipy(l, m, d):
    theta = np.arccos(np.clip(d[2], -1, 1))
    ph = np.arctan2(d[1], d[0])
    y = sps.sph_harm_y(l, abs(m), theta, ph)
    if m == 0:
        return y.real
    return math.sqrt(2) * (y.real if m > 0 else y.imag)


def test_sh_basis_matches_scipy_and_its_gradient_matches_fd():
    rng = np.random.default_rng(3)
    for _ in range(10):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        Y, dY = O.sh_basis(3, d)
        k = 0
        for l in range(4):
            for m in range(-l, l + 1):
                assert abs(Y[k] - _real_sh_scipy(l, m, d)) < 1e-12
                k += 1
        # tangential gradient vs central differences on the sphere
        P = np.eye(3) - np.outer(d, d)
        for j in range(3):
            h = 1e-6
            dp, dm = d + h * P[j], d - h * P[j]
            fd = (O.sh_basis(3, dp / np.linalg.norm(dp))[0] - O.sh_basis(3, dm / np.linalg.norm(dm))[0]) / (2 * h)
            np.testing.assert_allclose((P @ dY.T).T @ P[j], fd, atol=1e-7)


def test_phi_properties():
    assert O.phi(2.0, 0.1, 1)[0] == 1.0
    for b in (0.5, 1.0, 3.0, 6.0):
        assert O.phi(b, 0.0, 1)[0] == 1.0
        assert O.phi(b, 0.1, 0) == (1.0, 0.0)
        for mode in (1, 2):
            h = 1e-6
            fd = (O.phi(b + h, 0.1, mode)[0] - O.phi(b - h, 0.1, mode)[0]) / (2 * h)
            assert abs(fd - O.phi(b, 0.1, mode)[1]) < 1e-8
    assert 0.0 < O.phi(2.0, 0.1, 2)[0] < 0.05  # the literal Eq. 7 collapses scales at beta = 2
    assert O.phi(1.0, 0.1, 1)[0] < 1.0 < O.phi(6.0, 0.1, 1)[0]


def test_phi_is_a_scale_multiplier():
    """Centred phi == phi off with every scale multiplied by phi(beta)."""
    rng = np.random.default_rng(12)
    n = 40
    sc = make_scene(n, 12, "uniform", -1)
    cam = look_at((0.2, -3.5, 0.5), (0, 0, 0), 48, 40).as_dict()
    a = O.render(sc, cam, oracle_cfg(phi_mode=1))
    sc2 = Scene(sc.pos_op, sc.lscale_beta.astype(np.float64).copy(), sc.quat, sc.color, -1)
    for i in range(n):
        sc2.lscale_beta[i, :3] += math.log(O.phi(float(sc.lscale_beta[i, 3]), 0.1, 1)[0])
    b = O.render(sc2, cam, oracle_cfg(phi_mode=0))
    np.testing.assert_allclose(a["color"], b["color"], atol=1e-12)


def test_sh_colour_degree0_and_clamp():
    cam = axis_camera(16, 16, 15.0)
    sc = make_splats([[0, 0, 2.0]], [-1.5, -1.5, -1.5], 2.0, 0.99)
    Y0 = 0.5 / math.sqrt(math.pi)
    for dc in (-1.0, 0.3, 2.0):
        sc2 = Scene(sc.pos_op, sc.lscale_beta, sc.quat, np.full((1, 1, 3), dc, np.float32), 0)
        pre = O.preprocess(sc2, cam, oracle_cfg())
        np.testing.assert_allclose(pre["rgb"][0], max(0.0, Y0 * float(np.float32(dc)) + 0.5), rtol=1e-12)


# ----------------------------------------------------------------- DRT, Eq. 15
def test_drt_schedule():
    assert ODRT.scale(0, 100, 0.26, 1.0) == pytest.approx(0.26)
    assert ODRT.scale(100, 100, 0.26, 1.0) == pytest.approx(1.0)
    assert ODRT.scale(50, 100, 0.26, 1.0) == pytest.approx(0.63)
    s = [ODRT.scale(i, 100, 0.26, 1.0) for i in range(101)]
    assert all(b >= a for a, b in zip(s, s[1:]))
    sizes8 = ODRT.batch_sizes(1600, 1040, 8)
    assert sizes8[0] == (400, 260) and sizes8[-1] == (1600, 1040)
    assert sum(w * h for w, h in sizes8) == 6_252_862
    sizes16 = ODRT.batch_sizes(1920, 1080, 16)
    assert sizes16[0] == (480, 270) and sizes16[-1] == (1920, 1080)
    assert sum(w * h for w, h in sizes16) == 15_437_124


# ----------------------------------------------------------------- binning reading
def test_rect_min_q_against_dense_grid():
    rng = np.random.default_rng(4)
    for _ in range(200):
        A = rng.normal(size=(2, 2))
        cov = A @ A.T + 0.3 * np.eye(2)
        inv = np.linalg.inv(cov)
        a, b, c = inv[0, 0], inv[0, 1], inv[1, 1]
        X0, Y0 = rng.uniform(-6, 6, 2)
        X1, Y1 = X0 + rng.uniform(0, 8), Y0 + rng.uniform(0, 8)
        got = float(OB.rect_min_q(a, b, c, X0, X1, Y0, Y1))
        gx, gy = np.meshgrid(np.linspace(X0, X1, 301), np.linspace(Y0, Y1, 301))
        dense = (a * gx * gx + 2 * b * gx * gy + c * gy * gy).min()
        assert got <= dense * (1 + 1e-5) + 1e-6
        assert got >= dense - 1e-3 * (1 + dense)


def test_tile_lists_cover_the_exact_support():
    """Every pixel whose FP64 Q is within q_cut lies in a tile the float32 reading lists."""
    sc = make_scene(150, 13, "uniform", -1)
    W, H, tw, th = 90, 70, 16, 8
    cam = look_at((0.3, -3.2, 0.6), (0, 0, 0), W, H).as_dict()
    pre = O.preprocess(sc, cam, oracle_cfg())
    xs, ys = pixel_grid(W, H)
    tiles_x = (W + tw - 1) // tw
    checked = 0
    for i in np.nonzero(pre["visible"])[0]:
        u, v = pre["uvz"][i, :2]
        a, b, c = pre["conic"][i]
        q = pre["qcut"][i]
        qm = np.float32(np.float32(q) * OB.QM)
        ext_x = np.sqrt(np.float32(pre["cov2d"][i, 0]) * qm)
        ext_y = np.sqrt(np.float32(pre["cov2d"][i, 2]) * qm)
        tiles = set(OB.splat_tiles(u, v, a, b, c, q, ext_x, ext_y, W, H, tw, th))
        dx, dy = xs - u, ys - v
        Q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        inside = np.nonzero(Q <= q)[0]
        for p in inside:
            px, py = p % W, p // W
            assert (py // th) * tiles_x + px // tw in tiles
        checked += len(inside)
    assert checked > 1000


# ---------------------------------------------------------------- the oracle's cell index
@pytest.mark.parametrize("kind,sh,cell,w,h", [("object", 3, 1, 203, 151), ("object", 3, 7, 203, 151),
                                              ("uniform", -1, 16, 203, 151), ("uniform", -1, 64, 203, 151),
                                              ("object", 3, 16, 1600, 1040)])
def test_cell_index_gives_the_brute_force_result(kind, sh, cell, w, h):
    """Walking a pixel's cell list instead of every visible splat leaves out only splats whose step
    of the per-pixel loop does nothing, so the forward (every output and flag) is identical bit for
    bit, and the gradient equal up to the order of its FP64 sums. The uniform scene has splats
    whose boxes cover many cells and reach past the image border; at 1600x1040 the borderline
    bands, which grow with the float32 rounding of the screen centres, are widest."""
    sc = make_scene(2500, 17, kind, sh)
    cam = look_at((0.4, -2.6, 0.9), (0, 0, 0), w, h).as_dict()
    base = oracle_cfg()
    ref = O.render(sc, cam, base)
    got = O.render(sc, cam, dict(base, cell=cell))
    for k in ref:
        np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
    assert (ref["n_contrib"] > 0).mean() > 0.3  # the scene covers the image
    rng = np.random.default_rng(cell)
    P = cam["width"] * cam["height"]
    g = [rng.standard_normal((P, 3)), rng.standard_normal(P), rng.standard_normal(P), rng.standard_normal((P, 3))]
    gb = O.backward(sc, cam, base, *g)
    gc = O.backward(sc, cam, dict(base, cell=cell), *g)
    for k in ("g2d", "g_pos_op", "g_lscale_beta", "g_quat", "g_color"):
        np.testing.assert_allclose(gc[k], gb[k], rtol=1e-11, atol=1e-11 * np.abs(gb[k]).max(), err_msg=k)


def test_sample_shift_moves_the_sample_point():
    """The shift of the sample points moves them relative to the splats: a single splat rendered
    with the sample points shifted by (sx, sy) equals the splat moved by (-sx, -sy) on screen
    (here by moving it in the world along the image axes of an axis-aligned camera; its extent
    along z is negligible, so the projected covariance does not depend on where it sits)."""
    cam = axis_camera(31, 23, 40.0)
    cfg = oracle_cfg()
    sx, sy, Z = 0.3, -0.2, 2.0
    a = O.render(make_splats([[0.05, -0.02, Z]], [-2.5, -2.8, -14.0], 2.7, 0.7), cam, dict(cfg, shift=(sx, sy)))
    b = O.render(make_splats([[0.05 - sx * Z / 40.0, -0.02 - sy * Z / 40.0, Z]], [-2.5, -2.8, -14.0], 2.7, 0.7),
                 cam, cfg)
    np.testing.assert_allclose(a["color"], b["color"], atol=1e-9)
    np.testing.assert_array_equal(a["n_contrib"], b["n_contrib"])


def test_cusp_flag_marks_pixels_near_the_centre_of_a_low_beta_splat():
    """Reading D16: a blended splat with beta < 2 whose centre lies within 0.25 px of a pixel's
    sample point flags that pixel; beta >= 2, or farther away, does not."""
    cam = axis_camera(9, 9, 40.0)
    for beta, off, flagged in ((1.5, 0.1, True), (1.5, 0.3, False), (2.0, 0.1, False), (3.0, 0.0, False)):
        # centre at x = 4.5 + off px, y = 4.5 px (pixel (4, 4)'s sample point), depth 2
        u = (4.5 + off - 4.5) * 2.0 / 40.0
        sc = make_splats([[u, 0.0, 2.0]], [-3.0, -3.0, -3.0], beta, 0.8)
        out = O.render(sc, cam, oracle_cfg())
        f = out["flags"].reshape(9, 9)[4, 4]
        assert bool(f & O.FLAG_CUSP) == flagged, (beta, off, f)
        assert out["n_contrib"].reshape(9, 9)[4, 4] == 1


def test_cell_index_keeps_a_splat_whose_support_band_flags_a_pixel_past_its_box():
    """A splat whose support-edge band (which widens with the float32 rounding of its screen
    centre, about 4e-4 px on a 1601-px view) reaches a pixel centre just beyond the box of
    Q <= qcut (1 + flag_eps): the brute-force loop flags that pixel, so the cell index must list
    the splat there too. The splat is axis-aligned on the centre row of an odd-height view; its
    x is solved so that its box edge falls 1e-4 px short of the pixel centre."""
    W, H, f = 1601, 41, 1200.0
    cam = axis_camera(W, H, f)
    cfg = oracle_cfg()
    eps = cfg["flag_eps"]
    k = 1400  # the pixel column past the box
    Z, s = 4.0, np.log(0.01)

    def splat(X):
        return make_splats([[X, 0.0, Z]], [s, s, -12.0], 2.0, 0.8)

    X = (k - 0.5 * W) * Z / f
    for _ in range(6):  # Newton steps on the box edge u + ex - 1/2 = k - 1e-4
        pre = O.preprocess(splat(X), cam, cfg)
        u, S00, qc = pre["uvz"][0, 0], pre["cov2d"][0, 0], pre["qcut"][0]
        ex = np.sqrt(S00 * qc * (1 + eps))
        X += ((k - 1e-4) - (u + ex - 0.5)) * Z / f
    pre = O.preprocess(splat(X), cam, cfg)
    u, S00, qc = pre["uvz"][0, 0], pre["cov2d"][0, 0], pre["qcut"][0]
    edge = u + np.sqrt(S00 * qc * (1 + eps)) - 0.5
    assert k - 2e-4 < edge < k, edge  # pixel k is outside the box by about 1e-4 px
    assert abs(pre["uvz"][0, 1] - (H // 2 + 0.5)) < 1e-12  # on the centre row's sample points
    ref = O.render(splat(X), cam, cfg)
    assert ref["flags"].reshape(H, W)[H // 2, k] & O.FLAG_SUPPORT  # the band reaches it
    for cell in (1, 16):
        got = O.render(splat(X), cam, dict(cfg, cell=cell))
        np.testing.assert_array_equal(got["flags"], ref["flags"])
    # sample points moved by a few 1e-4 px: the cell index still equals the brute-force loop
    for shift in ((3e-4, 0.0), (0.0, -5e-4)):
        ref = O.render(splat(X), cam, dict(cfg, shift=shift))
        got = O.render(splat(X), cam, dict(cfg, shift=shift, cell=16))
        for key in ref:
            np.testing.assert_array_equal(got[key], ref[key], err_msg=key)
