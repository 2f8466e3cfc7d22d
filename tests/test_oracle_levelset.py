"""Pins of the level-set extraction oracle (oracle/levelset.py): the ray and its start point
against the camera projection, the crossing of an isolated flat splat against its closed form,
its normal, sigma_g(v) along a principal axis, the cases without a point, the normal against
central differences of the density, and the choice of the rising crossing."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import levelset as OLS


def _cam(w=64, h=48, f=50.0, R=np.eye(3), t=np.array([0.0, 0.0, 4.0])):
    vm = np.concatenate([R, t[:, None]], 1)
    return dict(width=w, height=h, fx=f, fy=f, cx=w / 2, cy=h / 2, viewmat=vm.reshape(-1))


def _scene(centre, ls, q, o=1.0, beta=2.0):
    # splat 0 at the centre, 16 far splats of zero opacity
    pos = np.zeros((17, 4))
    pos[0, :3], pos[0, 3] = centre, o
    pos[1:, :3] = 100.0 + np.arange(16)[:, None]
    lsb = np.zeros((17, 4))
    lsb[:, :3], lsb[:, 3] = ls, beta
    return pos, lsb, np.tile(q, (17, 1))


def test_start_point_projects_to_the_pixel_at_the_rendered_depth():
    R = Rotation.from_euler("xyz", [0.2, -0.3, 0.1]).as_matrix()
    cam = _cam(R=R, t=np.array([0.1, -0.2, 3.5]))
    pos, lsb, q = _scene([0.0, 0.0, 0.0], [-2.0, -2.0, -2.0], [1.0, 0, 0, 0])
    out = OLS.extract(pos, lsb, q, cam, depth=1.8, alpha=0.6, px=20, py=31)
    pc = R @ out["x0"] + np.array([0.1, -0.2, 3.5])
    assert abs(pc[2] - 3.0) < 1e-12  # D / A
    np.testing.assert_allclose([50 * pc[0] / pc[2] + 32, 50 * pc[1] / pc[2] + 24], [20.5, 31.5], atol=1e-10)


def test_isolated_flat_splat_crossing_and_normal():
    # a flat Gaussian splat facing the camera, its centre on the optical axis at depth 4: along
    # the axis d(t) = o exp(-(t / s)^2 / 2), first reaching 0.3 at t = -s sqrt(2 ln(o / 0.3))
    o, s = 0.9, 0.02
    pos, lsb, q = _scene([0.0, 0.0, 0.0], [np.log(0.5), np.log(0.5), np.log(s)], [1.0, 0, 0, 0], o=o)
    cam = _cam(w=64, h=64)
    # pixel (31, 31)'s centre is 0.5 px off the axis: at depth 4 that is 0.04, far inside the 0.5 scales
    out = OLS.extract(pos, lsb, q, cam, depth=4.0, alpha=1.0, px=32, py=32, n_steps=4001, phi_mode=0)
    assert out["valid"] and not out["flag"]
    _, v, _ = OLS.ray(cam, 32, 32)
    x0 = out["x0"]
    # along this slightly oblique ray the flat axis is z: d = o exp(-1/2 (Q_inplane + (z / s)^2))
    qin = (x0[0] + out["t"] * v[0]) ** 2 / 0.25 + (x0[1] + out["t"] * v[1]) ** 2 / 0.25
    z = x0[2] + out["t"] * v[2]
    d = o * np.exp(-0.5 * (qin + (z / s) ** 2))
    assert abs(d - 0.3) < 2e-4
    assert z < 0  # the camera side: the camera sits at z = -4 in the world
    # normal: -grad d points away from the splat, toward the camera side
    A = np.diag([4.0, 4.0, 1 / s ** 2])
    g = A @ out["point"]
    np.testing.assert_allclose(out["normal"], g / np.linalg.norm(g), atol=1e-10)


def test_sigma_along_a_principal_axis():
    R = Rotation.from_euler("z", 0.7).as_matrix()
    q = Rotation.from_matrix(R).as_quat()[[3, 0, 1, 2]]
    pos, lsb, _ = _scene([0.0, 0.0, 0.0], [np.log(0.3), np.log(0.2), np.log(0.05)], q)
    q = np.tile(q, (17, 1))
    cam = _cam(w=64, h=64)
    out = OLS.extract(pos, lsb, q, cam, depth=4.0, alpha=1.0, px=32, py=32, phi_mode=0)
    _, v, _ = OLS.ray(cam, 32, 32)
    loc = R.T @ v
    np.testing.assert_allclose(out["sigma"], np.sqrt(((loc * [0.3, 0.2, 0.05]) ** 2).sum()), rtol=1e-12)


def test_no_point_without_coverage_or_crossing():
    pos, lsb, q = _scene([0.0, 0.0, 0.0], [-2.0, -2.0, -4.0], [1.0, 0, 0, 0], o=0.2)  # peak below the level
    cam = _cam(w=64, h=64)
    assert not OLS.extract(pos, lsb, q, cam, depth=4.0, alpha=1.0, px=32, py=32)["valid"]
    assert not OLS.extract(pos, lsb, q, cam, depth=4.0, alpha=5e-5, px=32, py=32)["valid"]


def test_normal_is_the_finite_difference_gradient_of_the_density():
    # several overlapping rotated splats of different beta: -grad d by central differences of
    # density_at must have the direction normal_at reports, anywhere (not only on the level set)
    rng = np.random.default_rng(4)
    n = 17
    pos = np.concatenate([rng.normal(0, 0.05, (n, 3)), rng.uniform(0.3, 1.0, (n, 1))], 1)
    lsb = np.concatenate([rng.normal(-2.5, 0.3, (n, 3)), rng.uniform(1.2, 5.0, (n, 1))], 1)
    q = Rotation.random(n, random_state=5).as_quat()[:, [3, 0, 1, 2]]
    nb = np.arange(16)
    for x in rng.normal(0, 0.08, (6, 3)):
        h = 1e-6
        grad = np.array([(OLS.density_at(pos, lsb, q, nb, x + h * e) - OLS.density_at(pos, lsb, q, nb, x - h * e))
                         / (2 * h) for e in np.eye(3)])
        nrm, cond = OLS.normal_at(pos, lsb, q, nb, x)
        np.testing.assert_allclose(nrm, -grad / np.linalg.norm(grad), atol=1e-6)
        assert cond >= 1.0


def test_first_crossing_from_the_camera_side():
    # a flat splat facing the camera on its axis at z = -0.2 (another far behind it, at z = +0.2):
    # d rises through the level in front of the near splat and falls through it again behind;
    # the point is the rising crossing, on the camera side
    s = 0.01
    pos = np.zeros((18, 4))
    pos[0, :3], pos[0, 3] = [0.0, 0.0, -0.2], 0.9
    pos[1, :3], pos[1, 3] = [0.0, 0.0, 0.2], 0.9
    pos[2:, :3] = 100.0 + np.arange(16)[:, None]
    lsb = np.zeros((18, 4))
    lsb[:, :3] = [np.log(0.5), np.log(0.5), np.log(s)]
    lsb[:, 3] = 2.0
    q = np.tile([1.0, 0, 0, 0], (18, 1))
    cam = _cam(w=64, h=64)
    # start just behind the near splat (camera depth 4 is z = 0): sigma_g along the axis is s, so
    # +-3 sigma covers both of its crossings
    out = OLS.extract(pos, lsb, q, cam, depth=3.8 + 0.5 * s, alpha=1.0, px=32, py=32, n_steps=2001, phi_mode=0)
    assert out["valid"]
    z = out["point"][2]
    assert -0.2 - 4 * s < z < -0.2, z  # on the camera side of the near splat
    d = OLS.density_at(pos, lsb, q, out["neighbours"], out["point"], phi_mode=0)
    assert abs(d - 0.3) < 1e-3


def _axis_splat(ls_flat):
    # a flat beta = 2 splat facing a 65x65 camera whose centre pixel (32, 32) looks straight down
    # the optical axis: along that ray the splat's spread is its flat scale exactly
    pos, lsb, q = _scene([0.0, 0.0, 0.0], [np.log(0.5), np.log(0.5), ls_flat], [1.0, 0, 0, 0], o=0.9)
    return pos, lsb, q, _cam(w=65, h=65)


def test_march_samples_the_printed_range_of_sigma():
    # Sec. 3.3: t_k runs over [-3 sigma_g(v), 3 sigma_g(v)] (k = 3 from the golden fixture);
    # sigma_g(v) here is the flat scale s in closed form (v is the splat's flat axis)
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
    k = gold["march_half_width_sigmas"]["value"]
    s = 0.02
    pos, lsb, q, cam = _axis_splat(np.log(s))
    for n_steps in (2, 7, 32):
        out = OLS.extract(pos, lsb, q, cam, depth=4.0, alpha=1.0, px=32, py=32, n_steps=n_steps, phi_mode=0)
        ts = out["ts"]
        assert len(ts) == n_steps
        np.testing.assert_allclose([ts[0], ts[-1]], [-k * s, k * s], rtol=1e-12)
        np.testing.assert_allclose(np.diff(ts), 2 * k * s / (n_steps - 1), rtol=1e-9)


def test_crossing_between_two_and_three_sigma_is_found_and_beyond_three_is_not():
    # start x0 on the camera side of the splat at world z = -c s (camera depth 4 - c s). Along the
    # axis d(z) = 0.9 exp(-(z / s)^2 / 2) first reaches the level 0.3 at z = -s sqrt(2 ln 3), so
    # the crossing lies at t = (c - sqrt(2 ln 3)) s from x0: 2.52 s for c = 4 (inside +-3 sigma,
    # outside +-2 sigma) and 3.22 s for c = 4.7 (outside +-3 sigma, inside +-4 sigma)
    s = 0.02
    zc = np.sqrt(2.0 * np.log(0.9 / 0.3))
    pos, lsb, q, cam = _axis_splat(np.log(s))
    out = OLS.extract(pos, lsb, q, cam, depth=4.0 - 4.0 * s, alpha=1.0, px=32, py=32, n_steps=601, phi_mode=0)
    assert out["valid"] and not out["flag"]
    assert abs(out["t"] - (4.0 - zc) * s) < 1e-3 * s
    np.testing.assert_allclose(out["point"], [0.0, 0.0, -zc * s], atol=1e-3 * s)
    out = OLS.extract(pos, lsb, q, cam, depth=4.0 - 4.7 * s, alpha=1.0, px=32, py=32, n_steps=601, phi_mode=0)
    assert not out["valid"] and out["hit"] == -1
