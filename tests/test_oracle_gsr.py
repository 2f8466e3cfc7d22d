"""Pins of the GSR oracle (oracle/gsr.py): KNN against scipy's k-d tree, rotations against
scipy, the density of single splats in closed form, the ideal flat splat (zero SDF and normal
losses), the normal direction of an isolated splat in closed form, and the gradient against
central finite differences."""
import numpy as np
import pytest
import torch
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from oracle import gsr as OG


def _scene(n, seed, flat=False):
    rng = np.random.default_rng(seed)
    pos = np.concatenate([rng.uniform(-1, 1, (n, 3)), rng.uniform(0.3, 0.95, (n, 1))], 1)
    ls = rng.normal(-2.5, 0.4, (n, 3))
    if flat:
        ls[:, 2] = -7.0
    lsb = np.concatenate([ls, rng.uniform(1.0, 4.0, (n, 1))], 1)
    q = rng.normal(size=(n, 4))
    return pos, lsb, q


def test_knn_matches_kd_tree():
    pos, _, _ = _scene(3000, 0)
    idx = OG.knn(pos)
    dist, ref = cKDTree(pos[:, :3]).query(pos[:, :3], k=16)
    assert (idx[:, 0] == np.arange(3000)).all()
    np.testing.assert_allclose(OG.knn_distances(pos, idx), dist, rtol=0, atol=1e-12)
    # equal index sets wherever the 16th and 17th distances are apart
    d17 = cKDTree(pos[:, :3]).query(pos[:, :3], k=17)[0][:, 16]
    sep = d17 - dist[:, 15] > 1e-9
    assert all(set(a) == set(b) for a, b in zip(idx[sep], ref[sep]))


def test_rotation_matches_scipy():
    q = np.random.default_rng(1).normal(size=(50, 4))
    R = OG.rotation(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()  # scipy takes (x, y, z, w)
    np.testing.assert_allclose(R, ref, rtol=0, atol=1e-12)


def test_density_of_one_isotropic_gaussian_splat():
    # 16 copies of one splat would sum; use one splat far from 15 others of zero opacity
    n = 16
    pos = np.zeros((n, 4))
    pos[1:, :3] = 50.0 + np.arange(15)[:, None]
    pos[0, 3] = 0.7
    lsb = np.zeros((n, 4))
    lsb[:, :3] = np.log(0.2)
    lsb[:, 3] = 2.0  # beta = 2: Gaussian, phi(2) = 1 in mode 1
    q = np.tile([1.0, 0, 0, 0], (n, 1))
    knn = np.tile(np.arange(n), (n, 1))
    z = np.array([[0.5, -1.0, 0.25]])
    out = OG.evaluate(pos, lsb, q, knn, [0], z, with_grad=False)
    x = 0.2 * z[0]
    np.testing.assert_allclose(out["x"][0], x, rtol=0, atol=1e-15)
    np.testing.assert_allclose(out["d"][0], 0.7 * np.exp(-0.5 * (x @ x) / 0.04), rtol=1e-13)


def test_ideal_flat_splat_has_zero_sdf_and_normal_loss():
    # opacity 1, a very flat splat, the sample on its normal axis: d = dbar exactly
    n = 16
    pos = np.zeros((n, 4))
    pos[1:, :3] = 50.0 + np.arange(15)[:, None]
    pos[:, 3] = 1.0
    pos[1:, 3] = 0.0
    lsb = np.zeros((n, 4))
    lsb[:, :3] = [np.log(0.3), np.log(0.25), np.log(0.01)]
    lsb[:, 3] = 3.0
    q = np.tile(Rotation.from_euler("xyz", [0.3, -0.2, 0.5]).as_quat()[[3, 0, 1, 2]], (n, 1))
    knn = np.tile(np.arange(n), (n, 1))
    z = np.array([[0.0, 0.0, 0.8]])  # along the smallest axis only
    out = OG.evaluate(pos, lsb, q, knn, [0], z, with_grad=False)
    assert abs(out["f"][0] - out["fbar"][0]) < 1e-12
    assert abs(out["cos"][0] - 1.0) < 1e-12
    assert out["l_sdf"] < 1e-12 and out["l_nor"] < 1e-12


def test_normal_direction_of_an_isolated_gaussian_is_the_mahalanobis_gradient():
    n = 16
    pos = np.zeros((n, 4))
    pos[1:, :3] = 50.0 + np.arange(15)[:, None]
    pos[0, 3] = 0.9
    lsb = np.zeros((n, 4))
    lsb[:, :3] = [np.log(0.3), np.log(0.2), np.log(0.05)]
    lsb[:, 3] = 2.0
    qv = np.array([0.9, 0.2, -0.3, 0.1])
    q = np.tile(qv, (n, 1))
    knn = np.tile(np.arange(n), (n, 1))
    z = np.array([[0.7, -0.4, 1.1]])
    out = OG.evaluate(pos, lsb, q, knn, [0], z, with_grad=False)
    R = Rotation.from_quat(qv[[1, 2, 3, 0]]).as_matrix()
    s = np.exp(lsb[0, :3])
    x = R @ (s * z[0])
    A = R @ np.diag(1 / s ** 2) @ R.T
    u = A @ x / np.linalg.norm(A @ x)
    nrm = R[:, 2] * np.sign(R[:, 2] @ x)
    np.testing.assert_allclose(out["cos"][0], u @ nrm, rtol=0, atol=1e-12)


@pytest.mark.parametrize("phi_mode", [1, 0])
def test_gradient_matches_central_differences(phi_mode):
    n = 60
    pos, lsb, q = _scene(n, 3, flat=True)
    knn = OG.knn(pos)
    rng = np.random.default_rng(4)
    js = rng.integers(0, n, 40)
    z = rng.normal(size=(40, 3))
    out = OG.evaluate(pos, lsb, q, knn, js, z, phi_mode=phi_mode, lambda_sdf=1.0, lambda_nor=0.5)
    assert not out["flags"].any()
    h = 1e-6
    for name, arr, g in (("pos", pos, out["grads"]["g_pos_op"]), ("lsb", lsb, out["grads"]["g_lscale_beta"]),
                         ("quat", q, out["grads"]["g_quat"])):
        for (i, c) in [(int(js[0]), 0), (int(js[1]), 3), (int(knn[js[2], 5]), 1), (int(js[3]), 2)]:
            ap, am = arr.copy(), arr.copy()
            ap[i, c] += h
            am[i, c] -= h
            args = dict(pos_op=pos, lscale_beta=lsb, quat=q)
            key = {"pos": "pos_op", "lsb": "lscale_beta", "quat": "quat"}[name]
            lp = OG.evaluate(**{**args, key: ap}, knn_idx=knn, sample_splat=js, sample_z=z, phi_mode=phi_mode,
                             lambda_sdf=1.0, lambda_nor=0.5, with_grad=False)["loss"]
            lm = OG.evaluate(**{**args, key: am}, knn_idx=knn, sample_splat=js, sample_z=z, phi_mode=phi_mode,
                             lambda_sdf=1.0, lambda_nor=0.5, with_grad=False)["loss"]
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i, c]) <= 1e-6 * max(1.0, abs(fd)), (name, i, c, fd, g[i, c])


def test_normal_direction_is_minus_the_density_gradient():
    # the explicit direction sum against autograd of the density itself, where nothing underflows
    n = 80
    pos, lsb, q = _scene(n, 8)
    lsb[:, :3] += 1.0  # wide splats: every sample sees several neighbours
    knn = OG.knn(pos)
    rng = np.random.default_rng(9)
    js, z = rng.integers(0, n, 30), 0.5 * rng.normal(size=(30, 3))
    out = OG.evaluate(pos, lsb, q, knn, js, z, with_grad=False)
    po, ls, qt = (torch.tensor(a, dtype=torch.float64) for a in (pos, lsb, q))
    R = OG.rotation(qt)
    sp = OG.phi(ls[:, 3], 0.1, 1)[:, None] * torch.exp(ls[:, :3])
    for k in range(30):
        x = torch.tensor(out["x"][k], requires_grad=True)
        d = 0.0
        for i in knn[js[k]]:
            loc = (R[i].T @ (x - po[i, :3])) / sp[i]
            d = d + po[i, 3] * torch.exp(-0.5 * (loc @ loc) ** (ls[i, 3] / 2))
        (gd,) = torch.autograd.grad(d, x)
        u = -gd / torch.linalg.norm(gd)
        g = int(knn[js[k]][out["gstar"][k]])
        nrm = R[g][:, int(torch.argmin(ls[g, :3]))]
        nrm = nrm * torch.sign(nrm @ (x.detach() - po[g, :3]))
        assert abs(float(u @ nrm) - out["cos"][k]) < 1e-10


def test_far_sample_with_underflowing_density_keeps_a_defined_normal():
    # |z|^2 = 200 and beta = 6: the density is exp(-4e6), zero in any float format, yet the
    # direction of -grad d is that of the splat's own term
    n = 16
    pos = np.zeros((n, 4))
    pos[1:, :3] = 50.0 + np.arange(15)[:, None]
    pos[0, 3] = 0.9
    lsb = np.zeros((n, 4))
    lsb[:, :3] = [np.log(0.3), np.log(0.2), np.log(0.05)]
    lsb[:, 3] = 6.0
    qv = np.array([0.9, 0.2, -0.3, 0.1])
    q = np.tile(qv, (n, 1))
    knn = np.tile(np.arange(n), (n, 1))
    z = np.array([[10.0, -6.0, 7.48331477]])
    out = OG.evaluate(pos, lsb, q, knn, [0], z, with_grad=False)
    assert out["d"][0] == 0.0 and np.isfinite(out["f"][0]) and np.isfinite(out["l_nor"])
    R = Rotation.from_quat(qv[[1, 2, 3, 0]]).as_matrix()
    s = np.exp(lsb[0, :3]) * 2 / (1 + np.exp(-0.1 * 4.0))
    x = R @ (s * z[0])
    A = R @ np.diag(1 / s ** 2) @ R.T
    u = A @ x / np.linalg.norm(A @ x)
    nrm = R[:, 2] * np.sign(R[:, 2] @ x)
    np.testing.assert_allclose(out["cos"][0], u @ nrm, rtol=0, atol=1e-12)


def test_losses_are_the_means_of_eq12_and_eq13_over_samples():
    # Eq. 12 and Eq. 13 average over the sample points. Two isolated axis-aligned splats (phi off,
    # identity rotations, smallest scale on z), each listed with 15 far splats of zero opacity, and
    # three samples x = mu + s * z. For one splat of opacity o and shape beta: Q = |z|^2, d =
    # o exp(-Q^(beta/2) / 2), so f = s_z sqrt(Q^(beta/2) - 2 ln o); e = s_z |z_3| gives
    # fbar = s_z |z_3|^(beta/2); -grad d is along Sigma^-1 (x - mu) = z / s, and n* = (0, 0, sign z_3).
    n = 17
    pos = np.zeros((n, 4))
    pos[1, :3] = [5.0, 0.0, 0.0]
    pos[2:, :3] = 100.0 + 3.0 * np.arange(15)[:, None]
    pos[0, 3], pos[1, 3] = 0.8, 0.6
    lsb = np.zeros((n, 4))
    lsb[:, :3] = np.log([0.3, 0.2, 0.05])
    lsb[0, 3], lsb[1, 3], lsb[2:, 3] = 2.0, 4.0, 2.0
    q = np.tile([1.0, 0, 0, 0], (n, 1))
    knn = np.zeros((n, 16), np.int64)
    knn[:, 1:] = np.arange(2, 17)
    knn[1, 0] = 1
    js = np.array([0, 0, 1])
    z = np.array([[0.4, -0.3, 0.5], [-0.2, 0.1, -0.25], [0.3, 0.2, 0.6]])
    s = np.array([0.3, 0.2, 0.05])
    o, beta = pos[js, 3], lsb[js, 3]
    Q = (z ** 2).sum(1)
    f = s[2] * np.sqrt(Q ** (beta / 2) - 2 * np.log(o))
    fbar = s[2] * np.abs(z[:, 2]) ** (beta / 2)
    u = (z / s) / np.linalg.norm(z / s, axis=1, keepdims=True)
    nstar = np.zeros((3, 3))
    nstar[:, 2] = np.sign(z[:, 2])
    want_sdf = np.mean(np.abs(fbar - f))
    want_nor = np.mean(((u - nstar) ** 2).sum(1))
    out = OG.evaluate(pos, lsb, q, knn, js, z, phi_mode=0, lambda_sdf=1.0, lambda_nor=0.5, with_grad=False)
    np.testing.assert_allclose(out["f"], f, rtol=1e-12)
    np.testing.assert_allclose(out["fbar"], fbar, rtol=1e-12)
    np.testing.assert_allclose(out["cos"], (u * nstar).sum(1), rtol=1e-12)
    np.testing.assert_allclose(out["l_sdf"], want_sdf, rtol=1e-12)
    np.testing.assert_allclose(out["l_nor"], want_nor, rtol=1e-12)
    np.testing.assert_allclose(out["loss"], want_sdf + 0.5 * want_nor, rtol=1e-12)
    assert not out["flags"].any()
