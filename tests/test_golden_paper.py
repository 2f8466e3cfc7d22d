"""The oracle against the constants the paper prints (tests/golden/paper_constants.json, each
value with its passage): its defaults for rho, the neighbour count and the level; the march
range of +-3 sigma_g(v) covering the printed 99.7 % of a beta = 2 splat's distribution along
v, with sigma_g(v) as the oracle computes it (reading LS3: the standard deviation of the
splat's marginal along v), checked by sampling the splat through the oracle's own frame; and
the Eq. 15 schedule at the printed start and end scales."""
import inspect
import json
import os

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import drt as ODRT
from oracle import gsr as OG
from oracle import levelset as OLS

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _default(fn, name):
    return inspect.signature(fn).parameters[name].default


def test_oracle_defaults_are_the_printed_constants():
    assert _default(OLS.extract, "rho") == GOLD["rho"]["value"]
    assert _default(OLS.extract, "level") == GOLD["level_alpha"]["value"]
    assert _default(OG.evaluate, "rho") == GOLD["rho"]["value"]
    assert OG.K == GOLD["knn_k"]["value"]
    pos = np.random.default_rng(0).normal(size=(40, 4))
    nb, _ = OLS.nearest(pos, np.zeros(3))
    assert len(nb) == GOLD["knn_k"]["value"]


def test_three_sigma_range_covers_the_printed_fraction():
    # one anisotropic beta = 2 splat (a Gaussian) and a few directions: the fraction of its
    # distribution whose offset along v lies within +-3 sigma_g(v) is the printed 99.7 %
    rng = np.random.default_rng(1)
    k = GOLD["march_half_width_sigmas"]["value"]
    for trial in range(4):
        q = Rotation.random(random_state=trial).as_quat()[[3, 0, 1, 2]]
        pos = np.zeros((17, 4))
        pos[0, 3] = 1.0
        pos[1:, :3] = 50.0 + np.arange(16)[:, None]
        lsb = np.zeros((17, 4))
        lsb[:, :3] = np.log([0.3, 0.1, 0.03])
        lsb[:, 3] = 2.0
        quat = np.tile(q, (17, 1))
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        sigma = OLS.march(pos, lsb, quat, np.zeros(3), v, phi_mode=0)["sigma"]
        N = OLS._Neighbours(pos, lsb, quat, np.array([0]), 0.1, 0)  # the oracle's own frame
        z = rng.standard_normal((400_000, 3))
        x = (z * N.sp[0]) @ N.R[0].T  # mu + R diag(s') z
        frac = np.mean(np.abs(x @ v) <= k * sigma)
        assert abs(frac - GOLD["march_coverage"]["value"]) < 1.5e-3, (trial, frac)
        # and the density the oracle marches is that distribution's: exp(-Q/2) at a sample
        # equals the Gaussian's exp(-|z|^2/2)
        for j in range(5):
            assert abs(OLS.density_at(pos, lsb, quat, np.arange(16), x[j], phi_mode=0)
                       - np.exp(-0.5 * (z[j] ** 2).sum())) < 1e-9


def test_eq15_schedule_at_the_printed_scales():
    start, end = GOLD["drt_start_scale"]["value"], GOLD["drt_end_scale"]["value"]
    total = GOLD["drt_fraction_of_training"]["value"] * 30000  # any training length
    assert abs(ODRT.scale(0, total, start, end) - start) < 1e-12
    assert abs(ODRT.scale(total, total, start, end) - end) < 1e-12
    mids = [ODRT.scale(t, total, start, end) for t in np.linspace(0, total, 50)]
    assert all(a <= b + 1e-15 for a, b in zip(mids, mids[1:]))  # rises monotonically
