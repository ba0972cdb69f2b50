"""Pins of the oracle's LM loop (Section 4.1) and the claim of Section 4.4."""
import numpy as np

from oracle import camera, lm
from tests._problems import scene


def test_lm_decreases_cost_to_noise_level():
    sc = scene("tiny")
    m = lm.measurements(sc)
    tr = lm.lm(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, solver="pcg")
    assert np.all(np.diff(tr.costs) <= 0)
    F_true = camera.cost(sc.cams_true, sc.pts_true, sc.obs_cam, sc.obs_pt, m)
    # the optimum fits the noise at least as well as the true parameters do
    assert tr.costs[-1] <= F_true * (1 + 1e-6)


def test_pcg_and_mcg_give_the_same_cost_each_iteration():
    """Section 4.4: "MCG and PCG give the same error at each BA iteration"."""
    sc = scene("tiny")
    m = lm.measurements(sc)
    a = lm.lm(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, solver="pcg", max_iters=8)
    b = lm.lm(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, solver="mcg", n_dirs=8, tau=3.0, max_iters=8)
    n = min(len(a.costs), len(b.costs))
    assert n >= 4
    rel = np.abs(np.array(a.costs[:n]) - np.array(b.costs[:n])) / np.array(a.costs[:n])
    assert rel.max() < 1e-6
