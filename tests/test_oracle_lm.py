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
    """Section 4.4: MCG and PCG reach the same error at every BA iteration."""
    sc = scene("tiny")
    m = lm.measurements(sc)
    a = lm.lm(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, solver="pcg", max_iters=8)
    b = lm.lm(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, solver="mcg", n_dirs=8, tau=3.0, max_iters=8)
    n = min(len(a.costs), len(b.costs))
    assert n >= 4
    rel = np.abs(np.array(a.costs[:n]) - np.array(b.costs[:n])) / np.array(a.costs[:n])
    assert rel.max() < 1e-6


def test_lambda_schedule_on_rejected_and_accepted_steps():
    """The LM lambda rule read for Section 4.1: accept when F decreases and divide lambda by 10,
    otherwise keep the state and multiply lambda by 10 (clamped to [1e-12, 1e16])."""
    sc = scene("tiny")
    m = lm.measurements(sc)
    rng = np.random.default_rng(3)
    # a 20 % perturbation with no damping to start from: the first Gauss-Newton steps overshoot
    cams0 = sc.cams0 + 0.2 * np.abs(sc.cams0) * rng.standard_normal(sc.cams0.shape)
    tr = lm.lm(cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, solver="pcg", lam0=1e-12, max_iters=10)
    assert not all(tr.accepted) and any(tr.accepted)
    for i, ok in enumerate(tr.accepted):
        if i + 1 < len(tr.lambdas):
            want = max(tr.lambdas[i] / 10, 1e-12) if ok else min(tr.lambdas[i] * 10, 1e16)
            assert tr.lambdas[i + 1] == want, (i, tr.lambdas)
        if ok:
            assert tr.costs[i + 1] < tr.costs[i]
        else:
            assert tr.costs[i + 1] == tr.costs[i]
