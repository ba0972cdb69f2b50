"""Pins of the oracle's camera model (Section 3.1, Eqs. 1-4; BAL model reading)."""
import os

import numpy as np
import pytest

from oracle import camera
from tests._problems import random_cameras


def _fd_jacobians(cams, pts, obs_cam, obs_pt, h_rel=1e-6):
    """Central finite differences of the residual, one parameter at a time (brute force)."""
    n = obs_cam.size
    Jp = np.zeros((n, 2, 9))
    Jl = np.zeros((n, 2, 3))
    for k in range(9):
        h = h_rel * np.maximum(1.0, np.abs(cams[obs_cam, k]))
        cp, cm = cams[obs_cam].copy(), cams[obs_cam].copy()
        cp[:, k] += h
        cm[:, k] -= h
        idx = np.arange(n)
        fp = camera.project(cp, pts[obs_pt], idx, idx)
        fm = camera.project(cm, pts[obs_pt], idx, idx)
        Jp[:, :, k] = (fp - fm) / (2 * h)[:, None]
    for k in range(3):
        h = h_rel * np.maximum(1.0, np.abs(pts[obs_pt, k]))
        xp, xm = pts[obs_pt].copy(), pts[obs_pt].copy()
        xp[:, k] += h
        xm[:, k] -= h
        idx = np.arange(n)
        fp = camera.project(cams[obs_cam], xp, idx, idx)
        fm = camera.project(cams[obs_cam], xm, idx, idx)
        Jl[:, :, k] = (fp - fm) / (2 * h)[:, None]
    return Jp, Jl


def jacobian_fd_error(jac_fn=camera.jacobians, seed=0, angle_scale=1.0, n=200):
    rng = np.random.default_rng(seed)
    cams = random_cameras(rng, n, angle_scale)
    pts = rng.uniform(-1, 1, size=(n, 3))
    idx = np.arange(n)
    Jp, Jl = jac_fn(cams, pts, idx, idx)
    Fp, Fl = _fd_jacobians(cams, pts, idx, idx)
    scale_p = np.maximum(np.abs(Fp).max(axis=(1, 2), keepdims=True), 1e-3)
    scale_l = np.maximum(np.abs(Fl).max(axis=(1, 2), keepdims=True), 1e-3)
    return max(np.abs((Jp - Fp) / scale_p).max(), np.abs((Jl - Fl) / scale_l).max())


@pytest.mark.parametrize("angle_scale", [1.0, 1e-3, 2.5])
def test_jacobians_match_central_differences(angle_scale):
    assert jacobian_fd_error(angle_scale=angle_scale) < 1e-6


def test_jacobian_small_angle_branch():
    # |omega| below 1e-8 takes the first-order rotation; its derivative is -[X]_x
    rng = np.random.default_rng(3)
    cams = random_cameras(rng, 50, angle_scale=1e-10)
    pts = rng.uniform(-1, 1, size=(50, 3))
    idx = np.arange(50)
    Jp, Jl = camera.jacobians(cams, pts, idx, idx)
    Fp, Fl = _fd_jacobians(cams, pts, idx, idx, h_rel=1e-7)
    assert np.abs(Jp - Fp).max() / np.abs(Fp).max() < 1e-6
    assert np.abs(Jl - Fl).max() / np.abs(Fl).max() < 1e-6


def test_rotation_is_orthonormal_and_proper():
    rng = np.random.default_rng(1)
    R = camera.rotation_matrix(rng.normal(size=(100, 3)) * 2)
    eye = np.eye(3)[None]
    assert np.abs(np.einsum("nji,njk->nik", R, R) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-13


def test_rotation_about_z_closed_form():
    th = 0.7
    R = camera.rotation_matrix(np.array([[0.0, 0.0, th]]))[0]
    c, s = np.cos(th), np.sin(th)
    assert np.allclose(R, [[c, -s, 0], [s, c, 0], [0, 0, 1]], atol=1e-15)


def test_rotation_fixes_its_axis_and_inverts():
    rng = np.random.default_rng(2)
    w = rng.normal(size=(20, 3))
    R = camera.rotation_matrix(w)
    assert np.abs(np.einsum("nij,nj->ni", R, w) - w).max() < 1e-13
    Rm = camera.rotation_matrix(-w)
    assert np.abs(np.einsum("nij,njk->nik", R, Rm) - np.eye(3)[None]).max() < 1e-13


def test_projection_pinhole_closed_form():
    # identity pose, f = 1, no distortion: pi = -(X/Z, Y/Z)
    cams = np.array([[0, 0, 0, 0, 0, 0, 1.0, 0, 0]])
    pts = np.array([[0.3, -0.2, -2.0], [1.0, 2.0, -4.0]])
    out = camera.project(cams, pts, np.array([0, 0]), np.array([0, 1]))
    assert np.allclose(out, [[0.15, -0.1], [0.25, 0.5]], atol=1e-15)


def test_projection_distortion_closed_form():
    # p = (0.5, 0): rho = 1 + k1/4 + k2/16, translated camera
    k1, k2, f = 0.1, -0.05, 300.0
    cams = np.array([[0, 0, 0, 0, 0, -3.0, f, k1, k2]])
    pts = np.array([[-1.0, 0.0, 1.0]])  # P = (-1, 0, -2) -> p = (-0.5, 0)
    out = camera.project(cams, pts, np.array([0]), np.array([0]))
    rho = 1 + k1 * 0.25 + k2 * 0.0625
    assert np.allclose(out, [[f * rho * -0.5, 0.0]], atol=1e-12)


def test_residual_and_cost_definition():
    rng = np.random.default_rng(4)
    cams = random_cameras(rng, 3)
    pts = rng.uniform(-1, 1, size=(5, 3))
    oc = np.array([0, 1, 2, 0])
    op = np.array([0, 1, 2, 4])
    m = rng.normal(size=(4, 2))
    r = camera.residuals(cams, pts, oc, op, m)
    # each residual depends only on its own camera and point
    for i in range(4):
        pi = camera.project(cams[oc[i]:oc[i] + 1], pts[op[i]:op[i] + 1], np.array([0]), np.array([0]))
        assert np.allclose(r[i], pi[0] - m[i], atol=1e-12)
    assert np.isclose(camera.cost(cams, pts, oc, op, m), np.sum(r ** 2))


def test_planted_sign_error_is_caught():
    """A sign flip in one Jacobian column must fail the finite-difference pin."""

    def broken(*a):
        Jp, Jl = camera.jacobians(*a)
        Jp = Jp.copy()
        Jp[:, :, 7] *= -1
        return Jp, Jl

    assert jacobian_fd_error(broken) > 1e-3


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "bal_projection_worked_example.txt")


def test_projection_matches_hand_worked_example():
    # rows: camera (9), point (3), projection worked out by hand in the file's header
    rows = np.loadtxt(GOLDEN)
    for r in rows:
        pi = camera.project(r[None, :9], r[None, 9:12], np.array([0]), np.array([0]))[0]
        assert np.allclose(pi, r[12:14], rtol=1e-14, atol=1e-12), (pi, r[12:14])
