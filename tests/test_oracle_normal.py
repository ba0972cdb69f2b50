"""Pins of the oracle's damped normal equation (Section 3.1, Eqs. 5-11)."""
import numpy as np
import pytest

from oracle import camera, lm, normal
from tests._problems import micro


def _setup(lam=1e-2, damping="marquardt", seed=0):
    sc = micro(seed)
    m = lm.measurements(sc)
    r = camera.residuals(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m)
    Jp, Jl = camera.jacobians(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt)
    ne = normal.normal_equation(Jp, Jl, r, sc.obs_cam, sc.obs_pt, sc.n_cams, sc.n_pts, lam, damping)
    return sc, r, Jp, Jl, ne


def test_blocks_equal_dense_JtJ():
    sc, r, Jp, Jl, ne = _setup(lam=0.0)
    J = normal.dense_jacobian(Jp, Jl, sc.obs_cam, sc.obs_pt, sc.n_cams, sc.n_pts)
    H_dense = J.T @ J
    b_dense = J.T @ r.ravel()
    H, b = normal.dense_H(ne, sc.n_cams, sc.n_pts)
    scale = np.abs(H_dense).max()
    assert np.abs(H - H_dense).max() < 1e-12 * scale
    assert np.abs(b - b_dense).max() < 1e-12 * np.abs(b_dense).max()


def damped_lstsq_error(normal_fn=normal.normal_equation, lam=1e-2, damping="marquardt"):
    """|dx(H dx = -b) - argmin |r + J dx|^2 + lam |D dx|^2| / |dx| (Eq. 5 vs Eq. 6)."""
    sc = micro(1)
    m = lm.measurements(sc)
    r = camera.residuals(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m)
    Jp, Jl = camera.jacobians(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt)
    J = normal.dense_jacobian(Jp, Jl, sc.obs_cam, sc.obs_pt, sc.n_cams, sc.n_pts)
    # D^T D from the definition of the damping reading, on the dense J
    d = np.sum(J * J, axis=0)
    dd = np.clip(d, 1e-6, 1e32) if damping == "marquardt" else np.ones_like(d)
    A = np.vstack([J, np.sqrt(lam) * np.diag(np.sqrt(dd))])
    rhs = -np.concatenate([r.ravel(), np.zeros(d.size)])
    dx_ls = np.linalg.lstsq(A, rhs, rcond=None)[0]
    ne = normal_fn(Jp, Jl, r, sc.obs_cam, sc.obs_pt, sc.n_cams, sc.n_pts, lam, damping)
    H, b = normal.dense_H(ne, sc.n_cams, sc.n_pts)
    dx = np.linalg.solve(H, -b)
    return np.linalg.norm(dx - dx_ls) / np.linalg.norm(dx_ls)


@pytest.mark.parametrize("damping", ["marquardt", "identity"])
@pytest.mark.parametrize("lam", [1e-4, 1e-1, 10.0])
def test_normal_solution_is_damped_least_squares(damping, lam):
    assert damped_lstsq_error(lam=lam, damping=damping) < 1e-8


def test_marquardt_damping_scales_the_diagonal():
    lam = 0.25
    sc, r, Jp, Jl, ne0 = _setup(lam=0.0)
    _, _, _, _, ne = _setup(lam=lam)
    iu = np.arange(9)
    d = ne0.U[:, iu, iu]
    assert np.allclose(ne.U[:, iu, iu], d + lam * np.clip(d, 1e-6, 1e32), rtol=1e-14)
    assert (d < 1e-6).any()  # the clamp is exercised (the k2 column of a small image)
    off = ~np.eye(9, dtype=bool)
    assert np.array_equal(ne.U[:, off], ne0.U[:, off])
    il = np.arange(3)
    dv = ne0.V[:, il, il]
    assert np.allclose(ne.V[:, il, il], dv + lam * np.clip(dv, 1e-6, 1e32), rtol=1e-14)


def test_planted_missing_damping_is_caught():
    def broken(Jp, Jl, r, oc, op, nc, npt, lam, damping):
        return normal.normal_equation(Jp, Jl, r, oc, op, nc, npt, 0.0, damping)

    assert damped_lstsq_error(broken, lam=1.0) > 1e-4


def test_planted_sign_error_in_b_is_caught():
    def broken(*a):
        ne = normal.normal_equation(*a)
        ne.b_l = -ne.b_l
        return ne

    assert damped_lstsq_error(broken) > 1e-4
