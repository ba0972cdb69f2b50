"""Pins of the oracle's reduced camera system (Section 3.1, Eqs. 12-15)."""
import numpy as np
import pytest

from oracle import camera, lm, normal, schur
from tests._problems import micro, scene


def _micro_ne(seed=0, lam=1e-4, n_cams=4, n_pts=12):
    sc = micro(seed, n_cams, n_pts)
    m = lm.measurements(sc)
    lin = lm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, lam)
    return sc, lin


def schur_vs_dense_error(schur_fn=schur.schur_complement, seed=0):
    sc, lin = _micro_ne(seed, n_cams=5, n_pts=30)
    H, b = normal.dense_H(lin.ne, sc.n_cams, sc.n_pts)
    S_ref, bt_ref = schur.dense_schur(H, b, sc.n_cams)
    S, bt = schur_fn(lin.ne, sc.n_cams, sc.n_pts)
    S = S.toarray()
    return (np.abs(S - S_ref).max() / np.abs(S_ref).max(),
            np.abs(bt - bt_ref).max() / np.abs(bt_ref).max())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_schur_equals_dense_elimination(seed):
    eS, eb = schur_vs_dense_error(seed=seed)
    assert eS < 1e-9 and eb < 1e-9


def test_reduced_solution_equals_full_solve():
    sc, lin = _micro_ne(3, lam=1e-2)
    H, b = normal.dense_H(lin.ne, sc.n_cams, sc.n_pts)
    dx = np.linalg.solve(H, -b)
    dxp = np.linalg.solve(lin.S.toarray(), -lin.btilde)
    m = 9 * sc.n_cams
    assert np.linalg.norm(dxp - dx[:m]) < 1e-8 * np.linalg.norm(dx[:m])
    # and back-substitution (Eq. 15, sign corrected) gives the landmark part
    dxl = lm.back_substitute(lin.ne, dxp, sc.n_pts)
    assert np.linalg.norm(dxl.ravel() - dx[m:]) < 1e-8 * np.linalg.norm(dx[m:])


def test_paper_sign_of_eq15_is_wrong():
    """The printed -V^{-1}(-b_l + W^T dx_p) does not solve the second block row of Eq. 6."""
    sc, lin = _micro_ne(3, lam=1e-2)
    H, b = normal.dense_H(lin.ne, sc.n_cams, sc.n_pts)
    dx = np.linalg.solve(H, -b)
    m = 9 * sc.n_cams
    ne = lin.ne
    acc = -ne.b_l.copy()
    np.add.at(acc, ne.obs_pt, np.einsum("nij,ni->nj", ne.W, dx[:m].reshape(-1, 9)[ne.obs_cam]))
    printed = -np.linalg.solve(ne.V, acc[:, :, None])[:, :, 0]
    assert np.linalg.norm(printed.ravel() - dx[m:]) > 1e-3 * np.linalg.norm(dx[m:])


def test_single_blocks_match_the_sparse_product():
    sc = scene("tiny")
    m = lm.measurements(sc)
    lin = lm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, 1e-4)
    S = lin.S.toarray()
    for j, k in [(0, 0), (0, 5), (7, 3), (15, 15)]:
        blk = schur.schur_block(lin.ne, j, k)
        ref = S[9 * j:9 * j + 9, 9 * k:9 * k + 9]
        assert np.abs(blk - ref).max() < 1e-10 * np.abs(S).max()
    for j in [0, 9]:
        assert np.allclose(schur.btilde_block(lin.ne, j), lin.btilde[9 * j:9 * j + 9], rtol=1e-10, atol=1e-10)


def test_schur_is_symmetric_and_zero_off_covisibility():
    sc = scene("sequential", n_cams=60, n_pts=3000)
    m = lm.measurements(sc)
    lin = lm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, 1e-4)
    S = lin.S.toarray()
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    # S_jk = 0 unless cameras j and k share a landmark (Section 3.2)
    share = np.zeros((sc.n_cams, sc.n_cams), bool)
    cams_of = {}
    for c, p in zip(sc.obs_cam, sc.obs_pt):
        cams_of.setdefault(p, []).append(c)
    for cs in cams_of.values():
        for a in cs:
            share[a, cs] = True
    blocks = np.abs(S.reshape(sc.n_cams, 9, sc.n_cams, 9)).max(axis=(1, 3))
    assert np.all(blocks[~share] == 0)
    assert np.all(blocks[share] > 0)


def test_planted_sign_error_in_btilde_is_caught():
    def broken(ne, n_cams, n_pts):
        S, bt = schur.schur_complement(ne, n_cams, n_pts)
        W = schur.W_matrix(ne, n_cams, n_pts)
        Vinv = schur.block_diag_matrix(np.linalg.inv(ne.V))
        return S, ne.b_p.ravel() + W @ Vinv @ ne.b_l.ravel()

    eS, eb = schur_vs_dense_error(broken)
    assert eb > 1e-3


def test_planted_dropped_inverse_is_caught():
    def broken(ne, n_cams, n_pts):
        W = schur.W_matrix(ne, n_cams, n_pts)
        S = schur.block_diag_matrix(ne.U) - W @ W.T
        return S.tocsr(), ne.b_p.ravel() - W @ ne.b_l.ravel()

    eS, eb = schur_vs_dense_error(broken)
    assert eS > 1e-3
