"""Oracle: reduced camera system (Section 3.1, Eqs. 12-14).

Test infrastructure only (see ``oracle/__init__``).

    S dx_p = -b~,   S = U_lambda - W V_lambda^{-1} W^T,   b~ = b_p - W V_lambda^{-1} b_l

W is the sparse (9 n_p x 3 n_l) matrix whose (camera j, landmark l) block is
the sum of J_p^T J_l over the observations of l by j; V_lambda^{-1} is block
diagonal.  The products are library sparse matrix products (scipy.sparse).
S_jk is nonzero only when cameras j and k share a landmark (Section 3.2).

Pins: S and b~ against the textbook dense elimination of the landmark block
of H (``dense_schur``), and the solution of S dx_p = -b~ against the camera
part of the dense solve of the whole H dx = -b (Eq. 6).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .normal import NormalEquation


def W_matrix(ne: NormalEquation, n_cams: int, n_pts: int) -> sp.csr_matrix:
    n = ne.W.shape[0]
    rows = (9 * ne.obs_cam[:, None, None] + np.arange(9)[None, :, None]).repeat(3, axis=2)
    cols = (3 * ne.obs_pt[:, None, None] + np.arange(3)[None, None, :]).repeat(9, axis=1)
    return sp.csr_matrix((ne.W.ravel(), (rows.ravel(), cols.ravel())), shape=(9 * n_cams, 3 * n_pts))


def block_diag_matrix(blocks: np.ndarray) -> sp.csr_matrix:
    n, k, _ = blocks.shape
    rows = (k * np.arange(n)[:, None, None] + np.arange(k)[None, :, None]).repeat(k, axis=2)
    cols = (k * np.arange(n)[:, None, None] + np.arange(k)[None, None, :]).repeat(k, axis=1)
    return sp.csr_matrix((blocks.ravel(), (rows.ravel(), cols.ravel())), shape=(n * k, n * k))


def schur_complement(ne: NormalEquation, n_cams: int, n_pts: int):
    """(S, b~) of Eqs. 13-14; S as a scipy CSR matrix of size 9 n_p."""
    W = W_matrix(ne, n_cams, n_pts)
    Vinv = block_diag_matrix(np.linalg.inv(ne.V))
    WVinv = W @ Vinv
    S = block_diag_matrix(ne.U) - WVinv @ W.T
    btilde = ne.b_p.ravel() - WVinv @ ne.b_l.ravel()
    return S.tocsr(), btilde


def schur_block(ne: NormalEquation, j: int, k: int) -> np.ndarray:
    """One 9x9 block S_jk = delta_jk U_j - sum_l W_jl V_l^{-1} W_kl^T (Eq. 13).

    The sum runs over the landmarks l observed by both cameras; W_jl sums
    the observation blocks of the pair (j, l).
    """
    S = ne.U[j].copy() if j == k else np.zeros((9, 9))
    on_j = ne.obs_cam == j
    on_k = ne.obs_cam == k
    common = np.intersect1d(ne.obs_pt[on_j], ne.obs_pt[on_k])
    for l in common:
        Wjl = ne.W[on_j & (ne.obs_pt == l)].sum(axis=0)
        Wkl = ne.W[on_k & (ne.obs_pt == l)].sum(axis=0)
        S -= Wjl @ np.linalg.solve(ne.V[l], Wkl.T)
    return S


def btilde_block(ne: NormalEquation, j: int) -> np.ndarray:
    """b~_j = b_p,j - sum_l W_jl V_l^{-1} b_l (Eq. 14)."""
    out = ne.b_p[j].copy()
    on_j = ne.obs_cam == j
    for i in np.nonzero(on_j)[0]:
        l = ne.obs_pt[i]
        out -= ne.W[i] @ np.linalg.solve(ne.V[l], ne.b_l[l])
    return out


def dense_schur(H: np.ndarray, b: np.ndarray, n_cams: int):
    """Textbook elimination of the landmark unknowns from the dense H (Eq. 6)."""
    m = 9 * n_cams
    Hpp, Hpl, Hll = H[:m, :m], H[:m, m:], H[m:, m:]
    X = np.linalg.solve(Hll, np.concatenate([Hpl.T, b[m:, None]], axis=1))
    S = Hpp - Hpl @ X[:, :-1]
    bt = b[:m] - Hpl @ X[:, -1]
    return S, bt


def density(S: sp.spmatrix, n_cams: int) -> float:
    """Fraction of nonzero 9x9 blocks of S (the paper's density d, read as nnzb / n_p^2)."""
    A = sp.csr_matrix(S)
    r, c = A.nonzero()
    blocks = np.unique((r // 9).astype(np.int64) * n_cams + c // 9)
    return blocks.size / float(n_cams * n_cams)
