"""Oracle: damped normal equation (Section 3.1, Eqs. 5-11).

Test infrastructure only (see ``oracle/__init__``).

    H = [[U_lambda, W], [W^T, V_lambda]],  H (dx_p, dx_l) = -(b_p, b_l)
    U_lambda = J_p^T J_p + lambda D_p^T D_p
    V_lambda = J_l^T J_l + lambda D_l^T D_l
    W = J_p^T J_l,  b_p = J_p^T r0,  b_l = J_l^T r0

J is block sparse: observation i = (j, l) touches camera j's 9 columns and
landmark l's 3 columns only, so U and V are block diagonal (9x9 per camera,
3x3 per landmark) and W has one 9x3 block per (camera, landmark) pair.

The damping matrices D are not specified by the paper ("diagonal damping
matrices", Eq. 5).  Reading used: Marquardt's scaling,
D^T D = diag(J^T J) with each entry clamped to [1e-6, 1e32]; ``damping =
"identity"`` gives Levenberg's D = I instead.

Pins: the assembled blocks against a dense J^T J of the explicitly stacked
dense Jacobian, and the normal-equation solution against the least-squares
solution of the damped problem (Eq. 5) computed by ``numpy.linalg.lstsq``
from J and r alone, which fixes every sign and the lambda placement.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

DIAG_MIN = 1e-6
DIAG_MAX = 1e32


@dataclass
class NormalEquation:
    U: np.ndarray        # (n_p, 9, 9) U_lambda
    V: np.ndarray        # (n_l, 3, 3) V_lambda
    W: np.ndarray        # (n_obs, 9, 3) J_p^T J_l of each observation
    b_p: np.ndarray      # (n_p, 9)
    b_l: np.ndarray      # (n_l, 3)
    obs_cam: np.ndarray
    obs_pt: np.ndarray


def damping_diagonal(diag: np.ndarray, damping: str) -> np.ndarray:
    """Diagonal of D^T D for the blocks whose J^T J diagonal is ``diag``."""
    if damping == "marquardt":
        return np.clip(diag, DIAG_MIN, DIAG_MAX)
    if damping == "identity":
        return np.ones_like(diag)
    raise ValueError(damping)


def normal_equation(Jp, Jl, r, obs_cam, obs_pt, n_cams, n_pts, lam, damping="marquardt") -> NormalEquation:
    """U_lambda, V_lambda, W, b_p, b_l of Eqs. 7-11 from per-observation blocks."""
    U = np.zeros((n_cams, 9, 9))
    V = np.zeros((n_pts, 3, 3))
    np.add.at(U, obs_cam, np.einsum("nki,nkj->nij", Jp, Jp))
    np.add.at(V, obs_pt, np.einsum("nki,nkj->nij", Jl, Jl))
    W = np.einsum("nki,nkj->nij", Jp, Jl)
    b_p = np.zeros((n_cams, 9))
    b_l = np.zeros((n_pts, 3))
    np.add.at(b_p, obs_cam, np.einsum("nki,nk->ni", Jp, r))
    np.add.at(b_l, obs_pt, np.einsum("nki,nk->ni", Jl, r))
    iu = np.arange(9)
    il = np.arange(3)
    U[:, iu, iu] += lam * damping_diagonal(U[:, iu, iu].copy(), damping)
    V[:, il, il] += lam * damping_diagonal(V[:, il, il].copy(), damping)
    return NormalEquation(U, V, W, b_p, b_l, np.asarray(obs_cam), np.asarray(obs_pt))


def dense_jacobian(Jp, Jl, obs_cam, obs_pt, n_cams, n_pts) -> np.ndarray:
    """The full J (2 n_obs, 9 n_p + 3 n_l) with the blocks in their places."""
    n = Jp.shape[0]
    J = np.zeros((2 * n, 9 * n_cams + 3 * n_pts))
    for i in range(n):
        j, l = int(obs_cam[i]), int(obs_pt[i])
        J[2 * i:2 * i + 2, 9 * j:9 * j + 9] = Jp[i]
        J[2 * i:2 * i + 2, 9 * n_cams + 3 * l:9 * n_cams + 3 * l + 3] = Jl[i]
    return J


def dense_H(ne: NormalEquation, n_cams: int, n_pts: int) -> tuple[np.ndarray, np.ndarray]:
    """Assemble the dense H and b = (b_p, b_l) of Eq. 6 from the blocks."""
    npar = 9 * n_cams + 3 * n_pts
    H = np.zeros((npar, npar))
    for j in range(n_cams):
        H[9 * j:9 * j + 9, 9 * j:9 * j + 9] = ne.U[j]
    o = 9 * n_cams
    for l in range(n_pts):
        H[o + 3 * l:o + 3 * l + 3, o + 3 * l:o + 3 * l + 3] = ne.V[l]
    for i in range(ne.W.shape[0]):
        j, l = int(ne.obs_cam[i]), int(ne.obs_pt[i])
        H[9 * j:9 * j + 9, o + 3 * l:o + 3 * l + 3] += ne.W[i]
        H[o + 3 * l:o + 3 * l + 3, 9 * j:9 * j + 9] += ne.W[i].T
    b = np.concatenate([ne.b_p.ravel(), ne.b_l.ravel()])
    return H, b
