"""Oracle: block-Jacobi PCG (Algorithm 1) and MCG (Algorithm 2), Section 3.2.

Test infrastructure only (see ``oracle/__init__``).

Both solve S dx_p = -b~ (Eq. 12/16) from x0 = 0 (the paper leaves x0 open;
zero is the reading used).  The stop test, r_{i+1} against eps * r0, is read as the
Euclidean norm of the recursive (unpreconditioned) residual, eps = 1e-6 and
imax = 1000 by default (Section 4.1).

Readings of points the paper leaves open:

* D(S)^{-1} is the inverse of each 9x9 diagonal block of S (Section 3.2),
  here ``numpy.linalg.inv`` of the block.
* Delta_i = Q_i^T P_i is symmetrised, (Delta + Delta^T) / 2, before its
  pseudo-inverse; it is symmetric in exact arithmetic.
* The pseudo-inverse (the paper uses Eigen's) drops eigenvalues at or below
  w * 2^-52 * lambda_max of the w x w symmetric Delta; for a full-rank Delta it
  is the inverse and for w = 1 a division.
* The poses are split into subsets of s = ceil(n_p / N) consecutive poses,
  the last holding the remainder (the paper makes N - 1 equal subsets and puts
  the leftover poses in the last, end of Section 3.2); ceil(n_p / s) <= N of
  them are non-empty.
* The tau-test is strict: t_i < tau takes the N local directions, otherwise a
  single global direction (a PCG step).
* Eq. 18 prints Q_i = S Z_i - sum_{j<i} Q_j beta_{i,j}; applying S to the P
  update of Algorithm 2 pairs Z_{i+1} with beta_{i,j}, j = 0..i, which is what
  ``q_trick=True`` computes.  ``q_trick=False`` instead takes Q_i = S P_i as
  Algorithm 2 states it.

Pins: the solutions against a dense Cholesky solve of S; MCG with N = 1 or
tau = 0 against PCG iterate by iterate; non-increasing S-energy error; t_i of the
tau-test against the energy decrease of each step over the preconditioned norm of the
new residual, both formed independently, and a hand-worked two-camera value;
S-conjugacy of the search blocks; finite termination of PCG; the
pseudo-inverse against the Moore-Penrose identities and an SVD pseudo-inverse.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp


def diagonal_blocks(S, n_cams: int) -> np.ndarray:
    """The 9x9 diagonal blocks S_jj, (n_p, 9, 9)."""
    if sp.issparse(S):
        B = sp.bsr_matrix(S, blocksize=(9, 9))
        out = np.zeros((n_cams, 9, 9))
        for j in range(n_cams):
            for q in range(B.indptr[j], B.indptr[j + 1]):
                if B.indices[q] == j:
                    out[j] += B.data[q]
        return out
    S = np.asarray(S)
    return np.stack([S[9 * j:9 * j + 9, 9 * j:9 * j + 9] for j in range(n_cams)])


def block_jacobi_inverse(S, n_cams: int) -> np.ndarray:
    """D(S)^{-1} as its n_p inverse 9x9 blocks (Section 3.2)."""
    return np.linalg.inv(diagonal_blocks(S, n_cams))


def apply_block_diag(Dinv: np.ndarray, r: np.ndarray) -> np.ndarray:
    """D(S)^{-1} r, blockwise."""
    n = Dinv.shape[0]
    return np.einsum("nij,nj->ni", Dinv, r.reshape(n, 9)).ravel()


def pinv_sym(A: np.ndarray) -> np.ndarray:
    """Pseudo-inverse of a symmetric w x w matrix through its eigendecomposition."""
    w = A.shape[0]
    lam, V = np.linalg.eigh(A)
    top = max(float(lam.max()), 0.0) if w else 0.0
    thr = w * 2.0 ** -52 * top
    keep = lam > thr
    inv = np.zeros_like(lam)
    inv[keep] = 1.0 / lam[keep]
    return (V * inv[None, :]) @ V.T


def subsets(n_cams: int, n_dirs: int) -> tuple[np.ndarray, int]:
    """Pose -> subset index and the number of non-empty subsets (end of Section 3.2)."""
    s = -(-n_cams // max(1, n_dirs))
    sub = np.arange(n_cams) // s
    return sub, int(-(-n_cams // s))


def tau_ratio(gamma: np.ndarray, alpha: np.ndarray, r_next: np.ndarray, z_next: np.ndarray) -> float:
    """The adaptive tau-test quantity of Algorithm 2 (Section 3.2):

        t_i = gamma_i^T alpha_i / (r_{i+1}^T D(S)^{-1} r_{i+1}),

    the decrease of the S-energy error made by step i over the preconditioned norm of the new
    residual (z_next = D(S)^{-1} r_next)."""
    return float(gamma @ alpha) / float(r_next @ z_next)


@dataclass
class SolveResult:
    x: np.ndarray
    iters: int
    rel_res: list = field(default_factory=list)     # |r_{i+1}| / |r_0| after each step
    widths: list = field(default_factory=list)      # width of P_i used by step i
    local_steps: int = 0
    xs: list = field(default_factory=list)          # iterates x_{i+1} when recorded
    P: list = field(default_factory=list)           # search blocks when recorded
    t: list = field(default_factory=list)           # MCG: t_i of every step that reached the tau-test
    converged: bool = False


def pcg(S, btilde, Dinv, eps=1e-6, imax=1000, record=False) -> SolveResult:
    """Algorithm 1: block-Jacobi preconditioned conjugate gradients on S dx = -b~."""
    n = btilde.size
    x = np.zeros(n)
    r = -btilde - S @ x
    rn0 = np.linalg.norm(r)
    res = SolveResult(x, 0)
    if rn0 == 0.0:
        res.converged = True
        return res
    Z = apply_block_diag(Dinv, r)
    P = Z
    i = 0
    while i < imax:
        Q = S @ P
        Delta = Q @ P
        gamma = P @ r
        alpha = gamma / Delta
        x = x + alpha * P
        r = r - alpha * Q
        i += 1
        res.rel_res.append(np.linalg.norm(r) / rn0)
        res.widths.append(1)
        if record:
            res.xs.append(x.copy())
            res.P.append(P[:, None].copy())
        if np.linalg.norm(r) < eps * rn0:
            res.converged = True
            break
        Z = apply_block_diag(Dinv, r)
        Phi = Q @ Z
        beta = Phi / Delta
        P = Z - beta * P
    res.x = x
    res.iters = i
    return res


def mcg(S, btilde, Dinv, n_dirs, tau, eps=1e-6, imax=1000, q_trick=True, record=False) -> SolveResult:
    """Algorithm 2: multidirectional conjugate gradients on S dx = -b~.

    Search blocks P_j, their images Q_j = S P_j and the pseudo-inverses of
    Delta_j are kept for the full reorthogonalisation over j = 0..i.
    """
    n = btilde.size
    n_cams = n // 9
    sub, n_eff = subsets(n_cams, n_dirs)
    row_sub = np.repeat(sub, 9)
    x = np.zeros(n)
    r = -btilde - S @ x
    rn0 = np.linalg.norm(r)
    res = SolveResult(x, 0)
    if rn0 == 0.0:
        res.converged = True
        return res
    Z = apply_block_diag(Dinv, r)[:, None]
    Ps = [Z]
    Qs = [S @ Z]
    Dps = []
    i = 0
    while i < imax:
        P_i, Q_i = Ps[-1], Qs[-1]
        Delta = Q_i.T @ P_i
        Delta = 0.5 * (Delta + Delta.T)
        gamma = P_i.T @ r
        Dp = pinv_sym(Delta)
        Dps.append(Dp)
        alpha = Dp @ gamma
        x = x + P_i @ alpha
        r = r - Q_i @ alpha
        i += 1
        res.rel_res.append(np.linalg.norm(r) / rn0)
        res.widths.append(P_i.shape[1])
        if record:
            res.xs.append(x.copy())
            res.P.append(P_i.copy())
        if np.linalg.norm(r) < eps * rn0:
            res.converged = True
            break
        z = apply_block_diag(Dinv, r)
        t = tau_ratio(gamma, alpha, r, z)
        res.t.append(t)
        if t < tau:
            Z = np.zeros((n, n_eff))
            Z[np.arange(n), row_sub] = z
            res.local_steps += 1
        else:
            Z = z[:, None]
        betas = [Dps[j] @ (Qs[j].T @ Z) for j in range(len(Ps))]
        P_next = Z - sum(Ps[j] @ betas[j] for j in range(len(Ps)))
        if q_trick:
            Q_next = S @ Z - sum(Qs[j] @ betas[j] for j in range(len(Ps)))
        else:
            Q_next = S @ P_next
        Ps.append(P_next)
        Qs.append(np.asarray(Q_next))
    res.x = x
    res.iters = i
    return res


def dense_solve(S, btilde) -> np.ndarray:
    """Exact reference: Cholesky solve of the dense S dx = -b~ (textbook)."""
    import scipy.linalg as sla
    A = S.toarray() if sp.issparse(S) else np.asarray(S)
    c = sla.cho_factor(A)
    return sla.cho_solve(c, -btilde)


def true_rel_residual(S, btilde, x) -> float:
    """|-b~ - S x| / |b~| in float64 (the reported solve metric)."""
    return float(np.linalg.norm(-btilde - S @ x) / np.linalg.norm(btilde))
