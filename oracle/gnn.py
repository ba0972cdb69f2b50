"""Oracle: the learned pose grouping for MCG (message passing over the camera co-visibility graph).

Test infrastructure only (see ``oracle/__init__``).

The paper splits the poses into N subsets of consecutive poses and notes that the best
decomposition is not obvious (Section 3.2); it has no learned component.  This module states,
in float64, the small network the library trains to choose the subsets, so that the library's
float32 forward pass, loss and gradients can be checked against it:

Graph of one reduced camera system S (Eq. 13), nodes = cameras:
    Lam_j   = diag(S_jj)^(-1/2) (Jacobi scaling, per scalar row)
    c_jk    = |Lam_j S_jk Lam_k|_F for every stored block with j != k, c_jj = 0
    d_j     = sum_k c_jk                                   (coupling degree)
Node features (8 per camera) from the current camera parameters (omega, t, ...):
    centre  C_j = -R(omega_j)^T t_j, standardised per axis over the cameras (mean removed,
            divided by that axis' root mean square)                               (3)
    axis    the third row of R(omega_j), the viewing axis                          (3)
    log(1 + d_j), standardised (mean removed, divided by its standard deviation)  (1)
    1                                                                               (1)
Three message-passing layers, widths 8 -> 64 -> 64 -> 64:
    H^l = relu(H^{l-1} W_s^l + (A H^{l-1}) W_n^l + b^l),  A = D^{-1} C (row-normalised coupling)
and a linear read-out s = H^3 w_o + b_o (one score per camera).
Loss: the Rayleigh quotient of the coupling Laplacian,
    u = s - (d^T s / sum d),   L(s) = u^T (D - C) u / u^T D u,
whose minimum over s is the second generalised eigenvalue of (D - C, D) (the Fiedler value):
a low L puts strongly coupled cameras next to each other.  Grouping: sort the cameras by s and
cut the order into the paper's N subsets of consecutive positions.

Parameter vector (float, this order): per layer W_s (in x out, row-major), W_n (in x out), b
(out); then w_o (64), b_o (1).

Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8) with bias correction.

Pins (tests/test_oracle_gnn.py): the loss on a cycle graph against its closed-form spectrum;
the gradient of the whole network against central finite differences; the features against
their definitions on hand-made cameras.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .camera import rotation_matrix

N_FEATURES = 8
HIDDEN = 64
LAYERS = 3


def layer_shapes(in_features: int = N_FEATURES, hidden: int = HIDDEN, layers: int = LAYERS):
    shapes = []
    fi = in_features
    for _ in range(layers):
        shapes.append(("Ws", (fi, hidden)))
        shapes.append(("Wn", (fi, hidden)))
        shapes.append(("b", (hidden,)))
        fi = hidden
    shapes.append(("wo", (hidden,)))
    shapes.append(("bo", (1,)))
    return shapes


def param_count(**kw) -> int:
    return int(sum(np.prod(s) for _, s in layer_shapes(**kw)))


def unpack(theta: np.ndarray, **kw) -> list[np.ndarray]:
    out, o = [], 0
    for _, shp in layer_shapes(**kw):
        n = int(np.prod(shp))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(shp))
        o += n
    return out


def coupling(S, n_cams: int) -> sp.csr_matrix:
    """C with c_jk = |Lam_j S_jk Lam_k|_F (j != k), from the sparse float64 S (9 n x 9 n)."""
    S = sp.csr_matrix(S)
    lam = 1.0 / np.sqrt(S.diagonal())
    Sh = sp.diags(lam) @ S @ sp.diags(lam)
    B = sp.bsr_matrix(Sh, blocksize=(9, 9))
    B.sort_indices()
    rows = np.repeat(np.arange(n_cams), np.diff(B.indptr))
    vals = np.sqrt((B.data ** 2).sum(axis=(1, 2)))
    vals[rows == B.indices] = 0.0
    C = sp.csr_matrix((vals, B.indices, B.indptr), shape=(n_cams, n_cams))
    return C


def features(cams: np.ndarray, C: sp.csr_matrix) -> np.ndarray:
    """The 8 node features of every camera (see the module text)."""
    R = rotation_matrix(cams[:, :3])
    t = cams[:, 3:6]
    centre = -np.einsum("nji,nj->ni", R, t)          # -R^T t
    centre = centre - centre.mean(axis=0)
    rms = np.sqrt((centre ** 2).mean(axis=0))
    centre = centre / np.where(rms > 0, rms, 1.0)
    axis = R[:, 2, :]
    d = np.asarray(C.sum(axis=1)).ravel()
    ld = np.log1p(d)
    ld = ld - ld.mean()
    sd = np.sqrt((ld ** 2).mean())
    ld = ld / sd if sd > 0 else ld
    return np.concatenate([centre, axis, ld[:, None], np.ones((cams.shape[0], 1))], axis=1)


def forward(theta: np.ndarray, X: np.ndarray, C: sp.csr_matrix):
    """Scores s and the activations needed by ``backward``."""
    P = unpack(theta)
    d = np.asarray(C.sum(axis=1)).ravel()
    A = sp.diags(1.0 / np.maximum(d, 1e-30)) @ C
    H = [X]
    AH, Z = [], []
    for l in range(LAYERS):
        Ws, Wn, b = P[3 * l], P[3 * l + 1], P[3 * l + 2]
        ah = A @ H[-1]
        z = H[-1] @ Ws + ah @ Wn + b
        AH.append(ah)
        Z.append(z)
        H.append(np.maximum(z, 0.0))
    s = H[-1] @ P[-2] + P[-1][0]
    return s, {"H": H, "AH": AH, "Z": Z, "A": A, "P": P}


def loss(s: np.ndarray, C: sp.csr_matrix) -> float:
    d = np.asarray(C.sum(axis=1)).ravel()
    u = s - (d @ s) / d.sum()
    num = u @ (d * u) - u @ (C @ u)
    den = u @ (d * u)
    return float(num / den)


def loss_grad_s(s: np.ndarray, C: sp.csr_matrix):
    """L(s) and dL/ds.  The centring drops out of the gradient because d^T u = 0."""
    d = np.asarray(C.sum(axis=1)).ravel()
    u = s - (d @ s) / d.sum()
    Cu = C @ u
    den = u @ (d * u)
    num = den - u @ Cu
    L = num / den
    g = (2.0 * (d * u - Cu) - 2.0 * L * d * u) / den
    return float(L), g


def backward(theta: np.ndarray, cache: dict, g_s: np.ndarray) -> np.ndarray:
    """dL/dtheta from dL/ds (the layout of the parameter vector)."""
    P, H, AH, Z, A = cache["P"], cache["H"], cache["AH"], cache["Z"], cache["A"]
    grads = [None] * len(P)
    grads[-2] = H[-1].T @ g_s
    grads[-1] = np.array([g_s.sum()])
    dH = np.outer(g_s, P[-2])
    for l in range(LAYERS - 1, -1, -1):
        Ws, Wn = P[3 * l], P[3 * l + 1]
        dZ = dH * (Z[l] > 0.0)
        grads[3 * l] = H[l].T @ dZ
        grads[3 * l + 1] = AH[l].T @ dZ
        grads[3 * l + 2] = dZ.sum(axis=0)
        dH = dZ @ Ws.T + A.T @ (dZ @ Wn.T)
    return np.concatenate([g.ravel() for g in grads])


def loss_and_grad(theta: np.ndarray, X: np.ndarray, C: sp.csr_matrix):
    s, cache = forward(theta, X, C)
    L, g_s = loss_grad_s(s, C)
    return L, backward(theta, cache, g_s), s


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new theta, m, v."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def order(s: np.ndarray) -> np.ndarray:
    """Cameras sorted by score (ties by index): the grouping's camera order."""
    return np.lexsort((np.arange(s.size), s))
