"""Training and use of the pose-grouping network (``ba_gnn_*`` in include/ba.h).

The network scores the cameras of a built reduced camera system; its camera order, cut into the
paper's N subsets of consecutive poses, is the grouping of Algorithm 2.  Everything computed
here runs in the library's kernels; this module only drives them:

* ``init_params``   Glorot-uniform weights, zero biases, from the seeded generator.
* ``harvest_train`` trains on the normal equations that Levenberg-Marquardt iterations of
                    synthetic problems generate (one Adam step per normal equation).
* ``grouped``       the scene renumbered in the network's camera order.
* ``solve_grouped`` MCG on the grouped problem, with plain MCG on the original camera order as
                    the fallback when the grouped solve does not converge.
"""
from __future__ import annotations

import numpy as np

from . import problem as pb
from . import synthetic as sy
from .binding import GNN, BA_OK, BAError

N_FEATURES, HIDDEN, LAYERS = 8, 64, 3


def layer_shapes():
    shapes, fi = [], N_FEATURES
    for _ in range(LAYERS):
        shapes += [("Ws", (fi, HIDDEN)), ("Wn", (fi, HIDDEN)), ("b", (HIDDEN,))]
        fi = HIDDEN
    return shapes + [("wo", (HIDDEN,)), ("bo", (1,))]


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights (bound sqrt(6 / (fan_in + fan_out))) and zero biases."""
    s = sy.Stream(seed, "gnn/init")
    out = []
    for name, shp in layer_shapes():
        n = int(np.prod(shp))
        if name in ("b", "bo"):
            out.append(np.zeros(n))
        else:
            fan_out = shp[1] if len(shp) > 1 else 1
            bound = np.sqrt(6.0 / (shp[0] + fan_out))
            out.append((2.0 * s.uniform(n) - 1.0) * bound)
    return np.concatenate(out).astype(np.float32)


def training_scene(kind: str, seed: int) -> sy.Scene:
    """One shuffled training problem of the sequential or clustered-dense family (camera order
    random, sizes drawn from the seed)."""
    s = sy.Stream(seed, "gnn/sizes")
    u = s.uniform(2)
    if kind == "sequential":
        n = int(80 + 160 * u[0])
        sc = sy.sequential(seed, n_cams=n, n_pts=60 * n, window=int(12 + 20 * u[1]))
    else:
        n = int(60 + 120 * u[0])
        sc = sy.dense(seed, n_cams=n, n_pts=100 * n, n_clusters=max(2, n // 30))
    return sy.shuffled(sc, seed)


def harvest_train(gnn: GNN, seeds, kinds=("sequential",), lm_steps: int = 4, lr: float = 3e-3, epochs: int = 1,
                  precision: str = "mixed", log=None) -> list[float]:
    """Adam steps on the normal equations of ``lm_steps`` LM iterations of each training problem.

    For every problem (seed, kind) the LM loop runs from the perturbed start; before each LM
    iteration the system is built at the current lambda and the network takes one training step
    on it.  Returns the losses in order.
    """
    losses = []
    for ep in range(epochs):
        for seed in seeds:
            for kind in kinds:
                sc = training_scene(kind, int(seed))
                p = pb.from_scene(sc, precision=precision)
                lam = 1e-4
                for _ in range(lm_steps):
                    p.ba_build_normal(lam)
                    losses.append(gnn.ba_gnn_train_step(p, lr))
                    st = p.ba_lm_step("pcg", lambda0=lam, tol=1e-2, max_iters=200)
                    lam = st["lambda_next"]
                p.close()
                if log:
                    log(ep, seed, kind, losses[-1])
    return losses


def grouped(gnn: GNN, sc: sy.Scene, precision: str = "mixed", bf16: bool = False, lam: float = 1e-4):
    """The scene renumbered in the network's camera order, and that order."""
    p = pb.from_scene(sc, precision=precision)
    p.ba_build_normal(lam)
    order, _ = gnn.ba_gnn_order(p, bf16=bf16)
    p.close()
    return sy.permute_cameras(sc, order), order


def solve_grouped(gnn: GNN, sc: sy.Scene, n_dirs: int, tau: float, precision: str = "mixed", tol: float = 1e-6,
                  max_iters: int = 1000, lam: float = 1e-4, bf16: bool = False) -> dict:
    """MCG with the learned grouping; plain MCG on the given camera order when that fails.

    Returns the solve stats, the camera-space solution in the scene's own camera order and which
    grouping produced it.
    """
    sg, order = grouped(gnn, sc, precision=precision, bf16=bf16, lam=lam)
    p = pb.from_scene(sg, precision=precision)
    p.ba_build_normal(lam)
    used = "learned"
    try:
        st = p.ba_solve_mcg(tol, max_iters, n_dirs, tau)
        x = p.ba_get_delta()
    except BAError as e:
        st = {"status": e.code, "true_rel_residual": float("inf")}
        x = None
    p.close()
    if st["status"] != BA_OK or not st["true_rel_residual"] <= tol:
        q = pb.from_scene(sc, precision=precision)
        q.ba_build_normal(lam)
        st = q.ba_solve_mcg(tol, max_iters, n_dirs, tau)
        x = q.ba_get_delta()
        q.close()
        used = "fallback"
    else:
        xs = np.empty_like(x)
        xs[order] = x
        x = xs
    return {"stats": st, "x": x, "grouping": used, "order": order}
