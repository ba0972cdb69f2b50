"""Shared set-up of the GPU parity tests: each side forms its own measurements."""
import functools

import numpy as np
import scipy.sparse as sp

from oracle import lm as olm
from oracle import solvers as osol
from paper_2110_04015_gb300 import synthetic as sy

CASES = {
    # name: (generator, kwargs) - sizes the oracle handles in seconds, several tiles and ragged tails
    "tiny": ("tiny", {}),
    "tiny-s3": ("tiny", {"n_cams": 13, "n_pts": 777}),
    "seq-small": ("sequential", {"n_cams": 120, "n_pts": 8000}),
    "dense-small": ("dense", {"n_cams": 150, "n_pts": 20000, "n_clusters": 5}),
    "sequential": ("sequential", {}),
}


@functools.lru_cache(maxsize=None)
def scene(case, seed=0):
    gen, kw = CASES[case]
    return sy.make(gen, seed, **kw)


@functools.lru_cache(maxsize=None)
def oracle_system(case, seed=0, lam=1e-4, damping="marquardt"):
    sc = scene(case, seed)
    m = olm.measurements(sc)
    lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, lam, damping)
    Dinv = osol.block_jacobi_inverse(lin.S, sc.n_cams)
    return m, lin, Dinv


def bsr_from_gpu(row_ptr, col, blocks, n_cams):
    return sp.bsr_matrix((blocks, col.astype(np.int64), row_ptr), shape=(9 * n_cams, 9 * n_cams)).tocsr()


def rel_max(a, b):
    """max |a - b| relative to max |b| (elementwise comparison against the oracle)."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def energy_err(S, x, ref):
    d = x - ref
    return float(np.sqrt(d @ (S @ d) / (ref @ (S @ ref))))
