"""Small seeded problems shared by the oracle pins."""
import functools

import numpy as np

from paper_2110_04015_gb300 import synthetic as sy


@functools.lru_cache(maxsize=None)
def scene(name="tiny", seed=0, **kw):
    return sy.make(name, seed, **dict(kw))


def micro(seed=0, n_cams=4, n_pts=12):
    """A problem small enough for dense H and a dense Jacobian."""
    return sy.tiny(seed=seed, n_cams=n_cams, n_pts=n_pts, track_min=2, track_max=min(4, n_cams))


def random_cameras(rng, n, angle_scale=1.0):
    omega = rng.normal(size=(n, 3)) * angle_scale
    t = rng.normal(size=(n, 3)) + np.array([0.0, 0.0, -8.0])
    intr = np.stack([500 + 50 * rng.normal(size=n), 1e-2 * rng.normal(size=n), 1e-2 * rng.normal(size=n)], 1)
    return np.concatenate([omega, t, intr], 1)
