"""Seeded synthetic bundle-adjustment scenes: inputs only.

This module draws everything random that a solve needs as input: the true
cameras and landmarks, which cameras observe which landmark (the tracks), the
pixel noise, and the 1 % perturbation of the parameters that gives the initial
state of the first Levenberg-Marquardt iteration.  It computes none of the
method's arithmetic: no projection, residual, Jacobian, normal equation, Schur
complement or solve.  A consumer of a scene forms the measurements with its
own projection, ``m = pi(c_true, X_true) + noise``, and starts from
``(cams0, pts0)``.

Camera parameters follow the BAL layout used by the paper's datasets
(Section 3, d_p = 9 with intrinsics): angle-axis rotation (3), translation (3),
focal length, radial distortion k1, k2.  A camera looks down its own -z axis.

Random numbers come from a counter-based generator (SplitMix64, Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
one independent stream per named quantity, and normals from the Box-Muller
transform, so a scene depends only on (config, seed) and not on numpy's own
generators.

Workloads (shapes of the paper's Table 1 problems, which are not available):

* ``tiny``: 16 cameras on a circle of radius 10 facing the origin, 1,000
  landmarks uniform in the centred unit cube, tracks of 3..6 distinct cameras.
* ``sequential``: 1,000 cameras along a helix looking along its tangent,
  100,000 landmarks each seen only by cameras within a sliding window of 32,
  tracks Poisson(5) + 2 (about 700k observations): a banded, sparse S.
* ``dense``: 1,936 cameras on a sphere of radius 10 facing a unit-cube scene,
  about 1.3M landmarks with geometric track lengths (2 + Geom, mean 4, capped
  at 200) drawn mostly from 64 co-visibility clusters (about 5.2M
  observations): a dense S shaped like the paper's largest problem (F-1936).
* ``batched``: many independent problems of 50..600 cameras each with
  300 landmarks per camera and long tracks (mean 8).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _mix_int(z: int) -> int:
    z &= _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _fnv1a(name: str) -> int:
    h = 0xCBF29CE484222325
    for ch in name.encode():
        h = ((h ^ ch) * 0x100000001B3) & _MASK
    return h


class Stream:
    """One SplitMix64 stream: value k is mix(key + (k + 1) * gamma)."""

    def __init__(self, seed: int, name: str):
        self.key = _mix_int((int(seed) * _GAMMA) ^ _fnv1a(name))
        self.ctr = 0

    def bits(self, n: int) -> np.ndarray:
        k = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix(np.uint64(self.key) + k * np.uint64(_GAMMA))

    def uniform(self, n: int) -> np.ndarray:
        """Doubles in the open interval (0, 1)."""
        return ((self.bits(n) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive)."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)

    def poisson(self, mean: float, n: int) -> np.ndarray:
        """Poisson(mean) by inversion of its cumulative distribution."""
        kmax = int(mean + 20 * np.sqrt(mean) + 20)
        k = np.arange(kmax + 1)
        logp = -mean + k * np.log(mean) - np.cumsum(np.log(np.maximum(k, 1)))
        cdf = np.cumsum(np.exp(logp))
        return np.minimum(np.searchsorted(cdf, self.uniform(n)), kmax)

    def geometric(self, mean: float, n: int) -> np.ndarray:
        """Failures before the first success, P(G = g) = p (1 - p)^g, E[G] = mean."""
        p = 1.0 / (1.0 + mean)
        return np.floor(np.log(self.uniform(n)) / np.log1p(-p)).astype(np.int64)


# ---------------------------------------------------------------------------
# geometry helpers for placing cameras (not part of the method)


def _look_rotation(backward: np.ndarray, up: np.ndarray) -> np.ndarray:
    """World-to-camera rotations whose camera +z axis is ``backward``.

    Rows are the camera's right, up and backward axes in world coordinates, so
    a camera looks along -backward.
    """
    b = backward / np.linalg.norm(backward, axis=1, keepdims=True)
    right = np.cross(up, b)
    bad = np.linalg.norm(right, axis=1) < 1e-6
    if bad.any():
        right[bad] = np.cross(np.array([1.0, 0.0, 0.0]), b[bad])
    right /= np.linalg.norm(right, axis=1, keepdims=True)
    cam_up = np.cross(b, right)
    return np.stack([right, cam_up, b], axis=1)


def _log_rotation(R: np.ndarray) -> np.ndarray:
    """Angle-axis vectors of rotation matrices (the inverse of Rodrigues)."""
    n = R.shape[0]
    tr = np.trace(R, axis1=1, axis2=2)
    cos_t = np.clip((tr - 1.0) / 2.0, -1.0, 1.0)
    theta = np.arccos(cos_t)
    vee = np.stack([R[:, 2, 1] - R[:, 1, 2], R[:, 0, 2] - R[:, 2, 0], R[:, 1, 0] - R[:, 0, 1]], axis=1)
    out = np.zeros((n, 3))
    sin_t = np.sin(theta)
    generic = sin_t > 1e-6
    out[generic] = vee[generic] * (theta[generic] / (2.0 * sin_t[generic]))[:, None]
    near_pi = (~generic) & (cos_t < 0)
    for i in np.nonzero(near_pi)[0]:
        # R = 2 a a^T - I at theta = pi: the axis is the dominant column of R + I
        B = R[i] + np.eye(3)
        c = int(np.argmax(np.linalg.norm(B, axis=0)))
        a = B[:, c] / np.linalg.norm(B[:, c])
        out[i] = a * theta[i]
    # theta ~ 0: out stays (almost) zero, to first order vee / 2
    small = (~generic) & (cos_t >= 0)
    out[small] = vee[small] / 2.0
    return out


def _intrinsics(stream: Stream, n: int) -> np.ndarray:
    f = 500.0 + 50.0 * stream.normal(n)
    k1 = 1e-3 * stream.normal(n)
    k2 = 1e-3 * stream.normal(n)
    return np.stack([f, k1, k2], axis=1)


def _cameras_from_poses(R: np.ndarray, C: np.ndarray, intr: np.ndarray) -> np.ndarray:
    t = -np.einsum("nij,nj->ni", R, C)
    return np.concatenate([_log_rotation(R), t, intr], axis=1)


def _distinct_from_mask(stream: Stream, eligible: np.ndarray, t: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Pick t[i] distinct columns of row i among its eligible ones, uniformly.

    Returns (row, column) index arrays grouped by row.
    """
    n, m = eligible.shape
    keys = stream.uniform(n * m).reshape(n, m)
    keys[~eligible] = 2.0
    order = np.argsort(keys, axis=1, kind="stable")
    t = np.minimum(t, eligible.sum(axis=1))
    take = np.arange(m)[None, :] < t[:, None]
    rows = np.repeat(np.arange(n), t)
    cols = order[take]
    return rows, cols


@dataclass
class Scene:
    """One synthetic problem.

    ``obs_cam``/``obs_pt`` list the observations in BAL file order (by camera,
    then landmark).  ``noise`` is the pixel noise already scaled by sigma.
    """

    name: str
    seed: int
    cams_true: np.ndarray
    pts_true: np.ndarray
    obs_cam: np.ndarray
    obs_pt: np.ndarray
    noise: np.ndarray
    cams0: np.ndarray
    pts0: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_cams(self) -> int:
        return int(self.cams_true.shape[0])

    @property
    def n_pts(self) -> int:
        return int(self.pts_true.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.obs_cam.shape[0])


def _finish(name, seed, cams, pts, rows, cols, sigma, rel_perturb, meta) -> Scene:
    """Sort observations into BAL order, draw noise and the initial state."""
    obs_pt = rows.astype(np.int64)
    obs_cam = cols.astype(np.int64)
    order = np.lexsort((obs_pt, obs_cam))
    obs_cam = obs_cam[order].astype(np.int32)
    obs_pt = obs_pt[order].astype(np.int32)
    s_noise = Stream(seed, name + "/noise")
    noise = sigma * s_noise.normal(2 * obs_cam.size).reshape(-1, 2)
    s_pert = Stream(seed, name + "/perturb")
    xi_c = s_pert.normal(cams.size).reshape(cams.shape)
    xi_p = s_pert.normal(pts.size).reshape(pts.shape)
    cams0 = cams + rel_perturb * np.abs(cams) * xi_c
    pts0 = pts + rel_perturb * np.abs(pts) * xi_p
    return Scene(name, seed, cams, pts, obs_cam, obs_pt, noise, cams0, pts0, meta)


def tiny(seed: int = 0, n_cams: int = 16, n_pts: int = 1000, track_min: int = 3, track_max: int = 6,
         sigma: float = 1.0, rel_perturb: float = 0.01) -> Scene:
    """Cameras on a circle of radius 10 in z = 0 facing the origin."""
    name = "tiny"
    s = Stream(seed, name + "/scene")
    ang = 2.0 * np.pi * np.arange(n_cams) / n_cams
    C = np.stack([10.0 * np.cos(ang), 10.0 * np.sin(ang), np.zeros(n_cams)], axis=1)
    R = _look_rotation(C, np.tile([0.0, 0.0, 1.0], (n_cams, 1)))
    cams = _cameras_from_poses(R, C, _intrinsics(s, n_cams))
    pts = s.uniform(3 * n_pts).reshape(n_pts, 3) - 0.5
    t = s.integers(track_min, min(track_max, n_cams), n_pts)
    rows, cols = _distinct_from_mask(s, np.ones((n_pts, n_cams), bool), t)
    return _finish(name, seed, cams, pts, rows, cols, sigma, rel_perturb,
                   {"track": f"U{{{track_min}..{track_max}}}"})


def sequential(seed: int = 0, n_cams: int = 1000, n_pts: int = 100_000, window: int = 32,
               track_mean_extra: float = 5.0, sigma: float = 1.0, rel_perturb: float = 0.01) -> Scene:
    """Cameras along a helix (radius 20, rise 2 per 100 cameras) looking along its tangent.

    Each landmark is anchored at a uniformly drawn camera c, at depth U(5, 20)
    in front of it with lateral offsets up to +-0.4 depth, and is seen by
    min(Poisson(5) + 2, 32) distinct cameras of the window [c - 16, c + 15]
    that have it at least 2 in front of them and within 40 degrees of their
    viewing direction.
    """
    name = "sequential"
    s = Stream(seed, name + "/scene")
    j = np.arange(n_cams)
    phi = 2.0 * np.pi * j / 100.0
    C = np.stack([20.0 * np.cos(phi), 20.0 * np.sin(phi), 0.02 * j], axis=1)
    T = np.stack([-20.0 * np.sin(phi) * 2.0 * np.pi / 100.0, 20.0 * np.cos(phi) * 2.0 * np.pi / 100.0,
                  np.full(n_cams, 0.02)], axis=1)
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    R = _look_rotation(-T, np.tile([0.0, 0.0, 1.0], (n_cams, 1)))
    cams = _cameras_from_poses(R, C, _intrinsics(s, n_cams))

    half_lo, half_hi = window // 2, window // 2 - 1
    anchor = s.integers(0, n_cams - 1, n_pts)
    depth = 5.0 + 15.0 * s.uniform(n_pts)
    lat = 0.8 * (s.uniform(2 * n_pts).reshape(n_pts, 2) - 0.5) * depth[:, None]
    pts = C[anchor] + depth[:, None] * T[anchor] + lat[:, :1] * R[anchor, 0] + lat[:, 1:] * R[anchor, 1]
    cand = anchor[:, None] + np.arange(-half_lo, half_hi + 1)[None, :]
    valid = (cand >= 0) & (cand < n_cams)
    candc = np.clip(cand, 0, n_cams - 1)
    ray = pts[:, None, :] - C[candc]
    along = np.einsum("nwk,nwk->nw", ray, T[candc])
    # visible: at least 2 in front and within 40 degrees of the viewing direction
    front = (along > 2.0) & (along > np.cos(np.radians(40.0)) * np.linalg.norm(ray, axis=2))
    eligible = valid & front
    t = np.minimum(s.poisson(track_mean_extra, n_pts) + 2, window)
    rows, cols = _distinct_from_mask(s, eligible, t)
    cams_idx = candc[rows, cols]
    return _finish(name, seed, cams, pts, rows, cams_idx, sigma, rel_perturb,
                   {"window": window, "track": "min(Poisson(5)+2, 32)"})


def _fibonacci_sphere(n: int, radius: float) -> np.ndarray:
    k = np.arange(n) + 0.5
    z = 1.0 - 2.0 * k / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = np.pi * (3.0 - np.sqrt(5.0))
    a = ga * np.arange(n)
    return radius * np.stack([r * np.cos(a), r * np.sin(a), z], axis=1)


def _clustered_tracks(s: Stream, n_cams: int, n_pts: int, n_clusters: int, t: np.ndarray,
                      p_uniform: float) -> tuple[np.ndarray, np.ndarray]:
    """Distinct cameras per landmark: from its cluster with prob 1 - p_uniform, else uniform."""
    bounds = (np.arange(n_clusters + 1) * n_cams) // n_clusters
    csize = np.diff(bounds)
    cluster = s.integers(0, n_clusters - 1, n_pts)
    rows = np.repeat(np.arange(n_pts), t)
    nslot = rows.size
    uni = s.uniform(nslot) < p_uniform
    cl = cluster[rows]
    cams = np.empty(nslot, np.int64)

    def draw(idx, uniform_slot):
        u = s.uniform(idx.size)
        c_cl = bounds[cl[idx]] + np.floor(u * csize[cl[idx]]).astype(np.int64)
        c_un = np.floor(u * n_cams).astype(np.int64)
        return np.where(uniform_slot, c_un, c_cl)

    cams[:] = draw(np.arange(nslot), uni)
    for attempt in range(64):
        key = rows * n_cams + cams
        order = np.argsort(key, kind="stable")
        dup_sorted = np.zeros(nslot, bool)
        dup_sorted[1:] = key[order][1:] == key[order][:-1]
        dup = order[dup_sorted]
        if dup.size == 0:
            break
        # after a few rounds a slot whose cluster is exhausted falls back to uniform
        force_uniform = uni[dup] | (attempt >= 8)
        uni[dup] = force_uniform
        cams[dup] = draw(dup, force_uniform)
    else:  # pragma: no cover - vanishingly unlikely
        raise RuntimeError("could not draw distinct cameras")
    return rows, cams


def dense(seed: int = 0, n_cams: int = 1936, n_pts: int = 1_300_000, n_clusters: int = 64,
          track_extra_mean: float = 2.0, track_cap: int = 200, p_uniform: float = 0.25,
          sigma: float = 1.0, rel_perturb: float = 0.01) -> Scene:
    """Cameras on a sphere of radius 10 facing a unit-cube scene; clustered tracks.

    Track length is 2 + Geom(mean 2) capped at 200, so the mean is 4 and the
    observation count about 4 n_pts.  A fraction ``p_uniform`` of the track
    slots picks any camera, which couples clusters and sets the density of S
    (0.25 gives d ~ 0.9 at the default sizes, as for F-1936).
    """
    name = "dense"
    s = Stream(seed, name + "/scene")
    C = _fibonacci_sphere(n_cams, 10.0)
    R = _look_rotation(C, np.tile([0.0, 0.0, 1.0], (n_cams, 1)))
    cams = _cameras_from_poses(R, C, _intrinsics(s, n_cams))
    pts = s.uniform(3 * n_pts).reshape(n_pts, 3) - 0.5
    t = np.minimum(2 + s.geometric(track_extra_mean, n_pts), min(track_cap, n_cams))
    rows, cols = _clustered_tracks(s, n_cams, n_pts, n_clusters, t, p_uniform)
    return _finish(name, seed, cams, pts, rows, cols, sigma, rel_perturb,
                   {"clusters": n_clusters, "p_uniform": p_uniform, "track": "2+Geom(mean 2), cap 200"})


def batched(seed: int = 0, n_problems: int = 64, cams_lo: int = 50, cams_hi: int = 600,
            pts_per_cam: int = 300, track_extra_mean: float = 6.0, p_uniform: float = 0.3,
            scale: float = 1.0) -> list[Scene]:
    """Independent uneven problems (sphere geometry, clustered long tracks, mean 8).

    Tracks are capped at half the problem's cameras so that distinct cameras can always be drawn.
    ``scale`` shrinks the landmark count for quick tests.
    """
    s = Stream(seed, "batched/sizes")
    sizes = s.integers(cams_lo, cams_hi, n_problems)
    out = []
    for b, n_c in enumerate(sizes):
        n_c = int(n_c)
        n_l = max(8, int(pts_per_cam * n_c * scale))
        n_cl = max(1, n_c // 30)
        sc = dense(seed=seed * 1000 + b, n_cams=n_c, n_pts=n_l, n_clusters=n_cl,
                   track_extra_mean=track_extra_mean, track_cap=min(200, n_c // 2), p_uniform=p_uniform)
        sc.name = f"batched[{b}]"
        out.append(sc)
    return out


def permute_cameras(sc: Scene, order: np.ndarray) -> Scene:
    """The same scene with its cameras renumbered: new camera i is old camera order[i].

    Observations keep their measurements and noise (the rows are only relabelled), so the problem
    is the same one in another camera order.
    """
    order = np.asarray(order, dtype=np.int64)
    inv = np.empty_like(order)
    inv[order] = np.arange(order.size)
    return Scene(sc.name, sc.seed, sc.cams_true[order], sc.pts_true, inv[sc.obs_cam].astype(np.int32),
                 sc.obs_pt, sc.noise, sc.cams0[order], sc.pts0, dict(sc.meta, camera_order="permuted"))


def shuffled(sc: Scene, seed: int) -> Scene:
    """The scene with its cameras in a seeded random order (as in collections whose camera
    numbering carries no geometry)."""
    s = Stream(seed, "shuffle")
    return permute_cameras(sc, np.argsort(s.uniform(sc.n_cams), kind="stable"))


CONFIGS = {
    "tiny": tiny,
    "sequential": sequential,
    "dense": dense,
}


def make(config: str, seed: int = 0, **kw) -> Scene:
    return CONFIGS[config](seed=seed, **kw)

