"""Build library problems from seeded scenes, measurements synthesised on the device.

The measurements of a synthetic scene are m = pi(c_true, X_true) + noise; here
pi is the library's own camera model (``ba_project``), so no code outside the
CUDA library evaluates the method.
"""
from __future__ import annotations

import numpy as np

from .binding import Problem, ba_project
from .synthetic import Scene


def device_measurements(scene: Scene, device: str = "cuda"):
    import torch

    cams = torch.from_numpy(np.ascontiguousarray(scene.cams_true)).to(device)
    pts = torch.from_numpy(np.ascontiguousarray(scene.pts_true)).to(device)
    oc = torch.from_numpy(scene.obs_cam.astype(np.int32)).to(device)
    op = torch.from_numpy(scene.obs_pt.astype(np.int32)).to(device)
    xy = torch.empty((scene.n_obs, 2), dtype=torch.float64, device=device)
    ba_project(cams, pts, oc, op, xy)
    xy += torch.from_numpy(scene.noise).to(device)
    torch.cuda.synchronize()
    return xy


def from_scene(scene: Scene, precision: str = "fp64", device: str = "cuda", xy=None, **kw) -> Problem:
    """A ``Problem`` at the scene's initial (perturbed) state."""
    if xy is None:
        xy = device_measurements(scene, device)
    return Problem(scene.cams0, scene.pts0, scene.obs_cam, scene.obs_pt, xy, precision=precision, **kw)
