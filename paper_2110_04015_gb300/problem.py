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


def concat_offsets(scenes: list[Scene]) -> tuple[np.ndarray, np.ndarray]:
    """Camera offsets (n + 1) and landmark offsets (n + 1) of scenes laid end to end."""
    cam_off = np.zeros(len(scenes) + 1, np.int64)
    pt_off = np.zeros(len(scenes) + 1, np.int64)
    for b, sc in enumerate(scenes):
        cam_off[b + 1] = cam_off[b] + sc.n_cams
        pt_off[b + 1] = pt_off[b] + sc.n_pts
    return cam_off, pt_off


def from_scenes(scenes: list[Scene], precision: str = "fp64", device: str = "cuda", **kw) -> Problem:
    """One batched ``Problem`` over independent scenes (``ba_batch_create``): cameras, landmarks and
    observations concatenated in scene order, each scene's indices shifted by the sizes before it."""
    import torch

    cam_off, pt_off = concat_offsets(scenes)
    cams = np.concatenate([sc.cams0 for sc in scenes])
    pts = np.concatenate([sc.pts0 for sc in scenes])
    oc = np.concatenate([sc.obs_cam.astype(np.int64) + cam_off[b] for b, sc in enumerate(scenes)])
    op = np.concatenate([sc.obs_pt.astype(np.int64) + pt_off[b] for b, sc in enumerate(scenes)])
    xy = torch.cat([device_measurements(sc, device) for sc in scenes])
    return Problem(cams, pts, oc, op, xy, precision=precision, cam_off=cam_off.astype(np.int32), **kw)
