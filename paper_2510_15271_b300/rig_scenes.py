"""Seeded synthetic multi-camera rig scenes: the inputs of rig bundle
adjustment with extrinsic refinement.

This module only synthesises data.  A vehicle carrying a rig of cameras
drives along a gently curving street between two facades; each camera's
world-to-camera pose is its vehicle-to-camera extrinsic composed with the
vehicle's world-to-vehicle pose.  Points on the facades and the road are
measured, through each camera's 3 x 4 projection matrix, by a random subset
of the cameras that see them, with pixel noise.  The start state perturbs the
vehicle poses, the extrinsics (a calibration error) and the points.  Nothing
here evaluates a residual, a Jacobian or a cost of the solver.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial.transform import Rotation

from .pose_graphs import _rig_extrinsics
from .scenes import _image, _in_view, _intrinsics, _measure, _pick_views, _projection_matrices, _rng

__all__ = ["RigScene", "make_rig_scene"]


@dataclasses.dataclass
class RigScene:
    intrinsics: np.ndarray   # (R, 4) fx, fy, cx, cy
    obs_frame: np.ndarray    # (N,) int32
    obs_rc: np.ndarray       # (N,) int32 rig camera
    obs_pt: np.ndarray       # (N,) int32
    obs_uv: np.ndarray       # (N, 2)
    Rv: np.ndarray           # (F, 3, 3) start: world -> vehicle
    tv: np.ndarray
    Re: np.ndarray           # (R, 3, 3) start: vehicle -> camera
    te: np.ndarray
    X: np.ndarray            # (P, 3) start
    Rv_gt: np.ndarray
    tv_gt: np.ndarray
    Re_gt: np.ndarray
    te_gt: np.ndarray
    X_gt: np.ndarray
    frame_fixed: np.ndarray  # (F,) uint8
    rc_fixed: np.ndarray     # (R,) uint8

    @property
    def n_frames(self):
        return int(self.Rv.shape[0])

    @property
    def n_rc(self):
        return int(self.Re.shape[0])

    @property
    def n_pts(self):
        return int(self.X.shape[0])

    @property
    def n_obs(self):
        return int(self.obs_pt.shape[0])


def _perturb(rng, R, t, rot_sigma, pos_sigma, keep):
    dR = Rotation.from_rotvec(rng.normal(0.0, rot_sigma, size=(R.shape[0], 3))).as_matrix()
    R2 = dR @ R
    t2 = t + rng.normal(0.0, pos_sigma, size=t.shape)
    R2[keep] = R[keep]
    t2[keep] = t[keep]
    return R2, t2


def make_rig_scene(seed: int = 1, n_frames: int = 12, rig: int = 3, n_pts: int = 300, *,
                   spacing: float = 1.0, f: float = 500.0, width: int = 640, height: int = 480,
                   sigma: float = 0.5, track=(2, 6), veh_sigma=(0.005, 0.03),
                   ext_sigma=(0.01, 0.02), pt_sigma: float = 0.03) -> RigScene:
    rng = _rng(seed)
    K = _intrinsics(f, width, height)
    # vehicle: x forward, y left, z up; a gentle left curve
    s = np.arange(n_frames) * spacing
    yaw = 0.01 * s
    Cv = np.stack([s, 0.05 * s * s * 0.01, np.zeros(n_frames)], axis=1)
    fwd = np.stack([np.cos(yaw), np.sin(yaw), np.zeros(n_frames)], axis=1)
    left = np.stack([-np.sin(yaw), np.cos(yaw), np.zeros(n_frames)], axis=1)
    up = np.broadcast_to([0.0, 0.0, 1.0], fwd.shape)
    Rwv = np.stack([fwd, left, up], axis=2)         # vehicle -> world rotation
    Rv = np.transpose(Rwv, (0, 2, 1))               # world -> vehicle
    tv = -np.einsum("fab,fb->fa", Rv, Cv)
    Re, te = _rig_extrinsics(rig)                   # vehicle -> camera
    # composite cameras (frame-major: camera f * rig + c)
    Rc = np.einsum("cab,fbd->fcad", Re, Rv).reshape(-1, 3, 3)
    tc = (np.einsum("cab,fb->fca", Re, tv) + te[None]).reshape(-1, 3)
    Cc = -np.einsum("nba,nb->na", Rc, tc)
    Pm = _projection_matrices(K, Rc, Cc)
    # points: two facades and the road along the drive
    x = rng.uniform(-5.0, s[-1] + 15.0, n_pts)
    side = rng.integers(0, 3, n_pts)
    y = np.where(side == 0, rng.uniform(5.0, 9.0, n_pts),
                 np.where(side == 1, -rng.uniform(5.0, 9.0, n_pts), rng.uniform(-4.0, 4.0, n_pts)))
    z = np.where(side == 2, 0.0, rng.uniform(0.0, 6.0, n_pts))
    X = np.stack([x, y + 0.05 * x * x * 0.01, z], axis=1)
    uv, w = _image(Pm[None, :, :, :], X[:, None, :])
    vis = _in_view(uv, w, width, height, 0.5, 40.0)
    nvis = vis.sum(axis=1)
    keep = nvis >= 2
    X, vis, nvis = X[keep], vis[keep], nvis[keep]
    L = np.minimum(rng.integers(track[0], track[1] + 1, X.shape[0]), nvis)
    sel = _pick_views(rng, vis, L)
    obs_cam, obs_pt = [], []
    for j in range(X.shape[0]):
        for c in sel[j]:
            if c >= 0:
                obs_cam.append(int(c))
                obs_pt.append(j)
    obs_cam = np.array(obs_cam, dtype=np.int64)
    obs_pt = np.array(obs_pt, dtype=np.int64)
    uvm, _ = _measure(rng, K, Rc, Cc, X, obs_cam, obs_pt, sigma, 0.0, width, height)
    frame_fixed = np.zeros(n_frames, dtype=np.uint8)
    frame_fixed[0] = 1
    rc_fixed = np.zeros(rig, dtype=np.uint8)
    Rv0, tv0 = _perturb(rng, Rv, tv, veh_sigma[0], veh_sigma[1], frame_fixed.astype(bool))
    Re0, te0 = _perturb(rng, Re, te, ext_sigma[0], ext_sigma[1], rc_fixed.astype(bool))
    X0 = X + rng.normal(0.0, pt_sigma, size=X.shape)
    intr = np.tile([K[0, 0], K[1, 1], K[0, 2], K[1, 2]], (rig, 1))
    return RigScene(intr, (obs_cam // rig).astype(np.int32), (obs_cam % rig).astype(np.int32),
                    obs_pt.astype(np.int32), np.ascontiguousarray(uvm), Rv0, tv0, Re0, te0, X0,
                    Rv, tv, Re, te, X, frame_fixed, rc_fixed)
