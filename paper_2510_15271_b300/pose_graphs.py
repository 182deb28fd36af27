"""Seeded synthetic pose graphs: the inputs of pose-graph optimisation.

This module only synthesises data.  A vehicle carrying a rig of cameras
drives a route; every camera of every frame is a node.  A simulated
relative-pose sensor measures, for each edge (i, j), the pose of camera i in
camera j from the true poses (as 4 x 4 homogeneous matrices) and perturbs it
with a small random rotation and translation.  The starting state is the
dead-reckoned trajectory: the true frame-to-frame motion of the vehicle with
a small random error per step, composed from the first frame.  Nothing here
evaluates a residual, a Jacobian or a cost of the solver.

Edges, as the three constraint kinds of cuSfM's pose graph (Sec. 4.2):
  * sequential: camera c of frame f and of frame f + k, k = 1 .. seq_k;
  * extrinsic: every pair of cameras of one frame (one rig);
  * loop closure: the first cameras of two frames at least ``loop_gap``
    frames apart whose centres lie within ``loop_radius`` metres and which
    face the same way, at most one per later frame, every ``loop_every``-th
    candidate kept.

Workload ``pose_graph`` (the default sizes): 3,000 frames of a 3-camera rig
(9,000 nodes) at 2 m spacing on a random route over a 3 km x 3 km street
grid (revisits included), sequential edges with k = 1, 2, rig edges and loop
closures; the cameras of frame 0 are fixed.  Edge weights are 1 / sigma_t^2
of the edge kind's translation noise.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from .scenes import _grid_route, _look_rotation, _pose_vector, _rng

__all__ = ["PoseGraphScene", "make_pose_graph", "EDGE_SEQ", "EDGE_RIG", "EDGE_LOOP"]

EDGE_SEQ, EDGE_RIG, EDGE_LOOP = 0, 1, 2


@dataclasses.dataclass
class PoseGraphScene:
    name: str
    seed: int
    node_qt_true: np.ndarray   # (n, 7) world -> camera
    node_qt_init: np.ndarray   # (n, 7) drifted start
    edge_ij: np.ndarray        # (E, 2) int32
    edge_qt: np.ndarray        # (E, 7) measured pose of node i in node j
    edge_w: np.ndarray         # (E,)
    edge_kind: np.ndarray      # (E,) EDGE_SEQ / EDGE_RIG / EDGE_LOOP
    fixed: np.ndarray          # (n,) uint8
    n_frames: int
    rig: int
    lm_iters: int = 20

    @property
    def n_nodes(self) -> int:
        return int(self.node_qt_init.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edge_ij.shape[0])


def _homog(R, t):
    T = np.zeros(R.shape[:-2] + (4, 4))
    T[..., :3, :3] = R
    T[..., :3, 3] = t
    T[..., 3, 3] = 1.0
    return T


def _rig_extrinsics(rig):
    """Camera-from-vehicle rotations and translations of a rig: camera 0
    looks forward, the others are spread in yaw around it, 0.5 m apart."""
    yaw = np.linspace(0.0, 2.0 * np.pi, rig, endpoint=False)
    yaw = np.where(yaw > np.pi, yaw - 2.0 * np.pi, yaw) * (0.5 if rig > 2 else 1.0)
    Rv = []
    tv = []
    for a in yaw:
        # vehicle axes: x forward, y left, z up; camera axes: x right, y down, z forward
        fwd = np.array([np.cos(a), np.sin(a), 0.0])
        Rcv = _look_rotation(fwd[None])[0]          # vehicle -> camera rotation
        pos = 0.5 * np.array([np.cos(a), np.sin(a), 0.0]) + np.array([0.0, 0.0, 1.5])
        Rv.append(Rcv)
        tv.append(-Rcv @ pos)
    return np.array(Rv), np.array(tv)


def _noisy(rng, T, rot_sigma, pos_sigma):
    """Left-perturb 4 x 4 poses by a random rotation and translation."""
    n = T.shape[0]
    dR = Rotation.from_rotvec(rng.normal(0.0, rot_sigma, size=(n, 3))).as_matrix()
    out = T.copy()
    out[:, :3, :3] = dR @ T[:, :3, :3]
    out[:, :3, 3] = np.einsum("nab,nb->na", dR, T[:, :3, 3]) + rng.normal(0.0, pos_sigma, (n, 3))
    return out


def _qt_of(T):
    R = T[:, :3, :3]
    C = -np.einsum("nba,nb->na", R, T[:, :3, 3])   # centre -R^T t
    return _pose_vector(R, C)


def make_pose_graph(seed: int = 7, n_frames: int = 3000, rig: int = 3, *, spacing: float = 2.0,
                    extent: float = 3000.0, block: float = 250.0, seq_k: int = 2,
                    loop_radius: float = 4.0, loop_gap: int = 50, loop_every: int = 1,
                    drift_rot: float = 2e-4, drift_pos: float = 0.02,
                    seq_sigma=(1e-3, 0.01), rig_sigma=(5e-4, 0.005), loop_sigma=(2e-3, 0.05),
                    lm_iters: int = 20, route: str = "grid") -> PoseGraphScene:
    rng = _rng(seed)
    if route == "grid":
        Cv, H, _ = _grid_route(rng, n_frames, spacing, extent, block)
    else:   # a straight line (small test graphs without loops)
        Cv = np.stack([np.arange(n_frames) * spacing, np.zeros(n_frames), np.zeros(n_frames)], 1)
        H = np.tile([1.0, 0.0, 0.0], (n_frames, 1))
    # vehicle -> world: x forward (heading), y left, z up
    fwd = H / np.linalg.norm(H, axis=1, keepdims=True)
    left = np.cross(np.array([0.0, 0.0, 1.0]), fwd)
    Rwv = np.stack([fwd, left, np.broadcast_to([0.0, 0.0, 1.0], fwd.shape)], axis=2)
    T_wv = _homog(Rwv, Cv)
    Rcv, tcv = _rig_extrinsics(rig)
    T_cv = _homog(Rcv, tcv)
    # true node poses (world -> camera), node = f * rig + c
    T_vw = np.linalg.inv(T_wv)
    T_cw = np.einsum("cab,fbd->fcad", T_cv, T_vw).reshape(-1, 4, 4)
    # drifted start: dead reckoning, the true frame-to-frame motion of the
    # vehicle composed with a small random error in the vehicle frame per step
    noise = _noisy(rng, np.broadcast_to(np.eye(4), (n_frames, 4, 4)).copy(), drift_rot,
                   drift_pos)
    T_wv0 = np.empty_like(T_wv)
    T_wv0[0] = T_wv[0]
    for f in range(1, n_frames):
        step = np.linalg.inv(T_wv[f - 1]) @ T_wv[f]
        T_wv0[f] = T_wv0[f - 1] @ step @ noise[f]
    T_cw0 = np.einsum("cab,fbd->fcad", T_cv, np.linalg.inv(T_wv0)).reshape(-1, 4, 4)
    # edges
    ei, ej, kind, sig = [], [], [], []
    node = lambda f, c: f * rig + c
    for k in range(1, seq_k + 1):
        f = np.arange(n_frames - k)
        for c in range(rig):
            ei.append(node(f, c))
            ej.append(node(f + k, c))
            kind.append(np.full(f.size, EDGE_SEQ))
            sig.append(np.tile(seq_sigma, (f.size, 1)))
    for a in range(rig):
        for b in range(a + 1, rig):
            f = np.arange(n_frames)
            ei.append(node(f, a))
            ej.append(node(f, b))
            kind.append(np.full(f.size, EDGE_RIG))
            sig.append(np.tile(rig_sigma, (f.size, 1)))
    if n_frames > loop_gap:
        tree = cKDTree(Cv[:, :2])
        li, lj = [], []
        for f2 in range(loop_gap, n_frames):
            cand = [f1 for f1 in tree.query_ball_point(Cv[f2, :2], loop_radius)
                    if f1 <= f2 - loop_gap and float(fwd[f1] @ fwd[f2]) > 0.9]
            if cand:
                f1 = min(cand, key=lambda q: float(np.sum((Cv[q] - Cv[f2]) ** 2)))
                li.append(f1)
                lj.append(f2)
        li = np.array(li[::loop_every], dtype=np.int64)
        lj = np.array(lj[::loop_every], dtype=np.int64)
        if li.size:
            ei.append(node(li, 0))
            ej.append(node(lj, 0))
            kind.append(np.full(li.size, EDGE_LOOP))
            sig.append(np.tile(loop_sigma, (li.size, 1)))
    ei = np.concatenate(ei).astype(np.int32)
    ej = np.concatenate(ej).astype(np.int32)
    kind = np.concatenate(kind).astype(np.int8)
    sig = np.concatenate(sig)
    # measured pose of node i in node j: T_cw,j T_wc,i, perturbed
    M = np.einsum("eab,ebc->eac", T_cw[ej], np.linalg.inv(T_cw[ei]))
    Mn = np.empty_like(M)
    for kk in (EDGE_SEQ, EDGE_RIG, EDGE_LOOP):
        sel = kind == kk
        if sel.any():
            s = sig[sel][0]
            Mn[sel] = _noisy(rng, M[sel], s[0], s[1])
    w = 1.0 / sig[:, 1] ** 2
    fixed = np.zeros(n_frames * rig, dtype=np.uint8)
    fixed[:rig] = 1
    return PoseGraphScene("pose_graph", seed, _qt_of(T_cw), _qt_of(T_cw0), np.stack([ei, ej], 1),
                          _qt_of(Mn), w, kind, fixed, n_frames, rig, lm_iters)
