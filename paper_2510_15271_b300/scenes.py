"""Seeded synthetic bundle-adjustment scenes: the inputs both solvers consume.

This module only synthesises data: camera poses, 3D points, and pixel
measurements of those points with noise, outliers and a perturbed starting
state.  Measurements are made by a simulated pinhole camera through its 3x4
projection matrix P = K [R | t] applied to homogeneous points; nothing here
evaluates a residual, a Jacobian, a cost or any other part of the solver.
Rotations are converted with scipy's ``Rotation`` (a library routine).

Conventions of the solver boundary that the data follows:
  * a pose maps world to camera, x_c = R X + t, stored as the 7 numbers
    (qw, qx, qy, qz, tx, ty, tz) with a unit quaternion;
  * a pixel is (fx x/z + cx, fy y/z + cy); camera axes are x right, y down,
    z forward.

Workloads (sizes are the defaults; every builder accepts smaller ones):
  * ``ring``     20 cameras on a 5 m circle looking inward, 640x480, f=500;
                 2,000 points in a 4 m cube, 5 views each; 0.5 px noise.
  * ``driving``  1,000 forward-facing 1920x1080 f=1000 cameras along a 2 km
                 smooth road at 1.5 m height; 200k points on the road plane
                 and on facades 8-15 m to either side; geometric track
                 lengths (mean 6, 2..30) over consecutive cameras; 0.7 px
                 noise; 2 % outliers.
  * ``city``     5,000 cameras driving a random route on a 3 km x 3 km street
                 grid (revisits included); 1M points; Zipf(1.5) track
                 lengths on 2..40 over all cameras that see the point; 1 px
                 noise; 1 % outliers.
  * ``window``   one local-BA window: a ring scene with C cameras, P points
                 and uniform 3..10 track lengths (the batched workload draws
                 512 of them with C in 10..60 and P in 500..8,000).
  * ``request``  one served request: a ring scene with C log-uniform in
                 10..200, P log-uniform in 1k..40k, track length 2+Geom(3).
"""
from __future__ import annotations

import dataclasses
import itertools
import math
from typing import List, Optional

import numpy as np
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

__all__ = ["Scene", "make_scene", "make_windows", "make_request", "poisson_arrivals",
           "WORKLOADS"]


@dataclasses.dataclass
class Scene:
    """One bundle-adjustment problem plus its ground truth and solve settings."""
    name: str
    seed: int
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    cam_qt: np.ndarray        # (C, 7) float64, initial (perturbed) poses
    pts: np.ndarray           # (P, 3) float64, initial (perturbed) points
    cam_qt_gt: np.ndarray     # (C, 7) float64, true poses
    pts_gt: np.ndarray        # (P, 3) float64, true points
    obs_cam: np.ndarray       # (N,) int32
    obs_pt: np.ndarray        # (N,) int32
    obs_uv: np.ndarray        # (N, 2) float64 pixels
    obs_inlier: np.ndarray    # (N,) bool, False for injected outliers
    cam_fixed: np.ndarray     # (C,) uint8, 1 = pose held fixed
    huber_delta: float        # px; 0 means plain least squares
    lm_iters: int
    solver: str               # "dense" | "pcg"
    pcg_tol: float
    pcg_max_iters: int
    precision: str            # "fp64" | "fp32"
    refine: bool              # FP64 iterative refinement of the PCG solve

    @property
    def n_cams(self) -> int:
        return int(self.cam_qt.shape[0])

    @property
    def n_pts(self) -> int:
        return int(self.pts.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.obs_cam.shape[0])

    def intrinsics(self):
        return (self.fx, self.fy, self.cx, self.cy)


# --------------------------------------------------------------------------- helpers

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _look_rotation(forward: np.ndarray, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """World->camera rotations whose rows are the camera's right, down and
    forward axes in world coordinates.  forward: (n, 3)."""
    f = forward / np.linalg.norm(forward, axis=1, keepdims=True)
    upv = np.broadcast_to(np.asarray(up, dtype=np.float64), f.shape)
    right = np.cross(f, upv)
    right /= np.linalg.norm(right, axis=1, keepdims=True)
    down = np.cross(f, right)
    return np.stack([right, down, f], axis=1)


def _projection_matrices(K: np.ndarray, R: np.ndarray, C: np.ndarray) -> np.ndarray:
    """P = K [R | -R C] for each camera (R world->camera, C camera centre)."""
    t = -np.einsum("nij,nj->ni", R, C)
    Rt = np.concatenate([R, t[:, :, None]], axis=2)
    return np.einsum("ij,njk->nik", K, Rt)


def _image(Pm: np.ndarray, X: np.ndarray):
    """Homogeneous image of points X (..., 3) through matrices Pm (..., 3, 4).
    Returns pixel coordinates (..., 2) and the third homogeneous coordinate,
    which for P = K[R|t] with K[2] = (0, 0, 1) is the depth along the axis."""
    Xh = np.concatenate([X, np.ones(X.shape[:-1] + (1,))], axis=-1)
    h = np.einsum("...ij,...j->...i", Pm, Xh)
    w = h[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        uv = h[..., :2] / w[..., None]
    return uv, w


def _pose_vector(R: np.ndarray, C: np.ndarray) -> np.ndarray:
    """(qw, qx, qy, qz, tx, ty, tz) of world->camera poses from rotations and
    camera centres."""
    q_xyzw = Rotation.from_matrix(R).as_quat()
    q = np.concatenate([q_xyzw[:, 3:4], q_xyzw[:, :3]], axis=1)
    q *= np.where(q[:, :1] < 0, -1.0, 1.0)
    t = -np.einsum("nij,nj->ni", R, C)
    return np.concatenate([q, t], axis=1)


def _perturb_poses(rng, R, C, rot_sigma, pos_sigma, fixed):
    """Rotate each camera by a random small rotation (left-applied, rotation
    vector ~ N(0, rot_sigma^2) per component) and move its centre by
    N(0, pos_sigma^2) per component; fixed cameras keep their true pose."""
    n = R.shape[0]
    dR = Rotation.from_rotvec(rng.normal(0.0, rot_sigma, size=(n, 3))).as_matrix()
    R2 = np.einsum("nij,njk->nik", dR, R)
    C2 = C + rng.normal(0.0, pos_sigma, size=(n, 3))
    keep = fixed.astype(bool)
    R2[keep] = R[keep]
    C2[keep] = C[keep]
    return R2, C2


def _measure(rng, K, R, C, X, obs_cam, obs_pt, sigma, outlier_frac, width, height):
    """Noisy pixel measurements of point obs_pt in camera obs_cam."""
    Pm = _projection_matrices(K, R, C)
    uv, _ = _image(Pm[obs_cam], X[obs_pt])
    uv = uv + rng.normal(0.0, sigma, size=uv.shape)
    n = obs_cam.shape[0]
    inlier = np.ones(n, dtype=bool)
    if outlier_frac > 0:
        # A wrong match replaces one measurement of a track that still has at
        # least three good ones (shorter tracks with a wrong match would not
        # survive triangulation); tracks are drawn so that outlier_frac of all
        # observations are outliers.
        L = np.bincount(obs_pt, minlength=int(obs_pt.max()) + 1)
        long_tracks = np.nonzero(L >= 4)[0]
        p = min(1.0, outlier_frac * n / max(long_tracks.size, 1))
        chosen = long_tracks[rng.random(long_tracks.size) < p]
        start = np.concatenate([[0], np.cumsum(L)[:-1]])     # obs are grouped by point
        pick = start[chosen] + (rng.random(chosen.size) * L[chosen]).astype(np.int64)
        inlier[pick] = False
        k = pick.size
        uv[pick, 0] = rng.uniform(0.0, width, size=k)
        uv[pick, 1] = rng.uniform(0.0, height, size=k)
    return uv, inlier


def _finish(name, seed, rng, K, width, height, R, C, X, obs_cam, obs_pt, *, sigma,
            outlier_frac, rot_sigma, pos_sigma, pt_sigma, fixed, settings):
    uv, inlier = _measure(rng, K, R, C, X, obs_cam, obs_pt, sigma, outlier_frac, width, height)
    R0, C0 = _perturb_poses(rng, R, C, rot_sigma, pos_sigma, fixed)
    X0 = X + rng.normal(0.0, pt_sigma, size=X.shape)
    # observations arrive in no particular order
    order = rng.permutation(obs_cam.shape[0])
    return Scene(
        name=name, seed=seed, fx=float(K[0, 0]), fy=float(K[1, 1]), cx=float(K[0, 2]),
        cy=float(K[1, 2]), width=width, height=height,
        cam_qt=_pose_vector(R0, C0), pts=X0.copy(),
        cam_qt_gt=_pose_vector(R, C), pts_gt=X.copy(),
        obs_cam=obs_cam[order].astype(np.int32), obs_pt=obs_pt[order].astype(np.int32),
        obs_uv=np.ascontiguousarray(uv[order]), obs_inlier=inlier[order],
        cam_fixed=fixed.astype(np.uint8), **settings)


def _intrinsics(f, width, height):
    return np.array([[f, 0.0, width / 2.0], [0.0, f, height / 2.0], [0.0, 0.0, 1.0]])


def _in_view(uv, depth, width, height, dmin, dmax):
    return ((depth > dmin) & (depth < dmax) & (uv[..., 0] >= 0) & (uv[..., 0] < width)
            & (uv[..., 1] >= 0) & (uv[..., 1] < height))


def _pick_views(rng, vis: np.ndarray, L: np.ndarray) -> np.ndarray:
    """For each row of the visibility mask choose L[row] distinct visible
    columns uniformly at random.  Returns a (rows, max L) array padded with -1."""
    keys = rng.random(vis.shape)
    keys[~vis] = 2.0
    order = np.argsort(keys, axis=1)
    Lmax = int(L.max()) if L.size else 0
    sel = order[:, :Lmax].copy()
    sel[np.arange(Lmax)[None, :] >= L[:, None]] = -1
    return sel


# --------------------------------------------------------------------------- ring scenes

def _ring_scene(name, seed, n_cams, n_pts, track_len, *, radius=5.0, cube=2.0, f=500.0,
                width=640, height=480, sigma=0.5, outlier_frac=0.0, rot_sigma=0.01,
                pos_sigma=0.05, pt_sigma=0.05, settings=None):
    """Cameras evenly spaced on a circle in the z=0 plane looking at the
    origin; points uniform in a cube; each point seen by ``track_len(rng, n)``
    random cameras that have it in view (depth > 0.1, inside the image)."""
    rng = _rng(seed)
    K = _intrinsics(f, width, height)
    th = 2.0 * np.pi * np.arange(n_cams) / n_cams
    C = np.stack([radius * np.cos(th), radius * np.sin(th), np.zeros(n_cams)], axis=1)
    R = _look_rotation(-C)
    Pm = _projection_matrices(K, R, C)
    X = np.empty((n_pts, 3))
    L = np.empty(n_pts, dtype=np.int64)
    sel_rows = []
    todo = np.arange(n_pts)
    for attempt in range(50):
        Xi = rng.uniform(-cube, cube, size=(todo.size, 3))
        Li = np.minimum(track_len(rng, todo.size), n_cams)
        uv, w = _image(Pm[None, :, :, :], Xi[:, None, :])
        vis = _in_view(uv, w, width, height, 0.1, np.inf)
        nvis = vis.sum(axis=1)
        if attempt == 49:   # last attempt: shorten tracks that cannot be met
            Li = np.minimum(Li, np.maximum(nvis, 2))
        ok = nvis >= Li
        X[todo[ok]] = Xi[ok]
        L[todo[ok]] = Li[ok]
        sel_rows.append((todo[ok], _pick_views(rng, vis[ok], Li[ok])))
        todo = todo[~ok]
        if todo.size == 0:
            break
    if todo.size:
        raise RuntimeError("ring scene: could not place every point")
    obs_cam, obs_pt = _flatten_tracks(sel_rows)
    fixed = np.zeros(n_cams, dtype=np.uint8)
    fixed[0] = 1
    return _finish(name, seed, rng, K, width, height, R, C, X, obs_cam, obs_pt, sigma=sigma,
                   outlier_frac=outlier_frac, rot_sigma=rot_sigma, pos_sigma=pos_sigma,
                   pt_sigma=pt_sigma, fixed=fixed, settings=settings)


def _flatten_tracks(sel_rows):
    cams, pts = [], []
    for rows, sel in sel_rows:
        if rows.size == 0:
            continue
        valid = sel >= 0
        cams.append(sel[valid])
        pts.append(np.broadcast_to(rows[:, None], sel.shape)[valid])
    obs_cam = np.concatenate(cams).astype(np.int64)
    obs_pt = np.concatenate(pts).astype(np.int64)
    order = np.lexsort((obs_cam, obs_pt))
    return obs_cam[order], obs_pt[order]


# --------------------------------------------------------------------------- road scenes

def _road_points(rng, n, base, tangent, road_frac, road_half_width=6.0,
                 facade=(8.0, 15.0), facade_height=10.0):
    """Points on the road plane (z = 0) or on facades beside it, placed
    relative to base points and unit road tangents (both (n, 3))."""
    left = np.stack([-tangent[:, 1], tangent[:, 0], np.zeros(n)], axis=1)
    left /= np.linalg.norm(left, axis=1, keepdims=True)
    on_road = rng.random(n) < road_frac
    lat = np.where(on_road, rng.uniform(-road_half_width, road_half_width, n),
                   rng.choice([-1.0, 1.0], n) * rng.uniform(facade[0], facade[1], n))
    h = np.where(on_road, 0.0, rng.uniform(0.0, facade_height, n))
    X = base + lat[:, None] * left
    X[:, 2] = h
    return X


def _driving_scene(name, seed, n_cams=1000, n_pts=200_000, length_m=2000.0, *, f=1000.0,
                   width=1920, height=1080, cam_height=1.5, sigma=0.7, outlier_frac=0.02,
                   mean_track=6.0, max_track=30, max_depth=60.0, settings=None):
    """A smooth road; cameras at equal arc spacing face along it; each point
    is seen by L ~ Geometric(1/mean) (clamped to 2..max) consecutive cameras
    from the run of cameras that have it in view."""
    rng = _rng(seed)
    K = _intrinsics(f, width, height)
    a1, l1, a2, l2 = 20.0, 800.0, 6.0, 300.0
    phase = rng.uniform(0, 2 * np.pi)
    xs = np.linspace(0.0, length_m * 1.2, 400_001)
    ys = a1 * np.sin(2 * np.pi * xs / l1) + a2 * np.sin(2 * np.pi * xs / l2 + phase)
    arc = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(xs), np.diff(ys)))])

    def road_at(s):
        x = np.interp(s, arc, xs)
        y = a1 * np.sin(2 * np.pi * x / l1) + a2 * np.sin(2 * np.pi * x / l2 + phase)
        dy = (a1 * 2 * np.pi / l1 * np.cos(2 * np.pi * x / l1)
              + a2 * 2 * np.pi / l2 * np.cos(2 * np.pi * x / l2 + phase))
        p = np.stack([x, y, np.zeros_like(x)], axis=1)
        tg = np.stack([np.ones_like(x), dy, np.zeros_like(x)], axis=1)
        return p, tg / np.linalg.norm(tg, axis=1, keepdims=True)

    spacing = length_m / max(n_cams - 1, 1)
    s_cam = np.arange(n_cams) * spacing
    Cp, Ct = road_at(s_cam)
    C = Cp + np.array([0.0, 0.0, cam_height])
    R = _look_rotation(Ct)
    Pm = _projection_matrices(K, R, C)
    back = int(math.ceil((max_depth + 10.0) / spacing)) + 1
    window = back + 3

    X = np.empty((n_pts, 3))
    sel_rows = []
    todo = np.arange(n_pts)
    for attempt in range(60):
        m = todo.size
        s_p = rng.uniform(0.0, length_m + 0.5 * max_depth, m)
        bp, bt = road_at(s_p)
        Xi = _road_points(rng, m, bp, bt, road_frac=0.35)
        first = np.clip(np.floor(s_p / spacing).astype(np.int64) - back, 0, None)
        cand = first[:, None] + np.arange(window)[None, :]
        valid = cand < n_cams
        cand_c = np.minimum(cand, n_cams - 1)
        uv, w = _image(Pm[cand_c], Xi[:, None, :])
        vis = _in_view(uv, w, width, height, 1.0, max_depth) & valid
        # first run of consecutive cameras that see the point
        start = np.argmax(vis, axis=1)
        has = vis.any(axis=1)
        col = np.arange(window)[None, :]
        stop = (col > start[:, None]) & ~vis
        end = np.where(stop.any(axis=1), np.argmax(stop, axis=1), window)
        run = np.where(has, end - start, 0)
        L = np.clip(rng.geometric(1.0 / mean_track, size=m), 2, max_track)
        ok = run >= 2
        L = np.minimum(L, run)
        off = (rng.random(m) * (run - L + 1)).astype(np.int64)
        ok_idx = np.nonzero(ok)[0]
        X[todo[ok]] = Xi[ok]
        Lo = L[ok]
        Lmax = int(Lo.max()) if Lo.size else 0
        sel = cand[ok_idx, start[ok] + off[ok]][:, None] + np.arange(Lmax)[None, :]
        sel[np.arange(Lmax)[None, :] >= Lo[:, None]] = -1
        sel_rows.append((todo[ok], sel))
        todo = todo[~ok]
        if todo.size == 0:
            break
    if todo.size:
        raise RuntimeError("driving scene: could not place every point")
    obs_cam, obs_pt = _flatten_tracks(sel_rows)
    _check_cameras_seen(obs_cam, n_cams, "driving")
    fixed = np.zeros(n_cams, dtype=np.uint8)
    fixed[0] = 1
    return _finish(name, seed, rng, K, width, height, R, C, X, obs_cam, obs_pt, sigma=sigma,
                   outlier_frac=outlier_frac, rot_sigma=0.01, pos_sigma=0.05, pt_sigma=0.05,
                   fixed=fixed, settings=settings)


def _check_cameras_seen(obs_cam, n_cams, what):
    seen = np.bincount(obs_cam, minlength=n_cams)
    if (seen[1:] == 0).any():
        raise RuntimeError(f"{what} scene: a camera sees no point; use more points")


def _grid_route(rng, n_cams, spacing, extent, block):
    """A random drive on a square street grid (no U-turns), sampled every
    ``spacing`` metres.  Returns camera centres (z=0), headings and the
    visited street segments."""
    nodes = int(round(extent / block)) + 1
    pos = np.array([rng.integers(1, nodes - 1), rng.integers(1, nodes - 1)])
    dirs = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]])
    d = int(rng.integers(0, 4))
    need = n_cams * spacing + block
    pts, heads, segs = [], [], set()
    total = 0.0
    while total < need:
        choices = [d, (d + 1) % 4, (d + 3) % 4]
        rng.shuffle(choices)
        for nd in choices:
            nxt = pos + dirs[nd]
            if 0 <= nxt[0] < nodes and 0 <= nxt[1] < nodes:
                break
        else:
            nd = (d + 2) % 4
            nxt = pos + dirs[nd]
        a = pos * block
        b = nxt * block
        segs.add(tuple(sorted([tuple(pos), tuple(nxt)])))
        pts.append((a.astype(float), b.astype(float)))
        heads.append(dirs[nd].astype(float))
        total += block
        pos, d = nxt, nd
    s = np.arange(n_cams) * spacing + 0.5 * spacing
    seg_idx = np.minimum((s // block).astype(np.int64), len(pts) - 1)
    frac = (s - seg_idx * block) / block
    A = np.array([p[0] for p in pts])[seg_idx]
    B = np.array([p[1] for p in pts])[seg_idx]
    xy = A + frac[:, None] * (B - A)
    hd = np.array(heads)[seg_idx]
    C = np.concatenate([xy, np.zeros((n_cams, 1))], axis=1)
    H = np.concatenate([hd, np.zeros((n_cams, 1))], axis=1)
    return C, H, sorted(segs)


def _zipf_lengths(rng, n, s, lo, hi):
    k = np.arange(lo, hi + 1)
    p = k.astype(float) ** (-s)
    p /= p.sum()
    return rng.choice(k, size=n, p=p)


def _city_scene(name, seed, n_cams=5000, n_pts=1_000_000, *, extent=3000.0, block=250.0,
                spacing=2.0, f=1000.0, width=1920, height=1080, cam_height=1.5, sigma=1.0,
                outlier_frac=0.01, zipf_s=1.5, track_range=(2, 40), max_depth=100.0,
                settings=None):
    """A street-grid route with revisits; each point is seen by L ~ Zipf(s)
    on the track range cameras chosen at random among all that see it."""
    rng = _rng(seed)
    K = _intrinsics(f, width, height)
    C0, H, segs = _grid_route(rng, n_cams, spacing, extent, block)
    C = C0 + np.array([0.0, 0.0, cam_height])
    R = _look_rotation(H)
    Pm = _projection_matrices(K, R, C)
    tree = cKDTree(C)
    seg_a = np.array([[a[0] * block, a[1] * block, 0.0] for a, _ in segs])
    seg_b = np.array([[b[0] * block, b[1] * block, 0.0] for _, b in segs])
    X = np.empty((n_pts, 3))
    sel_rows = []
    todo = np.arange(n_pts)
    lo, hi = track_range
    for attempt in range(60):
        m = todo.size
        si = rng.integers(0, len(segs), m)
        u = rng.random(m)
        base = seg_a[si] + u[:, None] * (seg_b[si] - seg_a[si])
        tg = seg_b[si] - seg_a[si]
        tg /= np.linalg.norm(tg, axis=1, keepdims=True)
        Xi = _road_points(rng, m, base, tg, road_frac=0.35)
        L = _zipf_lengths(rng, m, zipf_s, lo, hi)
        if attempt == 59:
            L = np.full(m, lo)
        nb = tree.query_ball_point(Xi, r=max_depth + 1.0)
        ok = np.zeros(m, dtype=bool)
        rows_sel = []
        for chunk in range(0, m, 65536):
            idx = np.arange(chunk, min(m, chunk + 65536))
            lens = np.fromiter((len(nb[i]) for i in idx), dtype=np.int64, count=idx.size)
            maxc = int(lens.max()) if lens.size else 0
            if maxc == 0:
                continue
            # row r holds the neighbours of point idx[r] in the order the tree
            # returned them, padded with -1
            cand = np.full((idx.size, maxc), -1, dtype=np.int64)
            cand[np.arange(maxc)[None, :] < lens[:, None]] = np.fromiter(
                itertools.chain.from_iterable(nb[i] for i in idx), dtype=np.int64,
                count=int(lens.sum()))
            valid = cand >= 0
            cc = np.where(valid, cand, 0)
            uv, w = _image(Pm[cc], Xi[idx][:, None, :])
            vis = _in_view(uv, w, width, height, 1.0, max_depth) & valid
            nvis = vis.sum(axis=1)
            good = nvis >= L[idx]
            ok[idx[good]] = True
            pick = _pick_views(rng, vis[good], L[idx[good]])
            sel = np.where(pick >= 0, np.take_along_axis(cand[good], np.maximum(pick, 0), axis=1), -1)
            rows_sel.append((todo[idx[good]], sel))
        X[todo[ok]] = Xi[ok]
        sel_rows.extend(rows_sel)
        todo = todo[~ok]
        if todo.size == 0:
            break
    if todo.size:
        raise RuntimeError("city scene: could not place every point")
    obs_cam, obs_pt = _flatten_tracks(sel_rows)
    # a camera that sees nothing would make the problem ill-posed: hold it fixed
    seen = np.bincount(obs_cam, minlength=n_cams)
    fixed = (seen == 0).astype(np.uint8)
    fixed[0] = 1
    return _finish(name, seed, rng, K, width, height, R, C, X, obs_cam, obs_pt, sigma=sigma,
                   outlier_frac=outlier_frac, rot_sigma=0.01, pos_sigma=0.05, pt_sigma=0.05,
                   fixed=fixed, settings=settings)


# --------------------------------------------------------------------------- public API

_SETTINGS = {
    "ring": dict(huber_delta=0.0, lm_iters=10, solver="dense", pcg_tol=1e-6, pcg_max_iters=100,
                 precision="fp64", refine=False),
    "driving": dict(huber_delta=1.0, lm_iters=20, solver="pcg", pcg_tol=1e-6,
                    pcg_max_iters=100, precision="fp32", refine=False),
    "city": dict(huber_delta=1.5, lm_iters=15, solver="pcg", pcg_tol=1e-6, pcg_max_iters=100,
                 precision="fp32", refine=True),
    "window": dict(huber_delta=0.0, lm_iters=5, solver="dense", pcg_tol=1e-6,
                   pcg_max_iters=100, precision="fp32", refine=False),
    "request": dict(huber_delta=0.0, lm_iters=5, solver="dense", pcg_tol=1e-6,
                    pcg_max_iters=100, precision="fp32", refine=False),
}

WORKLOADS = tuple(_SETTINGS)


def _settings(name, overrides):
    s = dict(_SETTINGS[name])
    for k in list(overrides):
        if k in s:
            s[k] = overrides.pop(k)
    return s


def make_scene(name: str, seed: int = 1, **kw) -> Scene:
    """Build a seeded scene of the named workload.  Size keywords (n_cams,
    n_pts, ...) shrink it; solve-setting keywords (huber_delta, lm_iters,
    solver, pcg_tol, pcg_max_iters, precision, refine) override defaults."""
    settings = _settings(name, kw)
    if name == "ring":
        n_cams = kw.pop("n_cams", 20)
        n_pts = kw.pop("n_pts", 2000)
        views = kw.pop("views", 5)
        return _ring_scene(name, seed, n_cams, n_pts,
                           lambda rng, n: np.full(n, views, dtype=np.int64),
                           settings=settings, **kw)
    if name == "driving":
        return _driving_scene(name, seed, settings=settings, **kw)
    if name == "city":
        return _city_scene(name, seed, settings=settings, **kw)
    if name == "window":
        n_cams = kw.pop("n_cams", 30)
        n_pts = kw.pop("n_pts", 2000)
        lo, hi = kw.pop("track_range", (3, 10))
        return _ring_scene(name, seed, n_cams, n_pts,
                           lambda rng, n: rng.integers(lo, hi + 1, n),
                           settings=settings, **kw)
    if name == "request":
        return make_request(seed, **kw)
    raise ValueError(f"unknown workload {name!r}")


def make_windows(n_windows: int = 512, seed: int = 4, cams=(10, 60), pts=(500, 8000),
                 **kw) -> List[Scene]:
    """The batched local-BA workload: independent ring windows with cameras
    uniform in ``cams`` and points uniform in ``pts`` (inclusive)."""
    rng = _rng(seed)
    C = rng.integers(cams[0], cams[1] + 1, n_windows)
    P = rng.integers(pts[0], pts[1] + 1, n_windows)
    seeds = rng.integers(0, 2**31 - 1, n_windows)
    return [make_scene("window", int(s), n_cams=int(c), n_pts=int(p), **kw)
            for c, p, s in zip(C, P, seeds)]


def make_request(seed: int, cams=(10, 200), pts=(1000, 40000), **kw) -> Scene:
    """One served request: cameras and points log-uniform in the given ranges,
    track length 2 + Geometric(mean 3)."""
    settings = _settings("request", kw)
    rng = _rng(seed)
    C = int(round(math.exp(rng.uniform(math.log(cams[0]), math.log(cams[1])))))
    P = int(round(math.exp(rng.uniform(math.log(pts[0]), math.log(pts[1])))))
    return _ring_scene("request", seed, C, P,
                       lambda r, n: 2 + r.geometric(1.0 / 3.0, n),
                       settings=settings, **kw)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 5) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    rng = _rng(seed)
    n = rng.poisson(rate_hz * duration_s * 1.2 + 10)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    return t[t < duration_s]
