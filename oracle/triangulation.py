"""FP64 CPU oracle of the steps around bundle adjustment in cuSfM's mapping
loop: per-observation reprojection errors, outlier classification against a
pixel threshold, and DLT triangulation of points from their inlier
observations.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import, call or execute this module.  It
shares no code with the CUDA path and imports nothing from it.

What it computes (cuSfM, Sec. 4.3 "Iterative Triangulation and Mapping"):
  * the reprojection error e = || pi(K T X) - p_obs ||^2 of every observation
    (Sec. 4.3, the reprojection equation), +inf where the point is not in
    front of the camera (depth below Z_MIN);
  * after a BA round, observations whose error exceeds the outlier threshold
    are removed (Sec. 4.3, the alternation of triangulation and BA): here an
    observation is an inlier iff e <= threshold_px^2;
  * the DLT triangulation of Sec. 4.3, Eq. (dlt):
    X = argmin sum_j || P_j X - lambda_j p_j ||^2 over the homogeneous point
    X, with P_j = [R_j | t_j] and p_j the observation in normalised camera
    coordinates K^-1 (u, v, 1).  Eliminating lambda_j leaves two linear rows
    per observation, x P_j^(3) - P_j^(1) and y P_j^(3) - P_j^(2); with
    ||X|| = 1 the minimiser is the eigenvector of A^T A (A the stacked rows)
    of the smallest eigenvalue.

Readings where the paper is silent (listed with reasons in the design notes):
  * DLT in normalised camera coordinates (the paper allows image or
    normalised coordinates; normalised ones keep A^T A well scaled);
  * a point needs at least 2 inlier observations (status 1 otherwise); its
    homogeneous solution must not be at infinity, |X_4| > 1e-12 ||X||
    (status 2); and it must lie in front of every inlier camera, depth >=
    Z_MIN (status 3).  Status 0: triangulated.
"""
from __future__ import annotations

import numpy as np

from .ba_oracle import Z_MIN, Problem, State

__all__ = ["TRI_OK", "TRI_TOO_FEW", "TRI_AT_INFINITY", "TRI_BEHIND",
           "reprojection_errors", "classify_inliers", "triangulate_dlt"]

TRI_OK, TRI_TOO_FEW, TRI_AT_INFINITY, TRI_BEHIND = 0, 1, 2, 3


def reprojection_errors(prob: Problem, st: State) -> np.ndarray:
    """e_k = ||pi(K (R X + t)) - p_obs||^2 for every observation (Sec. 4.3,
    reprojection equation), +inf where the depth is below Z_MIN."""
    xc = np.einsum("nij,nj->ni", st.R[prob.obs_cam], st.X[prob.obs_pt]) + st.t[prob.obs_cam]
    z = xc[:, 2]
    front = z >= Z_MIN
    zs = np.where(front, z, 1.0)
    du = prob.fx * xc[:, 0] / zs + prob.cx - prob.obs_uv[:, 0]
    dv = prob.fy * xc[:, 1] / zs + prob.cy - prob.obs_uv[:, 1]
    e = du * du + dv * dv
    return np.where(front, e, np.inf)


def classify_inliers(err2: np.ndarray, threshold_px: float) -> np.ndarray:
    """Inlier iff the squared error is at most threshold_px^2 (Sec. 4.3:
    projections exceeding the outlier threshold are removed)."""
    return np.asarray(err2) <= threshold_px * threshold_px


def triangulate_dlt(prob: Problem, st: State, mask=None):
    """DLT triangulation (Sec. 4.3, Eq. dlt) of every point from its
    observations with mask True (all when mask is None), with the cameras'
    poses in st.  Returns (X (P, 3), status (P,) int8); X is NaN where the
    status is not TRI_OK."""
    P = prob.n_pts
    use = np.ones(prob.n_obs, dtype=bool) if mask is None else np.asarray(mask, dtype=bool)
    cam = prob.obs_cam[use]
    pt = prob.obs_pt[use]
    # normalised camera coordinates of the observations
    x = (prob.obs_uv[use, 0] - prob.cx) / prob.fx
    y = (prob.obs_uv[use, 1] - prob.cy) / prob.fy
    Pm = np.concatenate([st.R, st.t[:, :, None]], axis=2)[cam]  # (n, 3, 4) = [R | t]
    row1 = x[:, None] * Pm[:, 2, :] - Pm[:, 0, :]
    row2 = y[:, None] * Pm[:, 2, :] - Pm[:, 1, :]
    # A^T A per point: the sum over its observations of both rows' outer products
    outer = np.einsum("ni,nj->nij", row1, row1) + np.einsum("ni,nj->nij", row2, row2)
    AtA = np.zeros((P, 4, 4))
    np.add.at(AtA, pt, outer)
    count = np.bincount(pt, minlength=P)
    status = np.full(P, TRI_OK, dtype=np.int8)
    status[count < 2] = TRI_TOO_FEW
    # eigenvector of the smallest eigenvalue (eigh sorts them ascending)
    _, vecs = np.linalg.eigh(AtA)
    Xh = vecs[:, :, 0]
    w = Xh[:, 3]
    inf = np.abs(w) <= 1e-12 * np.linalg.norm(Xh, axis=1)
    status[(status == TRI_OK) & inf] = TRI_AT_INFINITY
    X = np.full((P, 3), np.nan)
    good = status == TRI_OK
    X[good] = Xh[good, :3] / w[good, None]
    # in front of every inlier camera
    Xo = np.where(np.isfinite(X[pt]), X[pt], 0.0)
    depth = np.einsum("nj,nj->n", st.R[cam, 2, :], Xo) + st.t[cam, 2]
    behind = np.zeros(P, dtype=bool)
    np.logical_or.at(behind, pt, depth < Z_MIN)
    status[good & behind] = TRI_BEHIND
    X[status != TRI_OK] = np.nan
    return X, status
