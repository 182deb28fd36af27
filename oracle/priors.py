"""FP64 CPU oracle of the pose-prior terms of the BA objective.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import, call or execute this module.  It
shares no code with the CUDA path and imports nothing from it.

What it computes (cuSfM):
  * the objective of the first optimisation stage (Sec. 4.3, objective L):
    L = sum rho(e_r) + lambda_c sum e_c + lambda_a sum e_a; with the oracle's
    F = L / 2 convention the priors add 1/2 lambda_c sum e_c + 1/2 lambda_a
    sum e_a to the reprojection cost;
  * the sequential constraint with adjacent frames (Sec. 4.2, Eq. seq, k = 1):
    the squared difference between the current relative pose of frames i and
    i + 1 and T_i^{i+1}, the relative pose measured on the initial trajectory
    ("derived from the initial trajectory", Sec. 4.2; the product order is a
    reading, below);
  * the absolute pose constraint (Sec. 4.3, Eq. abs):
    e_a^(i) = || T_i^w - T_{i,init}^w ||^2.

Readings where the paper is silent (listed with reasons in the design notes):
  * T_i^w is the camera-to-world matrix [R_i^T | -R_i^T t_i] of the solver's
    world-to-camera pose (R_i, t_i); the norms are Frobenius norms of the
    top 3 x 4 blocks (the bottom rows agree);
  * the relative pose T_i^{i+1} is the pose of frame i in frame i + 1, as the
    paper's notation defines it: (T_{i+1}^w)^-1 T_i^w = T_cw,{i+1} T_wc,i.
    The product as printed, T_i^w (T_{i+1}^w)^-1, changes when the world
    frame is moved rigidly (it becomes G Q G^-1), so a measurement "derived
    from the initial trajectory" would depend on the choice of world frame;
  * cameras are in trajectory order, so the adjacent frames of camera i are
    i - 1 and i + 1;
  * the terms enter the Gauss-Newton model like the reprojection term, with
    the same left perturbation T_cw <- Exp(xi) T_cw, xi = (v, omega) (so
    T_wc <- T_wc Exp(-xi)); with xi^ the 4 x 4 twist matrix and Q_i the
    relative pose,
        d e_a:   -T_wc,i xi_i^                  (12 x 6 Jacobian J_a),
        d e_c:   -Q_i xi_i^  +  xi_{i+1}^ Q_i   (J_c,i and J_c,i+1);
    fixed cameras contribute no columns.
"""
from __future__ import annotations

import numpy as np

from .ba_oracle import State, hat

__all__ = ["Priors", "cam_to_world", "relative_seq", "prior_residuals", "prior_cost",
           "prior_jacobians", "prior_blocks"]


def cam_to_world(st: State) -> np.ndarray:
    """Top 3 x 4 blocks of T^w = [R^T | -R^T t] (C, 3, 4)."""
    Rt = np.transpose(st.R, (0, 2, 1))
    c = -np.einsum("nij,nj->ni", Rt, st.t)
    return np.concatenate([Rt, c[:, :, None]], axis=2)


def relative_seq(st: State) -> np.ndarray:
    """Top 3 x 4 blocks of (T_{i+1}^w)^-1 T_i^w = [R_{i+1} R_i^T | t_{i+1} - R_{i+1} R_i^T t_i]
    for i = 0 .. C - 2 (C - 1, 3, 4)."""
    rot = st.R[1:] @ np.transpose(st.R[:-1], (0, 2, 1))
    tr = st.t[1:] - np.einsum("nij,nj->ni", rot, st.t[:-1])
    return np.concatenate([rot, tr[:, :, None]], axis=2)


class Priors:
    """Weights and the measurements taken from the initial state st0."""

    def __init__(self, st0: State, lam_c: float, lam_a: float):
        self.lam_c = float(lam_c)
        self.lam_a = float(lam_a)
        self.anchor = cam_to_world(st0)
        self.meas = relative_seq(st0) if st0.R.shape[0] > 1 else np.zeros((0, 3, 4))


def prior_residuals(st: State, pri: Priors):
    """(r_a (C, 12), r_c (C - 1, 12)): the entries of T_i^w - T_{i,init}^w and of
    (T_{i+1}^w)^-1 T_i^w - T_i^{i+1}, row-major over the top 3 x 4 blocks."""
    ra = (cam_to_world(st) - pri.anchor).reshape(-1, 12)
    rc = (relative_seq(st) - pri.meas).reshape(-1, 12) if st.R.shape[0] > 1 else np.zeros((0, 12))
    return ra, rc


def prior_cost(st: State, pri: Priors) -> float:
    """1/2 (lambda_a sum e_a + lambda_c sum e_c)."""
    ra, rc = prior_residuals(st, pri)
    return 0.5 * (pri.lam_a * float(np.sum(ra * ra)) + pri.lam_c * float(np.sum(rc * rc)))


def _twist(k: int) -> np.ndarray:
    """The 4 x 4 twist matrix of the unit vector e_k of xi = (v, omega)."""
    X = np.zeros((4, 4))
    if k < 3:
        X[k, 3] = 1.0
    else:
        X[:3, :3] = hat(np.eye(3)[k - 3])
    return X


def _homog(M34: np.ndarray) -> np.ndarray:
    H = np.zeros(M34.shape[:-2] + (4, 4))
    H[..., :3, :] = M34
    H[..., 3, 3] = 1.0
    return H


def prior_jacobians(st: State):
    """(J_a (C, 12, 6), Ji (C - 1, 12, 6), Jj (C - 1, 12, 6)): derivatives of
    the residual entries with respect to xi at 0: the absolute residual of
    camera i, and the sequential residual of pair (i, i + 1) with respect to
    camera i (Ji) and camera i + 1 (Jj)."""
    Twc = _homog(cam_to_world(st))
    C = st.R.shape[0]
    Q = _homog(relative_seq(st)) if C > 1 else np.zeros((0, 4, 4))
    Ja = np.zeros((C, 12, 6))
    Ji = np.zeros((max(C - 1, 0), 12, 6))
    Jj = np.zeros((max(C - 1, 0), 12, 6))
    for k in range(6):
        X = _twist(k)
        Ja[:, :, k] = -(Twc @ X)[:, :3, :].reshape(C, 12)
        if C > 1:
            Ji[:, :, k] = -(Q @ X)[:, :3, :].reshape(C - 1, 12)
            Jj[:, :, k] = (X @ Q)[:, :3, :].reshape(C - 1, 12)
    return Ja, Ji, Jj


def prior_blocks(st: State, pri: Priors, fixed: np.ndarray):
    """Gauss-Newton contributions of the priors over the cameras:
    dU (C, 6, 6), dg (C, 6) and the coupling blocks cpl (C - 1, 6, 6) of
    (i, i + 1) (zero where either camera is fixed; its transpose couples
    (i + 1, i)).  Fixed cameras get no contribution."""
    ra, rc = prior_residuals(st, pri)
    Ja, Ji, Jj = prior_jacobians(st)
    C = st.R.shape[0]
    free = ~np.asarray(fixed, dtype=bool)
    dU = pri.lam_a * np.einsum("nai,naj->nij", Ja, Ja)
    dg = pri.lam_a * np.einsum("nai,na->ni", Ja, ra)
    cpl = np.zeros((max(C - 1, 0), 6, 6))
    if C > 1:
        lc = pri.lam_c
        dU[:-1] += lc * np.einsum("nai,naj->nij", Ji, Ji)
        dU[1:] += lc * np.einsum("nai,naj->nij", Jj, Jj)
        dg[:-1] += lc * np.einsum("nai,na->ni", Ji, rc)
        dg[1:] += lc * np.einsum("nai,na->ni", Jj, rc)
        both = free[:-1] & free[1:]
        cpl[both] = lc * np.einsum("nai,naj->nij", Ji, Jj)[both]
    dU[~free] = 0.0
    dg[~free] = 0.0
    return dU, dg, cpl
