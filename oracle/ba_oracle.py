"""FP64 CPU oracle of the Levenberg-Marquardt bundle-adjustment iteration.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import, call or execute this module.  It
shares no code with the CUDA path and imports nothing from it.

What it computes (cuSfM, "Iterative Triangulation and Mapping"):
  * the reprojection error of point X seen by camera T (Sec. 4.3, the
    reprojection equation): e = || pi(K T X) - p_obs ||^2, with pi the
    perspective division and K the pinhole intrinsics (fixed);
  * the robust objective of the first optimisation stage (Sec. 4.3, the
    objective L = sum rho(e_r) + ...): here only the reprojection term, with
    rho = Huber on the squared norm, so F(x) = 1/2 sum_k rho(||r_k||^2);
  * fixed cameras (Sec. 4.3, absolute pose constraints: "arbitrary subsets
    of camera poses can be designated as fixed"), applied as a hard mask.

The paper says no more about its solver than that.  The solver steps follow
published textbook methods, named at each function:
  * Gauss-Newton normal equations with IRLS Huber weights, Schur complement
    on the point blocks: Triggs et al. 2000, "Bundle Adjustment - A Modern
    Synthesis", Sec. 4.3 and 6.1;
  * block-Jacobi preconditioned conjugate gradients on the reduced camera
    system: Agarwal et al. 2010, "Bundle Adjustment in the Large"; CG itself
    as in Hestenes & Stiefel 1952;
  * Levenberg-Marquardt with Marquardt's diagonal scaling, gain ratio and
    Nielsen's damping update: Madsen, Nielsen & Tingleff 2004, "Methods for
    Non-Linear Least Squares Problems", Sec. 3.2, eq. (3.13)-(3.16);
  * SE(3) left retraction through the exponential map (Rodrigues formula).

Readings where the paper is silent (listed with reasons in the design notes):
  * pose convention: world -> camera, x_c = R X + t, quaternion (w, x, y, z);
  * left perturbation: T <- Exp(xi) T with xi = (v, omega);
  * Huber: rho(s) = s for s <= delta^2, else 2 delta sqrt(s) - delta^2;
    weight w = rho'(s) = 1 or delta / sqrt(s); no rho'' term; delta <= 0
    means plain least squares;
  * observations with depth z < 1e-3 get weight 0 and leave the cost;
  * damping: (A + mu D) h = -g with D = diag(A) clamped to >= 1e-12,
    mu_0 = 1e-4, nu_0 = 2; accept iff dL > 0 and gain ratio > 0; optionally
    a floor mu >= mu_min after accepted steps (the reduced-precision path's
    schedule, for comparisons at equal algorithm; 0 by default);
  * PCG starts at x = 0 and stops when ||r|| <= tol ||b|| or after max
    iterations (or early, should p^T S p fail to be positive); the
    city-scale workload wraps it in iterative refinement (at most 5 outer
    steps on the FP64 residual, stop at ||b - S x|| <= 1e-6 ||b||);
  * a Cholesky factorisation that fails (S not numerically positive
    definite) counts as a rejected step.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import scipy.linalg
import scipy.sparse as sp

__all__ = [
    "Z_MIN", "DIAG_MIN", "Problem", "State", "LMOptions", "LMResult",
    "hat", "so3_exp", "so3_left_jacobian", "so3_log", "quat_to_rot", "rot_to_quat",
    "state_from_qt", "state_to_qt", "se3_retract", "retract",
    "huber_rho", "huber_weight", "residuals", "cost", "linearize", "block_sums",
    "damped_blocks", "schur_system", "back_substitute", "full_normal_equations",
    "pcg_block_jacobi", "pcg_refined", "solve_step", "model_decrease", "damping_update", "lm_solve",
    "rmse", "pose_errors", "umeyama_sim3",
]

Z_MIN = 1e-3      # smallest depth at which an observation counts
DIAG_MIN = 1e-12  # floor of the Marquardt scaling diagonal


# ----------------------------------------------------------------------------- rotations

def hat(w: np.ndarray) -> np.ndarray:
    """Skew-symmetric matrices [w]x with [w]x v = w x v.  w: (n, 3)."""
    w = np.asarray(w, dtype=np.float64)
    z = np.zeros(w.shape[:-1])
    return np.stack([
        np.stack([z, -w[..., 2], w[..., 1]], -1),
        np.stack([w[..., 2], z, -w[..., 0]], -1),
        np.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def _so3_coeffs(w):
    th2 = np.sum(w * w, axis=-1)
    th = np.sqrt(th2)
    small = th2 < 1e-10
    ths = np.where(small, 1.0, th)
    a = np.where(small, 1.0 - th2 / 6.0, np.sin(ths) / ths)
    b = np.where(small, 0.5 - th2 / 24.0, (1.0 - np.cos(ths)) / (ths * ths))
    c = np.where(small, 1.0 / 6.0 - th2 / 120.0, (ths - np.sin(ths)) / (ths ** 3))
    return a, b, c


def so3_exp(w: np.ndarray) -> np.ndarray:
    """Rodrigues: Exp(w) = I + sin(t)/t [w]x + (1 - cos t)/t^2 [w]x^2, t = |w|,
    with the Taylor coefficients when t^2 < 1e-10."""
    w = np.atleast_2d(np.asarray(w, dtype=np.float64))
    a, b, _ = _so3_coeffs(w)
    W = hat(w)
    return np.eye(3) + a[:, None, None] * W + b[:, None, None] * (W @ W)


def so3_left_jacobian(w: np.ndarray) -> np.ndarray:
    """V(w) = I + (1 - cos t)/t^2 [w]x + (t - sin t)/t^3 [w]x^2, the matrix that
    maps the translational part of a twist into SE(3)'s exponential."""
    w = np.atleast_2d(np.asarray(w, dtype=np.float64))
    _, b, c = _so3_coeffs(w)
    W = hat(w)
    return np.eye(3) + b[:, None, None] * W + c[:, None, None] * (W @ W)


def so3_log(R: np.ndarray) -> np.ndarray:
    """Rotation vectors of rotation matrices (angle in [0, pi])."""
    R = np.atleast_3d(np.asarray(R, dtype=np.float64)).reshape(-1, 3, 3)
    tr = np.trace(R, axis1=1, axis2=2)
    cos_t = np.clip((tr - 1.0) / 2.0, -1.0, 1.0)
    th = np.arccos(cos_t)
    vee = np.stack([R[:, 2, 1] - R[:, 1, 2], R[:, 0, 2] - R[:, 2, 0],
                    R[:, 1, 0] - R[:, 0, 1]], axis=1)
    out = np.empty((R.shape[0], 3))
    small = th < 1e-6
    near_pi = th > np.pi - 1e-6
    mid = ~(small | near_pi)
    out[small] = 0.5 * vee[small]
    out[mid] = (th[mid] / (2.0 * np.sin(th[mid])))[:, None] * vee[mid]
    for i in np.nonzero(near_pi)[0]:
        # axis from the column of R + I with the largest norm
        B = R[i] + np.eye(3)
        k = int(np.argmax(np.linalg.norm(B, axis=0)))
        axis = B[:, k] / np.linalg.norm(B[:, k])
        out[i] = th[i] * axis
    return out


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    """Rotation matrices of quaternions (w, x, y, z), normalised first."""
    q = np.atleast_2d(np.asarray(q, dtype=np.float64))
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def rot_to_quat(R: np.ndarray) -> np.ndarray:
    """Shepperd's method (1978): quaternion (w, x, y, z), w >= 0, from the
    largest of the four squared-component expressions."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3, 3)
    out = np.empty((R.shape[0], 4))
    for i, M in enumerate(R):
        tr = M[0, 0] + M[1, 1] + M[2, 2]
        cand = [tr, M[0, 0], M[1, 1], M[2, 2]]
        k = int(np.argmax(cand))
        if k == 0:
            s = 2.0 * np.sqrt(1.0 + tr)
            q = [0.25 * s, (M[2, 1] - M[1, 2]) / s, (M[0, 2] - M[2, 0]) / s,
                 (M[1, 0] - M[0, 1]) / s]
        elif k == 1:
            s = 2.0 * np.sqrt(1.0 + M[0, 0] - M[1, 1] - M[2, 2])
            q = [(M[2, 1] - M[1, 2]) / s, 0.25 * s, (M[0, 1] + M[1, 0]) / s,
                 (M[0, 2] + M[2, 0]) / s]
        elif k == 2:
            s = 2.0 * np.sqrt(1.0 + M[1, 1] - M[0, 0] - M[2, 2])
            q = [(M[0, 2] - M[2, 0]) / s, (M[0, 1] + M[1, 0]) / s, 0.25 * s,
                 (M[1, 2] + M[2, 1]) / s]
        else:
            s = 2.0 * np.sqrt(1.0 + M[2, 2] - M[0, 0] - M[1, 1])
            q = [(M[1, 0] - M[0, 1]) / s, (M[0, 2] + M[2, 0]) / s,
                 (M[1, 2] + M[2, 1]) / s, 0.25 * s]
        q = np.asarray(q)
        out[i] = q if q[0] >= 0 else -q
    return out


# ----------------------------------------------------------------------------- problem/state

@dataclasses.dataclass
class Problem:
    """Observations p_obs of point obs_pt in camera obs_cam (Sec. 4.3), the
    shared pinhole intrinsics and the fixed-camera mask (Sec. 4.3, absolute
    pose constraints)."""
    fx: float
    fy: float
    cx: float
    cy: float
    obs_cam: np.ndarray
    obs_pt: np.ndarray
    obs_uv: np.ndarray
    cam_fixed: np.ndarray
    n_cams: int
    n_pts: int

    @classmethod
    def from_arrays(cls, intrinsics, obs_cam, obs_pt, obs_uv, cam_fixed, n_cams, n_pts):
        fx, fy, cx, cy = (float(v) for v in intrinsics)
        fixed = (np.zeros(n_cams, dtype=bool) if cam_fixed is None
                 else np.asarray(cam_fixed).astype(bool))
        return cls(fx, fy, cx, cy, np.asarray(obs_cam, dtype=np.int64),
                   np.asarray(obs_pt, dtype=np.int64),
                   np.asarray(obs_uv, dtype=np.float64).reshape(-1, 2), fixed,
                   int(n_cams), int(n_pts))

    @property
    def n_obs(self):
        return int(self.obs_cam.shape[0])


@dataclasses.dataclass
class State:
    """Camera poses (world -> camera rotation R and translation t) and points."""
    R: np.ndarray   # (C, 3, 3)
    t: np.ndarray   # (C, 3)
    X: np.ndarray   # (P, 3)

    def copy(self):
        return State(self.R.copy(), self.t.copy(), self.X.copy())


def state_from_qt(cam_qt: np.ndarray, pts: np.ndarray) -> State:
    cam_qt = np.asarray(cam_qt, dtype=np.float64).reshape(-1, 7)
    return State(quat_to_rot(cam_qt[:, :4]), cam_qt[:, 4:].copy(),
                 np.asarray(pts, dtype=np.float64).reshape(-1, 3).copy())


def state_to_qt(st: State) -> np.ndarray:
    return np.concatenate([rot_to_quat(st.R), st.t], axis=1)


def se3_retract(R, t, xi):
    """Left retraction T <- Exp(xi) T for xi = (v, omega):
    R <- Exp(omega) R,  t <- Exp(omega) t + V(omega) v."""
    xi = np.atleast_2d(xi)
    v, om = xi[:, :3], xi[:, 3:]
    E = so3_exp(om)
    V = so3_left_jacobian(om)
    R2 = E @ R
    t2 = np.einsum("nij,nj->ni", E, t) + np.einsum("nij,nj->ni", V, v)
    return R2, t2


def retract(st: State, dc: np.ndarray, dp: np.ndarray) -> State:
    """x (+) h: every camera retracted by its 6-vector (zero for fixed cameras),
    every point moved by its 3-vector."""
    R2, t2 = se3_retract(st.R, st.t, dc.reshape(-1, 6))
    return State(R2, t2, st.X + dp.reshape(-1, 3))


# ----------------------------------------------------------------------------- residuals

def huber_rho(s: np.ndarray, delta: float) -> np.ndarray:
    """rho(s) = s for s <= delta^2, 2 delta sqrt(s) - delta^2 beyond (Huber
    applied to the squared norm s); delta <= 0: rho(s) = s."""
    s = np.asarray(s, dtype=np.float64)
    if delta <= 0:
        return s.copy()
    d2 = delta * delta
    return np.where(s <= d2, s, 2.0 * delta * np.sqrt(np.maximum(s, d2)) - d2)


def huber_weight(s: np.ndarray, delta: float) -> np.ndarray:
    """IRLS weight w = rho'(s): 1 for s <= delta^2, delta / sqrt(s) beyond."""
    s = np.asarray(s, dtype=np.float64)
    if delta <= 0:
        return np.ones_like(s)
    d2 = delta * delta
    return np.where(s <= d2, 1.0, delta / np.sqrt(np.maximum(s, d2)))


def residuals(prob: Problem, st: State):
    """r_k = pi(K (R X + t)) - p_obs for every observation (Sec. 4.3,
    reprojection equation) and the camera-frame points x_c.  Returns (r, xc,
    valid) with valid = depth >= Z_MIN; r is 0 where not valid."""
    R = st.R[prob.obs_cam]
    xc = np.einsum("nij,nj->ni", R, st.X[prob.obs_pt]) + st.t[prob.obs_cam]
    z = xc[:, 2]
    valid = z >= Z_MIN
    zs = np.where(valid, z, 1.0)
    u = prob.fx * xc[:, 0] / zs + prob.cx
    v = prob.fy * xc[:, 1] / zs + prob.cy
    r = np.stack([u, v], axis=1) - prob.obs_uv
    r[~valid] = 0.0
    return r, xc, valid


def cost(prob: Problem, st: State, delta: float) -> float:
    """F(x) = 1/2 sum_k rho(||r_k||^2) over observations in front of the camera."""
    r, _, valid = residuals(prob, st)
    s = np.sum(r * r, axis=1)
    return 0.5 * float(np.sum(huber_rho(s[valid], delta)))


def linearize(prob: Problem, st: State, delta: float):
    """Residuals, IRLS weights and analytic Jacobians of every observation.

    dr/dx_c = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]];
    camera: J_c = dr/dx_c [I | -[x_c]x] for the left perturbation
    x_c <- Exp(xi) x_c = x_c + v + omega x x_c (zero for fixed cameras);
    point:  J_p = dr/dx_c R.
    Returns r (N,2), w (N,), Jc (N,2,6), Jp (N,2,3)."""
    r, xc, valid = residuals(prob, st)
    s = np.sum(r * r, axis=1)
    w = np.where(valid, huber_weight(s, delta), 0.0)
    z = np.where(valid, xc[:, 2], 1.0)
    x, y = xc[:, 0], xc[:, 1]
    N = prob.n_obs
    D = np.zeros((N, 2, 3))
    D[:, 0, 0] = prob.fx / z
    D[:, 0, 2] = -prob.fx * x / (z * z)
    D[:, 1, 1] = prob.fy / z
    D[:, 1, 2] = -prob.fy * y / (z * z)
    D[~valid] = 0.0
    dxc = np.concatenate([np.broadcast_to(np.eye(3), (N, 3, 3)), -hat(xc)], axis=2)
    Jc = D @ dxc
    Jc[prob.cam_fixed[prob.obs_cam]] = 0.0
    Jp = D @ st.R[prob.obs_cam]
    return r, w, Jc, Jp


def _segment_sum(values: np.ndarray, index: np.ndarray, n: int) -> np.ndarray:
    """out[i] = sum of values[k] over k with index[k] == i (incidence product)."""
    N = values.shape[0]
    E = sp.csr_matrix((np.ones(N), (index, np.arange(N))), shape=(n, N))
    out = E @ values.reshape(N, -1)
    return np.asarray(out).reshape((n,) + values.shape[1:])


def block_sums(prob: Problem, r, w, Jc, Jp):
    """Blocks of A = sum w J^T J and g = sum w J^T r (Triggs 2000, Sec. 6.1):
    U_i = sum w Jc^T Jc, V_j = sum w Jp^T Jp, W_k = w Jc^T Jp (per observation),
    g_c,i = sum w Jc^T r, g_p,j = sum w Jp^T r."""
    wJc = w[:, None, None] * Jc
    wJp = w[:, None, None] * Jp
    U = _segment_sum(np.einsum("nai,naj->nij", wJc, Jc), prob.obs_cam, prob.n_cams)
    V = _segment_sum(np.einsum("nai,naj->nij", wJp, Jp), prob.obs_pt, prob.n_pts)
    W = np.einsum("nai,naj->nij", wJc, Jp)
    gc = _segment_sum(np.einsum("nai,na->ni", wJc, r), prob.obs_cam, prob.n_cams)
    gp = _segment_sum(np.einsum("nai,na->ni", wJp, r), prob.obs_pt, prob.n_pts)
    return U, V, W, gc, gp


def damped_blocks(U, V, mu):
    """Marquardt damping of the diagonal blocks: X* = X + mu diag(D), D the
    diagonal of X floored at DIAG_MIN.  Returns (U*, V*, Dc, Dp)."""
    Dc = np.maximum(np.diagonal(U, axis1=1, axis2=2), DIAG_MIN)
    Dp = np.maximum(np.diagonal(V, axis1=1, axis2=2), DIAG_MIN)
    Us = U + mu * (Dc[:, :, None] * np.eye(6))
    Vs = V + mu * (Dp[:, :, None] * np.eye(3))
    return Us, Vs, Dc, Dp


def _free_index(prob: Problem):
    free = np.nonzero(~prob.cam_fixed)[0]
    pos = np.full(prob.n_cams, -1, dtype=np.int64)
    pos[free] = np.arange(free.size)
    return free, pos


def _w_matrix(prob: Problem, W):
    """The 6F x 3P matrix whose (camera, point) block is the sum of W_k over the
    observations of that pair (F = number of free cameras)."""
    free, pos = _free_index(prob)
    keep = pos[prob.obs_cam] >= 0
    ci = pos[prob.obs_cam[keep]]
    pj = prob.obs_pt[keep]
    rows = (ci[:, None, None] * 6 + np.arange(6)[None, :, None]) * np.ones((1, 1, 3), dtype=np.int64)
    cols = (pj[:, None, None] * 3 + np.arange(3)[None, None, :]) * np.ones((1, 6, 1), dtype=np.int64)
    return sp.csr_matrix((W[keep].ravel(), (rows.ravel(), cols.ravel())),
                         shape=(6 * free.size, 3 * prob.n_pts))


def schur_system(prob: Problem, Us, Vs, W, gc, gp):
    """Reduced camera system of (A + mu D) h = -g after eliminating the points
    (Triggs 2000, Sec. 6.1; Agarwal 2010, Sec. 3):
        S = U* - W V*^-1 W^T,   b = -g_c + W V*^-1 g_p,
    over the free cameras.  Returns (S dense, b, V*^-1 (P,3,3), Wm)."""
    free, _ = _free_index(prob)
    Vinv = np.linalg.inv(Vs)
    Wm = _w_matrix(prob, W)
    P = prob.n_pts
    Vi = sp.bsr_matrix((Vinv, np.arange(P), np.arange(P + 1)), shape=(3 * P, 3 * P)).tocsr()
    WVi = Wm @ Vi
    S = scipy.linalg.block_diag(*Us[free]) if free.size else np.zeros((0, 0))
    S = S - (WVi @ Wm.T).toarray()
    b = -gc[free].ravel() + WVi @ gp.ravel()
    return S, b, Vinv, Wm


def back_substitute(prob: Problem, Vinv, Wm, gp, dc_free):
    """dp_j = V*_j^-1 (-g_p,j - sum_k W_k^T dc_i(k)) for every point."""
    rhs = -gp.ravel() - Wm.T @ dc_free
    return np.einsum("nij,nj->ni", Vinv, rhs.reshape(-1, 3))


def full_normal_equations(prob: Problem, st: State, delta: float):
    """Dense A = J^T diag(w) J and g = J^T diag(w) r over all unknowns (free
    cameras, then points), built from the stacked Jacobian.  For tiny problems."""
    r, w, Jc, Jp = linearize(prob, st, delta)
    free, pos = _free_index(prob)
    n = 6 * free.size + 3 * prob.n_pts
    J = np.zeros((2 * prob.n_obs, n))
    for k in range(prob.n_obs):
        i = pos[prob.obs_cam[k]]
        if i >= 0:
            J[2 * k:2 * k + 2, 6 * i:6 * i + 6] = Jc[k]
        j = prob.obs_pt[k]
        o = 6 * free.size + 3 * j
        J[2 * k:2 * k + 2, o:o + 3] = Jp[k]
    wr = np.repeat(w, 2)
    A = J.T @ (wr[:, None] * J)
    g = J.T @ (wr * r.ravel())
    return A, g


# ----------------------------------------------------------------------------- linear solvers

def pcg_block_jacobi(S: np.ndarray, b: np.ndarray, tol: float, max_iters: int, block: int = 6):
    """Conjugate gradients (Hestenes & Stiefel 1952) on S x = b preconditioned
    by M = blockdiag(S_ii)^-1 (6x6 diagonal blocks; Agarwal 2010).  Starts at
    x = 0; stops when ||r|| <= tol ||b|| or after max_iters products with S.
    Returns (x, iterations, ||r|| / ||b||)."""
    n = b.shape[0]
    nb = n // block
    Minv = np.stack([np.linalg.inv(S[i * block:(i + 1) * block, i * block:(i + 1) * block])
                     for i in range(nb)]) if nb else np.zeros((0, block, block))

    def precond(v):
        return np.einsum("nij,nj->ni", Minv, v.reshape(nb, block)).ravel()

    x = np.zeros(n)
    r = b.copy()
    bnorm = float(np.linalg.norm(b))
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    k = 0
    while k < max_iters and float(np.linalg.norm(r)) > tol * bnorm:
        q = S @ p
        pq = float(p @ q)
        if not pq > 0:
            break             # S not numerically positive definite along p
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    rel = float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0
    return x, k, rel


def pcg_refined(S: np.ndarray, b: np.ndarray, tol: float, max_iters: int, refine_max: int,
                refine_tol: float):
    """Iterative refinement around the PCG above (Carson & Higham 2018), the
    solver of the city-scale mapping workload (reading C11): from x = 0, at
    most refine_max times compute the residual r = b - S x, stop once
    ||r|| <= refine_tol ||b||, else solve S d = r by PCG (tol, max_iters) and
    set x = x + d.  With the residual in the same FP64 as everything else
    this is PCG restarted from the current iterate.  Returns (x, total
    products with S, ||b - S x|| / ||b||)."""
    x = np.zeros_like(b)
    bnorm = float(np.linalg.norm(b))
    total = 0
    for _ in range(refine_max):
        r = b - S @ x
        if float(np.linalg.norm(r)) <= refine_tol * bnorm:
            break
        d, k, _ = pcg_block_jacobi(S, r, tol, max_iters)
        x = x + d
        total += k
    rel = float(np.linalg.norm(b - S @ x)) / bnorm if bnorm > 0 else 0.0
    return x, total, rel


# ----------------------------------------------------------------------------- LM

@dataclasses.dataclass
class LMOptions:
    huber_delta: float = 0.0
    lm_iters: int = 10
    solver: str = "dense"        # "dense" (Schur + Cholesky), "pcg" (Schur + PCG), "full"
    pcg_tol: float = 1e-6
    pcg_max_iters: int = 100
    refine_max: int = 0          # > 0: PCG inside iterative refinement (pcg_refined)
    refine_tol: float = 1e-6
    mu0: float = 1e-4
    nu0: float = 2.0
    mu_min: float = 0.0          # damping floor after an accepted step (the FP32 path's, C15)
    prior_seq: float = 0.0       # lambda_c of the sequential pose prior (oracle/priors.py)
    prior_abs: float = 0.0       # lambda_a of the absolute pose prior


@dataclasses.dataclass
class LMResult:
    costs: np.ndarray        # F before the first and after every iteration (iters + 1)
    accepted: np.ndarray     # (iters,) bool
    mu: np.ndarray           # (iters,) damping used by each iteration's solve
    pcg_iters: np.ndarray    # (iters,) CG products (0 for direct solves)
    gain: np.ndarray         # (iters,) gain ratio (-inf where dL <= 0)
    dL: np.ndarray           # (iters,) model decrease
    state: State


def solve_step(prob: Problem, lin, mu: float, opts: LMOptions):
    """Solve (A + mu D) h = -g through the Schur complement (or densely, for
    solver == "full").  Returns (dc (C,6), dp (P,3), D (unknown order),
    g (unknown order), h (unknown order), cg iterations), or None when the
    Cholesky factorisation of S fails."""
    free, _ = _free_index(prob)
    if opts.solver == "full":
        A, g, st = lin["A"], lin["g"], None
        Dg = np.maximum(np.diag(A), DIAG_MIN)
        h = np.linalg.solve(A + mu * np.diag(Dg), -g)
        dc = np.zeros((prob.n_cams, 6))
        dc[free] = h[:6 * free.size].reshape(-1, 6)
        dp = h[6 * free.size:].reshape(-1, 3)
        return dc, dp, Dg, g, h, 0
    U, V, W, gc, gp = lin["U"], lin["V"], lin["W"], lin["gc"], lin["gp"]
    Us, Vs, Dc, Dp = damped_blocks(U, V, mu)
    S, b, Vinv, Wm = schur_system(prob, Us, Vs, W, gc, gp)
    if lin.get("cpl") is not None:
        # the sequential prior couples adjacent free cameras (undamped)
        _, pos = _free_index(prob)
        for i, B in enumerate(lin["cpl"]):
            a, c = pos[i], pos[i + 1]
            if a >= 0 and c >= 0:
                S[6 * a:6 * a + 6, 6 * c:6 * c + 6] += B
                S[6 * c:6 * c + 6, 6 * a:6 * a + 6] += B.T
    iters = 0
    if free.size == 0:
        dcf = np.zeros(0)
    elif opts.solver == "dense":
        try:
            dcf = scipy.linalg.cho_solve(scipy.linalg.cho_factor(S, lower=True), b)
        except np.linalg.LinAlgError:
            return None       # S not numerically positive definite: no step
    elif opts.solver == "pcg" and opts.refine_max > 0:
        dcf, iters, _ = pcg_refined(S, b, opts.pcg_tol, opts.pcg_max_iters, opts.refine_max,
                                    opts.refine_tol)
    elif opts.solver == "pcg":
        dcf, iters, _ = pcg_block_jacobi(S, b, opts.pcg_tol, opts.pcg_max_iters)
    else:
        raise ValueError(opts.solver)
    dp = back_substitute(prob, Vinv, Wm, gp, dcf)
    dc = np.zeros((prob.n_cams, 6))
    dc[free] = dcf.reshape(-1, 6)
    D = np.concatenate([Dc[free].ravel(), Dp.ravel()])
    g = np.concatenate([gc[free].ravel(), gp.ravel()])
    h = np.concatenate([dcf, dp.ravel()])
    return dc, dp, D, g, h, iters


def model_decrease(h, D, g, mu):
    """L(0) - L(h) = 1/2 h^T (mu D h - g) for the damped Gauss-Newton model
    (Madsen, Nielsen & Tingleff 2004, eq. 3.14 with D-scaled damping)."""
    return 0.5 * float(h @ (mu * D * h - g))


def damping_update(mu, nu, gain, accepted):
    """Nielsen's damping update (Madsen, Nielsen & Tingleff 2004, Sec. 3.2,
    eq. 3.16 with Nielsen's nu rule), returning the new (mu, nu).  After an
    accepted step mu shrinks by max(1/3, 1 - (2 gain - 1)^3): a third for a
    step the model predicted exactly (gain 1), unchanged at gain 1/2, doubled
    as gain tends to 0; nu restarts at 2.  After a rejected step mu grows by
    nu and nu doubles, so repeated rejections raise the damping
    geometrically faster."""
    if accepted:
        return mu * max(1.0 / 3.0, 1.0 - (2.0 * gain - 1.0) ** 3), 2.0
    return mu * nu, 2.0 * nu


def _linearization(prob, st, opts, pri=None):
    dU = dg = cpl = None
    if pri is not None:
        from .priors import prior_blocks
        dU, dg, cpl = prior_blocks(st, pri, prob.cam_fixed)
    if opts.solver == "full":
        A, g = full_normal_equations(prob, st, opts.huber_delta)
        if pri is not None:
            free, pos = _free_index(prob)
            for i in free:
                a = 6 * pos[i]
                A[a:a + 6, a:a + 6] += dU[i]
                g[a:a + 6] += dg[i]
            for i, B in enumerate(cpl):
                a, c = pos[i], pos[i + 1]
                if a >= 0 and c >= 0:
                    A[6 * a:6 * a + 6, 6 * c:6 * c + 6] += B
                    A[6 * c:6 * c + 6, 6 * a:6 * a + 6] += B.T
        return {"A": A, "g": g}
    r, w, Jc, Jp = linearize(prob, st, opts.huber_delta)
    U, V, W, gc, gp = block_sums(prob, r, w, Jc, Jp)
    if pri is not None:
        U = U + dU
        gc = gc + dg
    return {"U": U, "V": V, "W": W, "gc": gc, "gp": gp, "cpl": cpl}


def lm_solve(prob: Problem, st0: State, opts: LMOptions) -> LMResult:
    """Levenberg-Marquardt (Madsen, Nielsen & Tingleff 2004, Algorithm 3.16)
    for a fixed number of iterations; an iteration is one linear solve and
    one trial step, accepted or rejected.  A rejected step keeps the
    linearisation (the state did not change) and raises the damping."""
    st = st0.copy()
    mu, nu = opts.mu0, opts.nu0
    pri = None
    if opts.prior_seq > 0 or opts.prior_abs > 0:
        # pose priors (Sec. 4.2 Eq. seq, Sec. 4.3 Eq. abs), measured on st0
        from .priors import Priors, prior_cost
        pri = Priors(st0, opts.prior_seq, opts.prior_abs)
        F_of = lambda x: cost(prob, x, opts.huber_delta) + prior_cost(x, pri)
    else:
        F_of = lambda x: cost(prob, x, opts.huber_delta)
    F = F_of(st)
    costs, acc, mus, cg, gains, dLs = [F], [], [], [], [], []
    lin = None
    for _ in range(opts.lm_iters):
        if lin is None:
            lin = _linearization(prob, st, opts, pri)
        step = solve_step(prob, lin, mu, opts)
        if step is None:      # failed factorisation counts as a rejected step
            dL, F_new, iters = -np.inf, F, 0
        else:
            dc, dp, D, g, h, iters = step
            dL = model_decrease(h, D, g, mu)
            cand = retract(st, dc, dp)
            F_new = F_of(cand)
        gain = (F - F_new) / dL if dL > 0 else -np.inf
        mus.append(mu)
        cg.append(iters)
        gains.append(gain)
        dLs.append(dL)
        accept = bool(dL > 0 and gain > 0)
        mu, nu = damping_update(mu, nu, gain, accept)
        if accept:
            mu = max(mu, opts.mu_min)
            st, F = cand, F_new
            lin = None
        acc.append(accept)
        costs.append(F)
    return LMResult(np.array(costs), np.array(acc, dtype=bool), np.array(mus),
                    np.array(cg, dtype=np.int64), np.array(gains), np.array(dLs), st)


# ----------------------------------------------------------------------------- metrics

def rmse(prob: Problem, st: State, mask: Optional[np.ndarray] = None,
         threshold: Optional[float] = None) -> float:
    """sqrt(sum ||r_k||^2 / n) px over the observations in front of the camera
    (and in mask, when given).  With a threshold, observations whose
    reprojection error exceeds it are left out, as the mapping loop removes
    them after each BA round (Sec. 4.3, outlier removal)."""
    r, _, valid = residuals(prob, st)
    sel = valid if mask is None else (valid & np.asarray(mask, dtype=bool))
    if threshold is not None:
        sel = sel & (np.sum(r * r, axis=1) < threshold * threshold)
    if not sel.any():
        return 0.0
    return float(np.sqrt(np.sum(r[sel] ** 2) / sel.sum()))


def pose_errors(Ra, ta, Rb, tb):
    """Per-camera rotation error |Log(Ra Rb^T)| (rad) and camera-centre error
    |Ca - Cb| (m) with C = -R^T t."""
    rot = np.linalg.norm(so3_log(Ra @ np.transpose(Rb, (0, 2, 1))), axis=1)
    Ca = -np.einsum("nji,nj->ni", Ra, ta)
    Cb = -np.einsum("nji,nj->ni", Rb, tb)
    return rot, np.linalg.norm(Ca - Cb, axis=1)


def umeyama_sim3(src: np.ndarray, dst: np.ndarray):
    """Similarity (s, R, t) minimising sum |dst - (s R src + t)|^2
    (Umeyama 1991, eqs. 40-42)."""
    mu_s, mu_d = src.mean(0), dst.mean(0)
    xs, xd = src - mu_s, dst - mu_d
    cov = xd.T @ xs / src.shape[0]
    Uu, Dd, Vt = np.linalg.svd(cov)
    Sg = np.eye(3)
    if np.linalg.det(Uu) * np.linalg.det(Vt) < 0:
        Sg[2, 2] = -1.0
    R = Uu @ Sg @ Vt
    var_s = np.sum(xs * xs) / src.shape[0]
    s = float(np.trace(np.diag(Dd) @ Sg) / var_s)
    t = mu_d - s * R @ mu_s
    return s, R, t
