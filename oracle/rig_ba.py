"""FP64 CPU oracle of rig bundle adjustment with extrinsic refinement.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import, call or execute this module.  It
shares no code with the CUDA path and imports nothing from it.

What it computes (cuSfM, Sec. 4.4 "Extrinsic Refinement"):
  * every camera pose is the composition of a vehicle pose and a
    camera-to-vehicle extrinsic, T_c = T_c^v T_v^w, so the reprojection error
    of point X_i seen by rig camera c of frame f is
        e = || pi(K_c T_c^v T_{v_f}^w X_i) - p_obs ||^2;
  * the unknowns are the vehicle poses (one per frame), the extrinsics (one
    per rig camera, shared by all frames) and the points;
  * prior information on the extrinsics enters through absolute pose
    constraints on T_c^v, weighted by lambda_e (Sec. 4.4, Eq. abs applied to
    the extrinsics).

Readings where the paper is silent (listed with reasons in the design notes):
  * T_{v}^w maps world to vehicle coordinates and T_c^v vehicle to camera
    coordinates (the only order in which the printed composition maps world
    points into the camera); both are stored like BA poses (R, t);
  * the perturbations are left ones on both factors, V <- Exp(xi_V) V and
    E <- Exp(xi_E) E, so the composite camera moves by
        xi_cam = Ad(E) xi_V + xi_E,   Ad(E) = [[R_E, [t_E]x R_E], [0, R_E]]
    for xi = (v, omega): J_V = J_cam Ad(E), J_E = J_cam with J_cam the BA
    camera Jacobian of the composite pose;
  * the extrinsic prior is 1/2 lambda_e ||(T_c^v)^-1 - (T_c^v)_init^-1||^2 over
    the top 3 x 4 blocks (the camera-to-vehicle transform, compared like the
    absolute pose prior of the BA objective compares camera-to-world
    transforms), measured on the initial extrinsics;
  * the gauge: fixed frames keep their vehicle pose (fixing one removes the
    6-DoF freedom V -> H V, E -> E H^-1 as well as the rigid world motion;
    scale is left to the damping); fixed extrinsics keep theirs;
  * the solver is the BA oracle's Levenberg-Marquardt (Marquardt scaling,
    mu_0 = 1e-4, nu_0 = 2, accept iff dL > 0 and gain > 0, Huber IRLS,
    cheirality as in BA) on the full normal equations (small problems).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg

from . import ba_oracle as B
from . import priors as PR

__all__ = ["RigProblem", "RigState", "RigOptions", "RigResult", "adjoint", "composite",
           "rig_cost", "rig_jacobians", "rig_normal_equations", "rig_retract", "rig_lm_solve"]


@dataclasses.dataclass
class RigProblem:
    """Observation k: point obs_pt[k] seen by rig camera obs_rc[k] of frame
    obs_frame[k]; intrinsics per rig camera (R, 4) = (fx, fy, cx, cy)."""
    intrinsics: np.ndarray
    obs_frame: np.ndarray
    obs_rc: np.ndarray
    obs_pt: np.ndarray
    obs_uv: np.ndarray
    frame_fixed: np.ndarray
    rc_fixed: np.ndarray
    n_frames: int
    n_rc: int
    n_pts: int

    @property
    def n_obs(self) -> int:
        return int(self.obs_pt.shape[0])


@dataclasses.dataclass
class RigState:
    Rv: np.ndarray   # (F, 3, 3) world -> vehicle
    tv: np.ndarray   # (F, 3)
    Re: np.ndarray   # (R, 3, 3) vehicle -> camera
    te: np.ndarray   # (R, 3)
    X: np.ndarray    # (P, 3)

    def copy(self):
        return RigState(self.Rv.copy(), self.tv.copy(), self.Re.copy(), self.te.copy(),
                        self.X.copy())


def adjoint(R, t):
    """Ad(T) for poses T = (R, t) (R: (n, 3, 3)) acting on xi = (v, omega):
    [[R, [t]x R], [0, R]]."""
    n = R.shape[0]
    A = np.zeros((n, 6, 6))
    A[:, :3, :3] = R
    A[:, :3, 3:] = B.hat(t) @ R
    A[:, 3:, 3:] = R
    return A


def composite(prob: RigProblem, st: RigState):
    """Per observation: the composite camera pose (R_c, t_c) = E_c V_f."""
    Re, te = st.Re[prob.obs_rc], st.te[prob.obs_rc]
    Rv, tv = st.Rv[prob.obs_frame], st.tv[prob.obs_frame]
    Rc = Re @ Rv
    tc = np.einsum("nab,nb->na", Re, tv) + te
    return Rc, tc


def _linearize_obs(prob: RigProblem, st: RigState, delta: float):
    """Per observation, through the BA oracle on one virtual camera per
    observation (its composite pose and its rig camera's intrinsics):
    residual r (N, 2), IRLS weight w (N,), Jacobian of the composite camera
    Jc (N, 2, 6) and of the point Jp (N, 2, 3), and the validity mask."""
    Rc, tc = composite(prob, st)
    N = prob.n_obs
    r = np.zeros((N, 2))
    w = np.zeros(N)
    Jc = np.zeros((N, 2, 6))
    Jp = np.zeros((N, 2, 3))
    valid = np.zeros(N, dtype=bool)
    for c in range(prob.n_rc):
        sel = np.flatnonzero(prob.obs_rc == c)
        if sel.size == 0:
            continue
        vp = B.Problem.from_arrays(prob.intrinsics[c], np.arange(sel.size), prob.obs_pt[sel],
                                   prob.obs_uv[sel], None, sel.size, prob.n_pts)
        vs = B.State(Rc[sel], tc[sel], st.X)
        r[sel], w[sel], Jc[sel], Jp[sel] = B.linearize(vp, vs, delta)
        valid[sel] = B.residuals(vp, vs)[2]
    return r, w, Jc, Jp, valid


def _extrinsic_state(st: RigState) -> B.State:
    return B.State(st.Re, st.te, np.zeros((0, 3)))


def rig_cost(prob: RigProblem, st: RigState, delta: float, lam_e: float = 0.0,
             E0: RigState = None) -> float:
    """F = 1/2 sum_k rho(||r_k||^2) (+ 1/2 lambda_e sum_c ||T_vc,c - T_vc,c^init||^2)."""
    r, _, _, _, valid = _linearize_obs(prob, st, delta)
    s = np.sum(r * r, axis=1)
    F = 0.5 * float(np.sum(B.huber_rho(s[valid], delta)))
    if lam_e > 0:
        pri = PR.Priors(_extrinsic_state(E0), 0.0, lam_e)
        F += PR.prior_cost(_extrinsic_state(st), pri)
    return F


def rig_jacobians(prob: RigProblem, st: RigState, delta: float = 0.0):
    """(r, w, Jv, Je, Jp): per observation the Jacobians with respect to its
    frame's vehicle perturbation (J_cam Ad(E_c)), its rig camera's extrinsic
    perturbation (J_cam) and its point."""
    r, w, Jc, Jp, _ = _linearize_obs(prob, st, delta)
    Ad = adjoint(st.Re, st.te)[prob.obs_rc]
    Jv = Jc @ Ad
    return r, w, Jv, Jc, Jp


def _unknowns(prob: RigProblem):
    fv = np.flatnonzero(~prob.frame_fixed)
    fe = np.flatnonzero(~prob.rc_fixed)
    pv = -np.ones(prob.n_frames, dtype=np.int64)
    pv[fv] = np.arange(fv.size)
    pe = -np.ones(prob.n_rc, dtype=np.int64)
    pe[fe] = fv.size + np.arange(fe.size)
    return fv, fe, pv, pe


def rig_normal_equations(prob: RigProblem, st: RigState, delta: float, lam_e: float = 0.0,
                         E0: RigState = None):
    """Dense A = sum w J^T J and g = sum w J^T r over the unknowns [free
    vehicle poses (6 each), free extrinsics (6 each), points (3 each)], the
    extrinsic prior added to the extrinsic blocks."""
    fv, fe, pv, pe = _unknowns(prob)
    npose = 6 * (fv.size + fe.size)
    n = npose + 3 * prob.n_pts
    r, w, Jv, Je, Jp = rig_jacobians(prob, st, delta)
    N = prob.n_obs
    J = np.zeros((2 * N, n))
    for k in range(N):
        a = pv[prob.obs_frame[k]]
        if a >= 0:
            J[2 * k:2 * k + 2, 6 * a:6 * a + 6] = Jv[k]
        b = pe[prob.obs_rc[k]]
        if b >= 0:
            J[2 * k:2 * k + 2, 6 * b:6 * b + 6] += Je[k]
        j = prob.obs_pt[k]
        J[2 * k:2 * k + 2, npose + 3 * j:npose + 3 * j + 3] = Jp[k]
    sw = np.repeat(w, 2)
    A = J.T @ (sw[:, None] * J)
    g = J.T @ (sw * r.ravel())
    if lam_e > 0:
        pri = PR.Priors(_extrinsic_state(E0), 0.0, lam_e)
        dU, dg, _ = PR.prior_blocks(_extrinsic_state(st), pri, prob.rc_fixed)
        for c in fe:
            b = pe[c]
            A[6 * b:6 * b + 6, 6 * b:6 * b + 6] += dU[c]
            g[6 * b:6 * b + 6] += dg[c]
    return A, g


def rig_retract(prob: RigProblem, st: RigState, h: np.ndarray) -> RigState:
    """V_f <- Exp(xi_V) V_f, E_c <- Exp(xi_E) E_c (free ones), X <- X + dX."""
    fv, fe, pv, pe = _unknowns(prob)
    xv = np.zeros((prob.n_frames, 6))
    xe = np.zeros((prob.n_rc, 6))
    xv[fv] = h[:6 * fv.size].reshape(-1, 6)
    xe[fe] = h[6 * fv.size:6 * (fv.size + fe.size)].reshape(-1, 6)
    Rv, tv = B.se3_retract(st.Rv, st.tv, xv)
    Re, te = B.se3_retract(st.Re, st.te, xe)
    X = st.X + h[6 * (fv.size + fe.size):].reshape(-1, 3)
    return RigState(Rv, tv, Re, te, X)


@dataclasses.dataclass
class RigOptions:
    huber_delta: float = 0.0
    lm_iters: int = 10
    mu0: float = 1e-4
    nu0: float = 2.0
    lam_e: float = 0.0


@dataclasses.dataclass
class RigResult:
    costs: np.ndarray
    accepted: np.ndarray
    mu: np.ndarray
    gain: np.ndarray
    state: RigState


def rig_lm_solve(prob: RigProblem, st0: RigState, opts: RigOptions) -> RigResult:
    """The BA solver's Levenberg-Marquardt on the rig unknowns."""
    st = st0.copy()
    mu, nu = opts.mu0, opts.nu0
    F_of = lambda x: rig_cost(prob, x, opts.huber_delta, opts.lam_e, st0)
    F = F_of(st)
    costs, acc, mus, gains = [F], [], [], []
    lin = None
    for _ in range(opts.lm_iters):
        if lin is None:
            lin = rig_normal_equations(prob, st, opts.huber_delta, opts.lam_e, st0)
        A, g = lin
        D = np.maximum(np.diag(A), B.DIAG_MIN)
        try:
            h = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A + mu * np.diag(D), lower=True), -g)
            dL = 0.5 * float(h @ (mu * D * h - g))
            cand = rig_retract(prob, st, h)
            F_new = F_of(cand)
        except np.linalg.LinAlgError:
            dL, F_new = -np.inf, F
        gain = (F - F_new) / dL if dL > 0 else -np.inf
        mus.append(mu)
        gains.append(gain)
        accept = bool(dL > 0 and gain > 0)
        mu, nu = B.damping_update(mu, nu, gain, accept)
        if accept:
            st, F = cand, F_new
            lin = None
        acc.append(accept)
        costs.append(F)
    return RigResult(np.array(costs), np.array(acc, dtype=bool), np.array(mus),
                     np.array(gains), st)
