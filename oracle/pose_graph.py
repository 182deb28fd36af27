"""FP64 CPU oracle of pose-graph optimisation.

TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import, call or execute this module.  It
shares no code with the CUDA path and imports nothing from it.

What it computes (cuSfM, Sec. 4.2 "Pose Graph Optimization"):
  * nodes are camera poses; edges are relative-pose constraints of three
    kinds that share one form: sequential constraints between frames of the
    initial trajectory (Eq. seq), loop-closure constraints from the stereo
    relative-pose module, and extrinsic constraints between cameras of one
    vehicle rig (Eq. extrinsic).  Each edge (i, j) carries a measured pose
    M of frame i in frame j and a weight;
  * the objective min sum_e e_e^T Omega_e e_e over the node poses.

Readings where the paper is silent (listed with reasons in the design notes):
  * the error of edge (i, j) is the 12-vector of entries of the top 3 x 4
    blocks of T_cw,j T_wc,i - M (the pose of frame i in frame j, the same
    product order as the sequential pose prior, so the error does not
    depend on the choice of world frame), row-major;
  * Omega_e = w_e I_12 with a scalar weight w_e >= 0 per edge, and
    F = 1/2 sum_e w_e ||r_e||^2 (the halved convention of the BA cost);
  * node poses follow the BA convention (world -> camera, x_c = R X + t)
    and the same left perturbation T_cw <- Exp(xi) T_cw, xi = (v, omega);
    with X_k the 4 x 4 twist of e_k and Q = T_cw,j T_wc,i,
        d r / d xi_i = -(Q X_k),    d r / d xi_j = +(X_k Q);
  * the solver is the BA solver's Levenberg-Marquardt (Madsen, Nielsen &
    Tingleff 2004; Marquardt scaling D = diag(A) clamped to >= 1e-12,
    mu_0 = 1e-4, nu_0 = 2, accept iff dL > 0 and gain > 0) on the normal
    equations over the free nodes; fixed nodes keep their pose (the gauge of
    an otherwise free graph is fixed by fixing a node).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .ba_oracle import (DIAG_MIN, damping_update, hat, quat_to_rot, rot_to_quat,
                        se3_retract)

__all__ = ["PoseGraph", "PGOptions", "PGResult", "pose_graph_from_arrays", "relative_poses",
           "pg_residuals", "pg_cost", "pg_jacobians", "pg_normal_equations", "pg_lm_solve"]


@dataclasses.dataclass
class PoseGraph:
    """Edges (i, j) with the measured pose of frame i in frame j (top 3 x 4
    block) and a weight; a fixed mask over the nodes."""
    n_nodes: int
    edge_i: np.ndarray   # (E,) int
    edge_j: np.ndarray   # (E,) int
    meas: np.ndarray     # (E, 3, 4)
    weight: np.ndarray   # (E,)
    fixed: np.ndarray    # (n,) bool

    @property
    def n_edges(self) -> int:
        return int(self.edge_i.shape[0])


def _qt_to_rt(qt):
    qt = np.asarray(qt, dtype=np.float64).reshape(-1, 7)
    return quat_to_rot(qt[:, :4]), qt[:, 4:].copy()


def pose_graph_from_arrays(n_nodes, edge_ij, edge_qt, edge_w, fixed=None) -> PoseGraph:
    """A PoseGraph from the arrays of the C interface: edge_ij (E, 2),
    edge_qt (E, 7) = (qw, qx, qy, qz, tx, ty, tz) of the measured pose of
    frame i in frame j, edge_w (E,)."""
    ij = np.asarray(edge_ij, dtype=np.int64).reshape(-1, 2)
    Rm, tm = _qt_to_rt(edge_qt)
    meas = np.concatenate([Rm, tm[:, :, None]], axis=2)
    fx = np.zeros(n_nodes, dtype=bool) if fixed is None else np.asarray(fixed, dtype=bool)
    return PoseGraph(int(n_nodes), ij[:, 0].copy(), ij[:, 1].copy(), meas,
                     np.asarray(edge_w, dtype=np.float64).reshape(-1).copy(), fx.copy())


def relative_poses(R, t, i, j) -> np.ndarray:
    """Top 3 x 4 blocks of T_cw,j T_wc,i = [R_j R_i^T | t_j - R_j R_i^T t_i]
    for the index arrays i, j (the pose of frame i in frame j)."""
    rot = R[j] @ np.transpose(R[i], (0, 2, 1))
    tr = t[j] - np.einsum("nab,nb->na", rot, t[i])
    return np.concatenate([rot, tr[:, :, None]], axis=2)


def pg_residuals(pg: PoseGraph, R, t) -> np.ndarray:
    """(E, 12): entries of T_cw,j T_wc,i - M, row-major over the top 3 x 4."""
    if pg.n_edges == 0:
        return np.zeros((0, 12))
    return (relative_poses(R, t, pg.edge_i, pg.edge_j) - pg.meas).reshape(-1, 12)


def pg_cost(pg: PoseGraph, R, t) -> float:
    """F = 1/2 sum_e w_e ||r_e||^2."""
    r = pg_residuals(pg, R, t)
    return 0.5 * float(np.sum(pg.weight * np.sum(r * r, axis=1)))


def _twist(k: int) -> np.ndarray:
    """The 4 x 4 twist matrix of the unit vector e_k of xi = (v, omega)."""
    X = np.zeros((4, 4))
    if k < 3:
        X[k, 3] = 1.0
    else:
        X[:3, :3] = hat(np.eye(3)[k - 3])
    return X


def pg_jacobians(pg: PoseGraph, R, t):
    """(Ji, Jj), each (E, 12, 6): derivatives of the edge residuals with
    respect to xi of node i and of node j at xi = 0."""
    E = pg.n_edges
    Q = np.zeros((E, 4, 4))
    Q[:, :3, :] = relative_poses(R, t, pg.edge_i, pg.edge_j) if E else 0.0
    Q[:, 3, 3] = 1.0
    Ji = np.zeros((E, 12, 6))
    Jj = np.zeros((E, 12, 6))
    for k in range(6):
        X = _twist(k)
        Ji[:, :, k] = -(Q @ X)[:, :3, :].reshape(E, 12)
        Jj[:, :, k] = (X @ Q)[:, :3, :].reshape(E, 12)
    return Ji, Jj


def pg_normal_equations(pg: PoseGraph, R, t):
    """A = sum_e w_e J_e^T J_e and g = sum_e w_e J_e^T r_e over the free
    nodes (6 unknowns each, in node order), A as a scipy CSR matrix.
    Returns (A, g, free node indices)."""
    free = np.flatnonzero(~pg.fixed)
    pos = -np.ones(pg.n_nodes, dtype=np.int64)
    pos[free] = np.arange(free.size)
    r = pg_residuals(pg, R, t)
    Ji, Jj = pg_jacobians(pg, R, t)
    n = 6 * free.size
    g = np.zeros(n)
    rows, cols, vals = [], [], []
    w = pg.weight
    sides = ((pg.edge_i, Ji), (pg.edge_j, Jj))
    for na, Ja in sides:
        pa = pos[na]
        ga = np.einsum("e,eka,ek->ea", w, Ja, r)
        for e in np.flatnonzero(pa >= 0):
            g[6 * pa[e]:6 * pa[e] + 6] += ga[e]
        for nb, Jb in sides:
            pb = pos[nb]
            blk = np.einsum("e,eka,ekb->eab", w, Ja, Jb)
            ok = (pa >= 0) & (pb >= 0)
            for e in np.flatnonzero(ok):
                rr, cc = np.meshgrid(6 * pa[e] + np.arange(6), 6 * pb[e] + np.arange(6),
                                     indexing="ij")
                rows.append(rr.ravel())
                cols.append(cc.ravel())
                vals.append(blk[e].ravel())
    if rows:
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n)).tocsr()    # duplicate entries are summed
    else:
        A = sp.csr_matrix((n, n))
    return A, g, free


@dataclasses.dataclass
class PGOptions:
    lm_iters: int = 10
    solver: str = "dense"     # "dense" (Cholesky) or "sparse" (sparse LU, large graphs)
    mu0: float = 1e-4
    nu0: float = 2.0


@dataclasses.dataclass
class PGResult:
    costs: np.ndarray       # F before the first and after every iteration
    accepted: np.ndarray    # (iters,) bool
    mu: np.ndarray          # (iters,) damping of each iteration's solve
    gain: np.ndarray        # (iters,) gain ratio (-inf where dL <= 0)
    R: np.ndarray
    t: np.ndarray


def _solve(M, b, solver):
    if solver == "dense":
        Md = M.toarray()
        try:
            return scipy.linalg.cho_solve(scipy.linalg.cho_factor(Md, lower=True), b)
        except np.linalg.LinAlgError:
            return None
    if solver == "sparse":
        x = spla.spsolve(M.tocsc(), b)
        return x if np.all(np.isfinite(x)) else None
    raise ValueError(solver)


def pg_lm_solve(pg: PoseGraph, R0, t0, opts: PGOptions) -> PGResult:
    """Levenberg-Marquardt on F for a fixed number of iterations (one linear
    solve and one trial step each, as in the BA solver)."""
    R, t = np.array(R0, dtype=np.float64), np.array(t0, dtype=np.float64)
    mu, nu = opts.mu0, opts.nu0
    F = pg_cost(pg, R, t)
    costs, acc, mus, gains = [F], [], [], []
    lin = None
    for _ in range(opts.lm_iters):
        if lin is None:
            lin = pg_normal_equations(pg, R, t)
        A, g, free = lin
        D = np.maximum(A.diagonal(), DIAG_MIN)
        h = _solve(A + mu * sp.diags(D), -g, opts.solver) if free.size else np.zeros(0)
        if h is None:
            dL, F_new = -np.inf, F
        else:
            dL = 0.5 * float(h @ (mu * D * h - g))
            xi = np.zeros((pg.n_nodes, 6))
            xi[free] = h.reshape(-1, 6)
            R2, t2 = se3_retract(R, t, xi)
            F_new = pg_cost(pg, R2, t2)
        gain = (F - F_new) / dL if dL > 0 else -np.inf
        mus.append(mu)
        gains.append(gain)
        accept = bool(dL > 0 and gain > 0)
        mu, nu = damping_update(mu, nu, gain, accept)
        if accept:
            R, t, F = R2, t2, F_new
            lin = None
        acc.append(accept)
        costs.append(F)
    return PGResult(np.array(costs), np.array(acc, dtype=bool), np.array(mus), np.array(gains),
                    R, t)


def node_qt(R, t) -> np.ndarray:
    """(n, 7) = (qw, qx, qy, qz, tx, ty, tz) of world -> camera poses."""
    return np.concatenate([rot_to_quat(R), t], axis=1)
