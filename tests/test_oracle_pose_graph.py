"""Pins of the pose-graph oracle (Sec. 4.2, pose graph optimisation):
Jacobians and the gradient against central differences, the Gauss-Newton
matrix against the finite-difference Hessian at a zero-residual point, zero
cost at consistent measurements, invariance of a whole LM run to a rigid
change of the world frame (which holds for the left perturbation), a tree
graph solved exactly by composing its measurements, dense = sparse solves,
and agreement with the sequential pose prior of the BA objective."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from oracle import pose_graph as PG
from oracle import priors as PR
from paper_2510_15271_b300 import pose_graphs as G


def _random_poses(rng, n):
    R = Rotation.from_rotvec(rng.normal(0, 1.0, (n, 3))).as_matrix()
    t = rng.normal(0, 3.0, (n, 3))
    return R, t


def _T(R, t):
    T = np.zeros(R.shape[:-2] + (4, 4))
    T[..., :3, :3] = R
    T[..., :3, 3] = t
    T[..., 3, 3] = 1.0
    return T


def _graph(rng, n, edges, noise=0.0, R=None, t=None):
    """Edges measured from poses (R, t) as 4 x 4 products T_j inv(T_i),
    optionally perturbed."""
    if R is None:
        R, t = _random_poses(rng, n)
    ei = np.array([e[0] for e in edges])
    ej = np.array([e[1] for e in edges])
    T = _T(R, t)
    M = T[ej] @ np.linalg.inv(T[ei])
    if noise > 0:
        dR = Rotation.from_rotvec(rng.normal(0, noise, (len(edges), 3))).as_matrix()
        M[:, :3, :3] = dR @ M[:, :3, :3]
        M[:, :3, 3] += rng.normal(0, noise, (len(edges), 3))
    w = rng.uniform(0.5, 2.0, len(edges))
    fixed = np.zeros(n, bool)
    fixed[0] = True
    pg = PG.PoseGraph(n, ei, ej, M[:, :3, :], w, fixed)
    return pg, R, t


def _retract_node(R, t, i, xi):
    R2, t2 = O.se3_retract(R[i:i + 1], t[i:i + 1], xi[None])
    Ro, to = R.copy(), t.copy()
    Ro[i], to[i] = R2[0], t2[0]
    return Ro, to


EDGES = [(0, 1), (1, 2), (2, 3), (3, 4), (0, 2), (4, 1), (3, 0), (2, 4), (2, 4)]


def test_jacobians_match_central_differences():
    rng = np.random.default_rng(1)
    pg, _, _ = _graph(rng, 5, EDGES, noise=0.3)
    R, t = _random_poses(rng, 5)                 # away from the measurements
    Ji, Jj = PG.pg_jacobians(pg, R, t)
    h = 1e-6
    for node in range(5):
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            rp = PG.pg_residuals(pg, *_retract_node(R, t, node, e))
            rm = PG.pg_residuals(pg, *_retract_node(R, t, node, -e))
            d = (rp - rm) / (2 * h)
            for q in range(pg.n_edges):
                want = np.zeros(12)
                if pg.edge_i[q] == node:
                    want = want + Ji[q, :, k]
                if pg.edge_j[q] == node:
                    want = want + Jj[q, :, k]
                np.testing.assert_allclose(d[q], want, rtol=1e-6, atol=1e-7)


def test_gradient_matches_central_differences_of_the_cost():
    rng = np.random.default_rng(2)
    pg, _, _ = _graph(rng, 5, EDGES, noise=0.3)
    R, t = _random_poses(rng, 5)
    A, g, free = PG.pg_normal_equations(pg, R, t)
    h = 1e-6
    for a, node in enumerate(free):
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            Fp = PG.pg_cost(pg, *_retract_node(R, t, node, e))
            Fm = PG.pg_cost(pg, *_retract_node(R, t, node, -e))
            assert abs((Fp - Fm) / (2 * h) - g[6 * a + k]) <= 1e-6 * max(1.0, abs(g[6 * a + k]))


def test_gauss_newton_matrix_is_the_hessian_at_zero_residual():
    """With consistent measurements the residual vanishes at the true poses,
    where the Hessian of F is exactly J^T W J."""
    rng = np.random.default_rng(3)
    pg, R, t = _graph(rng, 4, [(0, 1), (1, 2), (2, 3), (3, 1), (0, 3)])
    A, g, free = PG.pg_normal_equations(pg, R, t)
    assert np.abs(g).max() < 1e-12
    h = 1e-4
    n = 6 * free.size
    H = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            def F(sa, sb):
                Rx, tx = R, t
                ea = np.zeros(6)
                ea[a % 6] = sa
                Rx, tx = _retract_node(Rx, tx, free[a // 6], ea)
                eb = np.zeros(6)
                eb[b % 6] = sb
                Rx, tx = _retract_node(Rx, tx, free[b // 6], eb)
                return PG.pg_cost(pg, Rx, tx)
            H[a, b] = (F(h, h) - F(h, -h) - F(-h, h) + F(-h, -h)) / (4 * h * h)
    Hs = 0.5 * (H + H.T)      # the retraction of one node twice is not symmetric in order
    np.testing.assert_allclose(A.toarray(), Hs, rtol=1e-5, atol=1e-5 * np.abs(Hs).max())


def test_zero_cost_at_consistent_measurements():
    rng = np.random.default_rng(4)
    pg, R, t = _graph(rng, 6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (1, 4)])
    assert PG.pg_cost(pg, R, t) < 1e-26
    assert PG.pg_cost(pg, *_random_poses(rng, 6)) > 1.0


def test_lm_run_is_invariant_to_a_rigid_world_change():
    """T_cw -> T_cw G for every node leaves every relative pose unchanged and,
    under the left perturbation, every LM step: the costs of the two runs
    agree iteration by iteration."""
    rng = np.random.default_rng(5)
    pg, _, _ = _graph(rng, 6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 0), (1, 4)],
                      noise=0.05)
    R, t = _random_poses(rng, 6)
    Gm = _T(Rotation.from_rotvec(rng.normal(0, 1, 3)).as_matrix(), rng.normal(0, 5, 3))
    T2 = _T(R, t) @ Gm
    R2, t2 = T2[:, :3, :3], T2[:, :3, 3]
    assert abs(PG.pg_cost(pg, R, t) - PG.pg_cost(pg, R2, t2)) <= 1e-11 * PG.pg_cost(pg, R, t)
    opts = PG.PGOptions(lm_iters=8)
    a = PG.pg_lm_solve(pg, R, t, opts)
    b = PG.pg_lm_solve(pg, R2, t2, opts)
    np.testing.assert_allclose(a.costs, b.costs, rtol=1e-9)
    assert (a.accepted == b.accepted).all()


def test_tree_graph_is_solved_by_composing_its_measurements():
    """A spanning tree with node 0 fixed has a zero-cost solution whatever
    the measurements: T_cw,j = M_ij T_cw,i along the tree's edges."""
    rng = np.random.default_rng(6)
    parent = [None, 0, 1, 1, 3, 0, 5]
    edges = []
    for j, p in enumerate(parent):
        if p is not None:
            edges.append((p, j) if j % 2 else (j, p))   # both edge orientations
    pg, Rtrue, ttrue = _graph(rng, len(parent), edges, noise=0.2)
    # composition from node 0 (fixed at its true pose)
    T = [None] * len(parent)
    T[0] = _T(Rtrue[0], ttrue[0])
    Mh = _T(pg.meas[:, :, :3], pg.meas[:, :, 3])
    for _ in range(len(parent)):
        for q in range(pg.n_edges):
            i, j = pg.edge_i[q], pg.edge_j[q]
            if T[i] is not None and T[j] is None:
                T[j] = Mh[q] @ T[i]                      # M = T_j inv(T_i)
            elif T[j] is not None and T[i] is None:
                T[i] = np.linalg.inv(Mh[q]) @ T[j]
    T = np.array(T)
    R0, t0 = Rtrue.copy(), ttrue.copy()
    R0[1:], t0[1:] = _random_poses(rng, len(parent) - 1)
    R0[1:] = (Rotation.from_rotvec(rng.normal(0, 0.05, (len(parent) - 1, 3))).as_matrix()
              @ T[1:, :3, :3])
    t0[1:] = T[1:, :3, 3] + rng.normal(0, 0.1, (len(parent) - 1, 3))
    res = PG.pg_lm_solve(pg, R0, t0, PG.PGOptions(lm_iters=40))
    assert res.costs[-1] < 1e-18
    np.testing.assert_allclose(res.R, T[:, :3, :3], atol=1e-9)
    np.testing.assert_allclose(res.t, T[:, :3, 3], atol=1e-9)
    assert np.array_equal(res.R[0], Rtrue[0]) and np.array_equal(res.t[0], ttrue[0])


def test_dense_and_sparse_solves_agree_and_cost_is_monotone():
    s = G.make_pose_graph(seed=11, n_frames=40, rig=2, route="line")
    pg = PG.pose_graph_from_arrays(s.n_nodes, s.edge_ij, s.edge_qt, s.edge_w, s.fixed)
    R, t = PG._qt_to_rt(s.node_qt_init)
    a = PG.pg_lm_solve(pg, R, t, PG.PGOptions(lm_iters=8, solver="dense"))
    b = PG.pg_lm_solve(pg, R, t, PG.PGOptions(lm_iters=8, solver="sparse"))
    np.testing.assert_allclose(a.costs, b.costs, rtol=1e-10)
    assert np.all(np.diff(a.costs) <= 0)
    # the drift is removed: at most the cost of the true poses (a feasible point)
    Rt, tt = PG._qt_to_rt(s.node_qt_true)
    assert a.costs[-1] <= PG.pg_cost(pg, Rt, tt)
    fixed = s.fixed.astype(bool)
    np.testing.assert_array_equal(a.R[fixed], R[fixed])
    np.testing.assert_array_equal(a.t[fixed], t[fixed])


def test_sequential_prior_is_a_pose_graph_of_adjacent_frames():
    """The sequential pose prior (lambda_c, measured on the initial state) is
    the pose graph of edges (i, i + 1) with weight lambda_c: the same cost,
    the same diagonal blocks and the same coupling blocks."""
    rng = np.random.default_rng(8)
    C = 6
    R0, t0 = _random_poses(rng, C)
    st0 = O.State(R0, t0, np.zeros((0, 3)))
    R, t = _random_poses(rng, C)
    st = O.State(R, t, np.zeros((0, 3)))
    lam = 3.5
    pri = PR.Priors(st0, lam, 0.0)
    ei = np.arange(C - 1)
    pg = PG.PoseGraph(C, ei, ei + 1, PG.relative_poses(R0, t0, ei, ei + 1),
                      np.full(C - 1, lam), np.zeros(C, bool))
    assert abs(PR.prior_cost(st, pri) - PG.pg_cost(pg, R, t)) <= 1e-12 * PG.pg_cost(pg, R, t)
    dU, dg, cpl = PR.prior_blocks(st, pri, np.zeros(C, bool))
    A, g, _ = PG.pg_normal_equations(pg, R, t)
    A = A.toarray()
    for i in range(C):
        np.testing.assert_allclose(A[6 * i:6 * i + 6, 6 * i:6 * i + 6], dU[i], rtol=1e-12,
                                   atol=1e-12)
        np.testing.assert_allclose(g[6 * i:6 * i + 6], dg[i], rtol=1e-12, atol=1e-12)
    for i in range(C - 1):
        np.testing.assert_allclose(A[6 * i:6 * i + 6, 6 * i + 6:6 * i + 12], cpl[i], rtol=1e-12,
                                   atol=1e-12)


def test_generator_graph_has_the_three_edge_kinds():
    s = G.make_pose_graph(seed=7, n_frames=400, rig=3, loop_gap=30, extent=200.0, block=50.0)
    assert s.n_nodes == 1200
    kinds = np.bincount(s.edge_kind, minlength=3)
    assert kinds[G.EDGE_SEQ] == 3 * (399 + 398) and kinds[G.EDGE_RIG] == 3 * 400
    assert kinds[G.EDGE_LOOP] > 0
    assert (s.edge_ij[:, 0] != s.edge_ij[:, 1]).all()
    np.testing.assert_allclose(np.linalg.norm(s.edge_qt[:, :4], axis=1), 1.0, atol=1e-12)
