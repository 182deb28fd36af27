"""Pose-graph optimisation (Sec. 4.2) on the GPU against the FP64 oracle:
per-iteration cost to 1e-9 with exact solves (dense Cholesky, PCG at
1e-13), the FP32 PCG path to the final-cost gate, fixed nodes, resumed
solves, input validation, and the full-size graph (9,000 nodes) in the
launch configuration the benchmark times: one iteration against the
oracle's sparse direct solve, and the reported cost against the oracle's
cost of the returned poses."""
import numpy as np
import pytest

from oracle import pose_graph as PG
from paper_2510_15271_b300 import ba, pose_graphs

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_15271_b300 import build
    build.build()
    ba.lib()


def _oracle_graph(s):
    return PG.pose_graph_from_arrays(s.n_nodes, s.edge_ij, s.edge_qt, s.edge_w, s.fixed)


def _oracle(s, iters, solver="dense"):
    pg = _oracle_graph(s)
    R, t = PG._qt_to_rt(s.node_qt_init)
    return PG.pg_lm_solve(pg, R, t, PG.PGOptions(lm_iters=iters, solver=solver))


def _gpu(s, precision="fp64", **kw):
    o = ba.ba_options_default(precision=ba.BA_FP32 if precision == "fp32" else ba.BA_FP64)
    for k, v in kw.items():
        setattr(o, k, v)
    with ba.ba_pg_create(o) as g:
        ba.ba_pg_set_graph(g, s.node_qt_init, s.edge_ij, s.edge_qt, s.edge_w, s.fixed)
        rep = ba.ba_pg_solve(g)
        q = ba.ba_pg_get_state(g, s.n_nodes)
    return rep, q


def _small(seed=21, n_frames=40, rig=2, **kw):
    return pose_graphs.make_pose_graph(seed=seed, n_frames=n_frames, rig=rig, route="line", **kw)


def _loops(seed=22, n_frames=250, rig=3):
    """A rig graph on a small street grid, with loop closures."""
    return pose_graphs.make_pose_graph(seed=seed, n_frames=n_frames, rig=rig, extent=100.0,
                                       block=50.0, loop_gap=30)


def test_fp64_dense_matches_oracle_per_iteration():
    s = _small()
    rep, q = _gpu(s, max_lm_iters=10, solver=ba.BA_SOLVER_DENSE)
    ref = _oracle(s, 10)
    rel = np.abs(rep["costs"] - ref.costs) / ref.costs
    assert rel.max() <= COST_RTOL, (rel, rep["costs"], ref.costs)
    assert (rep["accepted"] == ref.accepted).all()
    np.testing.assert_allclose(rep["mu"], ref.mu, rtol=1e-9)
    R, t = PG._qt_to_rt(q)
    np.testing.assert_allclose(R, ref.R, atol=1e-9)
    np.testing.assert_allclose(t, ref.t, atol=1e-8)


def test_fp64_dense_with_loop_closures_matches_oracle():
    s = _loops(seed=24, n_frames=200)           # 600 nodes: 6n = 3600 <= 4096
    assert (s.edge_kind == pose_graphs.EDGE_LOOP).any()
    rep, _ = _gpu(s, max_lm_iters=8, solver=ba.BA_SOLVER_DENSE)
    ref = _oracle(s, 8)
    rel = np.abs(rep["costs"] - ref.costs) / ref.costs
    assert rel.max() <= COST_RTOL, (rel, rep["costs"], ref.costs)
    assert (rep["accepted"] == ref.accepted).all()


def test_fp64_pcg_with_loop_closures_matches_oracle():
    """Loop closures and rig edges give off-diagonal blocks far from the
    diagonal; an exact-enough PCG (auto picks the standard recurrence at this
    tolerance) reproduces the oracle's direct LM path."""
    s = _loops()
    assert (s.edge_kind == pose_graphs.EDGE_LOOP).any()
    n = 6 * s.n_nodes
    rep, _ = _gpu(s, max_lm_iters=8, solver=ba.BA_SOLVER_PCG, pcg_tol=1e-13, pcg_max_iters=4 * n)
    assert (rep["pcg_rel_residual"] <= 1e-13).all()
    ref = _oracle(s, 8)
    rel = np.abs(rep["costs"] - ref.costs) / ref.costs
    assert rel.max() <= COST_RTOL, (rel, rep["costs"], ref.costs)
    assert (rep["accepted"] == ref.accepted).all()


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_fp64_pcg_variants_at_the_production_tolerance(variant):
    """Standard and pipelined PCG at tol 1e-6 / 100 iterations (an inexact
    LM: the capped solves slow it down on a graph with loop closures) reach
    the oracle's exact-LM final cost within the 1 % gate."""
    s = _loops(seed=23)
    rep, _ = _gpu(s, max_lm_iters=12, solver=ba.BA_SOLVER_PCG, pcg_variant=variant)
    ref = _oracle(s, 12)
    assert abs(rep["costs"][-1] - ref.costs[-1]) <= 1e-2 * ref.costs[-1], (rep["costs"],
                                                                         ref.costs)
    assert np.all(np.diff(rep["costs"]) <= 0)


def test_fp32_pcg_final_cost_gate():
    """FP32 system and PCG at the production settings (tol 1e-6, 100
    iterations): the final cost within 1 % of the oracle's exact LM."""
    s = _loops(seed=24)
    rep, _ = _gpu(s, "fp32", max_lm_iters=20, solver=ba.BA_SOLVER_PCG)
    ref = _oracle(s, 20)
    assert abs(rep["costs"][-1] - ref.costs[-1]) <= 0.01 * ref.costs[-1], (rep["costs"],
                                                                          ref.costs)
    assert np.all(np.diff(rep["costs"]) <= 0)


def test_fixed_nodes_keep_their_pose_and_resume_continues():
    s = _small(seed=25, n_frames=30, rig=3)
    fixed = s.fixed.copy()
    fixed[10:13] = 1
    s.fixed = fixed
    o = ba.ba_options_default(precision=ba.BA_FP64, solver=ba.BA_SOLVER_DENSE, max_lm_iters=4)
    with ba.ba_pg_create(o) as g:
        ba.ba_pg_set_graph(g, s.node_qt_init, s.edge_ij, s.edge_qt, s.edge_w, fixed)
        a = ba.ba_pg_solve(g)
        b = ba.ba_pg_solve(g)      # continues from the first solve's state and damping
        q = ba.ba_pg_get_state(g, s.n_nodes)
    ref = _oracle(s, 8)
    got = np.concatenate([a["costs"], b["costs"][1:]])
    rel = np.abs(got - ref.costs) / ref.costs
    assert rel.max() <= COST_RTOL, (got, ref.costs)
    R0, t0 = PG._qt_to_rt(s.node_qt_init)
    R, t = PG._qt_to_rt(q)
    keep = fixed.astype(bool)
    np.testing.assert_allclose(R[keep], R0[keep], atol=1e-14)
    np.testing.assert_allclose(t[keep], t0[keep], atol=1e-14)


def test_invalid_graphs_are_refused():
    s = _small(seed=26, n_frames=10, rig=1)
    o = ba.ba_options_default()
    with ba.ba_pg_create(o) as g:
        bad = s.edge_ij.copy()
        bad[0, 1] = s.n_nodes
        with pytest.raises(ba.BAError, match="out of range"):
            ba.ba_pg_set_graph(g, s.node_qt_init, bad, s.edge_qt, s.edge_w, s.fixed)
        bad = s.edge_ij.copy()
        bad[0, 1] = bad[0, 0]
        with pytest.raises(ba.BAError, match="i == j"):
            ba.ba_pg_set_graph(g, s.node_qt_init, bad, s.edge_qt, s.edge_w, s.fixed)
        w = s.edge_w.copy()
        w[0] = -1.0
        with pytest.raises(ba.BAError, match="negative weight"):
            ba.ba_pg_set_graph(g, s.node_qt_init, s.edge_ij, s.edge_qt, w, s.fixed)
        keep = ~((s.edge_ij == 5).any(axis=1))        # node 5 left without edges
        with pytest.raises(ba.BAError, match="no edge of positive weight"):
            ba.ba_pg_set_graph(g, s.node_qt_init, s.edge_ij[keep], s.edge_qt[keep],
                               s.edge_w[keep], s.fixed)
        with pytest.raises(ba.BAError, match="no graph"):
            ba.ba_pg_solve(g)
        # an isolated node is accepted when fixed
        fx = s.fixed.copy()
        fx[5] = 1
        ba.ba_pg_set_graph(g, s.node_qt_init, s.edge_ij[keep], s.edge_qt[keep], s.edge_w[keep],
                           fx)
        rep = ba.ba_pg_solve(g)
        assert rep["costs"][-1] < rep["costs"][0]


@pytest.fixture(scope="module")
def full_graph():
    return pose_graphs.make_pose_graph()


def test_full_size_first_iteration_matches_oracle_sparse_solve(full_graph):
    """The benchmark's graph (9,000 nodes, 27,495 edges): one FP64 LM
    iteration with a PCG at 1e-12 against the oracle's sparse direct solve."""
    s = full_graph
    rep, _ = _gpu(s, max_lm_iters=1, solver=ba.BA_SOLVER_PCG, pcg_tol=1e-12,
                  pcg_max_iters=20000)
    ref = _oracle(s, 1, solver="sparse")
    assert rep["pcg_rel_residual"][0] <= 1e-12
    rel = np.abs(rep["costs"] - ref.costs) / ref.costs
    assert rel.max() <= COST_RTOL, (rel, rep["costs"], ref.costs)


def test_full_size_fp32_solve_reports_the_cost_of_its_poses(full_graph):
    """The launch configuration the benchmark times (FP32, PCG tol 1e-6 /
    100, 20 iterations): costs non-increasing, the drift removed, and the
    reported final cost equal to the oracle's FP64 cost of the returned
    poses."""
    s = full_graph
    rep, q = _gpu(s, "fp32", max_lm_iters=s.lm_iters, solver=ba.BA_SOLVER_PCG)
    assert np.all(np.diff(rep["costs"]) <= 0)
    pg = _oracle_graph(s)
    Rt, tt = PG._qt_to_rt(s.node_qt_true)
    assert rep["costs"][-1] <= 1.5 * PG.pg_cost(pg, Rt, tt)
    R, t = PG._qt_to_rt(q)
    F = PG.pg_cost(pg, R, t)
    assert abs(F - rep["costs"][-1]) <= 1e-9 * F
    r = PG.pg_residuals(pg, R, t)
    assert abs(rep["rmse_px"] - np.sqrt(np.mean(r * r))) <= 1e-9 * rep["rmse_px"]
