"""Pins of the oracle's pose priors (Sec. 4.2 Eq. seq, Sec. 4.3 Eq. abs):
Jacobians against central finite differences of the residuals, zero at the
initial trajectory, invariance of the sequential term to a rigid change of
the world frame, Schur = full normal equations with the priors, and the LM
behaviour they induce."""
import numpy as np
import pytest

import oracle as O
from oracle import priors as PR
from paper_2510_15271_b300 import scenes


def _state(seed, C=6):
    rng = np.random.default_rng(seed)
    qt = np.zeros((C, 7))
    for i in range(C):
        q = rng.normal(size=4)
        qt[i, :4] = q / np.linalg.norm(q)
        qt[i, 4:] = rng.normal(size=3) * 2.0
    return O.state_from_qt(qt, rng.normal(size=(3, 3)))


def _perturb(st, i, xi):
    R2, t2 = O.se3_retract(st.R[i:i + 1], st.t[i:i + 1], xi[None])
    out = st.copy()
    out.R[i], out.t[i] = R2[0], t2[0]
    return out


def test_jacobians_match_central_differences():
    st0 = _state(1)
    st = _state(2)  # away from the measurements: non-zero residuals
    pri = PR.Priors(st0, 1.0, 1.0)
    Ja, Ji, Jj = PR.prior_jacobians(st)
    h = 1e-6
    for i in range(st.R.shape[0]):
        for k in range(6):
            e = np.zeros(6)
            e[k] = h
            ap, cp = PR.prior_residuals(_perturb(st, i, e), pri)
            am, cm = PR.prior_residuals(_perturb(st, i, -e), pri)
            da, dc = (ap - am) / (2 * h), (cp - cm) / (2 * h)
            np.testing.assert_allclose(da[i], Ja[i, :, k], rtol=1e-6, atol=1e-8)
            if i < st.R.shape[0] - 1:   # residual of pair (i, i + 1)
                np.testing.assert_allclose(dc[i], Ji[i, :, k], rtol=1e-6, atol=1e-8)
            if i > 0:                   # residual of pair (i - 1, i)
                np.testing.assert_allclose(dc[i - 1], Jj[i - 1, :, k], rtol=1e-6, atol=1e-8)
            # no other residual moves
            others = np.ones(st.R.shape[0] - 1, bool)
            others[max(i - 1, 0):i + 1] = False
            assert np.abs(dc[others]).max(initial=0.0) < 1e-8


def test_zero_at_the_initial_trajectory():
    st0 = _state(3)
    pri = PR.Priors(st0, 5.0, 7.0)
    ra, rc = PR.prior_residuals(st0, pri)
    assert np.abs(ra).max() == 0.0 and np.abs(rc).max() < 1e-15
    assert PR.prior_cost(st0, pri) < 1e-28
    dU, dg, _ = PR.prior_blocks(st0, pri, np.zeros(6, bool))
    assert np.abs(dg).max() < 1e-13


def test_sequential_term_ignores_a_rigid_change_of_world_frame():
    st0 = _state(4)
    pri = PR.Priors(st0, 1.0, 0.0)
    G = O.so3_exp(np.array([[0.3, -0.2, 0.5]]))[0]
    tg = np.array([1.0, -2.0, 0.5])
    # world points X' = G X + tg: world->camera poses become R G^T, t - R G^T tg
    moved = O.State(st0.R @ G.T, st0.t - np.einsum("nij,j->ni", st0.R @ G.T, tg), st0.X)
    _, rc = PR.prior_residuals(moved, pri)
    assert np.abs(rc).max() < 1e-12
    ra, _ = PR.prior_residuals(moved, PR.Priors(st0, 0.0, 1.0))
    assert np.abs(ra).max() > 0.1   # the absolute term is meant to anchor the world frame


def test_schur_step_equals_full_normal_equations_with_priors():
    s = scenes.make_scene("ring", seed=9, n_cams=6, n_pts=60)
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    st0 = O.state_from_qt(s.cam_qt_gt, s.pts_gt)   # measurements from the truth
    st = O.state_from_qt(s.cam_qt, s.pts)          # solve from the perturbed start
    pri = PR.Priors(st0, 3e3, 50.0)
    steps = {}
    for solver in ("dense", "full"):
        opts = O.LMOptions(solver=solver)
        lin = O.ba_oracle._linearization(prob, st, opts, pri)
        dc, dp, D, g, h, _ = O.solve_step(prob, lin, 1e-3, opts)
        steps[solver] = (dc, dp)
    np.testing.assert_allclose(steps["dense"][0], steps["full"][0], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(steps["dense"][1], steps["full"][1], rtol=1e-9, atol=1e-12)


def test_lm_with_priors_descends_and_strong_priors_hold_the_trajectory():
    s = scenes.make_scene("ring", seed=10, n_cams=10, n_pts=400)
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    st = O.state_from_qt(s.cam_qt, s.pts)
    drift = []
    for lam in (0.0, 1e2, 1e6):
        r = O.lm_solve(prob, st, O.LMOptions(solver="dense", lm_iters=8, prior_seq=lam,
                                             prior_abs=lam))
        acc = np.flatnonzero(r.accepted)
        assert np.all(np.diff(r.costs) <= 1e-12 * r.costs[0])   # monotone
        assert acc.size > 0
        drift.append(np.linalg.norm(r.state.t - st.t))
    assert drift[2] < drift[1] < drift[0]
