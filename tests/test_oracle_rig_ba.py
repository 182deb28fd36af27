"""Pins of the rig BA oracle (Sec. 4.4, extrinsic refinement): Jacobians of
the residuals with respect to the vehicle poses, the extrinsics and the points
against central differences through the retraction; the gradient against
differences of the cost; the reduction to plain BA for a one-camera rig with
the identity extrinsic; invariance of the cost to moving a rigid transform
between the vehicle poses and the extrinsics (which pins the composition
order); invariance of the cost to a rigid change of the world frame;
convergence below the cost of the true state; the extrinsic prior."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from oracle import rig_ba as RB
from paper_2510_15271_b300 import rig_scenes as RS


def _problem(s):
    return RB.RigProblem(s.intrinsics, s.obs_frame, s.obs_rc, s.obs_pt, s.obs_uv,
                         s.frame_fixed.astype(bool), s.rc_fixed.astype(bool), s.n_frames,
                         s.n_rc, s.n_pts)


def _start(s):
    return RB.RigState(s.Rv, s.tv, s.Re, s.te, s.X)


@pytest.fixture(scope="module")
def small():
    return RS.make_rig_scene(seed=3, n_frames=5, rig=3, n_pts=60)


def _move(st, which, i, xi):
    out = st.copy()
    if which == "v":
        R2, t2 = O.se3_retract(st.Rv[i:i + 1], st.tv[i:i + 1], xi[None])
        out.Rv[i], out.tv[i] = R2[0], t2[0]
    elif which == "e":
        R2, t2 = O.se3_retract(st.Re[i:i + 1], st.te[i:i + 1], xi[None])
        out.Re[i], out.te[i] = R2[0], t2[0]
    else:
        out.X[i] = st.X[i] + xi
    return out


def test_jacobians_match_central_differences(small):
    prob, st = _problem(small), _start(small)
    r0, w, Jv, Je, Jp = RB.rig_jacobians(prob, st)
    h = 1e-6
    res = lambda x: RB._linearize_obs(prob, x, 0.0)[0]
    for which, n, dim, J, idx in (("v", prob.n_frames, 6, Jv, prob.obs_frame),
                                  ("e", prob.n_rc, 6, Je, prob.obs_rc),
                                  ("x", 4, 3, Jp, prob.obs_pt)):
        for i in range(n):
            for k in range(dim):
                e = np.zeros(dim)
                e[k] = h
                d = (res(_move(st, which, i, e)) - res(_move(st, which, i, -e))) / (2 * h)
                mine = idx == i
                np.testing.assert_allclose(d[mine], J[mine][:, :, k], rtol=1e-5, atol=1e-5)
                assert np.abs(d[~mine]).max(initial=0.0) < 1e-7


def test_gradient_matches_differences_of_the_cost(small):
    prob, st = _problem(small), _start(small)
    A, g = RB.rig_normal_equations(prob, st, 0.0)
    fv, fe, pv, pe = RB._unknowns(prob)
    h = 1e-6
    F = lambda x: RB.rig_cost(prob, x, 0.0)
    for which, free, pos in (("v", fv, pv), ("e", fe, pe)):
        for i in free:
            for k in range(6):
                e = np.zeros(6)
                e[k] = h
                num = (F(_move(st, which, i, e)) - F(_move(st, which, i, -e))) / (2 * h)
                ana = g[6 * pos[i] + k]
                assert abs(num - ana) <= 1e-5 * max(1.0, abs(ana)), (which, i, k, num, ana)


def test_one_camera_rig_with_identity_extrinsic_is_plain_ba():
    s = RS.make_rig_scene(seed=4, n_frames=6, rig=1, n_pts=80)
    prob = _problem(s)
    prob.rc_fixed = np.ones(1, dtype=bool)
    # the vehicle frame re-expressed as the camera frame: V' = E V, E' = I
    st = _start(s)
    st.Rv = s.Re[0] @ s.Rv
    st.tv = np.einsum("ab,fb->fa", s.Re[0], s.tv) + s.te[0]
    st.Re = np.eye(3)[None].copy()
    st.te = np.zeros((1, 3))
    # the same observations as a BA problem over the frames' poses
    bp = O.Problem.from_arrays(s.intrinsics[0], s.obs_frame, s.obs_pt, s.obs_uv, s.frame_fixed,
                               s.n_frames, s.n_pts)
    bs = O.State(st.Rv.copy(), st.tv.copy(), st.X.copy())
    rig = RB.rig_lm_solve(prob, st, RB.RigOptions(lm_iters=6))
    ba = O.lm_solve(bp, bs, O.LMOptions(lm_iters=6, solver="full"))
    np.testing.assert_allclose(rig.costs, ba.costs, rtol=1e-10)
    assert (rig.accepted == ba.accepted).all()


def test_cost_is_unchanged_by_a_transform_moved_between_vehicle_and_extrinsics(small):
    """E_c -> E_c H^-1 and V_f -> H V_f for every camera and frame leave every
    composite camera E_c V_f unchanged."""
    prob, st = _problem(small), _start(small)
    rng = np.random.default_rng(5)
    Hr = Rotation.from_rotvec(rng.normal(0, 0.5, 3)).as_matrix()
    Ht = rng.normal(0, 2.0, 3)
    moved = st.copy()
    moved.Rv = Hr @ st.Rv
    moved.tv = np.einsum("ab,fb->fa", Hr, st.tv) + Ht
    Hinv_r = Hr.T
    moved.Re = st.Re @ Hinv_r
    moved.te = st.te - np.einsum("cab,b->ca", moved.Re, Ht)
    F0, F1 = RB.rig_cost(prob, st, 0.0), RB.rig_cost(prob, moved, 0.0)
    assert abs(F0 - F1) <= 1e-10 * F0
    # and the other order of composition would not be invariant
    wrong = st.copy()
    wrong.Re = Hr @ st.Re
    assert abs(RB.rig_cost(prob, wrong, 0.0) - F0) > 1e-3 * F0


def test_cost_is_invariant_to_a_rigid_change_of_the_world_frame(small):
    """X' = G X with T_vw' = T_vw G^-1 leaves every camera-frame point, and so
    the cost, unchanged.  (A whole LM run is not invariant: the points'
    Marquardt scaling diag(V_j) changes when the world frame rotates.)"""
    prob, st = _problem(small), _start(small)
    rng = np.random.default_rng(6)
    Gr = Rotation.from_rotvec(rng.normal(0, 1.0, 3)).as_matrix()
    Gt = rng.normal(0, 5.0, 3)
    moved = st.copy()
    moved.X = st.X @ Gr.T + Gt
    moved.Rv = st.Rv @ Gr.T
    moved.tv = st.tv - np.einsum("fab,b->fa", moved.Rv, Gt)
    F0 = RB.rig_cost(prob, st, 0.0)
    assert abs(RB.rig_cost(prob, moved, 0.0) - F0) <= 1e-10 * F0


def test_converges_below_the_cost_of_the_true_state():
    s = RS.make_rig_scene(seed=7)
    prob = _problem(s)
    res = RB.rig_lm_solve(prob, _start(s), RB.RigOptions(lm_iters=10))
    gt = RB.RigState(s.Rv_gt, s.tv_gt, s.Re_gt, s.te_gt, s.X_gt)
    assert res.costs[-1] <= RB.rig_cost(prob, gt, 0.0)
    assert np.all(np.diff(res.costs) <= 0)
    # fixed frame 0 kept
    np.testing.assert_array_equal(res.state.Rv[0], s.Rv[0])


def test_extrinsic_prior_is_zero_at_the_start_and_holds_the_extrinsics(small):
    prob, st = _problem(small), _start(small)
    assert RB.rig_cost(prob, st, 0.0, 1e6, st) == pytest.approx(RB.rig_cost(prob, st, 0.0),
                                                                 rel=1e-14)
    free = RB.rig_lm_solve(prob, st, RB.RigOptions(lm_iters=8))
    held = RB.rig_lm_solve(prob, st, RB.RigOptions(lm_iters=8, lam_e=1e9))
    d_free = np.abs(free.state.te - st.te).max() + np.abs(free.state.Re - st.Re).max()
    d_held = np.abs(held.state.te - st.te).max() + np.abs(held.state.Re - st.Re).max()
    assert d_held < 1e-2 * d_free


def test_generator_scene_is_consistent():
    """The seeded rig scene: indices in range, every point seen at least
    twice, the composite true cameras see their observations in front, and
    the noise-free reprojection of the true state is at the noise level."""
    s = RS.make_rig_scene(seed=2, n_frames=10, rig=3, n_pts=200)
    assert s.obs_frame.max() < s.n_frames and s.obs_rc.max() < s.n_rc and s.obs_pt.max() < s.n_pts
    assert np.bincount(s.obs_pt, minlength=s.n_pts).min() >= 2
    prob = _problem(s)
    gt = RB.RigState(s.Rv_gt, s.tv_gt, s.Re_gt, s.te_gt, s.X_gt)
    r, _, _, _, valid = RB._linearize_obs(prob, gt, 0.0)
    assert valid.all()
    rms = np.sqrt(np.mean(np.sum(r * r, axis=1)))
    assert 0.3 < rms < 1.0          # 0.5 px per axis of noise
    again = RS.make_rig_scene(seed=2, n_frames=10, rig=3, n_pts=200)
    np.testing.assert_array_equal(again.obs_uv, s.obs_uv)
