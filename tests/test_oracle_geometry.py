"""Pins of the oracle's geometry against library routines and closed forms.

Nothing here re-types an oracle formula: each check compares the oracle with
scipy (rotations, matrix exponential), with an exact textbook value, or with
the scene generator's own projection-matrix camera model.
"""
import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2510_15271_b300 import scenes


def _rng(seed=0):
    return np.random.Generator(np.random.PCG64(seed))


def test_so3_exp_matches_scipy_rotvec():
    w = _rng(1).normal(size=(200, 3)) * np.array([[0.1], [1.0], [3.0], [1e-6]] * 50)
    np.testing.assert_allclose(O.so3_exp(w), Rotation.from_rotvec(w).as_matrix(), atol=1e-14)


def test_so3_exp_textbook_quarter_turn():
    # a quarter turn about z maps x to y exactly
    R = O.so3_exp(np.array([[0.0, 0.0, np.pi / 2]]))[0]
    np.testing.assert_allclose(R, [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-15)


def test_so3_small_angle_branch_is_continuous():
    # either side of the Taylor switch (theta^2 = 1e-10) the maps agree
    axis = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    lo = axis * np.sqrt(1e-10) * (1 - 1e-9)
    hi = axis * np.sqrt(1e-10) * (1 + 1e-9)
    np.testing.assert_allclose(O.so3_exp(lo[None]), O.so3_exp(hi[None]), atol=1e-14)
    np.testing.assert_allclose(O.so3_left_jacobian(lo[None]), O.so3_left_jacobian(hi[None]),
                               atol=1e-14)


def test_se3_retraction_equals_matrix_exponential():
    """Exp(xi) T with xi = (v, w) is expm of the 4x4 twist [[w]x, v; 0, 0]."""
    rng = _rng(2)
    for _ in range(20):
        xi = rng.normal(size=6) * rng.choice([1e-7, 0.1, 1.0])
        R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
        t = rng.normal(size=3)
        R2, t2 = O.se3_retract(R[None], t[None], xi[None])
        tw = np.zeros((4, 4))
        tw[:3, :3] = O.hat(xi[3:])
        tw[:3, 3] = xi[:3]
        T = np.eye(4)
        T[:3, :3], T[:3, 3] = R, t
        E = scipy.linalg.expm(tw) @ T
        np.testing.assert_allclose(R2[0], E[:3, :3], atol=1e-12)
        np.testing.assert_allclose(t2[0], E[:3, 3], atol=1e-12)


def test_quaternion_conversions_match_scipy():
    rots = Rotation.random(500, random_state=3)
    q_xyzw = rots.as_quat()
    q = np.concatenate([q_xyzw[:, 3:], q_xyzw[:, :3]], axis=1)
    np.testing.assert_allclose(O.quat_to_rot(q), rots.as_matrix(), atol=1e-14)
    back = O.rot_to_quat(rots.as_matrix())
    sign = np.sign(np.sum(back * q, axis=1, keepdims=True))
    np.testing.assert_allclose(back, sign * q, atol=1e-14)
    assert (back[:, 0] >= 0).all()


def test_so3_log_matches_scipy():
    rots = Rotation.random(300, random_state=4)
    np.testing.assert_allclose(O.so3_log(rots.as_matrix()), rots.as_rotvec(), atol=1e-10)


@pytest.mark.parametrize("name,kw", [
    ("ring", dict(n_cams=12, n_pts=300)),
    ("driving", dict(n_cams=60, n_pts=4000, length_m=120.0)),
    ("city", dict(n_cams=300, n_pts=5000)),
])
def test_zero_residual_at_ground_truth_noise_free(name, kw):
    """The generator measures through P = K[R|t] in homogeneous coordinates;
    with no noise and no outliers the oracle's residuals at the true state are
    zero to rounding."""
    s = scenes.make_scene(name, seed=5, sigma=0.0, outlier_frac=0.0, **kw)
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    gt = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    r, _, valid = O.residuals(prob, gt)
    assert valid.all()
    assert np.abs(r).max() < 1e-8
    assert O.cost(prob, gt, 1.0) < 1e-15 * prob.n_obs * 1e6


def test_rmse_at_ground_truth_matches_noise_level():
    s = scenes.make_scene("ring", seed=6, sigma=0.5)
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    gt = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    # E||r||^2 = 2 sigma^2 for isotropic pixel noise
    assert abs(O.rmse(prob, gt) - 0.5 * np.sqrt(2.0)) < 0.02


def test_umeyama_recovers_similarity():
    rng = _rng(7)
    src = rng.normal(size=(50, 3))
    R = Rotation.random(random_state=8).as_matrix()
    s, t = 2.5, np.array([1.0, -2.0, 0.5])
    dst = s * src @ R.T + t
    s2, R2, t2 = O.umeyama_sim3(src, dst)
    assert abs(s2 - s) < 1e-12
    np.testing.assert_allclose(R2, R, atol=1e-12)
    np.testing.assert_allclose(t2, t, atol=1e-12)


def test_pose_errors_of_known_offsets():
    R = Rotation.random(10, random_state=9).as_matrix()
    t = _rng(10).normal(size=(10, 3))
    dR = O.so3_exp(np.tile([[0.0, 0.0, 0.01]], (10, 1)))
    # rotate each camera about its own z by 0.01 rad, keep the centre
    Ra = dR @ R
    Ca = -np.einsum("nji,nj->ni", R, t)
    ta = -np.einsum("nij,nj->ni", Ra, Ca + np.array([0.0, 0.2, 0.0]))
    rot, pos = O.pose_errors(Ra, ta, R, t)
    np.testing.assert_allclose(rot, 0.01, atol=1e-12)
    np.testing.assert_allclose(pos, 0.2, atol=1e-12)
