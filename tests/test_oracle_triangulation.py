"""Pins of the oracle's reprojection errors, outlier classification and DLT
triangulation (Sec. 4.3, Eq. dlt) against closed forms and noise-free
geometry."""
import numpy as np
import pytest

import oracle as O
from oracle import triangulation as T
from paper_2510_15271_b300 import scenes


def _prob(s, uv=None):
    return O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt,
                                 s.obs_uv if uv is None else uv, s.cam_fixed, s.n_cams, s.n_pts)


def _one_camera_problem(uv, pt_index=None, n_pts=1):
    K = (500.0, 400.0, 320.0, 240.0)
    n = len(uv)
    return O.Problem.from_arrays(K, np.zeros(n, np.int64),
                                 np.zeros(n, np.int64) if pt_index is None else pt_index,
                                 np.asarray(uv, float), None, 1, n_pts)


def test_reprojection_error_closed_form():
    # identity pose; X = (1, 2, 10) projects to (500*0.1 + 320, 400*0.2 + 240) = (370, 320)
    prob = _one_camera_problem([[373.0, 324.0]])
    st = O.State(np.eye(3)[None], np.zeros((1, 3)), np.array([[1.0, 2.0, 10.0]]))
    assert T.reprojection_errors(prob, st)[0] == 25.0  # 3^2 + 4^2
    # behind the camera: +inf, and never an inlier
    st.X[0, 2] = -10.0
    e = T.reprojection_errors(prob, st)
    assert np.isinf(e[0]) and not T.classify_inliers(e, 1e9)[0]


def test_classification_boundary_is_inclusive():
    e = np.array([24.999999, 25.0, 25.000001, np.inf])
    assert T.classify_inliers(e, 5.0).tolist() == [True, True, False, False]


def test_errors_vanish_at_ground_truth_and_match_the_cost():
    s = scenes.make_scene("ring", seed=5, sigma=0.0, outlier_frac=0.0)
    prob = _prob(s)
    gt = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    assert np.max(T.reprojection_errors(prob, gt)) < 1e-18 * 640 ** 2 + 1e-16
    st = O.state_from_qt(s.cam_qt, s.pts)
    e = T.reprojection_errors(prob, st)
    assert 0.5 * np.sum(e[np.isfinite(e)]) == pytest.approx(O.cost(prob, st, 0.0), rel=1e-12)


def test_two_view_triangulation_is_exact():
    R0, t0 = np.eye(3), np.zeros(3)
    c, s_ = np.cos(0.2), np.sin(0.2)
    R1 = np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]])
    t1 = -R1 @ np.array([1.0, 0.1, 0.0])
    X = np.array([0.3, -0.2, 4.0])
    fx, fy, cx, cy = 500.0, 400.0, 320.0, 240.0
    uv = []
    for R, t in ((R0, t0), (R1, t1)):
        xc = R @ X + t
        uv.append([fx * xc[0] / xc[2] + cx, fy * xc[1] / xc[2] + cy])
    prob = O.Problem.from_arrays((fx, fy, cx, cy), [0, 1], [0, 0], np.array(uv), None, 2, 1)
    st = O.State(np.stack([R0, R1]), np.stack([t0, t1]), np.zeros((1, 3)))
    Xt, status = T.triangulate_dlt(prob, st)
    assert status[0] == T.TRI_OK
    np.testing.assert_allclose(Xt[0], X, rtol=0, atol=1e-12)


def test_noise_free_scene_triangulates_to_the_truth_in_any_order():
    s = scenes.make_scene("ring", seed=6, sigma=0.0, outlier_frac=0.0)
    gt = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    X, status = T.triangulate_dlt(_prob(s), gt)
    assert np.all(status == T.TRI_OK)
    np.testing.assert_allclose(X, s.pts_gt, rtol=0, atol=1e-9)
    perm = np.random.default_rng(0).permutation(s.n_obs)
    prob_p = O.Problem.from_arrays(s.intrinsics(), s.obs_cam[perm], s.obs_pt[perm],
                                   s.obs_uv[perm], s.cam_fixed, s.n_cams, s.n_pts)
    Xp, status_p = T.triangulate_dlt(prob_p, gt)
    assert np.array_equal(status, status_p)
    np.testing.assert_allclose(Xp, X, rtol=0, atol=1e-10)


def test_mask_removes_a_gross_outlier():
    s = scenes.make_scene("ring", seed=7, sigma=0.0, outlier_frac=0.0)
    gt = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    uv = s.obs_uv.copy()
    k = int(np.flatnonzero(s.obs_pt == 3)[0])
    uv[k] += (40.0, -25.0)  # a wrong match of point 3
    prob = _prob(s, uv)
    e = T.reprojection_errors(prob, gt)
    mask = T.classify_inliers(e, 2.0)
    assert mask.sum() == s.n_obs - 1 and not mask[k]
    X_all, _ = T.triangulate_dlt(prob, gt)
    X_in, st_in = T.triangulate_dlt(prob, gt, mask)
    assert np.linalg.norm(X_all[3] - s.pts_gt[3]) > 1e-3  # the outlier pulls the point
    assert st_in[3] == T.TRI_OK
    np.testing.assert_allclose(X_in[3], s.pts_gt[3], rtol=0, atol=1e-9)


def test_status_too_few_behind_and_at_infinity():
    # one camera at the identity; point 0 seen once (too few); point 1 seen
    # twice from the same centre with the same ray (rank-deficient rows: the
    # solution set includes the point at infinity along the ray)
    fx, fy, cx, cy = 500.0, 400.0, 320.0, 240.0
    R = np.stack([np.eye(3), np.eye(3)])
    t = np.zeros((2, 3))
    prob = O.Problem.from_arrays((fx, fy, cx, cy), [0, 0, 1], [0, 1, 1],
                                 np.array([[320.0, 240.0], [330.0, 250.0], [330.0, 250.0]]),
                                 None, 2, 2)
    _, status = T.triangulate_dlt(prob, O.State(R, t, np.zeros((2, 3))))
    assert status[0] == T.TRI_TOO_FEW
    assert status[1] in (T.TRI_AT_INFINITY, T.TRI_BEHIND)
    # a point behind both cameras: DLT recovers it (the rows are projective),
    # the depth check rejects it
    c, s_ = np.cos(0.3), np.sin(0.3)
    R1 = np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]])
    t1 = -R1 @ np.array([1.0, 0.0, 0.0])
    Xb = np.array([0.2, 0.1, -5.0])
    uv = []
    for Rj, tj in ((np.eye(3), np.zeros(3)), (R1, t1)):
        xc = Rj @ Xb + tj
        uv.append([fx * xc[0] / xc[2] + cx, fy * xc[1] / xc[2] + cy])
    prob = O.Problem.from_arrays((fx, fy, cx, cy), [0, 1], [0, 0], np.array(uv), None, 2, 1)
    X, status = T.triangulate_dlt(prob, O.State(np.stack([np.eye(3), R1]),
                                                np.stack([np.zeros(3), t1]), np.zeros((1, 3))))
    assert status[0] == T.TRI_BEHIND and np.all(np.isnan(X[0]))


def test_triangulation_with_noise_is_close_to_the_truth():
    s = scenes.make_scene("ring", seed=8, sigma=0.5, outlier_frac=0.0)
    gt = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    X, status = T.triangulate_dlt(_prob(s), gt)
    assert np.all(status == T.TRI_OK)
    # 0.5 px at f = 500 and 5 m: a few millimetres
    assert np.median(np.linalg.norm(X - s.pts_gt, axis=1)) < 0.01
