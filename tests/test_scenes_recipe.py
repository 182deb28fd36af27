"""The seeded synthetic workloads follow their stated recipes (CPU).

Checked on the generators themselves, at full size for the small workloads and
at reduced size for the driving and city ones: camera model, track-length
distribution, outlier fraction, pixel noise of the inliers at the true state,
initial perturbation, the fixed gauge camera and the solve settings.  The
projection used here is written out in the test (pinhole of the world-to-camera
pose), independent of the generator's own.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2510_15271_b300 import scenes


def _project(s, qt, X, cam, pt):
    R = Rotation.from_quat(qt[:, [1, 2, 3, 0]])
    xc = R[cam].apply(X[pt]) + qt[cam, 4:]
    u = s.fx * xc[:, 0] / xc[:, 2] + s.cx
    v = s.fy * xc[:, 1] / xc[:, 2] + s.cy
    return np.stack([u, v], 1), xc[:, 2]


def _noise(s):
    """Inlier pixel errors at the true state (per coordinate)."""
    uv, z = _project(s, s.cam_qt_gt, s.pts_gt, s.obs_cam, s.obs_pt)
    assert np.all(z > 0)
    return (s.obs_uv - uv)[s.obs_inlier].ravel()


def _perturbation(s):
    Ra = Rotation.from_quat(s.cam_qt[:, [1, 2, 3, 0]])
    Rb = Rotation.from_quat(s.cam_qt_gt[:, [1, 2, 3, 0]])
    ang = (Ra * Rb.inv()).magnitude()
    Ca = -Ra.inv().apply(s.cam_qt[:, 4:])
    Cb = -Rb.inv().apply(s.cam_qt_gt[:, 4:])
    free = s.cam_fixed == 0
    return ang[free], (Ca - Cb)[free].ravel(), (s.pts - s.pts_gt).ravel()


def _track_lengths(s):
    return np.bincount(s.obs_pt, minlength=s.n_pts)


def test_ring_recipe():
    s = scenes.make_scene("ring", seed=3)
    assert (s.n_cams, s.n_pts, s.n_obs) == (20, 2000, 10000)
    assert (s.width, s.height, s.fx, s.fy, s.cx, s.cy) == (640, 480, 500.0, 500.0, 320.0, 240.0)
    assert np.all(_track_lengths(s) == 5)
    assert np.all(s.obs_inlier)
    Rgt = Rotation.from_quat(s.cam_qt_gt[:, [1, 2, 3, 0]])
    centres = -Rgt.inv().apply(s.cam_qt_gt[:, 4:])
    assert np.allclose(np.linalg.norm(centres[:, :2], axis=1), 5.0, atol=1e-9)
    assert np.all(np.abs(s.pts_gt) <= 2.0)
    uv, _ = _project(s, s.cam_qt_gt, s.pts_gt, s.obs_cam, s.obs_pt)
    assert np.all((uv >= 0) & (uv < [640, 480]))
    assert np.std(_noise(s)) == pytest.approx(0.5, rel=0.05)
    ang, dc, dx = _perturbation(s)
    assert np.sqrt(np.mean(ang ** 2)) == pytest.approx(0.01 * np.sqrt(3), rel=0.25)
    assert np.std(dc) == pytest.approx(0.05, rel=0.25)
    assert np.std(dx) == pytest.approx(0.05, rel=0.05)
    assert s.cam_fixed[0] == 1 and s.cam_fixed.sum() == 1
    assert (s.huber_delta, s.lm_iters, s.solver) == (0.0, 10, "dense")


def test_driving_recipe():
    s = scenes.make_scene("driving", seed=3, n_cams=200, n_pts=40000, length_m=400.0)
    assert (s.width, s.height, s.fx, s.cx, s.cy) == (1920, 1080, 1000.0, 960.0, 540.0)
    L = _track_lengths(s)
    assert L.min() >= 2 and L.max() <= 30
    assert L.mean() == pytest.approx(6.0, rel=0.05)  # geometric, mean 6, clamped to [2, 30]
    # each track is a run of consecutive cameras along the route
    o = np.lexsort((s.obs_cam, s.obs_pt))
    c = s.obs_cam[o].astype(np.int64)
    start = np.concatenate([[0], np.cumsum(L)[:-1]])
    span = np.maximum.reduceat(c, start) - np.minimum.reduceat(c, start) + 1
    assert np.all(span == L)
    assert 1.0 - s.obs_inlier.mean() == pytest.approx(0.02, rel=0.1)
    assert np.std(_noise(s)) == pytest.approx(0.7, rel=0.05)
    _, dc, _ = _perturbation(s)
    assert np.std(dc) == pytest.approx(0.05, rel=0.1)
    assert s.cam_fixed[0] == 1 and s.cam_fixed.sum() == 1
    assert (s.huber_delta, s.lm_iters, s.solver, s.pcg_tol, s.pcg_max_iters) == \
        (1.0, 20, "pcg", 1e-6, 100)


def test_city_recipe():
    s = scenes.make_scene("city", seed=3, n_cams=500, n_pts=100000)
    L = _track_lengths(s)
    assert L.min() >= 2 and L.max() <= 40
    l = np.arange(2, 41)
    zipf = l ** -1.5 / np.sum(l ** -1.5)  # Zipf, s = 1.5, on [2, 40]
    assert L.mean() == pytest.approx(np.sum(l * zipf), rel=0.05)
    assert np.mean(L == 2) == pytest.approx(zipf[0], rel=0.1)
    assert 1.0 - s.obs_inlier.mean() == pytest.approx(0.01, rel=0.1)
    assert np.std(_noise(s)) == pytest.approx(1.0, rel=0.05)
    assert s.cam_fixed[0] == 1
    assert (s.huber_delta, s.lm_iters, s.solver, s.refine) == (1.5, 15, "pcg", True)


def test_window_and_request_recipes():
    ws = scenes.make_windows(n_windows=24, seed=4)
    for w in ws:
        assert 10 <= w.n_cams <= 60 and 500 <= w.n_pts <= 8000
        L = _track_lengths(w)
        assert L.min() >= 3 and L.max() <= 10
        assert w.lm_iters == 5 and (w.width, w.height, w.fx) == (640, 480, 500.0)
    reqs = [scenes.make_request(5000 + k) for k in range(24)]
    for r in reqs:
        assert 10 <= r.n_cams <= 200 and 1000 <= r.n_pts <= 40000
        assert r.lm_iters == 5 and _track_lengths(r).min() >= 2
    # track length 2 + Geometric(mean 3): mean 5 over the pooled requests
    pooled = np.concatenate([_track_lengths(r) for r in reqs])
    assert pooled.mean() == pytest.approx(5.0, rel=0.05)
    # log-uniform sizes: the logs of the camera counts spread over [log 10, log 200]
    lc = np.log([r.n_cams for r in reqs])
    assert lc.min() < np.log(40) and lc.max() > np.log(60)


def test_generators_are_seeded():
    a = scenes.make_scene("driving", seed=9, n_cams=60, n_pts=6000, length_m=120.0)
    b = scenes.make_scene("driving", seed=9, n_cams=60, n_pts=6000, length_m=120.0)
    c = scenes.make_scene("driving", seed=10, n_cams=60, n_pts=6000, length_m=120.0)
    for f in ("cam_qt", "pts", "obs_cam", "obs_pt", "obs_uv", "obs_inlier"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert not np.array_equal(a.obs_uv, c.obs_uv) or a.n_obs != c.n_obs
