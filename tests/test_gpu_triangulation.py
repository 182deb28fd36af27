"""Reprojection errors, outlier classification and DLT triangulation on the
GPU (ba_reprojection_errors, ba_triangulate) against the FP64 oracle, and the
paper's two-stage mapping loop (Sec. 4.3) built from them and ba_solve."""
import numpy as np
import pytest

import oracle as O
from oracle import triangulation as OT
from paper_2510_15271_b300 import ba, scenes

pytestmark = pytest.mark.gpu

ERR_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_15271_b300 import build
    build.build()
    ba.lib()


def _prob(s, uv=None):
    return O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt,
                                 s.obs_uv if uv is None else uv, s.cam_fixed, s.n_cams, s.n_pts)


def _driving_small(seed=3, **kw):
    base = dict(n_cams=60, n_pts=6000, length_m=120.0)
    base.update(kw)
    return scenes.make_scene("driving", seed=seed, **base)


def _dlt_condition(s, st, mask):
    """lambda_max / (lambda_2 - lambda_1) of each point's A^T A (for the
    comparison tolerance only)."""
    use = np.ones(s.n_obs, bool) if mask is None else np.asarray(mask, bool)
    fx, fy, cx, cy = s.intrinsics()
    cam, pt = s.obs_cam[use], s.obs_pt[use]
    x = (s.obs_uv[use, 0] - cx) / fx
    y = (s.obs_uv[use, 1] - cy) / fy
    Pm = np.concatenate([st.R, st.t[:, :, None]], axis=2)[cam]
    r1 = x[:, None] * Pm[:, 2] - Pm[:, 0]
    r2 = y[:, None] * Pm[:, 2] - Pm[:, 1]
    M = np.zeros((s.n_pts, 4, 4))
    np.add.at(M, pt, np.einsum("ni,nj->nij", r1, r1) + np.einsum("ni,nj->nij", r2, r2))
    lam = np.linalg.eigvalsh(M)
    return lam[:, 3] / np.maximum(lam[:, 1] - lam[:, 0], 1e-300)


def _check_errors(s, cam_qt, pts, thresholds=(1.0, 2.0, 5.0)):
    st = O.state_from_qt(cam_qt, pts)
    ref = OT.reprojection_errors(_prob(s), st)
    for thr in thresholds:
        e, inl, n = ba.ba_reprojection_errors(cam_qt, pts, s.obs_cam, s.obs_pt, s.obs_uv,
                                              s.intrinsics(), thr)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(e), fin)
        # the camera-frame point R X + t is a difference of world-scale
        # numbers (up to ~2 km here): its rounding, ~1e-12 m, is ~1e-10 px at
        # the shortest depths, so e = du^2 + dv^2 may differ by about
        # 2 |d| 1e-10 between two orders of the same FP64 operations
        tol = 1e-9 * np.sqrt(ref[fin]) + ERR_RTOL * ref[fin] + 1e-18
        assert np.all(np.abs(e[fin] - ref[fin]) <= tol)
        assert np.array_equal(inl, OT.classify_inliers(ref, thr))
        assert n == int(inl.sum())


def test_errors_and_classification_match_the_oracle():
    s = _driving_small()
    _check_errors(s, s.cam_qt, s.pts)          # perturbed start: large errors
    _check_errors(s, s.cam_qt_gt, s.pts_gt)    # truth: noise and the outliers


def test_errors_at_full_driving_size():
    s = scenes.make_scene("driving", seed=2)
    _check_errors(s, s.cam_qt, s.pts, thresholds=(5.0,))


def test_noise_free_triangulation_recovers_the_truth():
    s = scenes.make_scene("ring", seed=6, sigma=0.0, outlier_frac=0.0)
    X, status = ba.ba_triangulate(s.cam_qt_gt, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(),
                                  s.n_pts)
    assert np.all(status == OT.TRI_OK)
    np.testing.assert_allclose(X, s.pts_gt, rtol=0, atol=1e-9)


@pytest.mark.parametrize("masked", [False, True])
def test_triangulation_matches_the_oracle(masked):
    s = _driving_small(seed=4)
    st = O.state_from_qt(s.cam_qt_gt, s.pts_gt)
    mask = None
    if masked:
        mask = OT.classify_inliers(OT.reprojection_errors(_prob(s), st), 3.0)
    X, status = ba.ba_triangulate(s.cam_qt_gt, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(),
                                  s.n_pts, mask)
    Xr, sr = OT.triangulate_dlt(_prob(s), st, mask)
    assert np.array_equal(status, sr)
    ok = sr == OT.TRI_OK
    assert ok.mean() > (0.95 if masked else 0.85)  # unmasked: the outliers spoil some points
    scale = 1.0 + np.linalg.norm(Xr[ok], axis=1)
    rel = np.max(np.abs(X[ok] - Xr[ok]), axis=1) / scale
    # the eigenvector moves by about eps ||A^T A|| / (gap of its two smallest
    # eigenvalues) (Davis-Kahan), and the point by about that times its
    # distance: a short baseline (a distant point seen along the direction of
    # travel) or rows made inconsistent by an outlier shrink the gap
    kappa = _dlt_condition(s, st, mask)[ok]
    assert np.median(rel) < 1e-12
    assert np.all(rel <= 1e-14 * kappa * scale + 1e-12), np.max(rel / (kappa * scale))
    assert np.all(np.isnan(X[~ok]))


def test_result_does_not_depend_on_the_observation_order():
    s = _driving_small(seed=5)
    perm = np.random.default_rng(1).permutation(s.n_obs)
    a = ba.ba_triangulate(s.cam_qt, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(), s.n_pts)
    b = ba.ba_triangulate(s.cam_qt, s.obs_cam[perm], s.obs_pt[perm], s.obs_uv[perm],
                          s.intrinsics(), s.n_pts)
    assert np.array_equal(a[1], b[1])
    assert np.array_equal(a[0], b[0], equal_nan=True)


def test_status_cases_match_the_oracle():
    # seen once; the same ray twice from one centre; behind both cameras
    fx, fy, cx, cy = 500.0, 400.0, 320.0, 240.0
    c, s_ = np.cos(0.3), np.sin(0.3)
    R1 = np.array([[c, 0, s_], [0, 1, 0], [-s_, 0, c]])
    t1 = -R1 @ np.array([1.0, 0.0, 0.0])
    Xb = np.array([0.2, 0.1, -5.0])
    uvb = []
    for Rj, tj in ((np.eye(3), np.zeros(3)), (R1, t1)):
        xc = Rj @ Xb + tj
        uvb.append([fx * xc[0] / xc[2] + cx, fy * xc[1] / xc[2] + cy])
    cam = np.array([0, 0, 0, 0, 1], np.int32)
    pt = np.array([0, 1, 1, 2, 2], np.int32)
    uv = np.array([[320.0, 240.0], [330.0, 250.0], [330.0, 250.0], uvb[0], uvb[1]])
    qt = np.zeros((2, 7))
    qt[0, 0] = 1.0
    qt[1, :4] = O.rot_to_quat(R1[None])[0]
    qt[1, 4:] = t1
    X, status = ba.ba_triangulate(qt, cam, pt, uv, (fx, fy, cx, cy), 3)
    prob = O.Problem.from_arrays((fx, fy, cx, cy), cam, pt, uv, None, 2, 3)
    _, sr = OT.triangulate_dlt(prob, O.state_from_qt(qt, np.zeros((3, 3))))
    assert status[0] == sr[0] == OT.TRI_TOO_FEW
    assert status[1] in (OT.TRI_AT_INFINITY, OT.TRI_BEHIND)
    assert status[2] == sr[2] == OT.TRI_BEHIND
    assert np.all(np.isnan(X))


def test_device_pointers_give_the_host_results():
    import torch
    s = _driving_small(seed=6)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")
    q, X0 = dev(s.cam_qt, torch.float64), dev(s.pts, torch.float64)
    oc, op = dev(s.obs_cam, torch.int32), dev(s.obs_pt, torch.int32)
    uv = dev(s.obs_uv, torch.float64)
    e = torch.empty(s.n_obs, dtype=torch.float64, device="cuda:0")
    inl = torch.empty(s.n_obs, dtype=torch.uint8, device="cuda:0")
    cnt = ba.c_int64()
    K = ba.Intrinsics(*s.intrinsics())
    st = ba.lib().ba_reprojection_errors(0, None, s.n_cams, s.n_pts, s.n_obs, q.data_ptr(),
                                         X0.data_ptr(), oc.data_ptr(), op.data_ptr(),
                                         uv.data_ptr(), ba.ctypes.byref(K), 2.0, e.data_ptr(),
                                         inl.data_ptr(), ba.ctypes.byref(cnt), ba.BA_MEM_DEVICE)
    assert st == ba.BA_OK
    eh, ih, nh = ba.ba_reprojection_errors(s.cam_qt, s.pts, s.obs_cam, s.obs_pt, s.obs_uv,
                                           s.intrinsics(), 2.0)
    assert np.array_equal(e.cpu().numpy(), eh) and np.array_equal(inl.cpu().numpy() != 0, ih)
    assert cnt.value == nh
    Xd = torch.empty((s.n_pts, 3), dtype=torch.float64, device="cuda:0")
    sd = torch.empty(s.n_pts, dtype=torch.int8, device="cuda:0")
    st = ba.lib().ba_triangulate(0, None, s.n_cams, s.n_pts, s.n_obs, q.data_ptr(), oc.data_ptr(),
                                 op.data_ptr(), uv.data_ptr(), ba.ctypes.byref(K), inl.data_ptr(),
                                 Xd.data_ptr(), sd.data_ptr(), ba.BA_MEM_DEVICE)
    assert st == ba.BA_OK
    Xh, sh = ba.ba_triangulate(s.cam_qt, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(), s.n_pts,
                               ih)
    assert np.array_equal(sd.cpu().numpy(), sh)
    assert np.array_equal(Xd.cpu().numpy(), Xh, equal_nan=True)


def test_invalid_arguments_are_refused():
    s = _driving_small(seed=7)
    bad = s.obs_pt.copy()
    bad[5] = s.n_pts
    with pytest.raises(ba.BAError, match="INVALID"):
        ba.ba_reprojection_errors(s.cam_qt, s.pts, s.obs_cam, bad, s.obs_uv, s.intrinsics(), 2.0)
    with pytest.raises(ba.BAError, match="INVALID"):
        ba.ba_triangulate(s.cam_qt, s.obs_cam, bad, s.obs_uv, s.intrinsics(), s.n_pts)
    with pytest.raises(ba.BAError, match="INVALID"):
        ba.ba_reprojection_errors(s.cam_qt, s.pts, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(),
                                  -1.0)
    # the device is usable afterwards
    ba.ba_triangulate(s.cam_qt, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics(), s.n_pts)


# --------------------------------------------------------------------------- the mapping loop

RELAXED_PX, STRICT_PX = 8.0, 3.0


def _keep(s, obs_keep, X, pt_ok):
    """The scene restricted to kept observations of triangulated points,
    points renumbered (host-side selection; no arithmetic)."""
    keep = obs_keep & pt_ok[s.obs_pt]
    # points that keep at least two observations
    cnt = np.bincount(s.obs_pt[keep], minlength=s.n_pts)
    live = cnt >= 2
    keep &= live[s.obs_pt]
    new_id = np.cumsum(live) - 1
    return (s.obs_cam[keep], new_id[s.obs_pt[keep]].astype(np.int32), s.obs_uv[keep],
            X[live], keep, live)


def test_two_stage_mapping_loop_matches_the_oracle():
    """Sec. 4.3: stage one with the robust loss and a relaxed outlier
    threshold; outliers removed and points re-triangulated from the
    remaining observations; stage two without a loss function and a strict
    threshold.  The GPU loop (ba_solve, ba_reprojection_errors,
    ba_triangulate) against the same loop on the oracle."""
    s = _driving_small(seed=8, outlier_frac=0.05)
    K = s.intrinsics()
    # stage one: Huber, relaxed threshold
    o1 = ba.options_for_scene(s, "fp64", max_lm_iters=8, solver=ba.BA_SOLVER_PCG)
    with ba.ba_create(o1) as h:
        ba.ba_set_problem(h, s.cam_qt, s.pts, s.obs_cam, s.obs_pt, s.obs_uv, K, s.cam_fixed)
        ba.ba_solve(h)
        q1, p1 = ba.ba_get_state(h, s.n_cams, s.n_pts)
    _, inl1, _ = ba.ba_reprojection_errors(q1, p1, s.obs_cam, s.obs_pt, s.obs_uv, K, RELAXED_PX)
    X1, st1 = ba.ba_triangulate(q1, s.obs_cam, s.obs_pt, s.obs_uv, K, s.n_pts, inl1)
    ok1 = st1 == OT.TRI_OK
    oc, op, uv, X2, keep, live = _keep(s, inl1, X1, ok1)
    # stage two: plain least squares
    o2 = ba.options_for_scene(s, "fp64", max_lm_iters=8, solver=ba.BA_SOLVER_PCG, huber_delta=0.0)
    with ba.ba_create(o2) as h:
        ba.ba_set_problem(h, q1, X2, oc, op, uv, K, s.cam_fixed)
        rep = ba.ba_solve(h)
        q2, p2 = ba.ba_get_state(h, s.n_cams, X2.shape[0])
    _, inl2, n2 = ba.ba_reprojection_errors(q2, p2, oc, op, uv, K, STRICT_PX)
    prob2 = O.Problem.from_arrays(K, oc, op, uv, s.cam_fixed, s.n_cams, X2.shape[0])
    rmse_gpu = O.rmse(prob2, O.state_from_qt(q2, p2), inl2)

    # the same loop on the oracle, with its own selections
    prob = _prob(s)
    r1 = O.lm_solve(prob, O.state_from_qt(s.cam_qt, s.pts),
                    O.LMOptions(huber_delta=s.huber_delta, lm_iters=8, solver="pcg",
                                pcg_tol=s.pcg_tol, pcg_max_iters=s.pcg_max_iters))
    m1 = OT.classify_inliers(OT.reprojection_errors(prob, r1.state), RELAXED_PX)
    Xo, so = OT.triangulate_dlt(prob, r1.state, m1)
    oc_r, op_r, uv_r, X2_r, keep_r, live_r = _keep(s, m1, Xo, so == OT.TRI_OK)
    prob2_r = O.Problem.from_arrays(K, oc_r, op_r, uv_r, s.cam_fixed, s.n_cams, X2_r.shape[0])
    r2 = O.lm_solve(prob2_r, O.State(r1.state.R, r1.state.t, X2_r),
                    O.LMOptions(huber_delta=0.0, lm_iters=8, solver="pcg",
                                pcg_tol=s.pcg_tol, pcg_max_iters=s.pcg_max_iters))
    m2 = OT.classify_inliers(OT.reprojection_errors(prob2_r, r2.state), STRICT_PX)
    rmse_ref = O.rmse(prob2_r, r2.state, m2)
    # the decisions agree but for observations at the thresholds
    assert np.mean(m1 != inl1) < 1e-3 and np.mean(so != st1) < 1e-3
    assert abs(int(keep.sum()) - int(keep_r.sum())) <= 0.002 * keep.sum()
    assert abs(rmse_gpu - rmse_ref) <= 0.01 * rmse_ref, (rmse_gpu, rmse_ref)
    assert abs(n2 - int(m2.sum())) <= 0.002 * n2
    # the injected outliers are gone after stage one
    injected = ~s.obs_inlier
    assert (~inl1[injected]).mean() > 0.9
    print(f"two-stage loop: kept {keep.sum()} of {s.n_obs} observations, {live.sum()} points; "
          f"strict inliers {n2}; RMSE {rmse_gpu:.4f} px (oracle {rmse_ref:.4f})")
