"""Full-size checks of the sparse workloads in the configuration the
benchmark times: driving (1,000 cameras, 200k points, ~1.21M observations,
FP32) and city (5,000 cameras, 1M points, ~7.9M observations, FP32 with FP64
refinement of the PCG residual).

Expected values come from tests/golden/<workload>_seed<seed>_oracle.json,
written by tests/golden/make_golden.py with the FP64 CPU oracle only.
"""
import glob
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2510_15271_b300 import ba, scenes

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDENS = sorted(glob.glob(os.path.join(HERE, "golden", "*_oracle.json")))


@pytest.fixture(scope="module", params=GOLDENS, ids=lambda p: os.path.basename(p).split("_")[0])
def golden(request):
    with open(request.param) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def scene(golden):
    from paper_2510_15271_b300 import build
    build.build()
    s = scenes.make_scene(golden["workload"], seed=golden["seed"])
    assert (s.n_cams, s.n_pts, s.n_obs) == (golden["n_cams"], golden["n_pts"], golden["n_obs"])
    return s


def _prob(s):
    return O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)


def test_initial_cost_matches_oracle(scene, golden):
    for prec, rtol in (("fp64", 1e-12), ("fp32", 1e-5)):
        rep, _, _ = ba.solve_scene(scene, prec, max_lm_iters=1, use_torch=True)
        assert rep["costs"][0] == pytest.approx(golden["costs"][0], rel=rtol), prec


def test_fp64_first_step_matches_oracle(scene, golden):
    """Same PCG settings on both sides: the first step's cost agrees to about
    the solve tolerance."""
    rep, _, _ = ba.solve_scene(scene, "fp64", max_lm_iters=2, use_torch=True)
    np.testing.assert_allclose(rep["costs"][:2], golden["costs"][:2], rtol=1e-6)
    assert rep["pcg_iters"][0] == golden["pcg_iters"][0]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_final_rmse_within_one_percent_of_oracle(scene, golden, prec):
    rep, q, p = ba.solve_scene(scene, prec, use_torch=True)
    prob = _prob(scene)
    st = O.state_from_qt(q, p)
    r = O.rmse(prob, st, scene.obs_inlier, golden["outlier_threshold_px"])
    r_ref = golden["rmse_inlier_trimmed_px"]
    assert abs(r - r_ref) <= 0.01 * r_ref, (prec, r, r_ref)
    # the gate on every generator inlier, untrimmed
    u = O.rmse(prob, st, scene.obs_inlier)
    u_ref = golden["rmse_inlier_px"]
    assert abs(u - u_ref) <= 0.01 * u_ref, (prec, u, u_ref)
    # the report's own RMSE is over every observation in front of the camera
    assert rep["rmse_px"] == pytest.approx(O.rmse(prob, st), rel=1e-6)
    assert rep["costs"][-1] <= 1.01 * golden["costs"][-1]
    print(f"{prec}: inlier rmse trimmed {r:.5f} (oracle {r_ref:.5f}), untrimmed {u:.5f} "
          f"(oracle {u_ref:.5f}), final cost {rep['costs'][-1]:.7e} "
          f"(oracle {golden['costs'][-1]:.7e})")
