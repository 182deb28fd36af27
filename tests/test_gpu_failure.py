"""Failure detection on the GPU without a fault: a grid-barrier wait that
nothing completes gives up after its limit, reports the time-out to the host
and leaves the device usable.  The PCG kernels wait at the same barrier."""
import numpy as np
import pytest

import oracle as O
from paper_2510_15271_b300 import ba, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_15271_b300 import build
    build.build()
    ba.lib()


def test_barrier_completes_when_every_cta_arrives():
    timed_out, ms = ba.ba_selftest_barrier(blocks=16, expected=16, limit_ms=200.0)
    assert not timed_out
    assert ms < 200.0


def test_barrier_wait_runs_out_and_is_reported():
    # one arrival more than there are CTAs: the count never reaches it
    timed_out, ms = ba.ba_selftest_barrier(blocks=4, expected=5, limit_ms=30.0)
    assert timed_out
    assert 30.0 <= ms < 1000.0


def test_device_usable_after_a_time_out():
    ba.ba_selftest_barrier(blocks=2, expected=3, limit_ms=10.0)
    s = scenes.make_scene("ring", seed=1)
    rep, _, _ = ba.solve_scene(s, "fp64", max_lm_iters=2)
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    ref = O.lm_solve(prob, O.state_from_qt(s.cam_qt, s.pts),
                     O.LMOptions(huber_delta=s.huber_delta, lm_iters=2, solver="dense"))
    np.testing.assert_allclose(rep["costs"], ref.costs, rtol=1e-9)
    # the PCG kernels' own barriers still complete (a time-out would raise)
    d = scenes.make_scene("driving", seed=3, n_cams=60, n_pts=6000, length_m=120.0)
    rep, _, _ = ba.solve_scene(d, "fp32", max_lm_iters=2, solver=ba.BA_SOLVER_PCG)
    assert np.all(np.isfinite(rep["costs"])) and rep["costs"][-1] < rep["costs"][0]


def test_selftest_rejects_bad_arguments():
    for kw in (dict(blocks=0), dict(blocks=65), dict(expected=0), dict(limit_ms=0.0),
               dict(limit_ms=5000.0)):
        with pytest.raises(ba.BAError, match="INVALID"):
            ba.ba_selftest_barrier(**kw)
