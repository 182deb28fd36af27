"""GPU test of ba_cost_noalloc, the entry point that allocates no device memory.

Some callers may not allocate device memory at the point of use: a vehicle or
robot process whose device memory plan is fixed at start-up, or a library
that owns every allocation of its CUDA context through its own pool.  They
pass their own device buffers to ba_cost_noalloc, which keeps its scratch in
a fixed device array inside the library.  This test checks, through the C
ABI, that two calls in a row give the cost that ba_solve reports for the
same state and the FP64 oracle's cost of it, with and without the Huber
loss (FP64, the tolerance of the other FP64 parity tests); that a call on
another problem in between leaves no trace; that once the first call on the
device has loaded the array, further calls leave the device's free memory
unchanged; and that sizes beyond the fixed capacity, bad indices and
non-finite values are refused.

This file is named so that pytest collects it after every other test file.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2510_15271_b300 import ba, scenes

pytestmark = pytest.mark.gpu

COST_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_15271_b300 import build
    build.build()
    ba.lib()


def _device_arrays(s):
    import torch
    dev = torch.device("cuda:0")
    return dict(q=torch.tensor(s.cam_qt, dtype=torch.float64, device=dev),
                p=torch.tensor(s.pts, dtype=torch.float64, device=dev),
                c=torch.tensor(s.obs_cam, dtype=torch.int32, device=dev),
                j=torch.tensor(s.obs_pt, dtype=torch.int32, device=dev),
                uv=torch.tensor(s.obs_uv, dtype=torch.float64, device=dev),
                out=torch.zeros(1, dtype=torch.float64, device=dev))


def _cost_noalloc(s, arr, n_cams=None, delta=None):
    import torch
    K = ba.Intrinsics(*s.intrinsics())
    st = ba.lib().ba_cost_noalloc(
        0, torch.cuda.current_stream().cuda_stream, n_cams or s.n_cams, s.n_pts, s.n_obs,
        arr["q"].data_ptr(), arr["p"].data_ptr(), arr["c"].data_ptr(), arr["j"].data_ptr(),
        arr["uv"].data_ptr(), ctypes.byref(K), s.huber_delta if delta is None else delta,
        arr["out"].data_ptr())
    return st, float(arr["out"].item())


def _reference_cost(s):
    rep, _, _ = ba.solve_scene(s, "fp64", max_lm_iters=1)
    return rep["costs"][0]


def _oracle_cost(s, delta):
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    return O.cost(prob, O.state_from_qt(s.cam_qt, s.pts), delta)


def test_two_calls_match_ba_solve():
    ring = scenes.make_scene("ring", seed=21, n_cams=15, n_pts=900)
    drive = scenes.make_scene("driving", seed=22, n_cams=40, n_pts=3000, length_m=80.0)
    arrays = {id(s): _device_arrays(s) for s in (ring, drive)}
    refs = {id(s): _reference_cost(s) for s in (ring, drive)}
    for s in (ring, drive, ring):      # another problem in between must leave no trace
        st1, c1 = _cost_noalloc(s, arrays[id(s)])
        st2, c2 = _cost_noalloc(s, arrays[id(s)])
        assert st1 == ba.BA_OK and st2 == ba.BA_OK, ba.ba_last_error(None)
        assert c1 == pytest.approx(refs[id(s)], rel=COST_RTOL)
        assert c2 == pytest.approx(refs[id(s)], rel=COST_RTOL)
        assert c1 == c2


@pytest.mark.parametrize("delta", [0.0, 1.0, 2.5])
def test_matches_the_oracle_cost_with_and_without_huber(delta):
    s = scenes.make_scene("driving", seed=24, n_cams=30, n_pts=2500, length_m=60.0,
                          outlier_frac=0.05)
    arr = _device_arrays(s)
    ref = _oracle_cost(s, delta)
    for _ in range(2):
        st, c = _cost_noalloc(s, arr, delta=delta)
        assert st == ba.BA_OK, ba.ba_last_error(None)
        assert c == pytest.approx(ref, rel=COST_RTOL)


def test_later_calls_take_no_device_memory():
    """The first call on the device loads the fixed array (the one point
    where device memory is taken); after it, calls on problems of any size
    up to the limit leave the driver's free-memory count unchanged."""
    import torch
    probs = [scenes.make_scene("ring", seed=25, n_cams=4, n_pts=60, views=3),
             scenes.make_scene("ring", seed=26, n_cams=16, n_pts=1500),
             scenes.make_scene("driving", seed=27, n_cams=50, n_pts=4000, length_m=100.0)]
    arrays = [_device_arrays(s) for s in probs]
    st, _ = _cost_noalloc(probs[0], arrays[0])          # the start-up call
    assert st == ba.BA_OK, ba.ba_last_error(None)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        for s, arr in zip(probs, arrays):
            st, c = _cost_noalloc(s, arr)
            assert st == ba.BA_OK, ba.ba_last_error(None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_refuses_sizes_beyond_capacity_and_bad_indices():
    s = scenes.make_scene("ring", seed=23, n_cams=6, n_pts=100, views=3)
    arr = _device_arrays(s)
    st, _ = _cost_noalloc(s, arr, n_cams=16385)
    assert st == ba.BA_ERR_INVALID_ARG
    assert "16384" in ba.ba_last_error(None)
    arr["c"][3] = s.n_cams  # out of range: skipped by the kernel and reported
    st, _ = _cost_noalloc(s, arr)
    assert st == ba.BA_ERR_INVALID_ARG
    assert "out of range" in ba.ba_last_error(None)
    arr["c"][3] = int(s.obs_cam[3])
    st, c = _cost_noalloc(s, arr)
    assert st == ba.BA_OK
    assert c == pytest.approx(_reference_cost(s), rel=COST_RTOL)


@pytest.mark.parametrize("key,index,value,msg", [
    ("q", (4, 5), float("nan"), "camera 4 has a non-finite pose"),
    ("q", (2, slice(0, 4)), 0.0, "camera 2 has a non-finite pose or a zero quaternion"),
    ("p", (17, 1), float("inf"), "point 17 is not finite"),
    ("uv", (9, 0), float("nan"), "observation 9 has a non-finite pixel"),
])
def test_refuses_non_finite_values_like_set_problem(key, index, value, msg):
    s = scenes.make_scene("ring", seed=28, n_cams=6, n_pts=100, views=3)
    arr = _device_arrays(s)
    good = arr[key][index].clone()
    arr[key][index] = value
    st, _ = _cost_noalloc(s, arr)
    assert st == ba.BA_ERR_INVALID_ARG
    assert msg in ba.ba_last_error(None)
    arr[key][index] = good   # the next call starts clean
    st, c = _cost_noalloc(s, arr)
    assert st == ba.BA_OK, ba.ba_last_error(None)
    assert c == pytest.approx(_oracle_cost(s, s.huber_delta), rel=COST_RTOL)
