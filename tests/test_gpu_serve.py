"""Served local BA (ba_create_server / ba_submit / ba_poll).

Requests of different sizes arrive while others run; each tick of the server
advances every resident request by one LM iteration.  A request's result must
be the same alone and in the mix, match the batched solver on the same
problem, and (FP64) match the oracle's per-iteration cost to 1e-9.
"""
import time

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


def _req(seed, cams=(10, 60), pts=(300, 3000)):
    return scenes.make_request(seed, cams=cams, pts=pts)


def _server(s, precision="fp32", **kw):
    o = ba.options_for_scene(s, precision, max_lm_iters=5)
    o.serve_arena_bytes = kw.pop("arena", 1 << 30)
    o.serve_slots = kw.pop("slots", 64)
    o.serve_queue = kw.pop("queue", 1024)
    for k, v in kw.items():
        setattr(o, k, v)
    return ba.ba_create_server(o)


def _wait(h, rid, timeout=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = ba.ba_poll(h, rid)
        if r is not None:
            return r
        time.sleep(0.0005)
    raise TimeoutError(rid)


def test_result_same_alone_and_in_the_mix():
    reqs = [_req(100 + i) for i in range(10)]
    target = reqs[3]
    ta = ba._ProblemArrays.from_scene(target, want_state=True)
    with _server(target) as h:
        alone = _wait(h, ba.ba_submit(h, ta))
        q_alone, p_alone = ta.q_out.copy(), ta.p_out.copy()
        # the same request among others, submitted while they run
        arrs = [ba._ProblemArrays.from_scene(s, want_state=True) for s in reqs]
        ids = []
        for i, a in enumerate(arrs):
            ids.append(ba.ba_submit(h, a))
            if i % 3 == 2:
                time.sleep(0.002)
        results = [_wait(h, rid) for rid in ids]
        stats = ba.ba_kernel_stats(h)
    mixed = results[3]
    assert mixed.status == ba.BA_OK and alone.status == ba.BA_OK
    assert np.array_equal(mixed.costs(), alone.costs())
    assert np.array_equal(arrs[3].q_out, q_alone) and np.array_equal(arrs[3].p_out, p_alone)
    assert all(r.status == ba.BA_OK and r.latency_ms > 0 for r in results)
    assert stats["serve_completed"][0] == 11
    assert stats["serve_tick"][0] >= 1


def test_served_matches_batched():
    reqs = [_req(200 + i, cams=(10, 40), pts=(300, 2000)) for i in range(4)]
    arrs = [ba._ProblemArrays.from_scene(s, want_state=True) for s in reqs]
    o = ba.options_for_scene(reqs[0], "fp32", max_lm_iters=5)
    with ba.ba_create(o) as h:
        batched = ba.ba_solve_batch(h, arrs)
    with _server(reqs[0]) as h:
        ids = [ba.ba_submit(h, a) for a in arrs]
        served = [_wait(h, rid) for rid in ids]
    for b, s in zip(batched, served):
        assert np.array_equal(b.costs(), s.costs())


def test_fp64_request_matches_oracle():
    s = _req(300, cams=(10, 20), pts=(300, 800))
    a = ba._ProblemArrays.from_scene(s, want_state=True)
    with _server(s, "fp64") as h:
        r = _wait(h, ba.ba_submit(h, a))
    prob = O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)
    ref = O.lm_solve(prob, O.state_from_qt(s.cam_qt, s.pts),
                     O.LMOptions(huber_delta=s.huber_delta, lm_iters=5, solver="dense"))
    rel = np.abs(r.costs() - ref.costs) / ref.costs
    assert rel.max() <= 1e-9, (rel, r.costs(), ref.costs)
    np.testing.assert_allclose(a.p_out, ref.state.X, atol=1e-7)


def test_admission_waits_for_memory():
    # an arena that holds about two of these requests at once: the rest wait
    # for memory and are admitted as earlier ones finish
    reqs = [_req(400 + i, cams=(20, 30), pts=(1500, 2000)) for i in range(6)]
    from paper_2510_15271_b300.ba import lib
    arrs = [ba._ProblemArrays.from_scene(s, want_state=True) for s in reqs]
    sizes = []
    for s in reqs:
        n = len(s.obs_cam)
        sizes.append(200 * n + 400 * s.n_pts + 4 * (6 * s.n_cams) ** 2 + 4 * 512 * s.n_cams)
    arena = int(2.5 * max(sizes)) + (4 << 20)
    with _server(reqs[0], arena=arena) as h:
        ids = [ba.ba_submit(h, a) for a in arrs]
        res = [_wait(h, rid) for rid in ids]
    assert all(r.status == ba.BA_OK for r in res)
    o = ba.options_for_scene(reqs[0], "fp32", max_lm_iters=5)
    with ba.ba_create(o) as h:
        batched = ba.ba_solve_batch(h, [ba._ProblemArrays.from_scene(s) for s in reqs])
    for b, r in zip(batched, res):
        assert np.array_equal(b.costs(), r.costs())


def test_request_larger_than_arena_is_refused():
    s = _req(500, cams=(30, 40), pts=(3000, 4000))
    with _server(s, arena=1 << 20) as h:
        with pytest.raises(ba.BAError, match="OOM"):
            ba.ba_submit(h, ba._ProblemArrays.from_scene(s))


def test_queue_full_is_busy():
    """One slot and a waiting queue of one: while the big request runs, a
    second request waits and the next submission is refused with BUSY."""
    big = _req(600, cams=(150, 160), pts=(20000, 25000))
    small = _req(601, cams=(10, 12), pts=(300, 400))
    sa = ba._ProblemArrays.from_scene(small)
    with _server(big, slots=1, queue=1) as h:
        ids = [ba.ba_submit(h, ba._ProblemArrays.from_scene(big))]
        busy = False
        for _ in range(8):  # submissions are microseconds apart; the big solve takes ms
            try:
                ids.append(ba.ba_submit(h, sa))
            except ba.BAError as e:
                assert e.status == ba.BA_ERR_BUSY
                busy = True
                break
        assert busy
        assert len(ids) <= 3
        assert all(_wait(h, rid).status == ba.BA_OK for rid in ids)


def test_poll_semantics_and_state_errors():
    s = _req(700, cams=(10, 12), pts=(300, 400))
    with _server(s) as h:
        rid = ba.ba_submit(h, ba._ProblemArrays.from_scene(s))
        _wait(h, rid)
        with pytest.raises(ba.BAError, match="INVALID"):
            ba.ba_poll(h, rid)           # collected already
        with pytest.raises(ba.BAError, match="INVALID"):
            ba.ba_poll(h, 987654321)
        with pytest.raises(ba.BAError, match="STATE"):
            ba.ba_set_problem(h, s.cam_qt, s.pts, s.obs_cam, s.obs_pt, s.obs_uv, s.intrinsics())
    with ba.ba_create(ba.options_for_scene(s, "fp32")) as h:
        with pytest.raises(ba.BAError, match="STATE"):
            ba.ba_submit(h, ba._ProblemArrays.from_scene(s))


def test_invalid_request_is_reported():
    s = _req(800, cams=(10, 12), pts=(300, 400))
    pt = s.obs_pt.copy()
    pt[0] = -1
    a = ba._ProblemArrays(s.cam_qt, s.pts, s.obs_cam, pt, s.obs_uv, s.intrinsics(), s.cam_fixed)
    with _server(s) as h:
        rid = ba.ba_submit(h, a)
        with pytest.raises(ba.BAError, match="INVALID"):
            _wait(h, rid)


def test_tick_budget_does_not_change_results():
    reqs = [_req(900 + i, cams=(10, 40), pts=(300, 2000)) for i in range(5)]
    arrs = [ba._ProblemArrays.from_scene(s) for s in reqs]
    out = []
    for budget in (0.0, 50.0):
        with _server(reqs[0], serve_tick_ms=budget) as h:
            ids = [ba.ba_submit(h, a) for a in arrs]
            out.append([_wait(h, rid) for rid in ids])
            ticks = ba.ba_kernel_stats(h)["serve_tick"][0]
        if budget == 0.0:
            assert ticks >= 5  # one iteration per tick
    for a, b in zip(*out):
        assert np.array_equal(a.costs(), b.costs())


def test_large_requests_run_beside_the_ticks():
    """Requests above 96 cameras run in launches of their own beside the
    small requests' ticks; every result still equals the batched solver's."""
    small = [_req(1000 + i, cams=(10, 40), pts=(300, 2000)) for i in range(6)]
    large = [_req(1100 + i, cams=(100, 130), pts=(3000, 6000)) for i in range(3)]
    reqs = [x for pair in zip(small, large + [None] * 3) for x in pair if x is not None]
    arrs = [ba._ProblemArrays.from_scene(s, want_state=True) for s in reqs]
    with _server(reqs[0]) as h:
        ids = []
        for i, a in enumerate(arrs):
            ids.append(ba.ba_submit(h, a))
            if i % 4 == 3:
                time.sleep(0.003)
        served = [_wait(h, rid) for rid in ids]
        stats = ba.ba_kernel_stats(h)
    assert stats["serve_large"][0] >= 1
    o = ba.options_for_scene(reqs[0], "fp32", max_lm_iters=5)
    with ba.ba_create(o) as h:
        batched = ba.ba_solve_batch(h, [ba._ProblemArrays.from_scene(s) for s in reqs])
    for b, r in zip(batched, served):
        assert r.status == ba.BA_OK
        assert np.array_equal(b.costs(), r.costs())
