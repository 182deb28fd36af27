"""Host logic of bench.py's multi-GPU leg (independent replicas, no data-path
collective): the max-over-ranks timing and the whole-job rate, run as two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        m = bench.max_over_ranks(ms, world, "cpu")
        v = bench.whole_job_value(1000, 4, world, m)
        out.put((rank, m, v, bench.replica_seed(7, rank)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, seed in res:
        assert m == 15.0
        assert v == pytest.approx(1000 * 4 * 2 / 0.015)
        assert seed == 7 + rank
    assert res[0][3] != res[1][3]


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_value(100, 2, 1, 50.0) == pytest.approx(4000.0)


def test_pose_difference_after_similarity_alignment():
    """Two pose sets that differ by a similarity of the world (rotation,
    scale, translation) differ by zero after the alignment, and not before;
    a perturbation of one camera shows up after it."""
    import numpy as np
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(3)
    n = 40
    Ra = Rotation.random(n, random_state=4)
    ta = rng.normal(size=(n, 3))
    qa = np.concatenate([Ra.as_quat()[:, [3, 0, 1, 2]], ta], 1)
    G = Rotation.from_rotvec([0.2, -0.4, 0.1])
    scale, shift = 1.7, np.array([3.0, -1.0, 0.5])
    Rb = Ra * G.inv()
    Cb = scale * G.apply(-Ra.inv().apply(ta)) + shift
    qb = np.concatenate([Rb.as_quat()[:, [3, 0, 1, 2]], -Rb.apply(Cb)], 1)
    rot, pos = bench.pose_errors_qt(qa, qb)
    assert rot.max() > 0.1 and pos.max() > 0.1
    rot, pos = bench.pose_errors_qt(qa, qb, align=True)
    assert rot.max() < 1e-12 and pos.max() < 1e-12
    qc = qb.copy()
    qc[7, 4] += 0.01  # move camera 7 by 1 cm (it also tilts the fitted similarity a little)
    rot, pos = bench.pose_errors_qt(qa, qc, align=True)
    assert int(np.argmax(pos)) == 7 and 0.005 < pos[7] < 0.011 and rot.max() < 1e-3


def test_measured_traffic_reads_the_matching_row_of_a_current_profile(tmp_path, monkeypatch):
    """The bench takes a kernel's DRAM traffic from the committed ncu summary
    only while the summary's source digest matches the sources, only from
    the row named exactly after the kernel, and reports none for a row
    without a full-size figure."""
    import types
    prof = tmp_path / "city_fp32_kernels.md"
    digest = bench.source_digest()
    prof.write_text(
        f"Source digest of the driving path's sources at capture: `{digest}`\n\n"
        "| kernel | a | b | c | traffic / launch (B) | rest |\n|---|---|---|---|---|---|\n"
        "| k_pcg_stream (0.4 scale) | 1 | 2 | 3 | 999 | x |\n"
        "| k_pcg_stream | 1 | 2 | 3 | 123456 | x |\n"
        "| k_schur | 1 | 2 | 3 | 777 | x |\n"
        "| k_backsub | 1 | 2 | 3 | — | x |\n")
    monkeypatch.setattr(bench, "profile_path", lambda name: str(prof))
    s = types.SimpleNamespace(name="city")
    assert bench.measured_traffic(s, "pcg") == 123456
    assert bench.measured_traffic(s, "schur") == 777
    assert bench.measured_traffic(s, "backsub") is None
    assert bench.measured_traffic(s, "lin_pt") is None
    prof.write_text(prof.read_text().replace(digest, "0" * 16))
    assert bench.measured_traffic(s, "pcg") is None
