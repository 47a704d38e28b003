"""Host-side logic of bench.py's multi-GPU launch (one replica per rank, no
collective on the data path), on CPU: the max-over-ranks timing and the
whole-job rate with two gloo ranks, and the reference arm under a
multi-rank launch (rank 0 alone prints, the others exit 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = bench.max_over_ranks(times[rank], dist, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, bench.whole_job_mlups(1000, 10, world, t)))


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    times = [0.25, 0.5]
    procs = [mp.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [0.5, 0.5]                          # every rank sees the slowest time
    assert all(abs(g[2] - 1000 * 10 * 2 / 0.5 / 1e6) < 1e-12 for g in got)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.3) == 0.3
    assert bench.whole_job_mlups(4096 * 4096, 300, 1, 6.27) == pytest.approx(802.6, rel=1e-3)


def _reference(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_non_zero_rank_exits_quietly():
    r = _reference({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"}, "--gpus", "2", "--steps", "2", "--warmup", "3")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_reference_arm_rank_zero_prints_one_line():
    r = _reference({"RANK": "0", "LOCAL_RANK": "0", "WORLD_SIZE": "2"}, "--gpus", "2", "--steps", "2", "--warmup", "3",
                   "--size", "256")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
