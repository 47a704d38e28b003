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


def test_gpus_flag_without_launcher_starts_that_many_ranks():
    """`bench.py --gpus 2` run directly starts two local ranks itself
    (torch.distributed.run on 127.0.0.1); the reference arm's rank 0 prints
    one line that reports both, the other rank prints nothing."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "MASTER_ADDR",
                                                           "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3", "--size", "256"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    assert json.loads(lines[0])["n_gpus"] == 2


def test_gpus_flag_must_match_the_launcher():
    r = _reference({"RANK": "0", "LOCAL_RANK": "0", "WORLD_SIZE": "1"}, "--gpus", "2", "--steps", "1",
                   "--warmup", "3")
    assert r.returncode != 0 and "WORLD_SIZE=1" in (r.stderr + r.stdout)


def test_summary_is_compact_and_complete():
    """The line's last key repeats every section's headline figure in a few
    hundred bytes (the part of the line a log tail keeps)."""
    sys.path.insert(0, ROOT)
    import bench
    roof = {"frac": 0.7, "bound": "alu", "fp64_pipe_frac": 0.9}
    line = {"value": 3000.0, "roofline": roof, "e2e": {"value": 2000.0}, "config": {"nx": 4096},
            "forms": {"f16n": {"value": 46000.0, "roofline": {"frac": 0.52}},
                      "f16s": {"value": 77000.0, "roofline": {"frac": 0.68}}},
            "accuracy": {"steps": 1000, **{k: {"rel_err_u": 1e-3, "err_u_over_uc": 2e-5, "max_abs_err_T": 1e-4,
                                               "rel_err_nu": 1e-5} for k in ("f16n", "f16s")}},
            "accuracy_2048": {"steps": 30000, **{k: {"rel_err_u": 1e-3, "err_u_over_uc": 2e-5,
                                                     "max_abs_err_T": 1e-4, "rel_err_nu": 1e-5}
                                                 for k in ("f16n", "f16s")}},
            "batch": {"value": 30000.0, "cases": 512, "mode": "persistent", "roofline": {"frac": 0.34},
                      "mlups_by_mode": {"graph": 29000.0, "persistent": 30000.0},
                      "validation": {"max_rel_nu_error": 1e-5}},
            "mrt_cost": {"ratio_clb_over_mrt": 1.1}, "cavity64": {"nu_hot": 1.49},
            "steady_state": {"forms": {"f64": {}, "f16n": {"rel_nu_converged_vs_f64": 1e-6, "speedup_vs_f64": 2.0}}},
            "cpu_baseline": {"cores": 16, "value": 38.0}, "cpu_baseline_1core": {"value": 3.0},
            "warm_start": {"steps_ratio_total": 0.8, "wall_speedup_total": 1.2, "max_rel_nu": 1e-5},
            "surrogate_training": {"roofline": {"achieved": 34.0}}}
    s = bench._summary(line)
    for k in ("f64_4096", "f16n_8192", "f16s_8192", "acc_8192", "acc_2048", "batch_512", "clb_over_mrt",
              "cavity64_nu", "steady_128", "oracle_mlups", "warm_start", "surrogate_tflops"):
        assert k in s, k
    assert len(json.dumps(s)) < 1400
    # keys name the measured sizes
    line["config"]["nx"] = 2048
    line["batch"]["cases"] = 128
    s = bench._summary(line)
    assert "f64_2048" in s and "batch_128" in s and "f64_4096" not in s
