"""CPU test of the multi-GPU replica logic of bench.py with two gloo ranks.

bench.py --gpus N runs one independent replica of the workload per GPU (the
solve does not shard across GPUs on this pool); its only cross-rank step is the
max over ranks of the timed region, and the whole-job value counts the solves
of every rank.  Both are exercised here on the CPU with world_size 2.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 100.0 + 50.0 * rank  # the slower rank decides the step time
    m = bench.reduce_max(ms, dist, device="cpu")
    out[rank] = (m, bench.replica_value(2, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 150.0
    # 2 solves per step on each of 2 ranks in 150 ms
    assert abs(out[0][1] - 4 / 0.150) < 1e-9


def test_single_rank_helpers():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert abs(bench.replica_value(2, 1, 250.0) - 8.0) < 1e-12


def test_reference_arm_json_contract(tmp_path):
    """bench.py --impl reference: one JSON line with the arm's metric, a measured value
    over the K timed steps (not extrapolated), the reference-arm keys, and nothing
    printed by ranks other than 0."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="0")
    p = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       cwd=root, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["higher_is_better"]
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert abs(d["ms_per_step"] - 1e3 / d["value"]) <= 1e-6 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    # other ranks exit 0 without work or output
    env1 = dict(os.environ, RANK="1")
    p1 = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference"],
                        capture_output=True, text=True, cwd=root, env=env1, timeout=120)
    assert p1.returncode == 0 and not [l for l in p1.stdout.splitlines() if l.startswith("{")]


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """A DRAM traffic figure taken once under ncu is reported only while the kernel it
    was measured on is unchanged: the bench hashes the kernel's source text and drops
    the figure (null) when the hash differs or the class has no record."""
    import bench
    k = "lu_gemm"
    rec = bench.TRAFFIC[k]
    assert bench.recorded_traffic(k) == rec["bytes_per_launch"]
    assert bench.recorded_traffic("no_such_class") is None
    src = open(os.path.join(bench.ROOT, rec["source"])).read()
    marker_line = next(ln for ln in src.split("\n") if rec["kernel"] in ln and "__global__" in ln)
    changed = src.replace(marker_line, marker_line + "  // edited", 1)
    (tmp_path / "src.cu").write_text(changed)
    monkeypatch.setitem(bench.TRAFFIC, k, dict(rec, source=str(tmp_path / "src.cu")))
    assert bench.recorded_traffic(k) is None
