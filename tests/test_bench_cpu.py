"""CPU tests of the benchmark driver: the reference arm (the oracle timed on
the host) and the replica aggregation used under torchrun, with world size 2
over gloo."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args, env_extra=None, timeout=600):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_line():
    r = _run(["--impl", "reference", "--size", "48", "--ref-side", "24", "--steps", "1",
              "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GB/s" and d["value"] > 0
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--size", "48", "--ref-side", "24", "--steps", "1"],
             {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    t = bench.slowest_rank(1.0 + rank, world, "cpu")  # rank r took 1 + r seconds
    v = bench.job_throughput(2e9, t, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_replicas_take_the_slowest_rank_gloo():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 2.0  # the slower rank's time on every rank
        assert v == pytest.approx(2 * 2e9 / 2.0 / 1e9)


def test_traffic_figure_keyed_on_source_hashes(tmp_path, monkeypatch):
    """The DRAM traffic figure of the bench line is reported only while the
    kernel's file and every header listed beside it are unchanged."""
    import hashlib
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    csrc = tmp_path / "paper_2505_00227_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (csrc / "k.cu").write_bytes(b"kernel")
    (csrc / "h.cuh").write_bytes(b"header")
    sha = {n: hashlib.sha256((csrc / n).read_bytes()).hexdigest() for n in ("k.cu", "h.cuh")}
    (tmp_path / "profiles" / "traffic.json").write_text(
        json.dumps({"k": {"source_sha256": sha, "dram_bytes_per_launch": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("k") == 123.0
    assert bench.traffic_for("other") is None
    (csrc / "h.cuh").write_bytes(b"header, changed")
    assert bench.traffic_for("k") is None
