"""Host logic of bench.py without a GPU: the reduction over ranks (gloo,
world size 2, on CPU, as torchrun would launch the replicas) and the
reference arm (the oracle) on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took 10 (r + 1) ms: every rank must see the slowest, 20 ms
    ms = bench.max_over_ranks(10.0 * (rank + 1), dist, "cpu")
    q.put((rank, ms, bench.whole_job_value(1000, world, ms)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value_world_size_2():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, v in got:
        assert ms == 20.0
        assert v == pytest.approx(2 * 1000 / 0.020)


def _run_reference(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--N", "3000", "--steps", "1",
           "--warmup", "0", "--ref-sample", "64", "--gpus", env_extra.get("WORLD_SIZE", "1")]
    return subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)


def test_reference_arm_prints_one_line_on_rank_0_only():
    r = _run_reference({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "targets/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    r = _run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_traffic_is_taken_only_from_a_summary_of_the_current_source(tmp_path):
    """roofline.traffic comes from a committed ncu summary only when the summary
    names the sha256 of the kernel's current source files; otherwise null."""
    import bench
    sha = bench.source_sha(bench.NEAR_SOURCES)
    (tmp_path / "near.md").write_text("source_sha256: %s\ndram_bytes_per_full_launch: 1.25e+08\n" % sha)
    (tmp_path / "stale.md").write_text("source_sha256: %s\ndram_bytes_per_full_launch: 1.25e+08\n" % ("0" * 64))
    (tmp_path / "no_bytes.md").write_text("source_sha256: %s\n" % sha)
    d = str(tmp_path)
    assert bench.kernel_traffic(bench.NEAR_SOURCES, "near.md", d) == 1.25e8
    assert bench.kernel_traffic(bench.NEAR_SOURCES, "stale.md", d) is None
    assert bench.kernel_traffic(bench.NEAR_SOURCES, "no_bytes.md", d) is None
    assert bench.kernel_traffic(bench.NEAR_SOURCES, "missing.md", d) is None
    assert bench.kernel_traffic(bench.FAR_SOURCES, "near.md", d) is None
