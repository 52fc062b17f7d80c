"""Host-side pieces of bench.py: the replica aggregation over ranks (gloo, two processes on the
CPU) and the reference arm's JSON line (the CPU oracle on a small sample)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [100.0, 250.0]
    t = bench.reduce_max(times[rank], dist, world, "cpu")
    v = bench.replica_throughput(world, 2.0 * 8192 ** 3, 6, t)
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks_gloo():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == 250.0  # the slowest replica sets the time
        assert abs(v - 2 * 2.0 * 8192 ** 3 * 6 / 0.25 / 1e12) < 1e-9


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1", "--cpu-sample", "256"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "TFLOP/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample", "64"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_defaults_cover_the_six_graphs(monkeypatch):
    """The default run: at least 3 warm-up steps, and the end-to-end line over six steps, one per
    graph of the n = 8192 workload (step i runs graph i mod 6), the mix of the timed steps."""
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    assert args.warmup >= 3 and args.steps >= 6
    assert args.e2e_steps == len(bench.workloads(64)) == 6
    for w in ("single", "batched", "batched-stack", "serving", "weighted", "update", "product", "mma-probe"):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", w])
        assert bench.parse().workload == w
