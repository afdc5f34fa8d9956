"""The N > 1 path of the benchmark on the CPU (gloo, world size 2): the
path does not shard (every rank runs its own frames, "replicas only"), so
the only cross-rank step is the timing: the job's time is its slowest
rank's, and the throughput counts the pixels of all ranks.  Also the
reference arm under a two-rank launch: rank 0 alone prints one line."""
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


def _worker(rank, world, port, ms, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.slowest_rank_ms(ms[rank], world)
        out.put((rank, got, bench.rank_frame(5, rank)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_disjoint_frames_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms = [1.5, 4.25]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [4.25, 4.25]       # both ranks see the slowest rank's time
    assert res[0][2] != res[1][2]                      # each rank seeds its own frames


def test_whole_job_rate():
    sys.path.insert(0, ROOT)
    import bench
    # 2 ranks x 10 frames x 2,073,600 pixels in 25 ms
    assert bench.whole_job_rate(10 * 2073600, 2, 25.0) == pytest.approx(1658.88)
    assert bench.slowest_rank_ms(3.0, 1) == 3.0


def test_reference_arm_two_ranks_prints_once():
    """`bench.py --impl reference` under a two-rank launch: rank 0 times the
    oracle and prints one JSON line, rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
