"""The N > 1 path of bench.py on CPU: two gloo ranks (one process each, as
torchrun launches them on a node).  The solver path shards by problem (every
rank solves its own replica, no exchange), so what crosses ranks is only the
barrier and the max-time / summed-units reduction; the reference arm runs on
rank 0 alone."""
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


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    got_ws, got_rank, _ = bench.dist_setup(None)
    assert dist.get_backend() == "gloo"
    bench.barrier(got_ws)
    # rank r took (10 + r) ms for (100 + 50 r) units
    ms_max, units, rate = bench.job_rate(got_ws, 10.0 + rank, 100.0 + 50 * rank, "cpu")
    out.put((got_rank, got_ws, ms_max, units, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_max_time_and_total_units():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, ms_max, units, rate in res:
        assert ws == 2 and ms_max == 11.0 and units == 250.0
        assert rate == pytest.approx(250.0 / 0.011)


def test_reference_arm_prints_one_line_from_rank_zero_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--grid-n", "33", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
