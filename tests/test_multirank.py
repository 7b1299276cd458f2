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


def _probs_small():
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2411_11041_gb300 import workloads as W
    rng = np.random.Generator(np.random.PCG64(31))
    return [W.random_problem(rng, int(n), mask=m)
            for n, m in ((17, "square"), (33, "disc"), (25, "L"), (21, "square"), (29, "disc"),
                         (19, "L"), (31, "square"), (23, "square"), (27, "disc"))]


def _batch_rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2411_11041_gb300 import partition as PT
    got_ws, got_rank, _ = bench.dist_setup(None)
    probs = _probs_small()
    parts, loads = PT.lpt_split([PT.work_estimate(p) for p in probs], got_ws)
    # this rank's share, solved here (the oracle stands in for the GPU batch)
    mine = {i: O.Oracle(probs[i], interp_weights=1).solve_stationary(tol=1e-8, max_iter=100000)[0]
            for i in parts[got_rank]}
    gathered = [None] * got_ws
    dist.all_gather_object(gathered, (got_rank, parts, loads, mine))
    if got_rank == 0:
        out.put(gathered)
    dist.destroy_process_group()


def test_batch_split_over_two_gloo_ranks_is_disjoint_complete_balanced_and_exact():
    """The batch workload's N > 1 split: every problem on exactly one rank,
    the estimated loads within the LPT bound, and every rank's answers equal
    to the same problems solved in one process."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2411_11041_gb300 import partition as PT
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    probs = _probs_small()
    works = [PT.work_estimate(p) for p in probs]
    parts, loads = gathered[0][1], gathered[0][2]
    assert all(g[1] == parts and g[2] == loads for g in gathered)  # the same split on every rank
    seen = sorted(i for part in parts for i in part)
    assert seen == list(range(len(probs)))  # complete and disjoint
    lower = max(sum(works) / 2, max(works))  # no split can beat this
    assert max(loads) <= 4.0 / 3.0 * lower
    assert sum(loads) == pytest.approx(sum(works))
    for rank, _, _, mine in gathered:
        assert sorted(mine) == parts[rank]
        for i, u in mine.items():
            ref = O.Oracle(probs[i], interp_weights=1).solve_stationary(tol=1e-8, max_iter=100000)[0]
            assert np.array_equal(u, ref)


def test_lpt_split_edge_cases():
    from paper_2411_11041_gb300 import partition as PT
    parts, loads = PT.lpt_split([5.0, 3.0, 3.0, 2.0, 2.0, 2.0], 3)
    assert sorted(i for p in parts for i in p) == list(range(6))
    assert max(loads) == 7.0  # the best any split of this list can do (17 over 3 ranks)
    parts, loads = PT.lpt_split([1.0, 1.0], 4)  # more ranks than problems: some idle
    assert sum(len(p) for p in parts) == 2 and loads.count(0.0) == 2
    with pytest.raises(ValueError):
        PT.lpt_split([1.0], 0)
