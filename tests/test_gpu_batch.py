"""Batched solves: one persistent launch per sweep stage over many problems of
uneven size and shape must give what each problem gives alone (and the
oracle's answer)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_11041_gb300 import build
    build.build()
    return torch


def _problems():
    rng = np.random.Generator(np.random.PCG64(77))
    probs = [W.random_problem(rng, int(n), mask=m)
             for n, m in ((17, "square"), (40, "disc"), (65, "L"), (33, "square"), (97, "disc"),
                          (23, "L"), (130, "square"))]
    probs.append(W.sheared(n=49))
    return probs


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_equals_individual_solves(torch_cuda, prec):
    from paper_2411_11041_gb300 import ADR_OK, Batch, Solver
    probs = _problems()
    solvers = [Solver(p, tol=1e-9, max_iter=20000, prec=prec) for p in probs]
    singles = [s.solve_stationary() for s in solvers]
    batch = Batch(solvers)
    for rep in range(2):  # the batch graph is reused
        outs, stats, st = batch.solve()
        assert st == ADR_OK
        for (u1, _, s1, _), u2, s2 in zip(singles, outs, stats):
            assert s2["iters"] == s1["iters"]
            d = (u2 - u1).abs().max().item() / max(u1.abs().max().item(), 1e-300)
            assert d <= 1e-13
    # and the oracle on two of them
    for k in (1, 7):
        ref, _, it, _, _ = O.Oracle(probs[k]).solve_stationary(tol=1e-9, max_iter=20000)
        # the reduced-precision mode's FP32 corrections may move the step that
        # reaches tol by a step or two
        assert abs(stats[k]["iters"] - it) <= (0 if prec == 0 else 2)
        err = np.abs(outs[k].cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= (1e-12 if prec == 0 else 1e-5)
    batch.close()


def test_batch_reports_problems_that_hit_max_iter(torch_cuda):
    from paper_2411_11041_gb300 import ADR_ENOCONV, Batch, Solver
    probs = _problems()[:3]
    solvers = [Solver(p, tol=1e-12, max_iter=(5 if i == 1 else 20000)) for i, p in enumerate(probs)]
    outs, stats, st = Batch(solvers).solve()
    assert st == ADR_ENOCONV
    assert stats[1]["iters"] == 5 and stats[0]["iters"] > 5 and stats[2]["iters"] > 5
    ref = O.Oracle(probs[1]).solve_stationary(tol=1e-12, max_iter=5)[0]
    assert np.abs(outs[1].cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_autotune_keeps_the_solution(torch_cuda, tmp_path, monkeypatch):
    from paper_2411_11041_gb300 import Solver, _tune_cache
    monkeypatch.setenv("ADR_TUNE_CACHE", str(tmp_path / "tune.json"))
    p = W.sheared(n=129)
    s0 = Solver(p, tol=1e-9)
    u0, _, st0, _ = s0.solve_stationary()
    s1 = Solver(p, tol=1e-9, autotune=True)
    r, m, ms = s1.tuned
    assert r in (4, 8, 16) and m in (2, 4, 8) and ms > 0
    u1, _, st1, _ = s1.solve_stationary()
    assert st1["iters"] == st0["iters"]
    assert (u1 - u0).abs().max().item() <= 1e-12 * u0.abs().max().item()
    assert len(_tune_cache()) == 1
    s2 = Solver(p, tol=1e-9, autotune=True)  # from the cache
    assert s2.tuned is None and s2.opts.rows_per_thread == r
    u2, _, _, _ = s2.solve_stationary()
    assert (u2 - u1).abs().max().item() <= 1e-12 * u0.abs().max().item()


def test_batch_autotune_keeps_the_answers(torch_cuda):
    """adr_batch_autotune regroups every handle for each candidate and
    rebuilds the batch; the solve after it takes the same steps to the same
    answers (the partitioned eliminations of other chunk sizes round
    differently, nothing more)."""
    from paper_2411_11041_gb300 import ADR_OK, Batch, Solver
    rng = np.random.Generator(np.random.PCG64(51))
    probs = [W.random_problem(rng, int(n)) for n in (70, 130, 257, 96)]
    b = Batch([Solver(p, tol=1e-10, max_iter=20000, interp_weights=1) for p in probs])
    before, sb, cb = b.solve()
    rows, ms = b.autotune(reps=3)
    assert rows in (4, 8, 16) and ms > 0
    after, sa, ca = b.solve()
    assert cb == ca == ADR_OK
    for x, y, s0, s1 in zip(before, after, sb, sa):
        assert abs(s0["iters"] - s1["iters"]) <= 1
        assert (x - y).abs().max().item() <= 1e-9 * y.abs().max().item()
