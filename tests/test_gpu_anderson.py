"""Anderson extrapolation of the stationary iteration (opts.anderson = m) on
the GPU against the oracle's: fixed step counts element by element (the
extrapolation weights come from sums taken in another order, so 1e-11 rather
than 1e-12), converged solves within 1e-12, the transfer through the grid and
the direct one, the parabolic slices, and the full-size sheared workload."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOL_STEPS = 1e-11


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_11041_gb300 import build
    build.build()
    return torch


def relerr(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    den = np.abs(b).max()
    return np.abs(a - b).max() / (den if den > 0 else 1.0)


PROBLEMS = {
    "manufactured33": lambda: W.manufactured(n=33),
    "L_mask": lambda: W.manufactured(n=41, beta=(0.3, 1.0), mask="L"),
    "sheared65": lambda: W.sheared(n=65),
    "data2d": lambda: W.data2d(33),
    "disc_rand": lambda: W.random_problem(np.random.Generator(np.random.PCG64(7)), 97, mask="disc"),
}


@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("transfer", [0, 1])
@pytest.mark.parametrize("m", [1, 3, 8])
def test_fixed_step_count_matches_oracle(torch_cuda, name, transfer, m):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = PROBLEMS[name]()
    iw = 1 if name == "disc_rand" else 0
    o = O.Oracle(p, interp_weights=iw, transfer=transfer, anderson=m)
    s = Solver(p, tol=0.0, max_iter=17, interp_weights=iw, transfer=transfer, anderson=m)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    ref, refit, it, rel, ost = o.solve_stationary(tol=0.0, max_iter=17)
    assert st == ADR_OK and ost == O.OK and stats["iters"] == it == 17
    assert relerr(u, ref) <= TOL_STEPS and relerr(uit, refit) <= TOL_STEPS
    assert abs(stats["rel_update"] - rel) <= 1e-8 * rel + 1e-13


@pytest.mark.parametrize("name", ["manufactured33", "sheared65", "L_mask"])
@pytest.mark.parametrize("transfer", [0, 1])
def test_converged_solve_matches_oracle(torch_cuda, name, transfer):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p, transfer=transfer, anderson=3)
    s = Solver(p, tol=1e-11, max_iter=20000, transfer=transfer, anderson=3)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    ref, refit, it, rel, ost = o.solve_stationary(tol=1e-11, max_iter=20000)
    plain, _, itp, _, _ = O.Oracle(p, transfer=transfer).solve_stationary(tol=1e-11, max_iter=20000)
    assert st == ADR_OK and ost == O.OK
    assert abs(stats["iters"] - it) <= 1 and stats["iters"] < itp
    assert relerr(u, ref) <= (TOL64 if stats["iters"] == it else 1e-10)
    assert relerr(u, plain) <= 1e-9  # the plain iteration's fixed point


def test_parabolic_slices_are_extrapolated_and_time_steps_are_not(torch_cuda):
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    p = W.parabolic(n=65)
    for mode in (0, 1):
        o = O.Oracle(p, anderson=3)
        s = Solver(p, tol=1e-9, max_iter=5000, anderson=3)
        u = torch.tensor(p.u0, device="cuda:0")
        stats, st = s.step_parabolic(u, 1e-3, 3, mode)
        ref, tot, ost = o.step_parabolic(p.u0, 1e-3, 3, mode, tol=1e-9, max_iter=5000)
        assert abs(stats["iters"] - tot) <= 3 * (mode == 1)
        assert relerr(u, ref) <= (TOL64 if mode == 0 else 1e-9)


def test_refusals(torch_cuda):
    from paper_2411_11041_gb300 import ADR_FP32_REFINE, AdrError, Solver
    p = W.manufactured(n=17)
    with pytest.raises(AdrError, match="EINVAL"):
        Solver(p, anderson=9)
    with pytest.raises(AdrError, match="EINVAL"):
        Solver(p, anderson=2, prec=ADR_FP32_REFINE)


def test_batch_with_mixed_depths_equals_the_problems_solved_one_by_one(torch_cuda):
    """A batch whose problems extrapolate over different depths (0, 1, 3, 5):
    every problem takes the steps and reaches the answer it reaches alone,
    and the oracle's."""
    from paper_2411_11041_gb300 import ADR_OK, Batch, Solver
    rng = np.random.Generator(np.random.PCG64(23))
    probs = [W.random_problem(rng, int(n), mask=m)
             for n, m in ((61, "square"), (97, "disc"), (45, "L"), (130, "square"), (77, "square"))]
    depths = [3, 0, 1, 5, 3]
    solo = []
    for p, m in zip(probs, depths):
        s = Solver(p, tol=1e-10, max_iter=20000, interp_weights=1, anderson=m)
        u, _, st, code = s.solve_stationary()
        assert code == ADR_OK
        solo.append((u, st["iters"]))
    batch = Batch([Solver(p, tol=1e-10, max_iter=20000, interp_weights=1, anderson=m)
                   for p, m in zip(probs, depths)])
    outs, stats, code = batch.solve()
    assert code == ADR_OK
    for i, (p, m) in enumerate(zip(probs, depths)):
        u, it = solo[i]
        assert stats[i]["iters"] == it, (i, m)
        assert (outs[i] - u).abs().max().item() <= 1e-13 * u.abs().max().item()
        if m:
            ref, _, oit, _, _ = O.Oracle(p, interp_weights=1, anderson=m).solve_stationary(
                tol=1e-10, max_iter=20000)
            assert abs(oit - it) <= 1
            if oit == it:
                assert relerr(outs[i], ref) <= TOL64


@pytest.fixture(scope="module")
def sheared2048_anderson():
    """The oracle's converged accelerated solve of the full-size sheared
    workload (2048^2, m = 3, tol 1e-8)."""
    p = W.sheared(n=2048)
    ref, refit, it, rel, st = O.Oracle(p, anderson=3).solve_stationary(tol=1e-8, max_iter=200000)
    assert st == O.OK
    return p, ref, it


def test_sheared_2048_accelerated_solve_matches_oracle(torch_cuda, sheared2048_anderson):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p, ref, it = sheared2048_anderson
    s = Solver(p, tol=1e-8, max_iter=200000, anderson=3)
    u, _, stats, st = s.solve_stationary()
    assert st == ADR_OK
    assert abs(stats["iters"] - it) <= 1
    assert relerr(u, ref) <= (TOL64 if stats["iters"] == it else 1e-7)
    s.close()


def test_direct_transfer_with_paper_start_and_extrapolation(torch_cuda):
    """The three options together: the direct transfer, the paper's initial
    state (the B-curve solutions as they stand) and the extrapolation."""
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = W.sheared(n=65)
    o = O.Oracle(p, transfer=1, anderson=3)
    for max_iter, tol in ((11, 0.0), (20000, 1e-11)):
        s = Solver(p, tol=tol, max_iter=max_iter, init=2, transfer=1, anderson=3)
        u, uit, stats, st = s.solve_stationary(want_iter=True)
        ref, refit, it, _, ost = o.solve_stationary(tol=tol, max_iter=max_iter, init=2)
        assert st == ADR_OK and ost == O.OK and abs(stats["iters"] - it) <= (0 if tol == 0.0 else 1)
        assert relerr(u, ref) <= (TOL_STEPS if stats["iters"] == it else 1e-10)


def test_extrapolation_from_a_caller_state_and_in_a_batch_with_paper_starts(torch_cuda):
    """ADR_INIT_USER and ADR_INIT_PAPER_U0 with the extrapolation, one by one
    and as one batch: the same steps and answers."""
    from paper_2411_11041_gb300 import ADR_OK, Batch, Solver
    torch = torch_cuda
    rng = np.random.Generator(np.random.PCG64(41))
    probs = [W.random_problem(rng, int(n), mask="square") for n in (49, 73, 88)]
    u0 = [torch.tensor(np.random.default_rng(i).normal(size=(p.ny, p.nx)), device="cuda:0")
          for i, p in enumerate(probs)]
    for init in (1, 2):
        solo = []
        for p, ui in zip(probs, u0):
            s = Solver(p, tol=1e-10, max_iter=20000, interp_weights=1, anderson=4, init=init)
            u, _, st, code = s.solve_stationary(u_init=ui if init == 1 else None)
            assert code == ADR_OK
            ref, _, it, _, _ = O.Oracle(p, interp_weights=1, anderson=4).solve_stationary(
                tol=1e-10, max_iter=20000, init=init, u_init=ui.cpu().numpy() if init == 1 else None)
            assert abs(st["iters"] - it) <= 1
            assert relerr(u, ref) <= (TOL64 if st["iters"] == it else 1e-9)
            solo.append((u, st["iters"]))
        b = Batch([Solver(p, tol=1e-10, max_iter=20000, interp_weights=1, anderson=4, init=init)
                   for p in probs])
        outs, stats, code = b.solve(u0 if init == 1 else None)
        assert code == ADR_OK
        for (u, it), o_, s_ in zip(solo, outs, stats):
            assert s_["iters"] == it
            assert (o_ - u).abs().max().item() <= 1e-13 * u.abs().max().item()


def test_extrapolation_caps_and_single_step(torch_cuda):
    """max_iter = 1 (no extrapolation happens), a cap reached before tol
    (ADR_ENOCONV, the state of the last step reported), and max_iter = 0."""
    from paper_2411_11041_gb300 import ADR_ENOCONV, ADR_OK, Solver
    p = W.sheared(n=65)
    o = O.Oracle(p, anderson=3)
    plain = O.Oracle(p)
    s1 = Solver(p, tol=0.0, max_iter=1, anderson=3)
    u1, _, st1, c1 = s1.solve_stationary()
    r1 = plain.solve_stationary(tol=0.0, max_iter=1)[0]
    assert c1 == ADR_OK and st1["iters"] == 1 and relerr(u1, r1) <= TOL64
    s2 = Solver(p, tol=1e-14, max_iter=9, anderson=3)
    u2, _, st2, c2 = s2.solve_stationary()
    r2, _, it2, _, oc2 = o.solve_stationary(tol=1e-14, max_iter=9)
    assert c2 == ADR_ENOCONV and oc2 == O.ENOCONV and st2["iters"] == it2 == 9
    assert relerr(u2, r2) <= TOL_STEPS
    s3 = Solver(p, tol=1e-10, max_iter=0, anderson=3)
    u3, _, st3, c3 = s3.solve_stationary()
    assert st3["iters"] == 0 and float(u3.abs().max()) == 0.0
