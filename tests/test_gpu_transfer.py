"""The direct curve-to-curve transfer (opts.transfer = 1) on the GPU against
the oracle's: crossing tables (indices exact, positions to 1e-12), single
split steps, fixed-step and converged solves, the paper's initial state,
parabolic steps, and the full-size sheared workload, all in FP64 within
max |u_gpu - u_oracle| / max |u_oracle| <= 1e-12."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


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


def _const(n, beta, mask="square", mu=0.1, sigma=1.0, nx=None, seed=0):
    nx = nx or n
    rng = np.random.default_rng(seed)
    X, Y = W.node_coords(nx, n)
    f = np.exp(-((X - 0.4) ** 2 + (Y - 0.55) ** 2) / 0.05) + 0.3 * rng.random((n, nx))
    m = W.make_mask(mask, nx, n) if nx == n else np.ones((n, nx), np.uint8)
    return W.Problem(nx, n, mu, sigma, np.full((n, nx), beta[0]), np.full((n, nx), beta[1]), f, m)


def _perforated(n, every):
    p = W.sheared(n=n)
    m = p.mask.copy()
    idx = np.arange(every // 2, n - 1, every)
    m[np.ix_(idx, idx)] = 0
    return W.Problem(n, n, p.mu, p.sigma, p.beta1, p.beta2, p.f, m, name=f"perforated{n}")


PROBLEMS = {
    "manufactured33": lambda: W.manufactured(n=33),
    "aligned17": lambda: W.manufactured(n=17, beta=(1.0, 0.0)),
    "rect_ragged": lambda: _const(19, (0.8, -0.35), nx=45),
    "L_mask": lambda: _const(41, (0.3, 1.0), mask="L"),
    "disc_mask": lambda: _const(47, (-0.9, 0.2), mask="disc", mu=1e-3),
    "sheared65": lambda: W.sheared(n=65),
    "data2d": lambda: W.data2d(33),
    "tiny3": lambda: _const(3, (1.0, 0.5)),
    # B curves of 4 097 unknowns (T = 512) crossed by 4 099 G curves of 3 unknowns
    "thin_m4097": lambda: _const(5, (1.0, 0.0), nx=4099, mu=1e-4),
    # oblique curves over 300^2 nodes: many crossings per cell
    "long_lines": lambda: _const(300, (1.0, 0.37), mu=1e-2),
    "perforated129": lambda: _perforated(129, 8),
}


@pytest.fixture(scope="module")
def pairs(torch_cuda):
    from paper_2411_11041_gb300 import Solver
    cache = {}

    def get(name):
        if name not in cache:
            p = PROBLEMS[name]()
            cache[name] = (p, O.Oracle(p, transfer=1), Solver(p, tol=0.0, max_iter=0, transfer=1))
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_transfer_tables_match_oracle(pairs, name):
    p, o, s = pairs(name)
    for fam in (0, 1):
        so, to, po = o.transfer_table(fam)
        sg, tg, pg = s.transfer_table(fam)
        assert np.array_equal(so, sg), f"family {fam}: crossed segments differ"
        assert np.abs(to - tg).max(initial=0) <= 1e-12 and np.abs(po - pg).max(initial=0) <= 1e-12


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_direct_split_step_matches_oracle(pairs, torch_cuda, name):
    from paper_2411_11041_gb300 import Solver
    p, o, s = pairs(name)
    torch = torch_cuda
    u = np.random.default_rng(11).normal(size=(p.ny, p.nx)) * o.interior()
    ug = torch.tensor(u, device="cuda:0")
    for theta, dt in ((0.5, o.default_dt()), (0.5, 0.3), (1.0, 0.01)):
        sv = s if theta == 0.5 else Solver(p, theta=theta, transfer=1)
        uh, un = sv.split_step(ug, dt)
        ouh, oun = o.split_step(theta, dt, u)
        assert relerr(uh, ouh) <= TOL64, (theta, dt)
        assert relerr(un, oun) <= TOL64, (theta, dt)


@pytest.mark.parametrize("name", ["manufactured33", "L_mask", "sheared65", "data2d", "tiny3",
                                  "long_lines", "perforated129"])
@pytest.mark.parametrize("theta", [0.5, 1.0])
def test_direct_fixed_step_count_solve_matches_oracle(torch_cuda, name, theta):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p, transfer=1)
    for init in (0, 2):
        s = Solver(p, tol=0.0, max_iter=23, init=init, theta=theta, transfer=1)
        u, uit, stats, st = s.solve_stationary(want_iter=True)
        ref, refit, it, rel, ost = o.solve_stationary(theta=theta, tol=0.0, max_iter=23, init=init)
        assert st == ADR_OK and ost == O.OK
        assert stats["iters"] == it == 23
        assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64
        assert abs(stats["rel_update"] - rel) <= 1e-9 * rel + 1e-13


@pytest.mark.parametrize("name", ["manufactured33", "aligned17", "disc_mask", "sheared65", "rect_ragged"])
def test_direct_converged_solve_matches_oracle(torch_cuda, name):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p, transfer=1)
    s = Solver(p, tol=1e-10, max_iter=20000, transfer=1)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    ref, refit, it, rel, ost = o.solve_stationary(tol=1e-10, max_iter=20000)
    assert st == ADR_OK and ost == O.OK
    assert stats["iters"] == it
    assert stats["rel_update"] <= 1e-10
    assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64


def test_direct_user_init_and_no_steps(torch_cuda):
    """A caller's initial state enters as its bilinear samples at the B nodes;
    with max_iter = 0 the output is those samples mapped back to the grid."""
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    p = W.sheared(n=65)
    o = O.Oracle(p, transfer=1)
    u0 = np.random.default_rng(3).normal(size=(65, 65))
    for steps in (0, 9):
        s = Solver(p, tol=0.0, max_iter=steps, init=1, transfer=1)
        u, uit, _, _ = s.solve_stationary(u_init=torch.tensor(u0, device="cuda:0"), want_iter=True)
        ref, refit, _, _, _ = o.solve_stationary(tol=0.0, max_iter=steps, init=1, u_init=u0)
        assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64, steps


@pytest.mark.parametrize("mode", [0, 1])
def test_direct_parabolic_matches_oracle(torch_cuda, mode):
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    p = W.parabolic(n=65)
    o = O.Oracle(p, transfer=1)
    s = Solver(p, tol=1e-9, max_iter=5000, transfer=1)
    u = torch.tensor(p.u0, device="cuda:0")
    stats, st = s.step_parabolic(u, 1e-3, 4, mode)
    ref, tot, ost = o.step_parabolic(p.u0, 1e-3, 4, mode, tol=1e-9, max_iter=5000)
    assert stats["iters"] == tot
    assert relerr(u, ref) <= TOL64


def test_direct_transfer_is_refused_where_it_does_not_apply(torch_cuda):
    from paper_2411_11041_gb300 import AdrError, Batch, Solver
    p = W.manufactured(n=17)
    with pytest.raises(AdrError, match="EINVAL"):
        Batch([Solver(p, transfer=1), Solver(p, transfer=1)])
    with pytest.raises(AdrError, match="EINVAL"):
        Solver(p).transfer_table(0)  # created without the transfer tables


def test_direct_kernel_timing_runs(torch_cuda):
    from paper_2411_11041_gb300 import Solver
    s = Solver(W.sheared(n=257), transfer=1)
    ms = s.time_kernels(reps=3)
    assert len(ms) == 6 and ms[0] == ms[3] == 0.0 and all(ms[k] > 0 for k in (1, 2, 4, 5))


@pytest.fixture(scope="module")
def sheared2048_direct():
    """The oracle's converged direct-transfer solve of the full-size sheared
    workload (2048^2, tol 1e-8; about a minute on one core)."""
    p = W.sheared(n=2048)
    o = O.Oracle(p, transfer=1)
    ref, refit, it, rel, st = o.solve_stationary(tol=1e-8, max_iter=200000)
    assert st == O.OK
    return p, o, ref, refit, it


def test_sheared_2048_direct_converged_solve_matches_oracle(torch_cuda, sheared2048_direct):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p, o, ref, refit, it = sheared2048_direct
    s = Solver(p, tol=1e-8, max_iter=200000, transfer=1)
    for fam in (0, 1):  # the tables at full size
        so, to, po = o.transfer_table(fam)
        sg, tg, pg = s.transfer_table(fam)
        assert np.array_equal(so, sg)
        assert np.abs(to - tg).max() <= 1e-12 and np.abs(po - pg).max() <= 1e-12
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    assert st == ADR_OK
    assert stats["iters"] == it
    assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64
    s.close()
