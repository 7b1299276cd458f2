"""CUDA path vs the FP64 CPU oracle, element by element, on seeded inputs.

Tolerance (FP64 mode): max |u_gpu - u_oracle| / max |u_oracle| <= 1e-12 over
the grid.  Geometry (curve counts, node counts, chosen crossings) must agree
exactly; coordinates to 1e-12 in index units.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12
TOL_REF = 1e-5


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
    """Sheared flow on the square with a mask-0 node every `every` nodes: one
    2 x 2-cell hole around each, so one boundary loop per hole.  The inflow
    walk keeps its successor table in shared memory up to about 46 000
    boundary edges and in global memory beyond."""
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
    "steep": lambda: _const(64, (0.02, 1.0), mu=1e-4),
    "long_lines": lambda: _const(300, (1.0, 0.37), mu=1e-2),
    "sheared65": lambda: W.sheared(n=65),
    "data2d": lambda: W.data2d(33),
    "tiny3": lambda: _const(3, (1.0, 0.5)),
    # lines of 4 100 nodes (4 098 unknowns): the 1024-thread curve solve.
    # mu is small so that dt mu / h^2 stays moderate at the test's largest dt
    # (with mu = 0.1 and dt = 0.3 it is 5e5, and the partitioned and the serial
    # eliminations then differ by 2e-12 from rounding alone)
    "thin_long": lambda: _const(5, (1.0, 0.0), nx=4100, mu=1e-4),
    # lines of m = nx - 2 unknowns at the chunking boundaries (8 rows per
    # thread): 32 (T = 32, 1 row each), 33, 2 048 (T = 256, 8 rows each, all
    # full) and 2 049 (the first length that takes T = 512)
    "thin_m32": lambda: _const(5, (1.0, 0.0), nx=34, mu=1e-3),
    "thin_m33": lambda: _const(5, (1.0, 0.0), nx=35, mu=1e-3),
    "thin_m2048": lambda: _const(5, (1.0, 0.0), nx=2050, mu=1e-4),
    "thin_m2049": lambda: _const(5, (1.0, 0.0), nx=2051, mu=1e-4),
    # the same for 16 rows per thread (the default): 4 096 (T = 256, 16 rows
    # each, all full), 4 097 (the first length that takes T = 512) and 8 193
    # (the first length that takes 1 024-thread blocks)
    "thin_m4096": lambda: _const(5, (1.0, 0.0), nx=4098, mu=1e-4),
    "thin_m4097": lambda: _const(5, (1.0, 0.0), nx=4099, mu=1e-4),
    "thin_m8193": lambda: _const(5, (1.0, 0.0), nx=8195, mu=1e-5),
    "perforated129": lambda: _perforated(129, 8),  # 2 560 boundary edges, 257 loops
    "perforated401": lambda: _perforated(401, 4),  # 81 600 boundary edges
}


@pytest.fixture(scope="module")
def pairs(torch_cuda):
    from paper_2411_11041_gb300 import Solver
    cache = {}

    def get(name):
        if name not in cache:
            p = PROBLEMS[name]()
            cache[name] = (p, O.Oracle(p), Solver(p, tol=0.0, max_iter=0))
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_geometry_matches_oracle(pairs, name):
    p, o, s = pairs(name)
    for fam in (0, 1):
        Lo, Lg = o.lines(fam), s.lines(fam)
        assert np.array_equal(Lo["off"], Lg["off"]), f"family {fam} curve layout differs"
        assert np.abs(Lo["xi"] - Lg["xi"]).max(initial=0) <= 1e-12
        assert np.abs(Lo["eta"] - Lg["eta"]).max(initial=0) <= 1e-12
        np.testing.assert_allclose(Lg["h"], Lo["h"], rtol=1e-13)
        so, to, po = o.crossings(fam)
        sg, tg, pg = s.crossings(fam)
        assert np.array_equal(so, sg), f"family {fam} crossings differ"
        assert np.abs(to - tg).max() <= 1e-12 and np.abs(po - pg).max() <= 1e-12


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_split_step_matches_oracle(pairs, torch_cuda, name):
    from paper_2411_11041_gb300 import Solver
    p, o, s = pairs(name)
    torch = torch_cuda
    u = np.random.default_rng(11).normal(size=(p.ny, p.nx)) * o.interior()
    ug = torch.tensor(u, device="cuda:0")
    for theta, dt in ((0.5, o.default_dt()), (0.5, 0.3), (1.0, 0.01)):
        sv = s if theta == 0.5 else Solver(p, theta=theta)
        uh, un = sv.split_step(ug, dt)
        ouh, oun = o.split_step(theta, dt, u)
        assert relerr(uh, ouh) <= TOL64, (theta, dt)
        assert relerr(un, oun) <= TOL64, (theta, dt)


@pytest.mark.parametrize("rows", [2, 4, 8])
def test_other_rows_per_thread_match_oracle(torch_cuda, rows):
    """Fewer rows per thread: more threads per curve, up to T = 1024 (with 2
    rows per thread every curve of more than 1 024 unknowns is capped at
    1 024 threads and takes more rows each)."""
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    for name in ("thin_long", "sheared65", "disc_mask"):
        p = PROBLEMS[name]()
        o = O.Oracle(p)
        s = Solver(p, rows_per_thread=rows)
        u = np.random.default_rng(5).normal(size=(p.ny, p.nx)) * o.interior()
        uh, un = s.split_step(torch.tensor(u, device="cuda:0"), o.default_dt())
        ouh, oun = o.split_step(0.5, o.default_dt(), u)
        assert relerr(uh, ouh) <= TOL64, (name, rows)
        assert relerr(un, oun) <= TOL64, (name, rows)
        s.close()


@pytest.mark.parametrize("name", ["manufactured33", "L_mask", "sheared65", "data2d", "tiny3",
                                  "long_lines"])
def test_fixed_step_count_solve_matches_oracle(torch_cuda, name):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p)
    for init in (0, 2):
        s = Solver(p, tol=0.0, max_iter=37, init=init)
        u, uit, stats, st = s.solve_stationary(want_iter=True)
        ref, refit, it, rel, ost = o.solve_stationary(tol=0.0, max_iter=37, init=init)
        assert st == ADR_OK and ost == O.OK  # tol <= 0: exactly max_iter steps
        assert stats["iters"] == it == 37
        assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64
        assert abs(stats["rel_update"] - rel) <= 1e-9 * rel + 1e-13


@pytest.mark.parametrize("name", ["manufactured33", "aligned17", "disc_mask", "sheared65"])
def test_converged_solve_matches_oracle(torch_cuda, name):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p)
    s = Solver(p, tol=1e-10, max_iter=20000)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    ref, refit, it, rel, ost = o.solve_stationary(tol=1e-10, max_iter=20000)
    assert st == ADR_OK and ost == O.OK
    assert stats["iters"] == it
    assert stats["rel_update"] <= 1e-10
    assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64


@pytest.mark.parametrize("name", ["manufactured33", "L_mask", "sheared65", "data2d", "thin_m4097",
                                  "thin_m8193"])
def test_min_pivot_matches_oracle_thomas(torch_cuda, name):
    """stats.min_pivot: the smallest |pivot| Thomas elimination meets on the
    curve systems of both families (the library factors them in parallel; the
    oracle runs Thomas curve by curve)."""
    from paper_2411_11041_gb300 import Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p)
    dt = o.default_dt()
    s = Solver(p, tol=0.0, max_iter=1)
    _, _, stats, _ = s.solve_stationary()
    u = np.zeros((p.ny, p.nx))
    ref = min(o.sweep_lines(0, 0.5, dt, u)[1], o.sweep_lines(1, 0.5, dt, u)[1])
    assert abs(stats["min_pivot"] - ref) <= 1e-10 * ref, (stats["min_pivot"], ref)
    assert stats["max_correction"] == 0.0  # FP64 mode


def test_user_init_and_paper_u0(torch_cuda):
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    p = W.sheared(n=65)
    o = O.Oracle(p)
    s = Solver(p)
    assert relerr(s.paper_u0(), o.paper_u0()) <= TOL64
    u0 = np.random.default_rng(3).normal(size=(65, 65))
    s2 = Solver(p, tol=0.0, max_iter=9, init=1)
    u, _, _, _ = s2.solve_stationary(u_init=torch.tensor(u0, device="cuda:0"))
    ref = o.solve_stationary(tol=0.0, max_iter=9, init=1, u_init=u0)[0]
    assert relerr(u, ref) <= TOL64


@pytest.mark.parametrize("mode", [0, 1])
def test_parabolic_matches_oracle(torch_cuda, mode):
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    p = W.parabolic(n=65)
    o = O.Oracle(p)
    s = Solver(p, tol=1e-9, max_iter=5000)
    u = torch.tensor(p.u0, device="cuda:0")
    stats, st = s.step_parabolic(u, 1e-3, 4, mode)
    ref, tot, ost = o.step_parabolic(p.u0, 1e-3, 4, mode, tol=1e-9, max_iter=5000)
    assert stats["iters"] == tot
    assert relerr(u, ref) <= TOL64


def test_sheared_2048_two_steps_match_oracle(torch_cuda):
    """Full-size sheared workload (2048^2 nodes, traced curves), two split
    steps from zero, every grid value compared."""
    from paper_2411_11041_gb300 import Solver
    p = W.sheared(n=2048)
    o = O.Oracle(p)
    s = Solver(p, tol=0.0, max_iter=2)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    ref, refit, it, rel, ost = o.solve_stationary(tol=0.0, max_iter=2)
    assert stats["iters"] == 2
    assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64


@pytest.fixture(scope="module")
def sheared2048_converged():
    """The oracle's converged solve of the full-size sheared workload (2048^2,
    traced curves, tol 1e-8; about a minute on one core)."""
    p = W.sheared(n=2048)
    ref, refit, it, rel, st = O.Oracle(p).solve_stationary(tol=1e-8, max_iter=200000)
    assert st == O.OK
    return p, ref, refit, it


@pytest.mark.parametrize("prec", [0, 1])
def test_sheared_2048_converged_solve_matches_oracle(torch_cuda, sheared2048_converged, prec):
    """The benchmarked solve at full size, to 1e-8, element by element against
    the oracle's converged solve: FP64 within 1e-12, FP32 + refinement within 1e-5."""
    from paper_2411_11041_gb300 import ADR_OK, Solver
    p, ref, refit, it = sheared2048_converged
    s = Solver(p, tol=1e-8, max_iter=200000, prec=prec)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    assert st == ADR_OK
    if prec == 0:
        assert stats["iters"] == it
        assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64
    else:
        assert abs(stats["iters"] - it) <= 2
        assert relerr(u, ref) <= TOL_REF
    s.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_parabolic_1024_first_steps_match_oracle(torch_cuda, mode):
    """The parabolic workload at full size (1024^2, dt = 1e-3): its first three
    time steps (mode 1: each slice solved to 1e-8) against the oracle's."""
    from paper_2411_11041_gb300 import Solver
    torch = torch_cuda
    p = W.parabolic(n=1024)
    o = O.Oracle(p)
    s = Solver(p, tol=1e-8, max_iter=200000)
    u = torch.tensor(p.u0, device="cuda:0")
    stats, st = s.step_parabolic(u, 1e-3, 3, mode)
    ref, tot, ost = o.step_parabolic(p.u0, 1e-3, 3, mode, tol=1e-8, max_iter=200000)
    assert ost == O.OK
    assert stats["iters"] == tot
    assert relerr(u, ref) <= TOL64


# ------------------------------------------------------------ FP32 + FP64 refinement


@pytest.mark.parametrize("name", ["manufactured33", "L_mask", "disc_mask", "long_lines", "sheared65",
                                  "data2d", "tiny3", "steep"])
def test_refine_split_step_matches_oracle(torch_cuda, name):
    from paper_2411_11041_gb300 import ADR_FP32_REFINE, Solver
    torch = torch_cuda
    p = PROBLEMS[name]()
    o = O.Oracle(p)
    s = Solver(p, prec=ADR_FP32_REFINE)
    u = np.random.default_rng(11).normal(size=(p.ny, p.nx)) * o.interior()
    for dt in (o.default_dt(), 0.3):
        uh, un = s.split_step(torch.tensor(u, device="cuda:0"), dt)
        ouh, oun = o.split_step(0.5, dt, u)
        assert relerr(uh, ouh) <= TOL_REF and relerr(un, oun) <= TOL_REF


@pytest.mark.parametrize("name", ["manufactured33", "sheared65", "disc_mask"])
def test_refine_converged_solve_matches_oracle(torch_cuda, name):
    from paper_2411_11041_gb300 import ADR_FP32_REFINE, ADR_OK, Solver
    p = PROBLEMS[name]()
    o = O.Oracle(p)
    s = Solver(p, tol=1e-8, max_iter=20000, prec=ADR_FP32_REFINE)
    u, _, stats, st = s.solve_stationary()
    ref, _, it, _, ost = o.solve_stationary(tol=1e-8, max_iter=20000)
    assert st == ADR_OK and ost == O.OK
    # FP32 corrections until the relative update reaches 100 tol, FP64 after
    assert abs(stats["iters"] - it) <= 2
    assert 0.5 * it <= stats["fp32_steps"] < stats["iters"]
    assert relerr(u, ref) <= TOL_REF


@pytest.mark.parametrize("name", ["sheared65", "L_mask"])
def test_refine_max_correction_is_the_step_increment(torch_cuda, name):
    """stats.max_correction of one refinement step from a given state: the
    largest |dt d| over both substeps, d the oracle's line increments."""
    from paper_2411_11041_gb300 import ADR_FP32_REFINE, Solver
    torch = torch_cuda
    p = PROBLEMS[name]()
    o = O.Oracle(p)
    dt = o.default_dt()
    u0 = np.random.default_rng(8).normal(size=(p.ny, p.nx)) * o.interior()
    s = Solver(p, tol=0.0, max_iter=1, init=1, prec=ADR_FP32_REFINE)
    _, _, stats, _ = s.solve_stationary(u_init=torch.tensor(u0, device="cuda:0"))
    uh, _ = o.split_step(0.5, dt, u0)
    ref = dt * max(np.abs(o.sweep_lines(0, 0.5, dt, u0)[0]).max(),
                   np.abs(o.sweep_lines(1, 0.5, dt, uh)[0]).max())
    assert abs(stats["max_correction"] - ref) <= 1e-5 * ref, (stats["max_correction"], ref)


def test_refine_paper_u0_and_parabolic(torch_cuda):
    from paper_2411_11041_gb300 import ADR_FP32_REFINE, Solver
    torch = torch_cuda
    p = W.parabolic(n=65)
    o = O.Oracle(p)
    s = Solver(p, tol=1e-9, max_iter=5000, prec=ADR_FP32_REFINE)
    assert relerr(s.paper_u0(), o.paper_u0()) <= TOL_REF
    u = torch.tensor(p.u0, device="cuda:0")
    s.step_parabolic(u, 1e-3, 3, 1)
    ref, _, _ = o.step_parabolic(p.u0, 1e-3, 3, 1, tol=1e-9, max_iter=5000)
    assert relerr(u, ref) <= TOL_REF


# ------------------------------------------------ inverse-gap weights, divergence

@pytest.mark.parametrize("name", ["manufactured33", "L_mask", "disc_mask", "sheared65", "steep"])
def test_weighted_map_mode_matches_oracle(torch_cuda, name):
    from paper_2411_11041_gb300 import ADR_OK, Solver
    torch = torch_cuda
    p = PROBLEMS[name]()
    o = O.Oracle(p, interp_weights=1)
    s = Solver(p, interp_weights=1, tol=1e-9, max_iter=20000)
    u = np.random.default_rng(2).normal(size=(p.ny, p.nx)) * o.interior()
    uh, un = s.split_step(torch.tensor(u, device="cuda:0"), 0.05)
    ouh, oun = o.split_step(0.5, 0.05, u)
    assert relerr(uh, ouh) <= TOL64 and relerr(un, oun) <= TOL64
    ug, _, stats, st = s.solve_stationary()
    ref, _, it, _, ost = o.solve_stationary(tol=1e-9, max_iter=20000)
    assert st == ADR_OK and ost == O.OK and stats["iters"] == it
    assert relerr(ug, ref) <= TOL64


def test_diverging_iteration_is_reported(torch_cuda):
    from paper_2411_11041_gb300 import ADR_ENOCONV, Solver, lib
    p = W.manufactured(n=17)
    s = Solver(p, theta=0.1, dt=5.0, tol=1e-8, max_iter=100000)
    u, _, stats, st = s.solve_stationary()
    _, _, it, _, ost = O.Oracle(p).solve_stationary(theta=0.1, dt=5.0, tol=1e-8, max_iter=100000)
    assert st == ADR_ENOCONV and ost == O.ENOCONV
    assert b"diverged" in lib().adr_last_error()
    assert abs(stats["iters"] - it) <= 2 and stats["iters"] < 2000


def test_data2d_paper_procedure_matches_oracle(torch_cuda):
    """eq. Data2D as the paper runs it: 50 steps of dt = 0.001 from the state
    of eq. u0stationary (61 x 61 nodes)."""
    from paper_2411_11041_gb300 import ADR_INIT_PAPER_U0, ADR_OK, Solver
    p = W.data2d(61)
    s = Solver(p, tol=0.0, max_iter=50, dt=1e-3, init=ADR_INIT_PAPER_U0)
    u, uit, stats, st = s.solve_stationary(want_iter=True)
    ref, refit, it, _, ost = O.Oracle(p).solve_stationary(theta=0.5, dt=1e-3, tol=0.0, max_iter=50,
                                                          init=2)
    assert st == ADR_OK and ost == O.OK and stats["iters"] == it == 50
    assert relerr(u, ref) <= TOL64 and relerr(uit, refit) <= TOL64


@pytest.mark.parametrize("name", ["aligned17", "steep", "L_mask", "sheared65", "data2d"])
def test_supg_mode_matches_oracle(torch_cuda, name):
    """SUPG on the B curves (opts.stabilize): the split step, the converged
    solve and the paper's initial state against the oracle's stabilised forms."""
    from paper_2411_11041_gb300 import ADR_OK, Solver
    torch = torch_cuda
    p = PROBLEMS[name]()
    o = O.Oracle(p, stabilize=1)
    s = Solver(p, tol=1e-10, max_iter=20000, stabilize=1)
    u = np.random.default_rng(12).normal(size=(p.ny, p.nx)) * o.interior()
    uh, un = s.split_step(torch.tensor(u, device="cuda:0"), o.default_dt())
    ouh, oun = o.split_step(0.5, o.default_dt(), u)
    assert relerr(uh, ouh) <= TOL64 and relerr(un, oun) <= TOL64
    out, _, stats, st = s.solve_stationary()
    ref, _, it, _, ost = o.solve_stationary(tol=1e-10, max_iter=20000)
    assert st == ADR_OK and ost == O.OK and stats["iters"] == it
    assert relerr(out, ref) <= TOL64
    assert relerr(s.paper_u0(), o.paper_u0()) <= TOL64


def test_supg_needs_fp64(torch_cuda):
    from paper_2411_11041_gb300 import AdrError, Solver
    with pytest.raises(AdrError, match="EINVAL"):
        Solver(W.manufactured(n=17), stabilize=1, prec=1)
