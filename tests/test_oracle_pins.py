"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties one step of the oracle to an independent fact: numerical
quadrature of the paper's bilinear forms, a closed-form 1D solution, a dense
direct solve, a library banded solver, exactness of interpolation on
polynomials, a dense 2D Q1 Galerkin solve, or the analytic integral curves of
a divergence-free field.
"""
import math

import numpy as np
import pytest
from scipy.linalg import solve_banded

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W


def _prob(n, beta=(1.0, 0.0), mu=0.1, sigma=1.0, f=None, mask="square", nx=None, box=None):
    nx = nx or n
    b1 = np.full((n, nx), float(beta[0]))
    b2 = np.full((n, nx), float(beta[1]))
    if f is None:
        f = np.ones((n, nx))
    m = W.make_mask(mask, nx, n) if nx == n else np.ones((n, nx), np.uint8)
    p = W.Problem(nx, n, mu, sigma, b1, b2, np.asarray(f, float), m)
    if box:
        p.x0, p.y0, p.x1, p.y1 = box
    return p


# ---------------------------------------------------------------- 1D forms

def _hat_quadrature_matrices(xs, bnodes, fnodes, mu, sigma):
    """Assemble s_i(u, w) and <l_i, w> by 40-point Gauss-Legendre quadrature of
    the integrands over every element (eq. SemiDiscrSplit1Dbeta1), with |beta|
    and f the piecewise-linear interpolants of the nodal values."""
    n = len(xs) - 1
    S = np.zeros((n + 1, n + 1))
    F = np.zeros(n + 1)
    gx, gw = np.polynomial.legendre.leggauss(40)
    for e in range(n):
        a, b = xs[e], xs[e + 1]
        h = b - a
        x = 0.5 * (a + b) + 0.5 * h * gx
        w = 0.5 * h * gw
        lam = (x - a) / h
        phi = [1 - lam, lam]
        dphi = [-1.0 / h * np.ones_like(x), 1.0 / h * np.ones_like(x)]
        bet = (1 - lam) * bnodes[e] + lam * bnodes[e + 1]
        fv = (1 - lam) * fnodes[e] + lam * fnodes[e + 1]
        for i in range(2):
            F[e + i] += np.sum(w * fv * phi[i])
            for j in range(2):
                S[e + i, e + j] += np.sum(w * (mu * dphi[j] * dphi[i] + bet * dphi[j] * phi[i]
                                               + sigma * phi[j] * phi[i]))
    return S, F


def test_line_system_matches_quadrature_of_the_forms():
    # a curved problem so that |beta| varies along every B line
    p = W.sheared(n=17, mu=0.05, sigma=0.7)
    o = O.Oracle(p)
    L = o.lines(0)
    rng = np.random.default_rng(1)
    theta, dt = 0.5, 0.03
    checked = 0
    for line in range(len(L["off"]) - 1):
        a0, a1 = L["off"][line], L["off"][line + 1]
        n = a1 - a0 - 1
        if n < 3:
            continue
        h = L["h"][line]
        xs = h * np.arange(n + 1)
        bn, fv = L["bnorm"][a0:a1], L["fval"][a0:a1]
        u = rng.normal(size=n + 1)
        u[0] = u[-1] = 0.0
        a, b, c, r = o.line_system(0, line, theta, dt, u, fv)
        S, F = _hat_quadrature_matrices(xs, bn, fv, p.mu, p.sigma)
        M, _ = _hat_quadrature_matrices(xs, np.zeros(n + 1), np.zeros(n + 1), 0.0, 1.0)
        A = M + theta * dt * S
        rhs = F - S @ u
        k = np.arange(1, n)
        np.testing.assert_allclose(b, A[k, k], rtol=1e-12)
        np.testing.assert_allclose(a[1:], A[k[1:], k[1:] - 1], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(c[:-1], A[k[:-1], k[:-1] + 1], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(r, rhs[1:-1], rtol=1e-10, atol=1e-13)
        checked += 1
    assert checked > 5


def test_gamma_line_system_is_pure_cross_diffusion():
    p = W.sheared(n=17, mu=0.05)
    o = O.Oracle(p)
    L = o.lines(1)
    line = int(np.argmax(np.diff(L["off"])))
    a0, a1 = L["off"][line], L["off"][line + 1]
    n = a1 - a0 - 1
    h = L["h"][line]
    xs = h * np.arange(n + 1)
    u = np.sin(np.linspace(0, 3, n + 1))
    u[0] = u[-1] = 0.0
    a, b, c, r = o.line_system(1, line, 0.5, 0.1, u, np.ones(n + 1))
    K, _ = _hat_quadrature_matrices(xs, np.zeros(n + 1), np.zeros(n + 1), p.mu, 0.0)
    M, _ = _hat_quadrature_matrices(xs, np.zeros(n + 1), np.zeros(n + 1), 0.0, 1.0)
    A = M + 0.05 * K
    k = np.arange(1, n)
    np.testing.assert_allclose(b, A[k, k], rtol=1e-12)
    np.testing.assert_allclose(r, -(K @ u)[1:-1], rtol=1e-10, atol=1e-13)


def _exact_1d(x, mu, beta, sigma, c, L=1.0):
    """-mu u'' + beta u' + sigma u = c, u(0) = u(L) = 0."""
    s = math.sqrt(beta * beta + 4 * mu * sigma)
    r1, r2 = (beta + s) / (2 * mu), (beta - s) / (2 * mu)
    # u = c/sigma (1 + A e^{r1 (x-L)} + B e^{r2 x})  (scaled to avoid overflow)
    M = np.array([[math.exp(-r1 * L), 1.0], [1.0, math.exp(r2 * L)]])
    A, B = np.linalg.solve(M, [-1.0, -1.0])
    return c / sigma * (1 + A * np.exp(r1 * (x - L)) + B * np.exp(r2 * x))


@pytest.mark.parametrize("beta", [1.0, 4.0])
def test_line_solve_converges_to_exact_exponential_solution(beta):
    """The stationary line solve s_i(u, w) = <l_i, w> (eq. u0stationary) on the
    grid rows of an aligned problem, against the closed form, at O(h^2)."""
    mu, sigma, c = 0.1, 1.0, 2.0
    errs = []
    for n in (33, 65, 129):
        p = _prob(n, beta=(beta, 0.0), mu=mu, sigma=sigma, f=np.full((n, n), c))
        o = O.Oracle(p)
        u0 = o.paper_u0()
        x = np.linspace(0, 1, n)
        ex = _exact_1d(x, mu, beta, sigma, c)
        row = u0[n // 2]
        errs.append(np.abs(row[1:-1] - ex[1:-1]).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] < 2e-3


# ---------------------------------------------------------- tridiagonal

@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 1023])
@pytest.mark.parametrize("kind", ["dominant", "advective"])
def test_thomas_matches_dense_lu_with_pivoting(n, kind):
    rng = np.random.default_rng(n)
    if kind == "dominant":
        a, c = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
        b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 1, n)
    else:  # strong advection: l*u < 0, not diagonally dominant
        a = -rng.uniform(1.0, 3.0, n)
        c = rng.uniform(0.0, 0.2, n)
        b = rng.uniform(0.5, 1.0, n)
    a[0] = 0.0
    c[-1] = 0.0
    r = rng.normal(size=n)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x_lu = O.dense_lu_solve(A, r)
    x_th = O.thomas(a, b, c, r)
    np.testing.assert_allclose(x_th, x_lu, rtol=1e-10, atol=1e-12 * np.abs(x_lu).max())
    np.testing.assert_allclose(x_lu, np.linalg.solve(A, r), rtol=1e-9, atol=1e-12)


def test_thomas_long_system_matches_banded_library_solver():
    n = 4097
    rng = np.random.default_rng(7)
    a, c = rng.uniform(-1, 1, n), rng.uniform(-1, 1, n)
    b = np.abs(a) + np.abs(c) + 0.05
    a[0] = c[-1] = 0.0
    r = rng.normal(size=n)
    ab = np.zeros((3, n))
    ab[0, 1:], ab[1], ab[2, :-1] = c[:-1], b, a[1:]
    np.testing.assert_allclose(O.thomas(a, b, c, r), solve_banded((1, 1), ab, r), rtol=1e-10,
                               atol=1e-12)


# ---------------------------------------------------------- interpolation

def test_bilinear_reproduces_bilinear_functions():
    p = _prob(9, nx=13, box=(0.0, 0.0, 1.5, 1.0))
    o = O.Oracle(p)
    xi, eta = np.meshgrid(np.arange(13.0), np.arange(9.0))
    g = 0.3 + 1.7 * xi - 0.4 * eta + 0.25 * xi * eta
    rng = np.random.default_rng(3)
    pts = list(zip(rng.uniform(0, 12, 50), rng.uniform(0, 8, 50)))
    pts += [(0.0, 0.0), (12.0, 8.0), (5.0, 3.5), (7.25, 8.0), (12.0, 0.3)]
    for x, y in pts:
        assert abs(o.bilinear(g, x, y) - (0.3 + 1.7 * x - 0.4 * y + 0.25 * x * y)) < 1e-12


@pytest.mark.parametrize("mask", ["square", "L", "disc"])
def test_maps_are_identity_for_grid_aligned_lines(mask):
    n = 21
    p = _prob(n, beta=(1.0, 0.0), mask=mask)
    o = O.Oracle(p)
    g = np.random.default_rng(0).normal(size=(n, n)) * o.interior()
    for fam in (0, 1):
        assert np.array_equal(o.map_to_grid(fam, o.gather(fam, g)), g)


@pytest.mark.parametrize("beta", [(1.0, 0.5), (-0.3, 1.0), (0.8, -0.6)])
def test_line_to_grid_reproduces_linear_functions(beta):
    n = 25
    p = _prob(n, beta=beta)
    o = O.Oracle(p)
    xi, eta = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    for fam in (0, 1):
        L = o.lines(fam)
        vals = 0.4 + 0.7 * L["xi"] - 1.3 * L["eta"]
        g = o.map_to_grid(fam, vals)
        seg, _, _ = o.crossings(fam)
        ok = o.interior() & np.all(seg >= 0, axis=2)
        assert ok.sum() > 0.5 * o.interior().sum()
        np.testing.assert_allclose(g[ok], (0.4 + 0.7 * xi - 1.3 * eta)[ok], atol=1e-12)


def test_round_trip_of_smooth_function_is_second_order():
    errs = []
    for n in (33, 65, 129):
        p = _prob(n, beta=(1.0, 0.45))
        o = O.Oracle(p)
        X, Y = W.node_coords(n, n)
        g = np.sin(math.pi * X) * np.sin(2 * math.pi * Y)
        e = 0.0
        for fam in (0, 1):
            e = max(e, np.abs(o.map_to_grid(fam, o.gather(fam, g)) - g).max())
        errs.append(e)
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


# ----------------------------------------------------- 2D brute force

@pytest.mark.parametrize("beta", [(1.0, 0.0), (-1.0, 0.0), (0.0, 1.0), (0.0, -2.0)])
@pytest.mark.parametrize("dt", [0.01, 0.2])
def test_aligned_midpoint_equals_dense_q1(beta, dt):
    """For grid-aligned flow the Crank-Nicolson split step's fixed point,
    taken at the midpoint (u_j + u_{j+1/2}) / 2, is the Q1 Galerkin solution of
    eqs. VP1/VP1a on the same grid, for every pseudo-step."""
    n = 17
    p = W.manufactured(n=n, mu=0.1, beta=beta)
    o = O.Oracle(p)
    u, _, it, rel, st = o.solve_stationary(theta=0.5, dt=dt, tol=1e-14, max_iter=20000)
    q = O.q1_dense(p)
    assert st == O.OK
    assert np.abs(u - q).max() <= 1e-11 * np.abs(q).max()


@pytest.mark.parametrize("along", ["x", "y"])
def test_aligned_midpoint_equals_dense_q1_on_rectangle(along):
    """With a general source the B lines' loads <l_i, w> only see f on the
    lines that carry unknowns, so the exact Q1 counterpart has f set to 0 on the
    two boundary grid lines parallel to the flow (there the Q1 mass coupling
    would pick it up)."""
    beta = (0.7, 0.0) if along == "x" else (0.0, -0.7)
    p = _prob(9, beta=beta, mu=0.05, nx=17, box=(0.0, 0.0, 2.0, 1.0))
    X, Y = W.node_coords(17, 9, 0.0, 0.0, 2.0, 1.0)
    p.f = np.exp(-((X - 0.6) ** 2 + (Y - 0.4) ** 2) / 0.1)
    o = O.Oracle(p)
    u, _, _, _, st = o.solve_stationary(theta=0.5, dt=0.05, tol=1e-14, max_iter=20000)
    ft = p.f.copy()
    if along == "x":
        ft[0, :] = ft[-1, :] = 0.0
    else:
        ft[:, 0] = ft[:, -1] = 0.0
    q = O.q1_dense(p, f=ft)
    assert st == O.OK and np.abs(u - q).max() <= 1e-11 * np.abs(q).max()
    # with the untouched source the two differ only near the boundary, O(h)
    assert np.abs(u - O.q1_dense(p)).max() < 0.05 * np.abs(q).max()


def test_implicit_euler_slice_equals_dense_q1_step():
    """Parabolic mode 1: every implicit-Euler slice, solved by the split
    iteration, equals the Q1 solve with sigma + 1/dt and f + u_n/dt."""
    n, dt = 17, 0.01
    p = W.manufactured(n=n, beta=(1.0, 0.0))
    o = O.Oracle(p)
    X, Y = W.node_coords(n, n)
    u0 = np.sin(math.pi * X) * np.sin(math.pi * Y) * 0.5
    u1, _, st = o.step_parabolic(u0, dt, 1, 1, tol=1e-14, max_iter=20000)
    q = O.q1_dense(p, sigma=p.sigma + 1 / dt, f=p.f + u0 / dt)
    assert np.abs(u1 - q).max() <= 1e-11 * np.abs(q).max()


def test_general_flow_iteration_reaches_the_affine_fixed_point():
    """The split step is affine, u -> T u + c.  Build T column by column and
    solve (I - T) u* = c densely; the iteration's u_{j+1} must reach u*."""
    n = 11
    p = W.sheared(n=n, mu=0.05)
    o = O.Oracle(p)
    inter = o.interior()
    idx = np.flatnonzero(inter.ravel())
    dt = o.default_dt()
    zero = np.zeros((n, n))
    _, c = o.split_step(0.5, dt, zero)
    T = np.zeros((len(idx), len(idx)))
    for j, k in enumerate(idx):
        e = np.zeros(n * n)
        e[k] = 1.0
        _, un = o.split_step(0.5, dt, e.reshape(n, n))
        T[:, j] = (un - c).ravel()[idx]
    ustar = np.linalg.solve(np.eye(len(idx)) - T, c.ravel()[idx])
    u, uit, it, rel, st = o.solve_stationary(theta=0.5, dt=dt, tol=1e-13, max_iter=100000)
    assert st == O.OK
    assert np.abs(uit.ravel()[idx] - ustar).max() <= 1e-10 * np.abs(ustar).max()
    full = np.zeros(n * n)
    full[idx] = ustar
    uh, _ = o.split_step(0.5, dt, full.reshape(n, n))
    assert np.abs(u - 0.5 * (full.reshape(n, n) + uh)).max() <= 1e-10 * np.abs(u).max()


def test_manufactured_solution_error_decreases_under_refinement():
    errs_aligned, errs_slanted = [], []
    for n in (17, 33, 65):
        ex = W.exact_manufactured(n)
        for beta, errs in (((1.0, 0.0), errs_aligned), ((1.0, 0.5), errs_slanted)):
            o = O.Oracle(W.manufactured(n=n, beta=beta))
            u, _, _, _, st = o.solve_stationary(tol=1e-11)
            assert st == O.OK
            errs.append(np.abs(u - ex).max())
    assert errs_aligned[0] / errs_aligned[1] > 3.5 and errs_aligned[1] / errs_aligned[2] > 3.5
    assert errs_slanted[0] / errs_slanted[1] > 1.7 and errs_slanted[1] / errs_slanted[2] > 1.7
    assert errs_slanted[2] < 0.03


def test_dense_references_converge_to_manufactured_solution():
    for fn in (O.q1_dense, O.p1_dense):
        e = [np.abs(fn(W.manufactured(n=n)) - W.exact_manufactured(n)).max() for n in (9, 17, 33)]
        assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.0, (fn, e)


# ------------------------------------------------------------ invariants

def test_linearity_in_f_and_zero_source():
    n = 21
    p1, p2 = W.sheared(n=n, seed=5), W.sheared(n=n, seed=6)
    o1, o2 = O.Oracle(p1), O.Oracle(p2)
    p3 = W.sheared(n=n, seed=5)
    p3.f = p1.f + 2.0 * p2.f
    o3 = O.Oracle(p3)
    dt = o1.default_dt()
    u1 = o1.solve_stationary(dt=dt, tol=0.0, max_iter=25)[0]
    u2 = o2.solve_stationary(dt=dt, tol=0.0, max_iter=25)[0]
    u3 = o3.solve_stationary(dt=dt, tol=0.0, max_iter=25)[0]
    np.testing.assert_allclose(u3, u1 + 2.0 * u2, atol=1e-13 * np.abs(u3).max())
    p0 = W.sheared(n=n)
    p0.f = np.zeros((n, n))
    assert np.all(O.Oracle(p0).solve_stationary(tol=1e-12)[0] == 0.0)


def test_dirichlet_nodes_stay_zero_on_masked_domains():
    for mask in ("disc", "L"):
        rng = np.random.default_rng(2)
        p = W.random_problem(rng, 41, mask=mask)
        o = O.Oracle(p)
        u, uit, _, _, _ = o.solve_stationary(tol=1e-9)
        assert np.all(u[~o.interior()] == 0.0) and np.all(uit[~o.interior()] == 0.0)
        assert np.abs(u).max() > 0


# -------------------------------------------------------------- curves

def test_traced_curves_of_sheared_field_are_vertical_translates():
    """beta = (1, 0.5 + 0.3 sin 2 pi x) has integral curves
    y = 0.5 x - 0.3/(2 pi) cos(2 pi x) + C (eq. CauchyBeta).  The traced curves
    (bilinear beta, RK4) follow them to O(h^2)."""
    devs = []
    for n in (33, 65):
        o = O.Oracle(W.sheared(n=n))
        assert not o.const_beta
        L = o.lines(0)
        h = 1.0 / (n - 1)
        dev = 0.0
        for line in range(len(L["off"]) - 1):
            a0, a1 = L["off"][line], L["off"][line + 1]
            x, y = L["xi"][a0:a1] * h, L["eta"][a0:a1] * h
            C = y - (0.5 * x - 0.3 / (2 * math.pi) * np.cos(2 * math.pi * x))
            dev = max(dev, C.max() - C.min())
        devs.append(dev)
    assert devs[1] < 1e-3 and devs[0] / devs[1] > 3.0, devs


def test_seed_spacing_is_the_transverse_measure():
    """On the left edge of the sheared problem b1 = 1/sqrt(1.25) is constant,
    so seeds there are h_s sqrt(1.25) apart in y."""
    n = 33
    o = O.Oracle(W.sheared(n=n))
    L = o.lines(0)
    starts = L["off"][:-1]
    left = sorted(L["eta"][starts][L["xi"][starts] == 0.0])
    gaps = np.diff(left)
    np.testing.assert_allclose(gaps, math.sqrt(1.25), rtol=1e-12)


def test_straight_lines_are_evenly_spaced_and_cover_the_square():
    n = 33
    o = O.Oracle(W.manufactured(n=n))
    assert o.const_beta
    b = np.array([1.0, 0.5]) / math.sqrt(1.25)
    pvec = np.array([b[1], -b[0]])
    L = o.lines(0)
    offs = []
    for line in range(len(L["off"]) - 1):
        a0, a1 = L["off"][line], L["off"][line + 1]
        P = np.stack([L["xi"][a0:a1], L["eta"][a0:a1]], 1) / (n - 1)
        q = P @ pvec
        assert np.ptp(q) < 1e-12  # straight, along b
        offs.append(q[0] * (n - 1))
        hh = np.linalg.norm(np.diff(P, axis=0), axis=1)
        assert np.all(hh <= 1.0 / (n - 1) + 1e-12)
    np.testing.assert_allclose(np.diff(sorted(set(np.round(offs, 9)))), 1.0, atol=1e-9)


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_one_split_step_equals_dense_directional_step(theta):
    """eq. SemiDiscrSplit for flow along x, built densely from 1D matrices
    assembled by quadrature: rows first (s with load), then columns (m), each
    (M + theta dt S) d = F - S u,  u <- u + dt d."""
    n, mu, sigma, b, dt = 13, 0.07, 0.9, 1.3, 0.04
    p = _prob(n, beta=(b, 0.0), mu=mu, sigma=sigma)
    X, Y = W.node_coords(n, n)
    p.f = 1.0 + X * Y
    o = O.Oracle(p)
    rng = np.random.default_rng(4)
    u = rng.normal(size=(n, n)) * o.interior()
    xs = np.linspace(0, 1, n)
    S, _ = _hat_quadrature_matrices(xs, np.full(n, b), np.zeros(n), mu, sigma)
    M, _ = _hat_quadrature_matrices(xs, np.zeros(n), np.zeros(n), 0.0, 1.0)
    K, _ = _hat_quadrature_matrices(xs, np.zeros(n), np.zeros(n), mu, 0.0)
    I = slice(1, n - 1)
    uh = np.zeros_like(u)
    for r in range(1, n - 1):
        F = M @ p.f[r]
        rhs = (F - S @ u[r])[I]
        d = np.linalg.solve((M + theta * dt * S)[I, I], rhs)
        uh[r, I] = u[r, I] + dt * d
    un = np.zeros_like(u)
    for i in range(1, n - 1):
        rhs = (-(K @ uh[:, i]))[I]
        d = np.linalg.solve((M + theta * dt * K)[I, I], rhs)
        un[I, i] = uh[I, i] + dt * d
    ouh, oun = o.split_step(theta, dt, u)
    np.testing.assert_allclose(ouh, uh, atol=1e-12 * np.abs(uh).max())
    np.testing.assert_allclose(oun, un, atol=1e-12 * np.abs(un).max())
    # the paper's parabolic scheme (mode 0) is this step repeated
    u2, _, _ = o.step_parabolic(u, dt, 2, 0, theta=theta)
    _, ref2 = o.split_step(theta, dt, oun)
    np.testing.assert_allclose(u2, ref2, atol=1e-14 * np.abs(ref2).max())


# ------------------------------------------- inverse-gap weighting, divergence

@pytest.mark.parametrize("mask", ["square", "L"])
def test_weighted_map_is_identity_for_aligned_lines(mask):
    n = 21
    o = O.Oracle(_prob(n, beta=(0.0, -1.0), mask=mask), interp_weights=1)
    g = np.random.default_rng(1).normal(size=(n, n)) * o.interior()
    for fam in (0, 1):
        assert np.array_equal(o.map_to_grid(fam, o.gather(fam, g)), g)


@pytest.mark.parametrize("beta", [(1.0, 0.5), (1.0, 0.03), (-0.2, 1.0)])
def test_weighted_map_reproduces_linear_functions(beta):
    n = 25
    o = O.Oracle(_prob(n, beta=beta), interp_weights=1)
    xi, eta = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
    for fam in (0, 1):
        L = o.lines(fam)
        g = o.map_to_grid(fam, 0.4 + 0.7 * L["xi"] - 1.3 * L["eta"])
        seg, _, _ = o.crossings(fam)
        ok = o.interior() & np.all(seg >= 0, axis=2)
        np.testing.assert_allclose(g[ok], (0.4 + 0.7 * xi - 1.3 * eta)[ok], atol=1e-12)


def test_weighted_map_prefers_the_denser_direction():
    """With flow at 1.5 degrees the row crossings of the B curves are far apart;
    the weighted value of a smooth function is far closer to it than the
    plain average."""
    n = 65
    X, Y = W.node_coords(n, n)
    g = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    errs = []
    for w in (0, 1):
        o = O.Oracle(_prob(n, beta=(1.0, np.tan(np.radians(1.5)))), interp_weights=w)
        errs.append(np.abs(o.map_to_grid(0, o.gather(0, g * o.interior())) - g * o.interior()).max())
    assert errs[1] < 0.2 * errs[0], errs


def test_diverging_iteration_stops_without_convergence():
    """theta = 0.1 with a large step amplifies stiff modes by about -(1-theta)/theta
    per step: the iteration must end as not converged once a norm overflows,
    long before max_iter, instead of reading 0/inf as convergence."""
    p = W.manufactured(n=17)
    o = O.Oracle(p)
    u, uit, it, rel, st = o.solve_stationary(theta=0.1, dt=5.0, tol=1e-8, max_iter=100000)
    assert st == O.ENOCONV and not np.isfinite(rel) and it < 2000


def test_flows_whose_curves_do_not_cover_the_domain_are_rejected():
    """The method needs both curve families to cover Omega_h (§3, §6).  A
    rotating flow leaves a disc around its centre that no inflow-seeded beta
    curve reaches; a source-like flow beta = x - c has no inflow boundary for
    its beta family at all.  Both are geometry errors, not silent zeros."""
    n = 34  # no node at the centre, so |beta| > 0 at every node
    X, Y = W.node_coords(n, n)
    sq = W.make_mask("square", n, n)
    one = np.ones((n, n))
    rot = W.Problem(n, n, 0.01, 1.0, -(Y - 0.5), X - 0.5, one, sq)
    src = W.Problem(n, n, 0.01, 1.0, X - 0.5, Y - 0.5, one, sq)
    for prob in (rot, src):
        with pytest.raises(O.OracleError) as e:
            O.Oracle(prob)
        assert e.value.status == O.EGEOM


def _exact_advection_1d(x, L, mu, b, c):
    """-mu u'' + b u' = c on [0, L], u(0) = u(L) = 0 (exponentials written to
    stay finite for large b L / mu)."""
    r = b / mu
    return c / b * (x - L * (np.exp(r * (x - L)) - np.exp(-r * L)) / (1.0 - np.exp(-r * L)))


@pytest.mark.parametrize("mu", [1e-3, 0.1])
def test_supg_line_solve_is_nodally_exact(mu):
    """With tau = h/(2b)(coth Pe - 1/Pe) the SUPG solution of -mu u'' + b u' = c
    is exact at the nodes (textbook result for linear elements), for large and
    small element Peclet numbers; Galerkin is not at large Pe."""
    n, b, c = 33, 1.0, 1.0
    p = W.Problem(n, n, mu, 1.0, np.full((n, n), b), np.zeros((n, n)), np.full((n, n), c),
                  W.make_mask("square", n, n))
    errs = {}
    for stab in (1, 0):
        o = O.Oracle(p, stabilize=stab)
        L = o.lines(0)
        line = len(L["off"]) // 2  # an interior grid row
        a0, a1 = L["off"][line], L["off"][line + 1]
        x = (L["xi"][a0:a1] - L["xi"][a0]) / (n - 1)
        u = np.zeros(a1 - a0)
        fl = np.full(a1 - a0, c)
        dt = 1e9  # theta = 1: dt d = (M/dt + S)^-1 (F - S u) -> S^-1 F
        a, bb, cc, r = o.line_system(0, line, 1.0, dt, u, fl, sigma=0.0)
        d = O.thomas(a, bb, cc, r)
        ex = _exact_advection_1d(x[1:-1], x[-1], mu, b, c)
        errs[stab] = np.abs(dt * d - ex).max() / np.abs(ex).max()
    assert errs[1] < 1e-7, errs
    if mu == 1e-3:  # Pe = 15.6: Galerkin is far from the nodal values
        assert errs[0] > 1e-2, errs


def test_supg_reduces_to_galerkin_as_pe_vanishes():
    """tau ~ h^2 / (12 mu) as Pe -> 0: the stabilised line systems differ from
    the Galerkin ones by O(Pe) relatively."""
    n = 33
    p = W.manufactured(n=n, mu=10.0, beta=(1.0, 0.5))  # Pe = |beta| h / (2 mu) ~ 2e-3
    u = np.random.default_rng(0).normal(size=40)
    out = []
    for stab in (0, 1):
        o = O.Oracle(p, stabilize=stab)
        L = o.lines(0)
        line = max(range(len(L["off"]) - 1), key=lambda l: L["off"][l + 1] - L["off"][l])
        m = L["off"][line + 1] - L["off"][line]
        out.append(np.concatenate(o.line_system(0, line, 0.5, 0.01, u[:m], np.ones(m))))
    rel = np.abs(out[1] - out[0]).max() / np.abs(out[0]).max()
    assert 0 < rel < 1e-2, rel


def test_supg_keeps_a_steep_solution_within_its_bounds():
    """Aligned flow with mu = 1e-4 on 33^2 nodes (Pe ~ 16): the Galerkin lines
    oscillate (the converged midpoint leaves [0, f / sigma] visibly), SUPG
    stays within the bounds of the maximum principle up to 1 %."""
    n = 33
    p = W.Problem(n, n, 1e-4, 1.0, np.ones((n, n)), np.zeros((n, n)), np.ones((n, n)),
                  W.make_mask("square", n, n))
    res = {}
    for stab in (0, 1):
        u, _, it, _, st = O.Oracle(p, stabilize=stab).solve_stationary(tol=1e-10, max_iter=20000)
        assert st == O.OK
        res[stab] = (u.min(), u.max())
    assert res[0][1] > 1.05 or res[0][0] < -0.05, res  # Galerkin over/undershoots
    assert res[1][0] > -0.01 and res[1][1] < 1.01, res
