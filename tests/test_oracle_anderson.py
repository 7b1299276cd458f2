"""Pins of the oracle's accelerated stationary iteration (Anderson
extrapolation over the last m split steps, opts.anderson = m), against facts
that do not come from the oracle:

* on a linear fixed-point map of size n, the extrapolation over m >= n steps
  ends in at most n + 2 maps (it then minimises the residual over the whole
  Krylov space, as GMRES does), where the plain iteration needs hundreds;
* the extrapolation leaves the fixed point in place: the accelerated solve
  converges to the plain solve's answer, through the grid and with the direct
  transfer, in fewer split steps;
* time stepping (adr_step_parabolic mode 0) is never extrapolated.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W


def _linear(n, radius, seed, symmetric=False):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(n, n))
    if symmetric:
        Q = Q + Q.T
    T = Q / np.abs(np.linalg.eigvals(Q)).max() * radius
    return T, rng.normal(size=n)


@pytest.mark.parametrize("n,seed,symmetric", [(3, 0, False), (6, 1, False), (8, 2, True)])
def test_full_depth_terminates_on_linear_maps(n, seed, symmetric):
    T, c = _linear(n, 0.97, seed, symmetric)
    exact = np.linalg.solve(np.eye(n) - T, c)
    x, k, res = O.anderson_linear(T, c, np.zeros(n), m=8, max_iter=200, tol=1e-12)
    assert k <= n + 2, (k, res)
    assert np.abs(x - exact).max() <= 1e-10 * np.abs(exact).max()
    xp, kp, _ = O.anderson_linear(T, c, np.zeros(n), m=0, max_iter=200, tol=1e-12)
    assert kp == 200  # the plain iteration is nowhere near in as many maps


def test_shallow_depth_still_converges_to_the_fixed_point():
    T, c = _linear(12, 0.95, 4)
    exact = np.linalg.solve(np.eye(12) - T, c)
    for m in (1, 2, 3):
        x, k, res = O.anderson_linear(T, c, np.zeros(12), m=m, max_iter=2000, tol=1e-13)
        assert res[-1] <= 1e-13
        assert np.abs(x - exact).max() <= 1e-10 * np.abs(exact).max(), m


@pytest.mark.parametrize("name", ["sheared", "slanted", "L"])
@pytest.mark.parametrize("transfer", [0, 1])
def test_accelerated_solve_keeps_the_fixed_point(name, transfer):
    prob = {"sheared": lambda: W.sheared(n=65),
            "slanted": lambda: W.manufactured(n=33),
            "L": lambda: W.manufactured(n=41, beta=(0.3, 1.0), mask="L")}[name]()
    u0, _, k0, _, s0 = O.Oracle(prob, transfer=transfer).solve_stationary(tol=1e-12)
    u3, _, k3, rel, s3 = O.Oracle(prob, transfer=transfer, anderson=3).solve_stationary(tol=1e-12)
    assert s0 == s3 == O.OK and rel <= 1e-12
    assert np.abs(u3 - u0).max() <= 1e-9 * np.abs(u0).max()
    assert k3 < 0.8 * k0, (k3, k0)


def test_time_steps_are_not_extrapolated():
    p = W.parabolic(n=33)
    for transfer in (0, 1):
        plain = O.Oracle(p, transfer=transfer).step_parabolic(p.u0, 1e-3, 5, 0)[0]
        acc = O.Oracle(p, transfer=transfer, anderson=3).step_parabolic(p.u0, 1e-3, 5, 0)[0]
        assert np.array_equal(plain, acc)
