"""Invalid inputs and degenerate problems: the library must refuse them with
the documented status (and the oracle with the same one), never fault or
return silent zeros.  Every case here is an input the host-side or the
device-side checks turn into an error before any sweep runs."""
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


def _status_of_create(prob):
    from paper_2411_11041_gb300 import AdrError, Solver
    try:
        Solver(prob).close()
        return 0
    except AdrError as e:
        return e.status


def _oracle_status(prob):
    try:
        O.Oracle(prob)
        return O.OK
    except O.OracleError as e:
        return e.status


def _degenerate():
    n = 34
    X, Y = W.node_coords(n, n)
    sq = W.make_mask("square", n, n)
    one = np.ones((n, n))
    rot = W.Problem(n, n, 0.01, 1.0, -(Y - 0.5), X - 0.5, one, sq, name="rotating")
    src = W.Problem(n, n, 0.01, 1.0, X - 0.5, Y - 0.5, one, sq, name="source")
    zb = W.manufactured(n=33)
    zb.beta1, zb.beta2 = zb.beta1.copy(), zb.beta2.copy()
    zb.beta1[10, 10] = zb.beta2[10, 10] = 0.0
    nanf = W.manufactured(n=33)
    nanf.f = nanf.f.copy()
    nanf.f[5, 7] = np.nan
    empty = W.manufactured(n=33)
    empty.mask = np.zeros((33, 33), np.uint8)
    return [(rot, 5), (src, 5), (zb, 1), (nanf, 1), (empty, 1)]


@pytest.mark.parametrize("case", range(5))
def test_degenerate_problems_are_refused_like_the_oracle(torch_cuda, case):
    prob, want = _degenerate()[case]
    assert _status_of_create(prob) == want, prob.name
    assert _oracle_status(prob) == want, prob.name


def test_solve_calls_reject_bad_arguments(torch_cuda):
    torch = torch_cuda
    import ctypes

    from paper_2411_11041_gb300 import (ADR_EINVAL, Batch, Solver, adr_stats, lib)
    s = Solver(W.manufactured(n=33), init=1)  # ADR_INIT_USER without u_init
    out = s._grid()
    st = lib().adr_solve_stationary(s.h, None, ctypes.c_void_p(out.data_ptr()), None, None)
    assert st == ADR_EINVAL and b"u_init" in lib().adr_last_error()
    u = s._grid()
    st = lib().adr_step_parabolic(s.h, 1e-3, 1, 7, ctypes.c_void_p(u.data_ptr()),
                                  ctypes.byref(adr_stats()))
    assert st == ADR_EINVAL
    ms = (ctypes.c_double * 4)()
    assert lib().adr_time_kernels(s.h, 0, ms) == ADR_EINVAL
    # a batch needs one precision mode
    a, b = Solver(W.manufactured(n=33)), Solver(W.manufactured(n=33), prec=1)
    from paper_2411_11041_gb300 import AdrError
    with pytest.raises(AdrError, match="EINVAL"):
        Batch([a, b])
    for x in (s, a, b):
        x.close()
