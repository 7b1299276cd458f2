"""The allocation-free cross-flow substep against the library's own substep.

adr_cross_substep_noalloc serves callers that cannot allocate device memory:
it takes the G-family curves and crossings from the caller and keeps its work
space in a fixed device array.  Here it is called through the C ABI (ctypes)
twice in a row and must reproduce the u_{j+1} that adr_split_step computes
from the same u_{j+1/2}.  This file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2411_11041_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _noalloc_fn():
    from paper_2411_11041_gb300 import lib
    fn = lib().adr_cross_substep_noalloc
    vp = C.c_void_p
    fn.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, vp, C.c_int, C.c_int,
                   vp, vp, vp, vp, vp, vp, vp, vp, vp]
    fn.restype = C.c_int
    return fn


def test_noalloc_substep_matches_split_step_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_11041_gb300 import ADR_OK, Solver, adr_split_step, build
    build.build()
    dev = torch.device("cuda:0")
    fn = _noalloc_fn()
    for name, prob in (("sheared", W.sheared(n=129)), ("slanted", W.manufactured(n=97))):
        s = Solver(prob, device=dev)
        L = s.lines(1)
        seg, t, pos = s.crossings(1)
        d = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
        off, h, xi, eta = d(L["off"], torch.int32), d(L["h"]), d(L["xi"]), d(L["eta"])
        seg_d, t_d, pos_d = d(seg.ravel(), torch.int32), d(t.ravel()), d(pos.ravel())
        n_lines, n_nodes = len(L["off"]) - 1, int(L["off"][-1])
        rng = np.random.default_rng(5)
        dt = 0.013
        for call in range(2):
            u = d(rng.normal(size=(prob.ny, prob.nx)))
            u_half = torch.zeros_like(u)
            u_next = torch.zeros_like(u)
            adr_split_step(s.h, dt, u, u_half, u_next)
            out = torch.full_like(u, float("nan"))
            st = fn(prob.nx, prob.ny, prob.mu, 0.5, dt, C.c_void_p(u_half.data_ptr()), n_lines,
                    n_nodes, C.c_void_p(off.data_ptr()), C.c_void_p(h.data_ptr()),
                    C.c_void_p(xi.data_ptr()), C.c_void_p(eta.data_ptr()),
                    C.c_void_p(seg_d.data_ptr()), C.c_void_p(t_d.data_ptr()),
                    C.c_void_p(pos_d.data_ptr()), C.c_void_p(out.data_ptr()),
                    C.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
            assert st == ADR_OK
            torch.cuda.synchronize(dev)
            ref = u_next.cpu().numpy()
            got = out.cpu().numpy()
            err = np.abs(got - ref).max() / np.abs(ref).max()
            assert err <= TOL64, (name, call, err)
        s.close()


def test_noalloc_rejects_sizes_beyond_its_work_space():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_11041_gb300 import ADR_EINVAL, lib
    fn = _noalloc_fn()
    p = C.c_void_p(16)
    st = fn(64, 64, 1.0, 0.5, 0.1, p, 10, (1 << 19) + 1, p, p, p, p, p, p, p, p, None)
    assert st == ADR_EINVAL
    assert b"524288" in lib().adr_last_error()
