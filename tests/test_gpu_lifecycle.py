"""Handle lifecycle on the device: problem buffers and setup temporaries come
from the library's stream-ordered pool and go back to it on destroy, so
creating and destroying the same problem again and again must not take more
device memory after the first round, and every round must give the same
answer."""
import pytest

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


def test_create_destroy_cycles_reuse_device_memory(torch_cuda):
    torch = torch_cuda
    from paper_2411_11041_gb300 import Solver
    prob = W.sheared(n=257)
    first, free_after = None, []
    for _ in range(12):
        s = Solver(prob, tol=1e-8, max_iter=200000)
        u, _, st, _ = s.solve_stationary()
        u = u.cpu()
        s.close()
        torch.cuda.synchronize()
        free_after.append(torch.cuda.mem_get_info()[0])
        if first is None:
            first = (u, st["iters"])
        else:
            assert st["iters"] == first[1]
            assert torch.equal(u, first[0])
    # after the first round the pool holds what a round needs; later rounds
    # reuse it (a leak of one round's buffers would be tens of MB each time)
    drift = free_after[1] - free_after[-1]
    assert drift < 8 << 20, f"free device memory fell by {drift} bytes over 10 rounds"
