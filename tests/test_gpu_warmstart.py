"""What the trained warm-start network gains: a network trained on the GPU on
solutions the method generated must cut the iterations to the same tolerance
on held-out problems (against u_0 = 0; against the paper's own initial state
it must not lose more than 5 %), and the answers from its initial states must
be the answers from u_0 = 0 (the iteration alone decides convergence)."""
import numpy as np
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


def test_trained_network_reduces_iterations_on_held_out_problems(torch_cuda):
    torch = torch_cuda
    from paper_2411_11041_gb300 import ADR_OK, Batch, Network, Solver
    from paper_2411_11041_gb300 import warmstart as WS
    train = W.learned(1024, n=256)
    hold = W.learned(48, n=256, seed=W.SEED_BASE + 5)
    net = Network(64)
    data = WS.generate(net, train)
    losses = WS.train(net, data, steps=2000, batch=32, log_every=500)
    hd = WS.generate(net, hold)
    zero_pred = 0.5 * (hd.t.double() ** 2).mean().item()
    held = net.loss_grad(hd.x[:32].contiguous(), hd.t[:32].contiguous())[0]
    assert held < 0.2 * zero_pred, (held, zero_pred, losses)
    res = WS.evaluate(net, hold)
    z, l = res["zero_iters"], res["learned_iters"]
    assert l.sum() < 0.97 * z.sum(), (l.sum(), z.sum())
    # against the paper's own initial state, which the network corrects: the
    # split iteration's slow modes are the smooth ones, so the network's
    # (smooth) residual error must be far below 1 % of u to gain much on it;
    # the trained network matches it rather than beats it
    ps = [Solver(p, init=2, **WS.solver_opts()) for p in hold]
    _, sp, stp = Batch(ps).solve()
    assert stp == ADR_OK
    paper = sum(x["iters"] for x in sp)
    assert l.sum() <= 1.05 * paper, (l.sum(), paper)
    # same answers: both runs stop at a relative update of 1e-8
    zs = [Solver(p, **WS.solver_opts()) for p in hold[:8]]
    ls = [Solver(p, init=1, **WS.solver_opts()) for p in hold[:8]]
    u0 = WS.initial_states(net, ls, WS.stack(hold[:8]))
    uz, _, stz = Batch(zs).solve()
    ul, _, stl = Batch(ls).solve(u0)
    assert stz == ADR_OK and stl == ADR_OK
    for a, b in zip(ul, uz):
        assert (a - b).abs().max().item() <= 1e-6 * b.abs().max().item()
