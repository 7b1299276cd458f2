"""What the trained warm-start network gains: a network trained on the GPU on
solutions the method generated, with its correction gated per class of
problems on a calibration set kept out of the training, must cut the
iterations to the same tolerance on held-out problems against u_0 = 0 and
against the paper's own initial state, and the answers from its initial
states must be the answers from u_0 = 0 (the iteration alone decides
convergence)."""
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
    draw = W.learned(2304, n=256)
    train, val = draw[:2048], draw[2048:]
    hold = W.learned(128, n=256, seed=W.SEED_BASE + 5)
    net = Network(128)
    data = WS.generate(net, train, anderson=3)
    losses = WS.train(net, data, steps=4000, batch=64, log_every=1000)
    hd = WS.generate(net, hold, anderson=3)
    zero_pred = 0.5 * (hd.t.double() ** 2).mean().item()
    held = net.loss_grad(hd.x[:64].contiguous(), hd.t[:64].contiguous())[0]
    assert held < 0.05 * zero_pred, (held, zero_pred, losses)
    gate = WS.calibrate_gate(net, val)
    use = WS.gate_of(gate, hold)
    opts = WS.solver_opts()
    zs = [Solver(p, **opts) for p in hold]
    ps = [Solver(p, init=2, **opts) for p in hold]  # eq. u0stationary
    ls = [Solver(p, init=1, **opts) for p in hold]
    _, sz, stz = Batch(zs).solve()
    _, sp, stp = Batch(ps).solve()
    _, sl, stl = Batch(ls).solve(WS.initial_states(net, ls, WS.stack(hold), use))
    assert stz == stp == stl == ADR_OK
    z = np.array([x["iters"] for x in sz])
    p = np.array([x["iters"] for x in sp])
    l = np.array([x["iters"] for x in sl])
    assert l.sum() < 0.9 * z.sum(), (l.sum(), z.sum())
    # against the paper's own initial state, which the network corrects: the
    # classes the gate keeps must gain, the others start from u0 unchanged
    assert any(gate.values()), gate
    assert l.sum() < p.sum(), (l.sum(), p.sum(), gate)
    for q, (a, b, u) in enumerate(zip(l, p, use)):
        if not u:
            assert a == b, q
    # same answers: both runs stop at a relative update of 1e-8
    zs = [Solver(p, **WS.solver_opts()) for p in hold[:8]]
    ls = [Solver(p, init=1, **WS.solver_opts()) for p in hold[:8]]
    u0 = WS.initial_states(net, ls, WS.stack(hold[:8]))
    uz, _, stz = Batch(zs).solve()
    ul, _, stl = Batch(ls).solve(u0)
    assert stz == ADR_OK and stl == ADR_OK
    for a, b in zip(ul, uz):
        assert (a - b).abs().max().item() <= 1e-6 * b.abs().max().item()


def test_init_learned_equals_the_manual_chain(torch_cuda):
    """ADR_INIT_LEARNED with a network attached by adr_set_warm_start runs the
    paper's u0, the features, the forward pass and the initial state inside
    the solve: the same iterations and answer, bit for bit, as the chain run by
    hand and passed with ADR_INIT_USER.  Without a network it is refused."""
    torch = torch_cuda
    from paper_2411_11041_gb300 import ADR_INIT_LEARNED, ADR_OK, AdrError, Network, Solver
    from paper_2411_11041_gb300 import warmstart as WS
    probs = W.learned(3, n=256, seed=W.SEED_BASE + 7)
    net = Network(4, W.cnn_init_params(seed=11, last_scale=1.0))
    for p in probs:
        man = Solver(p, init=1, **WS.solver_opts())
        u0 = WS.initial_states(net, [man], WS.stack([p]))[0]
        um, _, sm, cm = man.solve_stationary(u_init=u0)
        lrn = Solver(p, init=ADR_INIT_LEARNED, **WS.solver_opts())
        lrn.set_warm_start(net)
        ul, _, sl, cl = lrn.solve_stationary()
        assert cm == cl == ADR_OK
        assert sl["iters"] == sm["iters"]
        assert torch.equal(ul, um)
    bare = Solver(probs[0], init=ADR_INIT_LEARNED, **WS.solver_opts())
    with pytest.raises(AdrError, match="EINVAL"):
        bare.solve_stationary()
