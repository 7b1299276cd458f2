"""Learned warm start: data generation with the method's own solver, training
of the network on the GPU, and initial states for new problems.

The network (adr_cnn_* calls, ``Network``) maps a problem on a 256 x 256 grid
and the paper's initial state u0 of it (eq. u0stationary, one steady sweep
along the beta curves) to the cell means (4 x 4 nodes) of the correction
u - u0, scaled by max |u0|, u the converged iterate; ``adr_cnn_initial_state``
adds their bilinear interpolation to u0, giving u_0 for ADR_INIT_USER.  A
network that predicts zero starts from the paper's u0.  Only the smooth part
of the correction is predicted: smooth error modes are the slow ones of the
split iteration, and the grid-scale rest of u - u0 costs few iterations.  The solve itself is unchanged: it iterates from u_0 to the same
tolerance, so the answer meets the same test whatever the network predicts.

Every array lives on the GPU; the host only draws the seeded problems and
moves their nodal fields to the device once.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import ADR_OK, Batch, Network, Solver


def _torch():
    import torch
    return torch


def stack(probs, device="cuda:0"):
    """Nodal fields of equally sized problems as device tensors [B, n, n]."""
    torch = _torch()
    dev = torch.device(device)
    f = torch.as_tensor(np.stack([p.f for p in probs]), device=dev)
    b1 = torch.as_tensor(np.stack([p.beta1 for p in probs]), device=dev)
    b2 = torch.as_tensor(np.stack([p.beta2 for p in probs]), device=dev)
    m = torch.as_tensor(np.stack([p.mask for p in probs]).astype(np.uint8), device=dev)
    mu = torch.as_tensor([p.mu for p in probs], dtype=torch.float64, device=dev)
    sg = torch.as_tensor([p.sigma for p in probs], dtype=torch.float64, device=dev)
    return f, b1, b2, m, mu, sg


def solver_opts(tol=1e-8, prec=0, anderson=0):
    """Options of every solve of the warm-start workload (curve -> grid weights
    by crossing gaps: the flow directions are random, some near a grid axis;
    anderson: the accelerated iteration's depth, 0 for the plain one)."""
    return dict(tol=tol, max_iter=200000, prec=prec, interp_weights=1, anderson=anderson)


@dataclasses.dataclass
class Dataset:
    x: object  # bf16 [N, 64, 64, 40]
    t: object  # fp32 [N, 64, 64]
    iters: np.ndarray  # iterations of each generating solve (zero initial state)


def paper_states(solvers):
    """The paper's initial state (eq. u0stationary) of every solver, stacked."""
    torch = _torch()
    return torch.stack([s.paper_u0() for s in solvers])


def generate(net: Network, probs, chunk=128, tol=1e-8, prec=0, device="cuda:0", anderson=0):
    """Solve every problem with the batched solver from u_0 = 0 and keep the
    network's features (with the paper's u0) and targets: the cell means of
    u_{j+1} - u0 over max |u0|, u_{j+1} the iterate the solve converged to (its
    fixed point; for theta = 1/2 the reported solution is the midpoint of the
    last step, which differs from it by the splitting error).  The accelerated
    iteration (anderson > 0) reaches the same fixed point in fewer steps."""
    torch = _torch()
    xs, ts, its = [], [], []
    for k in range(0, len(probs), chunk):
        part = probs[k:k + chunk]
        solvers = [Solver(p, device=device, **solver_opts(tol, prec, anderson)) for p in part]
        b = Batch(solvers)
        outs, stats, st, its_u = b.solve(want_iter=True)
        if st != ADR_OK:
            raise RuntimeError("a generating solve did not converge")
        f, b1, b2, m, mu, sg = stack(part, device)
        u0 = paper_states(solvers)
        x, scale = net.features(f, b1, b2, m, mu, sg, u0)
        xs.append(x)
        ts.append(net.targets(torch.stack(its_u), scale, u0))
        its += [s["iters"] for s in stats]
        b.close()
        for s in solvers:
            s.close()
        del outs, its_u, f, b1, b2, m, u0
    return Dataset(torch.cat(xs), torch.cat(ts), np.asarray(its))


def train(net: Network, data: Dataset, steps, batch=32, lr=1e-3, lr_final=1e-4, seed=0,
          log_every=0):
    """Adam on random minibatches; the learning rate decays geometrically
    from lr to lr_final.  Returns the losses of the logged steps."""
    torch = _torch()
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = data.x.shape[0]
    batch = min(batch, n, net.max_batch)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).to(data.x.device)
        x = data.x.index_select(0, idx).contiguous()
        t = data.t.index_select(0, idx).contiguous()
        rate = lr * (lr_final / lr) ** (s / max(steps - 1, 1))
        want = bool(log_every) and (s % log_every == 0 or s == steps - 1)
        loss = net.train_step(x, t, rate, want_loss=want)
        if want:
            losses.append((s, loss))
    return losses


def mu_bin(mu):
    """The decade of mu a problem falls in (the gate's classes)."""
    return int(np.floor(np.log10(mu)))


def initial_states(net: Network, solvers, fields, use=None):
    """u_0 of every solver: the paper's state, the features, one network
    batch, and the corrected states.  fields = stack(problems).  use (a list
    of booleans, optional): where False the network's correction is left out
    and the problem starts from the paper's u0 as it stands."""
    u0 = paper_states(solvers)
    x, scale = net.features(*fields, u0)
    y = net.forward(x)
    zero = None
    out = []
    for i, s in enumerate(solvers):
        yi = y[i]
        if use is not None and not use[i]:
            if zero is None:
                zero = _torch().zeros_like(yi)
            yi = zero
        out.append(net.initial_state(s, yi, u0[i], scale[i:i + 1]))
    return out


def calibrate_gate(net: Network, probs, tol=1e-8, prec=0, device="cuda:0", chunk=256, anderson=0):
    """Which problem classes (decades of mu) gain from the network's
    correction, measured on problems the network was not trained on: the
    batched solves from the paper's u0 and from the corrected state, the
    iterations summed per class.  The correction is a 4 x 4-cell mean: where
    the solution has layers thinner than a cell (small mu) its interpolation
    adds error to an already close u0, and the class is better off without
    it.  Returns {bin: True/False} (True: use the correction)."""
    paper_it, learned_it = {}, {}
    chunk = min(chunk, net.max_batch)  # one network batch per chunk
    for k in range(0, len(probs), chunk):
        part = probs[k:k + chunk]
        opts = solver_opts(tol, prec, anderson)
        pp = [Solver(p, device=device, init=2, **opts) for p in part]
        ll = [Solver(p, device=device, init=1, **opts) for p in part]
        bp, bl = Batch(pp), Batch(ll)
        _, sp, st1 = bp.solve()
        _, sl, st2 = bl.solve(initial_states(net, ll, stack(part, device)))
        if st1 != ADR_OK or st2 != ADR_OK:
            raise RuntimeError("a calibration solve did not converge")
        for p, a, b in zip(part, sp, sl):
            key = mu_bin(p.mu)
            paper_it[key] = paper_it.get(key, 0) + a["iters"]
            learned_it[key] = learned_it.get(key, 0) + b["iters"]
        bp.close()
        bl.close()
        for q in pp + ll:
            q.close()
    return {key: learned_it[key] < paper_it[key] for key in paper_it}


def gate_of(gate, probs):
    """use-flags of problems from a gate (classes not seen: the correction)."""
    return [gate.get(mu_bin(p.mu), True) for p in probs]


def evaluate(net: Network, probs, tol=1e-8, prec=0, device="cuda:0", chunk=128, sequential=False):
    """Held-out comparison on the same GPU: batched solves from u_0 = 0 and
    from the network's u_0 (network time included), and optionally the plain
    method (one problem after another, u_0 = 0).  Wall times in seconds of
    the solve phase (handles and graphs are built before the clock starts)."""
    torch = _torch()
    res = {"zero_iters": [], "learned_iters": [], "zero_s": 0.0, "learned_s": 0.0,
           "plain_s": 0.0, "net_s": 0.0}
    for k in range(0, len(probs), chunk):
        part = probs[k:k + chunk]
        solvers = [Solver(p, device=device, **solver_opts(tol, prec)) for p in part]
        f, b1, b2, m, mu, sg = stack(part, device)
        learned = [Solver(p, device=device, init=1, **solver_opts(tol, prec)) for p in part]
        bz, bl = Batch(solvers), Batch(learned)
        bz.solve()  # warm-up: graph build
        bl.solve([s._grid() for s in learned])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, sz, stz = bz.solve()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u0 = initial_states(net, learned, (f, b1, b2, m, mu, sg))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        _, sl, stl = bl.solve(u0)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        if stz != ADR_OK or stl != ADR_OK:
            raise RuntimeError("a held-out solve did not converge")
        res["zero_s"] += t1 - t0
        res["learned_s"] += t3 - t1
        res["net_s"] += t2 - t1
        res["zero_iters"] += [s["iters"] for s in sz]
        res["learned_iters"] += [s["iters"] for s in sl]
        if sequential:
            for s in solvers:  # warm-up of each handle's graph
                s.solve_stationary()
            torch.cuda.synchronize()
            t4 = time.perf_counter()
            for s in solvers:
                s.solve_stationary()
            torch.cuda.synchronize()
            res["plain_s"] += time.perf_counter() - t4
        bz.close()
        bl.close()
        for s in solvers + learned:
            s.close()
    res["zero_iters"] = np.asarray(res["zero_iters"])
    res["learned_iters"] = np.asarray(res["learned_iters"])
    return res
