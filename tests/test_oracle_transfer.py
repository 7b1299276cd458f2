"""Pins of the oracle's direct curve-to-curve transfer (the alternative to
the intermediate grid that the paper's conclusions propose), against facts
that do not come from the oracle:

* the crossing tables equal a brute-force intersection of every element of
  the target curve with every segment of the other family;
* on straight families the transfer reproduces linear functions exactly
  wherever a node has a crossing on both sides;
* for grid-aligned flow the crossings sit on grid nodes, so the direct
  transfer and the transfer through the grid are the same map and the two
  iterations coincide;
* the direct iteration converges to the exact solution of a manufactured
  problem as the grid is refined.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W


def _brute_crossings(Lt, Ls):
    """Per interior node k of the target family: the nearest crossing at or
    before it and at or after it along its curve, as (pos, g, t) or None, and
    whether the choice is ambiguous (two crossings, or a crossing and the node,
    closer than 1e-9 in position)."""
    offs, xs, ys = Ls["off"], Ls["xi"], Ls["eta"]
    segs = np.concatenate([np.arange(offs[l], offs[l + 1] - 1) for l in range(len(offs) - 1)])
    Q0 = np.stack([xs[segs], ys[segs]], 1)
    q = np.stack([xs[segs + 1], ys[segs + 1]], 1) - Q0
    offt, xt, yt = Lt["off"], Lt["xi"], Lt["eta"]
    out = {}
    for l in range(len(offt) - 1):
        a, b = offt[l], offt[l + 1]
        n = b - a - 1
        cr = []
        for e in range(n):
            P0 = np.array([xt[a + e], yt[a + e]])
            d = np.array([xt[a + e + 1], yt[a + e + 1]]) - P0
            den = d[0] * q[:, 1] - d[1] * q[:, 0]
            w = Q0 - P0
            ok = den != 0.0
            sden = np.where(ok, den, 1.0)
            s = (w[:, 0] * q[:, 1] - w[:, 1] * q[:, 0]) / sden
            t = (w[:, 0] * d[1] - w[:, 1] * d[0]) / sden
            eps = 1e-12
            sel = ok & (s >= -eps) & (s <= 1 + eps) & (t >= -eps) & (t <= 1 + eps)
            for i in np.nonzero(sel)[0]:
                cr.append((e + min(max(s[i], 0.0), 1.0), int(segs[i]), min(max(t[i], 0.0), 1.0)))
        cr.sort()
        for kk in range(1, n):
            bef = [c for c in cr if c[0] <= kk]
            aft = [c for c in cr if c[0] >= kk]
            amb = any(abs(c[0] - kk) < 1e-9 for c in cr)
            amb |= len(bef) > 1 and bef[-1][0] - bef[-2][0] < 1e-9
            amb |= len(aft) > 1 and aft[1][0] - aft[0][0] < 1e-9
            out[a + kk] = (bef[-1] if bef else None, aft[0] if aft else None, amb, n)
    return out


@pytest.mark.parametrize("name", ["sheared", "data2d", "disc"])
def test_transfer_tables_equal_brute_force_intersections(name):
    prob = {"sheared": lambda: W.sheared(n=17),
            "data2d": lambda: W.data2d(17),
            "disc": lambda: W.random_problem(np.random.Generator(np.random.PCG64(5)), 21,
                                             mask="disc")}[name]()
    o = O.Oracle(prob, transfer=1)
    for tf in (0, 1):
        Lt, Ls = o.lines(tf), o.lines(1 - tf)
        seg, t, pos = o.transfer_table(tf)
        bf = _brute_crossings(Lt, Ls)
        checked = 0
        for k, (before, after, amb, n) in bf.items():
            if amb:
                continue
            checked += 1
            for side, c in ((0, before), (1, after)):
                if c is None:  # no crossing on that side: the curve's end
                    assert seg[k, side] == -1 and pos[k, side] == (0.0 if side == 0 else n)
                else:
                    assert seg[k, side] == c[1], (tf, k, side, c, seg[k, side])
                    assert t[k, side] == pytest.approx(c[2], abs=1e-9)
                    assert pos[k, side] == pytest.approx(c[0], abs=1e-9)
        assert checked > 0.9 * len(bf)
        off = Lt["off"]
        ends = np.concatenate([off[:-1], off[1:] - 1])
        assert np.all(seg[ends] == -2)


@pytest.mark.parametrize("beta,mask", [((1.0, 0.5), "square"), ((-0.6, 0.8), "disc")])
def test_transfer_reproduces_linear_functions_on_straight_families(beta, mask):
    """Straight curves with uniform nodes: a linear function sampled at the
    source nodes is linear along each source segment (exact at the crossing)
    and linear in position along the target curve (exact between crossings)."""
    o = O.Oracle(W.manufactured(n=19, beta=beta, mask=mask), transfer=1)
    for tf in (0, 1):
        Ls, Lt = o.lines(1 - tf), o.lines(tf)
        src = 0.3 + 1.7 * Ls["xi"] - 0.9 * Ls["eta"]
        want = 0.3 + 1.7 * Lt["xi"] - 0.9 * Lt["eta"]
        got = o.transfer(tf, src)
        seg, _, _ = o.transfer_table(tf)
        both = (seg[:, 0] >= 0) & (seg[:, 1] >= 0)
        assert both.sum() > 0.5 * len(got)
        np.testing.assert_allclose(got[both], want[both], rtol=0, atol=1e-11)
        off = Lt["off"]
        assert np.all(got[off[:-1]] == 0.0) and np.all(got[off[1:] - 1] == 0.0)


def test_aligned_flow_direct_transfer_equals_transfer_through_the_grid():
    """beta = (1, 0): the B curves are grid rows and the G curves grid
    columns, every crossing is a grid node, so both transfers are the
    identity on shared nodes and the two iterations are one."""
    prob = W.manufactured(n=17, beta=(1.0, 0.0))
    ug, _, itg, _, stg = O.Oracle(prob).solve_stationary(tol=1e-11)
    ud, _, itd, _, std = O.Oracle(prob, transfer=1).solve_stationary(tol=1e-11)
    assert stg == std == O.OK and itg == itd
    np.testing.assert_allclose(ud, ug, rtol=0, atol=1e-13 * np.abs(ug).max())


def test_direct_iteration_converges_to_the_exact_solution():
    """u = sin(pi x) sin(pi y) manufactured: the converged direct iteration's
    error falls at least first order as h halves."""
    errs = []
    for n in (17, 33, 65):
        u, _, _, _, st = O.Oracle(W.manufactured(n=n), transfer=1).solve_stationary(tol=1e-12)
        assert st == O.OK
        errs.append(np.abs(u - W.exact_manufactured(n)).max())
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8, errs
    assert errs[2] < 0.012, errs
