"""Pins of the oracle's traced curve families, their seeding and the
curve -> grid map on them, against facts that do not come from the oracle.

* G curves (§6 eq. CauchyGamma) of the sheared field follow its analytic
  cross-flow curves y + Y(x) = const, Y(x) = int_0^x dt / (0.5 + 0.3 sin 2 pi t),
  to O(h^2), oriented along p = (beta2, -beta1) / |beta|.
* For the paper's own field (§7 eq. Data2D) the G curves are exact rays out of
  (-1, -1) and the B curves circular arcs about it, run counter-clockwise.
* The curve -> grid map (§6, interpolation through the crossings) reproduces
  linear functions exactly on traced families too.
* Seeds (§6 eq. cauchyStartSets) on a domain with holes: counted, placed and
  spaced by the transverse inflow measure, computed here by an independent
  walk of the staircase boundary.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W


def _curves(L):
    off = L["off"]
    for line in range(len(off) - 1):
        yield line, off[line], off[line + 1]


# ------------------------------------------------------------ G curves

def _Y(x):
    """int_0^x dt / (0.5 + 0.3 sin 2 pi t), by adaptive quadrature."""
    return quad(lambda t: 1.0 / (0.5 + 0.3 * math.sin(2.0 * math.pi * t)), 0.0, x,
                epsabs=1e-13, epsrel=1e-13, limit=200)[0]


def test_gamma_curves_of_sheared_field_follow_the_analytic_cross_flow_curves():
    """gamma = (beta2, -beta1) = (0.5 + 0.3 sin 2 pi x, -1): dy/dx = -1/beta2,
    so y + Y(x) is constant on every G curve.  The traced curves (bilinear
    beta, RK4) follow that to O(h^2), and run with x increasing, y decreasing."""
    devs = []
    for n in (33, 65):
        o = O.Oracle(W.sheared(n=n))
        L = o.lines(1)
        h = 1.0 / (n - 1)
        xs = np.unique(L["xi"] * h)
        Ytab = {x: _Y(x) for x in xs}
        dev = 0.0
        for _, a0, a1 in _curves(L):
            x, y = L["xi"][a0:a1] * h, L["eta"][a0:a1] * h
            if a1 - a0 >= 2:
                assert np.all(np.diff(x) > 0) and np.all(np.diff(y) < 0)
            C = y + np.array([Ytab[v] for v in x])
            dev = max(dev, C.max() - C.min())
        devs.append(dev)
    assert devs[1] < 2e-3 and devs[0] / devs[1] > 3.0, devs


def test_gamma_curves_are_orthogonal_to_the_flow():
    """Chords of consecutive G nodes are orthogonal to the exact beta at their
    midpoints (sheared field).  The nodes sit on the chords between RK4
    points, O(ds^2 kappa) off the curve, so a chord's direction is first order
    in h (the positions are second order: the test above)."""
    errs = []
    for n in (33, 65, 129):
        o = O.Oracle(W.sheared(n=n))
        L = o.lines(1)
        h = 1.0 / (n - 1)
        worst = 0.0
        for _, a0, a1 in _curves(L):
            x, y = L["xi"][a0:a1] * h, L["eta"][a0:a1] * h
            dx, dy = np.diff(x), np.diff(y)
            ln = np.hypot(dx, dy)
            ok = ln > 0.25 * h  # the last element can be short
            xm = 0.5 * (x[1:] + x[:-1])
            b1, b2 = np.ones_like(xm), 0.5 + 0.3 * np.sin(2 * math.pi * xm)
            cosang = (dx * b1 + dy * b2) / (ln * np.hypot(b1, b2))
            if ok.any():
                worst = max(worst, np.abs(cosang[ok]).max())
        errs.append(worst)
    assert errs[2] < 5e-4 and errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8, errs


def _data2d_polar(L, n):
    h = 1.0 / (n - 1)
    for _, a0, a1 in _curves(L):
        x, y = L["xi"][a0:a1] * h + 1.0, L["eta"][a0:a1] * h + 1.0
        yield np.hypot(x, y), np.arctan2(y, x)


def test_data2d_gamma_curves_are_rays_and_beta_curves_are_arcs():
    """beta = (-5(y+1), 5(x+1)) is linear, so its bilinear interpolant is exact;
    gamma = 5 (x+1, y+1) is radial from (-1, -1).  G curves are straight rays
    run outward; B curves are circles about (-1, -1) run counter-clockwise.
    Their seed and exit points are RK4 points, on the circle; the nodes between
    sit on chords of RK4 steps ds = h_s / 2, at most ds^2 / (8 r) inside it."""
    n = 33
    o = O.Oracle(W.data2d(n=n))
    assert not o.const_beta
    nG = nB = 0
    for r, a in _data2d_polar(o.lines(1), n):
        assert np.ptp(a) < 1e-12
        assert np.all(np.diff(r) > 0)
        nG += 1
    for r, a in _data2d_polar(o.lines(0), n):
        ds = 0.5 / (n - 1)
        assert abs(r[-1] - r[0]) < 1e-9
        assert np.all(r <= r[0] + 1e-12) and np.all(r >= r[0] - ds * ds / (8 * r[0]) - 1e-12)
        assert np.all(np.diff(a) > 0)
        nB += 1
    assert nG > 20 and nB > 20


def test_data2d_seeds_lie_on_the_inflow_sides():
    """Inflow (n . dir < 0): B enters through the right and bottom edges of the
    square, G through the left and bottom edges."""
    n = 33
    o = O.Oracle(W.data2d(n=n))
    top = n - 1
    for fam, sides in ((0, ("right", "bottom")), (1, ("left", "bottom"))):
        L = o.lines(fam)
        s = L["off"][:-1]
        X, Y = L["xi"][s], L["eta"][s]
        on = {"left": X == 0.0, "right": X == top, "bottom": Y == 0.0, "top": Y == top}
        inflow = np.zeros(len(s), bool)
        for side in sides:
            inflow |= on[side]
        assert inflow.all()


# --------------------------------------------------- map on traced curves

@pytest.mark.parametrize("name", ["sheared", "data2d"])
def test_map_reproduces_linear_functions_on_traced_families(name):
    """A linear field sampled at the curve nodes is linear along every curve
    segment and along every grid row and column, so the crossing values and
    both directional interpolants are exact: the map returns it at every
    interior node whose four crossings lie on curves."""
    n = 41
    p = W.sheared(n=n) if name == "sheared" else W.data2d(n=n)
    for weights in (0, 1):
        o = O.Oracle(p, interp_weights=weights)
        xi, eta = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float))
        for fam in (0, 1):
            L = o.lines(fam)
            vals = 0.4 + 0.7 * L["xi"] - 1.3 * L["eta"]
            g = o.map_to_grid(fam, vals)
            seg, _, _ = o.crossings(fam)
            ok = o.interior() & np.all(seg >= 0, axis=2)
            assert ok.sum() > 0.5 * o.interior().sum()
            np.testing.assert_allclose(g[ok], (0.4 + 0.7 * xi - 1.3 * eta)[ok], atol=1e-11)


# ------------------------------------------------------------- seeding

def _perforated(n, every):
    p = W.sheared(n=n)
    m = p.mask.copy()
    idx = np.arange(every // 2, n - 1, every)
    m[np.ix_(idx, idx)] = 0
    return W.Problem(n, n, p.mu, p.sigma, p.beta1, p.beta2, p.f, m)


def _boundary_walk(mask):
    """Directed boundary edges of the staircase domain (a cell is active when
    its 4 corner nodes are in the mask), domain on the left, walked loop by
    loop: each loop from its lowest, then leftmost, edge running in +x, loops
    in the order of those edges; at a node with two ways on, turn left first.
    Edges are (i, r, dx, dy) from node (i, r) in index coordinates."""
    ny, nx = mask.shape
    m = mask.astype(bool)
    act = m[:-1, :-1] & m[:-1, 1:] & m[1:, :-1] & m[1:, 1:]

    def cell(i, r):
        return 0 <= i < nx - 1 and 0 <= r < ny - 1 and bool(act[r, i])

    out = {}  # node -> outgoing boundary edges
    for r in range(ny):
        for i in range(nx - 1):
            up, dn = cell(i, r), cell(i, r - 1)
            if up != dn:
                e = (i, r, 1, 0) if up else (i + 1, r, -1, 0)
                out.setdefault(e[:2], []).append(e)
    for r in range(ny - 1):
        for i in range(nx):
            lf, rt = cell(i - 1, r), cell(i, r)
            if lf != rt:
                e = (i, r, 0, 1) if lf else (i, r + 1, 0, -1)
                out.setdefault(e[:2], []).append(e)
    starts = sorted((e for es in out.values() for e in es if e[2] == 1), key=lambda e: (e[1], e[0]))
    seen, order = set(), []
    for e0 in starts:
        if e0 in seen:
            continue
        e = e0
        while e not in seen:
            seen.add(e)
            order.append(e)
            i, r, dx, dy = e
            end = (i + dx, r + dy)
            cand = {(c[2], c[3]): c for c in out.get(end, [])}
            nxt = None
            for d in ((-dy, dx), (dx, dy), (dy, -dx)):  # left, straight, right
                if d in cand:
                    nxt = cand[d]
                    break
            if nxt is None:
                break
            e = nxt
    return order


def _inflow_weight(p, fam, e):
    """max(0, -n . dir) |e|, dir from the nodal mean of beta over the edge."""
    i, r, dx, dy = e
    A, B = (r, i), (r + dy, i + dx)
    m1 = 0.5 * (p.beta1[A] + p.beta1[B])
    m2 = 0.5 * (p.beta2[A] + p.beta2[B])
    nm = math.hypot(m1, m2)
    vx, vy = (m1 / nm, m2 / nm) if fam == 0 else (m2 / nm, -m1 / nm)
    nxo, nyo = dy, -dx  # outward normal: right of the walking direction
    hx, hy = (p.x1 - p.x0) / (p.nx - 1), (p.y1 - p.y0) / (p.ny - 1)
    return max(0.0, -(nxo * vx + nyo * vy)) * (hx if dx else hy)


@pytest.mark.parametrize("fam", [0, 1])
@pytest.mark.parametrize("every", [8, 5])
def test_seeds_on_a_domain_with_holes_follow_the_inflow_measure(fam, every):
    """On the square with 2 x 2-cell holes (one boundary loop each): the seed
    count is #{k >= 0 : (k + 1/2) h_s < total inflow measure}; every seed lies
    inside an edge with n . dir < 0; the k-th seed sits at cumulative measure
    (k + 1/2) h_s along the walk, so consecutive seeds are h_s apart."""
    n = 49
    p = _perforated(n, every)
    o = O.Oracle(p)
    hs = min((p.x1 - p.x0) / (p.nx - 1), (p.y1 - p.y0) / (p.ny - 1))
    order = _boundary_walk(p.mask)
    # a hole around node i spans cells i-1 and i: it joins the outer loop when
    # it touches the border (i = 1 or i = n - 2)
    inner = [i for i in range(every // 2, n - 1, every) if 1 < i < n - 2]
    holes = len(inner) ** 2
    loops = sum(1 for k in range(len(order)) if k == 0 or
                (order[k - 1][0] + order[k - 1][2], order[k - 1][1] + order[k - 1][3]) != order[k][:2])
    assert loops == holes + 1
    w = [_inflow_weight(p, fam, e) for e in order]
    cum = np.concatenate([[0.0], np.cumsum(w)])
    total = cum[-1]
    L = o.lines(fam)
    s = L["off"][:-1]
    X, Y = L["xi"][s], L["eta"][s]
    expect = int(math.floor(total / hs - 0.5)) + 1
    if (expect - 0.5) * hs >= total:
        expect -= 1
    assert len(s) == expect
    index = {(e[0], e[1], e[2], e[3]): k for k, e in enumerate(order)}
    for k in range(len(s)):
        x, y = X[k], Y[k]
        hit = None
        for e in order:
            i, r, dx, dy = e
            if dy == 0 and y == r and min(i, i + dx) < x < max(i, i + dx):
                hit = e
            elif dx == 0 and x == i and min(r, r + dy) < y < max(r, r + dy):
                hit = e
            if hit:
                break
        assert hit is not None, (k, x, y)
        q = index[hit]
        assert w[q] > 0.0
        i, r, dx, dy = hit
        phi = (x - i) * dx + (y - r) * dy  # fraction of the edge walked
        np.testing.assert_allclose(cum[q] + phi * w[q], (k + 0.5) * hs, rtol=0, atol=1e-12)
