"""Pins of the warm-start network's CPU reference: central finite differences
of the loss, a brute-force convolution, the feature map, the targets and the
unpacking to the grid."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W

CNN = O.CNN


def _batch(n=2, seed=0, hw=64):
    rng = np.random.default_rng(seed)
    xs = rng.normal(size=(n, hw, hw, 40)) * 0.5
    ts = rng.normal(size=(n, hw, hw))
    return xs, ts


@pytest.fixture
def small_grid():
    CNN.set_size(16, 16)
    yield 16
    CNN.set_size(64, 64)


def test_parameter_count_is_about_half_a_million():
    ch = CNN.channels()
    assert ch[0] == 40 and ch[-1] == 8 and CNN.dilations() == [1, 2, 4, 8, 16, 32, 1, 1]
    n = CNN.num_params()
    assert n == sum(9 * a * b + b for a, b in zip(ch[:-1], ch[1:]))
    assert 450_000 < n < 600_000


def test_gradient_matches_central_differences(small_grid):
    """Central differences of the loss against the analytic gradient.  A
    sample whose forward and backward one-sided differences disagree sits next
    to a ReLU kink and is skipped; the others must agree to 2e-3 (the loss's
    own rounding, about 1e-12, limits the difference quotients).  Run on a
    16 x 16 grid (the layers do not depend on the size)."""
    xs, ts = _batch(2, hw=small_grid)
    p = CNN.init_params(3)
    loss, g = CNN.loss_grad(p, xs, ts)
    rng = np.random.default_rng(1)
    checked = 0
    for l in range(CNN.LAYERS):
        for bias in (False, True):
            lo = CNN.offset(l, bias)
            hi = CNN.offset(l, True) if not bias else CNN.offset(l + 1)
            cand = rng.integers(lo, hi, size=40)
            cand = cand[np.argsort(-np.abs(g[cand]))][:3]
            for k in cand:
                if abs(g[k]) < 1e-7:
                    continue
                eps = 1e-5 * max(1.0, abs(p[k]))
                q = p.copy()
                q[k] += eps
                lp, _ = CNN.loss_grad(q, xs, ts, False)
                q[k] -= 2 * eps
                lm, _ = CNN.loss_grad(q, xs, ts, False)
                fwd, bwd, fd = (lp - loss) / eps, (loss - lm) / eps, (lp - lm) / (2 * eps)
                if abs(fwd - bwd) > 2e-3 * abs(g[k]):
                    continue  # a kink within eps
                assert abs(fd - g[k]) <= 2e-3 * abs(g[k]), (l, bias, k, fd, g[k])
                checked += 1
    assert checked >= 12, checked


def test_first_layer_equals_brute_force_convolution():
    """One layer against a direct numpy convolution with zero padding."""
    xs, _ = _batch(1)
    x = xs[0]
    p = np.zeros(CNN.num_params())
    rng = np.random.default_rng(4)
    ch = CNN.channels()
    Wl = rng.normal(size=(3, 3, ch[0], ch[1]))
    bl = rng.normal(size=ch[1])
    p[CNN.offset(0):CNN.offset(0, True)] = Wl.reshape(-1)
    p[CNN.offset(0, True):CNN.offset(1)] = bl
    # identity-like rest: route channel 0 of layer 0 to output channel 0
    # through unit centre taps, so that the output equals relu(layer0)[..., 0]
    for l in range(1, CNN.LAYERS):
        w = np.zeros((3, 3, ch[l], ch[l + 1]))
        w[1, 1, 0, 0] = 1.0
        p[CNN.offset(l):CNN.offset(l, True)] = w.reshape(-1)
    out = CNN.forward(p, x)
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    ref = np.zeros((64, 64, ch[1]))
    for ky in range(3):
        for kx in range(3):
            ref += np.einsum("rci,io->rco", xp[ky:ky + 64, kx:kx + 64], Wl[ky, kx])
    ref += bl
    np.testing.assert_allclose(out[..., 0], np.maximum(ref[..., 0], 0.0), rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(out[..., 1:], 0.0)


def test_dilated_layer_reads_the_taps_it_should():
    """A single unit weight at tap (ky, kx) of the dilation-32 layer shifts
    the map by (ky - 1, kx - 1) * 32 cells (zero where the tap leaves the grid)."""
    ch = CNN.channels()
    assert CNN.dilations()[5] == 32
    rng = np.random.default_rng(5)
    x = np.abs(rng.normal(size=(64, 64, ch[0])))
    for ky, kx in ((0, 2), (2, 1)):
        p = np.zeros(CNN.num_params())
        for l in range(CNN.LAYERS):
            w = np.zeros((3, 3, ch[l], ch[l + 1]))
            if l == 5:
                w[ky, kx, 0, 0] = 1.0
            else:
                w[1, 1, 0, 0] = 1.0
            p[CNN.offset(l):CNN.offset(l, True)] = w.reshape(-1)
        out = CNN.forward(p, x)[..., 0]
        dy, dx = (ky - 1) * 32, (kx - 1) * 32
        ref = np.zeros((64, 64))
        for r in range(64):
            for c in range(64):
                if 0 <= r + dy < 64 and 0 <= c + dx < 64:
                    ref[r, c] = x[r + dy, c + dx, 0]
        np.testing.assert_allclose(out, ref, rtol=0, atol=0)


def test_features_target_and_upsampling():
    p = W.random_problem(np.random.default_rng(2), 256, mask="disc")
    u0 = np.random.default_rng(5).normal(size=(256, 256))
    s0 = np.abs(u0).max()
    assert CNN.scale(u0) == s0 and CNN.scale(None) == 1.0 and CNN.scale(0 * u0) == 1.0
    x = CNN.features(p, u0)
    blocks = lambda a: a.reshape(64, 4, 64, 4).transpose(0, 2, 1, 3)  # [r][c][a][b]
    np.testing.assert_array_equal(x[..., :16], blocks(p.f).reshape(64, 64, 16))
    np.testing.assert_array_equal(x[..., 16:32], blocks(u0 / s0).reshape(64, 64, 16))
    np.testing.assert_allclose(x[..., 32], blocks(p.beta1).mean(axis=(2, 3)), rtol=1e-14)
    np.testing.assert_allclose(x[..., 33], blocks(p.beta2).mean(axis=(2, 3)), rtol=1e-14)
    assert np.allclose(x[..., 34], (np.log10(p.mu) + 2.5) / 1.5) and np.allclose(x[..., 35], p.sigma - 1)
    np.testing.assert_allclose(x[..., 36], blocks(p.mask.astype(float)).mean(axis=(2, 3)))
    assert np.all(x[..., 37:] == 0)
    assert np.all(CNN.features(p)[..., 16:32] == 0)  # no first state: zeros
    # target: cell means of (u - u0) / s
    u = np.random.default_rng(3).normal(size=(256, 256))
    np.testing.assert_allclose(CNN.target(u, u0), blocks(u - u0).mean(axis=(2, 3)) / s0,
                               rtol=1e-12, atol=1e-14)
    # a bilinear correction d: its cell means are its values at the cell
    # centres, and the bilinear interpolation through them gives d back
    # inside (the outer half cells are clamped)
    X, Y = W.node_coords(256, 256)
    d = 0.3 + 2.0 * X - 1.5 * Y + 0.7 * X * Y
    t = CNN.target(u0 + d, u0)
    y = np.zeros((64, 64, 8))
    y[..., 0] = t
    y[..., 1:] = 123.0  # channels 1..7 are not read
    inter = (np.random.default_rng(4).random((256, 256)) < 0.7).astype(np.uint8)
    back = CNN.upsample(y, inter, u0)
    ref = np.where(inter == 1, u0 + d, 0.0)
    assert np.abs(back - ref)[2:-2, 2:-2].max() < 1e-12
