"""Pins of the warm-start network's CPU reference: central finite differences
of the loss, a brute-force convolution, the feature map and the upsampling."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_11041_gb300 import workloads as W

CNN = O.CNN


def _batch(n=2, seed=0, hw=64):
    rng = np.random.default_rng(seed)
    xs = rng.normal(size=(n, hw, hw, 8)) * 0.5
    ts = rng.normal(size=(n, hw, hw))
    return xs, ts


@pytest.fixture
def small_grid():
    CNN.set_size(16, 16)
    yield 16
    CNN.set_size(64, 64)


def test_parameter_count_is_about_half_a_million():
    ch = CNN.channels()
    assert ch[0] == 8 and ch[-1] == 8 and CNN.dilations() == [1, 2, 4, 8, 4, 2, 1, 1]
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
    Wl = rng.normal(size=(3, 3, 8, 64))
    bl = rng.normal(size=64)
    p[CNN.offset(0):CNN.offset(0, True)] = Wl.reshape(-1)
    p[CNN.offset(0, True):CNN.offset(1)] = bl
    # identity-like rest: route channel 0 of layer 0 to the output through
    # positive weights so that the output equals relu(layer0)[..., 0]
    ch = CNN.channels()
    for l in range(1, CNN.LAYERS):
        w = np.zeros((3, 3, ch[l], ch[l + 1]))
        w[1, 1, 0, 0] = 1.0
        p[CNN.offset(l):CNN.offset(l, True)] = w.reshape(-1)
    out = CNN.forward(p, x)
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    ref = np.zeros((64, 64, 64))
    for ky in range(3):
        for kx in range(3):
            ref += np.einsum("rci,io->rco", xp[ky:ky + 64, kx:kx + 64], Wl[ky, kx])
    ref += bl
    np.testing.assert_allclose(out, np.maximum(ref[..., 0], 0.0), rtol=1e-12, atol=1e-12)


def test_features_target_and_upsampling():
    p = W.random_problem(np.random.default_rng(2), 256, mask="square")
    x = CNN.features(p)
    assert np.allclose(x[..., 0], p.f.reshape(64, 4, 64, 4).mean(axis=(1, 3)))
    assert np.allclose(x[..., 3], (np.log10(p.mu) + 2.5) / 1.5) and np.allclose(x[..., 6:], 0)
    u = np.outer(np.linspace(0, 1, 256), np.linspace(0, 2, 256))
    t = CNN.target(u, 2.0)
    assert np.allclose(t, 2.0 * u.reshape(64, 4, 64, 4).mean(axis=(1, 3)))
    inter = np.ones((256, 256), np.uint8)
    up = CNN.upsample(t, 2.0, inter)
    # bilinear through the cell centres reproduces the bilinear field inside
    assert np.abs(up[4:-4, 4:-4] - u[4:-4, 4:-4]).max() < 1e-12
