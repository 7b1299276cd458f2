"""Seeded synthetic inputs for the 2D advection-diffusion-reaction workloads.

This module only draws and tabulates problem data (grids, masks, advection
fields, sources, initial states).  It holds none of the splitting method's
arithmetic, so both the CPU oracle's tests and the CUDA path's tests and bench
take their inputs from here.

Every array is row-major ``[ny][nx]`` over the nodes of a uniform grid that
includes the boundary nodes (an "N x N grid" means N x N nodes).
Random numbers come from numpy's PCG64 generator with an explicit seed.

Workloads (problem statement of the paper, §2, eqs. BVP1 / Parabolic1):

* ``manufactured``  -- 64^2, mu=0.1, sigma=1, beta=(1, 0.5), f such that
  u = sin(pi x) sin(pi y) solves -mu Lap u + beta.grad u + sigma u = f.
* ``sheared``       -- 2048^2, beta=(1, 0.5+0.3 sin 2 pi x) (divergence free),
  mu=1e-3, sigma=1, f = sum of 8 Gaussians of width 0.02 at seeded centres.
* ``parabolic``     -- 1024^2, beta as ``sheared``, mu=1e-2, sigma=0.5, f=0,
  u0 = Gaussian blob centred (0.25, 0.5) of width 0.05 (zero on the boundary).
* ``batch``         -- many problems with N uniform in 128..1024, masks from
  {square, disc, L}, mu = 10^U[-4,-1], sigma ~ U[0.1, 2], beta a constant unit
  vector of uniform direction, f = 8 Gaussians.
* ``learned``       -- 256^2 squares drawn like ``batch``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 2411
GAUSS_WIDTH = 0.02
N_GAUSS = 8
MASKS = ("square", "disc", "L")


@dataclasses.dataclass
class Problem:
    """One stationary or parabolic problem on a uniform grid of nodes."""

    nx: int
    ny: int
    mu: float
    sigma: float
    beta1: np.ndarray  # float64 [ny][nx]
    beta2: np.ndarray  # float64 [ny][nx]
    f: np.ndarray      # float64 [ny][nx]
    mask: np.ndarray   # uint8 [ny][nx]
    x0: float = 0.0
    y0: float = 0.0
    x1: float = 1.0
    y1: float = 1.0
    u0: np.ndarray | None = None
    name: str = ""

    @property
    def grid(self):
        return (self.nx, self.ny, self.x0, self.y0, self.x1, self.y1)


def node_coords(nx: int, ny: int, x0=0.0, y0=0.0, x1=1.0, y1=1.0):
    """Physical coordinates (X, Y) of the grid nodes, each [ny][nx]."""
    xs = x0 + (x1 - x0) * np.arange(nx, dtype=np.float64) / (nx - 1)
    ys = y0 + (y1 - y0) * np.arange(ny, dtype=np.float64) / (ny - 1)
    return np.meshgrid(xs, ys, indexing="xy")


def make_mask(kind: str, nx: int, ny: int) -> np.ndarray:
    """Node mask: 1 where the node lies in the closed domain."""
    X, Y = node_coords(nx, ny)
    if kind == "square":
        m = np.ones((ny, nx), dtype=bool)
    elif kind == "disc":
        m = (X - 0.5) ** 2 + (Y - 0.5) ** 2 <= 0.45 ** 2
    elif kind == "L":
        m = ~((X > 0.5) & (Y > 0.5))
    else:
        raise ValueError(kind)
    return m.astype(np.uint8)


def gaussian_sources(nx: int, ny: int, centres: np.ndarray, width=GAUSS_WIDTH):
    """Sum of unit-amplitude Gaussians exp(-|x-c|^2 / (2 w^2))."""
    X, Y = node_coords(nx, ny)
    f = np.zeros((ny, nx), dtype=np.float64)
    for cx, cy in centres:
        f += np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * width * width))
    return f


def sheared_beta(nx: int, ny: int):
    """beta = (1, 0.5 + 0.3 sin 2 pi x): divergence free."""
    X, _ = node_coords(nx, ny)
    return np.ones((ny, nx)), 0.5 + 0.3 * np.sin(2.0 * math.pi * X)


def manufactured(n=64, mu=0.1, sigma=1.0, beta=(1.0, 0.5), mask="square"):
    """f for the exact solution u = sin(pi x) sin(pi y)."""
    X, Y = node_coords(n, n)
    pi = math.pi
    u = np.sin(pi * X) * np.sin(pi * Y)
    ux = pi * np.cos(pi * X) * np.sin(pi * Y)
    uy = pi * np.sin(pi * X) * np.cos(pi * Y)
    f = 2.0 * mu * pi * pi * u + beta[0] * ux + beta[1] * uy + sigma * u
    return Problem(n, n, mu, sigma, np.full((n, n), float(beta[0])),
                   np.full((n, n), float(beta[1])), f, make_mask(mask, n, n),
                   name=f"manufactured{n}")


def exact_manufactured(n: int):
    X, Y = node_coords(n, n)
    return np.sin(math.pi * X) * np.sin(math.pi * Y)


def sheared(n=2048, mu=1e-3, sigma=1.0, seed=SEED_BASE + 1):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(0.1, 0.9, size=(N_GAUSS, 2))
    b1, b2 = sheared_beta(n, n)
    f = gaussian_sources(n, n, centres)
    return Problem(n, n, mu, sigma, b1, b2, f, make_mask("square", n, n),
                   name=f"sheared{n}")


def parabolic(n=1024, mu=1e-2, sigma=0.5):
    b1, b2 = sheared_beta(n, n)
    X, Y = node_coords(n, n)
    u0 = np.exp(-((X - 0.25) ** 2 + (Y - 0.5) ** 2) / (2.0 * 0.05 ** 2))
    u0[0, :] = u0[-1, :] = 0.0
    u0[:, 0] = u0[:, -1] = 0.0
    return Problem(n, n, mu, sigma, b1, b2, np.zeros((n, n)),
                   make_mask("square", n, n), u0=u0, name=f"parabolic{n}")


def random_problem(rng: np.random.Generator, n: int, mask: str | None = None):
    """One problem drawn as in the batched and learned workloads."""
    if mask is None:
        mask = MASKS[int(rng.integers(0, len(MASKS)))]
    mu = 10.0 ** rng.uniform(-4.0, -1.0)
    sigma = rng.uniform(0.1, 2.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    centres = rng.uniform(0.1, 0.9, size=(N_GAUSS, 2))
    f = gaussian_sources(n, n, centres)
    return Problem(n, n, float(mu), float(sigma),
                   np.full((n, n), math.cos(phi)), np.full((n, n), math.sin(phi)),
                   f, make_mask(mask, n, n), name=f"rand{n}{mask}")


def batch(count=256, nmin=128, nmax=1024, seed=SEED_BASE + 3):
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        out.append(random_problem(rng, n))
    return out


def learned(count, n=256, seed=SEED_BASE + 4):
    rng = np.random.Generator(np.random.PCG64(seed))
    return [random_problem(rng, n, mask="square") for _ in range(count)]


def random_field(rng: np.random.Generator, nx: int, ny: int, smooth=True):
    """A smooth random nodal field (sum of a few low Fourier modes)."""
    X, Y = node_coords(nx, ny)
    g = np.zeros((ny, nx))
    for _ in range(4):
        kx, ky = rng.integers(1, 4, size=2)
        a, px, py = rng.normal(), rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
        g += a * np.sin(kx * math.pi * X + px) * np.sin(ky * math.pi * Y + py)
    return g


# warm-start network: layer widths (input features ... output channels)
CNN_CHANNELS = (40, 64, 64, 128, 128, 128, 64, 64, 8)


def cnn_init_params(seed=SEED_BASE + 6, last_scale=0.1):
    """Initial parameters of the warm-start network, packed W_0, b_0, W_1, ...:
    He-normal weights (std sqrt(2 / (9 Cin))), zero biases, the last layer's
    weights scaled by ``last_scale``.  FP32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ch = CNN_CHANNELS
    parts = []
    for l in range(len(ch) - 1):
        n = 9 * ch[l] * ch[l + 1]
        std = math.sqrt(2.0 / (9 * ch[l])) * (last_scale if l == len(ch) - 2 else 1.0)
        parts.append(rng.normal(0.0, std, n))
        parts.append(np.zeros(ch[l + 1]))
    return np.concatenate(parts).astype(np.float32)


def data2d(n=61):
    """The paper's numerical experiment (eq. Data2D): unit square, mu = 1,
    beta = (-5(y+1), 5(x+1)), sigma = 1, f = 5, on n x n nodes."""
    X, Y = node_coords(n, n)
    return Problem(n, n, 1.0, 1.0, -5.0 * (Y + 1.0), 5.0 * (X + 1.0), np.full((n, n), 5.0),
                   make_mask("square", n, n), name=f"data2d{n}")
