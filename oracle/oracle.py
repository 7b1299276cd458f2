"""ctypes wrapper of the FP64 CPU oracle (``adr_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this module; the product package never imports
it.  Arrays are numpy float64 / uint8, row-major ``[ny][nx]``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "adr_oracle.c")
SRCS = [SRC, os.path.join(HERE, "cnn_oracle.c")]
LIB = os.path.join(HERE, "liboracle.so")

OK, EINVAL, ENOMEM, ENOCONV, EGEOM = 0, 1, 2, 4, 5
OUTSIDE, DIRICHLET, INTERIOR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    deps = SRCS + [os.path.join(HERE, "adr_oracle.h")]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(map(os.path.getmtime, deps)):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", LIB, *SRCS, "-lm"])
    return LIB


_lib = None
dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                 C.c_double, up, C.c_double, C.c_double, dp, dp, dp,
                                 C.POINTER(vp)]
        L.orc_destroy.argtypes = [vp]
        L.orc_const_beta.argtypes = [vp]
        L.orc_set_interp_weights.argtypes = [vp, C.c_int]
        L.orc_set_interp_weights.restype = None
        L.orc_set_stabilization.argtypes = [vp, C.c_int]
        L.orc_set_stabilization.restype = None
        L.orc_node_types.argtypes = [vp, up]
        L.orc_num_lines.argtypes = [vp, C.c_int]
        L.orc_num_line_nodes.argtypes = [vp, C.c_int]
        L.orc_lines.argtypes = [vp, C.c_int, ip, dp, dp, dp, dp, dp]
        L.orc_crossings.argtypes = [vp, C.c_int, ip, dp, dp]
        L.orc_bilinear.argtypes = [vp, dp, C.c_double, C.c_double]
        L.orc_bilinear.restype = C.c_double
        L.orc_gather.argtypes = [vp, C.c_int, dp, dp]
        L.orc_map_to_grid.argtypes = [vp, C.c_int, dp, dp]
        L.orc_line_system.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, dp,
                                      C.c_double, dp, dp, dp, dp, dp]
        L.orc_thomas.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.orc_dense_lu_solve.argtypes = [C.c_int, dp, dp]
        L.orc_sweep_lines.argtypes = [vp, C.c_int, C.c_double, C.c_double, dp, C.c_double,
                                      dp, vp, C.c_double, dp]
        L.orc_sweep_lines.restype = C.c_double
        L.orc_split_step.argtypes = [vp, C.c_double, C.c_double, C.c_double, vp, C.c_double,
                                     dp, dp, dp]
        L.orc_default_dt.argtypes = [vp, C.c_double]
        L.orc_default_dt.restype = C.c_double
        L.orc_solve_stationary.argtypes = [vp, C.c_double, C.c_double, C.c_double, C.c_int,
                                           C.c_int, vp, C.c_double, vp, C.c_double, dp, vp,
                                           C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.orc_paper_u0.argtypes = [vp, dp]
        L.orc_set_transfer.argtypes = [vp, C.c_int]
        L.orc_transfer.argtypes = [vp, C.c_int, dp, dp]
        L.orc_transfer.restype = None
        L.orc_transfer_table.argtypes = [vp, C.c_int, ip, dp, dp]
        L.orc_transfer_table.restype = None
        L.orc_sweep_line_values.argtypes = [vp, C.c_int, C.c_double, C.c_double, dp, C.c_double,
                                            vp, C.c_double, dp]
        L.orc_sweep_line_values.restype = C.c_double
        L.orc_set_anderson.argtypes = [vp, C.c_int]
        L.orc_anderson_linear.argtypes = [C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_double, dp]
        L.orc_step_parabolic.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.c_double,
                                         C.c_double, C.c_double, C.c_int, dp,
                                         C.POINTER(C.c_int)]
        L.cnn_num_params.restype = C.c_long
        L.cnn_set_size.argtypes = [C.c_int, C.c_int]
        L.cnn_set_size.restype = None
        L.cnn_param_offset.argtypes = [C.c_int, C.c_int]
        L.cnn_param_offset.restype = C.c_long
        L.cnn_channels.argtypes = [C.c_int]
        L.cnn_dilation.argtypes = [C.c_int]
        L.cnn_scale.argtypes = [C.c_int, vp]
        L.cnn_scale.restype = C.c_double
        L.cnn_features.argtypes = [C.c_int, dp, dp, dp, up, C.c_double, C.c_double, vp,
                                   C.c_double, dp]
        L.cnn_target.argtypes = [C.c_int, dp, vp, C.c_double, dp]
        L.cnn_forward.argtypes = [dp, dp, vp, dp]
        L.cnn_loss_grad.argtypes = [dp, C.c_int, dp, dp, vp]
        L.cnn_loss_grad.restype = C.c_double
        L.cnn_upsample.argtypes = [C.c_int, dp, vp, C.c_double, up, dp]
        for fn in ("orc_q1_dense", "orc_p1_dense"):
            getattr(L, fn).argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, up, C.c_double, C.c_double, dp, dp, dp, dp]
        _lib = L
    return _lib


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def _opt(a):
    return None if a is None else _c(a)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


class Oracle:
    """One problem in the oracle.  Mirrors the library's handle."""

    def __init__(self, prob, interp_weights=0, stabilize=0, transfer=0, anderson=0):
        self.prob = prob
        self.nx, self.ny = prob.nx, prob.ny
        self.mask = _c(prob.mask, np.uint8)
        self.beta1, self.beta2, self.f = _c(prob.beta1), _c(prob.beta2), _c(prob.f)
        h = C.c_void_p()
        st = lib().orc_create(prob.nx, prob.ny, prob.x0, prob.y0, prob.x1, prob.y1,
                              self.mask, prob.mu, prob.sigma, self.beta1, self.beta2,
                              self.f, C.byref(h))
        if st != OK:
            raise OracleError(st, "orc_create")
        self.h = h
        if interp_weights:
            lib().orc_set_interp_weights(h, 1)
        if stabilize:
            lib().orc_set_stabilization(h, 1)
        if transfer:
            st = lib().orc_set_transfer(h, int(transfer))
            if st != OK:
                raise OracleError(st, "orc_set_transfer")
        if anderson:
            st = lib().orc_set_anderson(h, int(anderson))
            if st != OK:
                raise OracleError(st, "orc_set_anderson")

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # geometry
    @property
    def const_beta(self):
        return bool(lib().orc_const_beta(self.h))

    def node_types(self):
        out = np.zeros((self.ny, self.nx), np.uint8)
        lib().orc_node_types(self.h, out)
        return out

    def interior(self):
        return self.node_types() == INTERIOR

    def lines(self, fam):
        L = lib()
        nl, nn = L.orc_num_lines(self.h, fam), L.orc_num_line_nodes(self.h, fam)
        off = np.zeros(nl + 1, np.int32)
        xi, eta, bn, fv = (np.zeros(nn) for _ in range(4))
        h = np.zeros(max(nl, 1))
        L.orc_lines(self.h, fam, off, xi, eta, bn, fv, h)
        return dict(off=off, xi=xi, eta=eta, bnorm=bn, fval=fv, h=h[:nl])

    def crossings(self, fam):
        n = 4 * self.nx * self.ny
        seg, t, pos = np.zeros(n, np.int32), np.zeros(n), np.zeros(n)
        lib().orc_crossings(self.h, fam, seg, t, pos)
        s = (self.ny, self.nx, 4)
        return seg.reshape(s), t.reshape(s), pos.reshape(s)

    def transfer_table(self, fam):
        """Direct-transfer crossings of family fam's nodes: (seg, t, pos), each
        [n_nodes, 2] (left, right)."""
        n = 2 * lib().orc_num_line_nodes(self.h, fam)
        seg, t, pos = np.zeros(n, np.int32), np.zeros(n), np.zeros(n)
        lib().orc_transfer_table(self.h, fam, seg, t, pos)
        return seg.reshape(-1, 2), t.reshape(-1, 2), pos.reshape(-1, 2)

    def transfer(self, to_fam, vals):
        out = np.zeros(lib().orc_num_line_nodes(self.h, to_fam))
        lib().orc_transfer(self.h, to_fam, _c(vals), out)
        return out

    def sweep_line_values(self, fam, theta, dt, u_vals, sigma=None):
        d = np.zeros(lib().orc_num_line_nodes(self.h, fam) + 1)
        sig = self.prob.sigma if sigma is None else sigma
        piv = lib().orc_sweep_line_values(self.h, fam, theta, dt, _c(u_vals), sig, None, 0.0, d)
        return d[:-1], piv

    # steps
    def bilinear(self, grid, xi, eta):
        return lib().orc_bilinear(self.h, _c(grid), float(xi), float(eta))

    def gather(self, fam, grid):
        out = np.zeros(lib().orc_num_line_nodes(self.h, fam))
        lib().orc_gather(self.h, fam, _c(grid), out)
        return out

    def map_to_grid(self, fam, vals):
        out = np.zeros((self.ny, self.nx))
        lib().orc_map_to_grid(self.h, fam, _c(vals), out)
        return out

    def line_system(self, fam, line, theta, dt, u_line, f_line, sigma=None):
        n = len(u_line) - 1
        m = max(n - 1, 1)
        a, b, c, r = (np.zeros(m) for _ in range(4))
        sig = self.prob.sigma if sigma is None else sigma
        k = lib().orc_line_system(self.h, fam, line, theta, dt, _c(u_line), sig, _c(f_line),
                                  a, b, c, r)
        return a[:k], b[:k], c[:k], r[:k]

    def sweep_lines(self, fam, theta, dt, u_grid, sigma=None):
        d = np.zeros(lib().orc_num_line_nodes(self.h, fam) + 1)
        sig = self.prob.sigma if sigma is None else sigma
        piv = lib().orc_sweep_lines(self.h, fam, theta, dt, _c(u_grid), sig, self.f, None,
                                    0.0, d)
        return d[:-1], piv

    def split_step(self, theta, dt, u, sigma=None, f_extra=None, fx_scale=0.0):
        uh, un = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        sig = self.prob.sigma if sigma is None else sigma
        fx = None if f_extra is None else _c(f_extra)
        lib().orc_split_step(self.h, theta, dt, sig, _ptr(fx), fx_scale, _c(u), uh, un)
        return uh, un

    def default_dt(self, sigma=None):
        return lib().orc_default_dt(self.h, self.prob.sigma if sigma is None else sigma)

    def paper_u0(self):
        out = np.zeros((self.ny, self.nx))
        lib().orc_paper_u0(self.h, out)
        return out

    def solve_stationary(self, theta=0.5, dt=0.0, tol=1e-10, max_iter=100000, init=0,
                         u_init=None, sigma=None, f_extra=None, fx_scale=0.0):
        """Returns (u_out, u_iter, iters, rel, status)."""
        out, it_out = np.zeros((self.ny, self.nx)), np.zeros((self.ny, self.nx))
        ui = None if u_init is None else _c(u_init)
        fx = None if f_extra is None else _c(f_extra)
        iters, rel = C.c_int(0), C.c_double(0)
        sig = self.prob.sigma if sigma is None else sigma
        st = lib().orc_solve_stationary(self.h, theta, dt, tol, max_iter, init, _ptr(ui), sig,
                                        _ptr(fx), fx_scale, out, _ptr(it_out), C.byref(iters),
                                        C.byref(rel))
        return out, it_out, iters.value, rel.value, st

    def step_parabolic(self, u0, dt, nsteps, mode, theta=0.5, pseudo_dt=0.0, tol=1e-8,
                       max_iter=100000):
        u = _c(u0).copy()
        tot = C.c_int(0)
        st = lib().orc_step_parabolic(self.h, dt, nsteps, mode, theta, pseudo_dt, tol, max_iter,
                                      u, C.byref(tot))
        return u, tot.value, st


def anderson_linear(T, c, x0, m, max_iter=200, tol=1e-13):
    """The oracle's Anderson extrapolation (depth m) on g(x) = T x + c from x0.
    Returns (x, number of maps applied, relative updates per map)."""
    n = len(c)
    x = _c(x0).copy()
    res = np.zeros(max_iter)
    k = lib().orc_anderson_linear(n, int(m), _c(T), _c(c), x, int(max_iter), float(tol), res)
    return x, k, res[:max(k, 0)]


def thomas(a, b, c, r):
    x = np.zeros(len(b))
    st = lib().orc_thomas(len(b), _c(a), _c(b), _c(c), _c(r), x)
    if st:
        raise OracleError(st, "thomas")
    return x


def dense_lu_solve(A, b):
    A2, b2 = _c(A).copy(), _c(b).copy()
    st = lib().orc_dense_lu_solve(len(b2), A2, b2)
    if st:
        raise OracleError(st, "dense_lu_solve")
    return b2


def _dense(fn, prob, mu=None, sigma=None, f=None):
    u = np.zeros((prob.ny, prob.nx))
    st = fn(prob.nx, prob.ny, prob.x0, prob.y0, prob.x1, prob.y1, _c(prob.mask, np.uint8),
            prob.mu if mu is None else mu, prob.sigma if sigma is None else sigma,
            _c(prob.beta1), _c(prob.beta2), _c(prob.f if f is None else f), u)
    if st:
        raise OracleError(st, "dense FEM")
    return u


def q1_dense(prob, **kw):
    return _dense(lib().orc_q1_dense, prob, **kw)


def p1_dense(prob, **kw):
    return _dense(lib().orc_p1_dense, prob, **kw)


# ------------------------------------------------------------ warm-start net

class CNN:
    """FP64 reference of the warm-start network (cnn_oracle.c)."""
    H = W = 64
    LAYERS = 8

    @staticmethod
    def num_params():
        return lib().cnn_num_params()

    @staticmethod
    def channels():
        return [lib().cnn_channels(l) for l in range(CNN.LAYERS + 1)]

    @staticmethod
    def dilations():
        return [lib().cnn_dilation(l) for l in range(CNN.LAYERS)]

    @staticmethod
    def offset(l, bias=False):
        return lib().cnn_param_offset(l, int(bias))

    @staticmethod
    def scale(u0):
        """max |u0| over the grid (1 for None or zero)."""
        u0c = _opt(u0)
        return lib().cnn_scale(0 if u0c is None else u0c.shape[0], _ptr(u0c))

    @staticmethod
    def features(prob, u0=None):
        """[H][W][40] features of a problem on a (4 H) x (4 W) grid, with its
        first initial state u0 (None: zeros)."""
        x = np.zeros((CNN.H, CNN.W, 40))
        u0c = _opt(u0)
        lib().cnn_features(prob.nx, _c(prob.f), _c(prob.beta1), _c(prob.beta2),
                           _c(prob.mask, np.uint8), prob.mu, prob.sigma, _ptr(u0c),
                           CNN.scale(u0), x)
        return x

    @staticmethod
    def target(u, u0=None):
        """[H][W]: the cell means of (u - u0) / max |u0|."""
        t = np.zeros((CNN.H, CNN.W))
        u0c = _opt(u0)
        lib().cnn_target(u.shape[0], _c(u), _ptr(u0c), CNN.scale(u0), t)
        return t

    @staticmethod
    def forward(params, x):
        """The last layer's output [H][W][8]."""
        out = np.zeros((CNN.H, CNN.W, 8))
        lib().cnn_forward(_c(params), _c(x), None, out)
        return out

    @staticmethod
    def set_size(h, w):
        CNN.H, CNN.W = int(h), int(w)
        lib().cnn_set_size(int(h), int(w))

    @staticmethod
    def loss_grad(params, xs, ts, want_grad=True):
        g = np.zeros(CNN.num_params()) if want_grad else None
        loss = lib().cnn_loss_grad(_c(params), len(xs), _c(xs), _c(ts), _ptr(g))
        return loss, g

    @staticmethod
    def upsample(y, interior, u0=None):
        """Initial state u0 + max|u0| * bilinear(y[..., 0]) on the (4 H) x (4 W)
        grid from one output [H][W][8]."""
        n = 4 * CNN.W
        u = np.zeros((4 * CNN.H, n))
        u0c = _opt(u0)
        lib().cnn_upsample(n, _c(y), _ptr(u0c), CNN.scale(u0), _c(interior, np.uint8), u)
        return u

    @staticmethod
    def init_params(seed=0):
        """He-normal weights, zero biases (the last layer scaled down)."""
        rng = np.random.default_rng(seed)
        p = np.zeros(CNN.num_params())
        ch = CNN.channels()
        for l in range(CNN.LAYERS):
            n = 9 * ch[l] * ch[l + 1]
            std = np.sqrt(2.0 / (9 * ch[l])) * (0.1 if l == CNN.LAYERS - 1 else 1.0)
            p[CNN.offset(l):CNN.offset(l) + n] = rng.normal(0, std, n)
        return p
