"""Python binding of the GB300 directional diffusion splitting library.

Thin ctypes marshalling over ``libadr.so`` (C ABI in ``include/adr.h``): the
functions below carry the C names and only move pointers, sizes and structs.
Every step of the method runs in the library's CUDA kernels; there is no CPU
path, and importing the binding fails loudly when the library is missing.

Device memory and streams come from PyTorch: arrays are CUDA tensors
(float64 grids ``[ny][nx]``, uint8 masks) and the stream is torch's current
CUDA stream unless one is given.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadr.so")

ADR_OK, ADR_EINVAL, ADR_ENOMEM, ADR_ECUDA, ADR_ENOCONV, ADR_EGEOM, ADR_ETIMEOUT = range(7)
ADR_FP64, ADR_FP32_REFINE = 0, 1
ADR_INIT_ZERO, ADR_INIT_USER, ADR_INIT_PAPER_U0, ADR_INIT_LEARNED = 0, 1, 2, 3
STATUS_NAMES = {0: "ADR_OK", 1: "ADR_EINVAL", 2: "ADR_ENOMEM", 3: "ADR_ECUDA", 4: "ADR_ENOCONV",
                5: "ADR_EGEOM", 6: "ADR_ETIMEOUT"}


class adr_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("x1", C.c_double), ("y1", C.c_double)]


class adr_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("theta", C.c_double), ("dt", C.c_double),
                ("tol", C.c_double), ("max_iter", C.c_int), ("init", C.c_int),
                ("rows_per_thread", C.c_int), ("map_blocks_per_sm", C.c_int),
                ("interp_weights", C.c_int), ("stabilize", C.c_int), ("transfer", C.c_int),
                ("anderson", C.c_int)]


class adr_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_update", C.c_double), ("ms", C.c_double),
                ("line_dofs", C.c_double), ("dt", C.c_double), ("min_pivot", C.c_double),
                ("max_correction", C.c_double), ("fp32_steps", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AdrError(RuntimeError):
    def __init__(self, status, what):
        msg = lib().adr_last_error().decode(errors="replace")
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libadr.so (built by ``paper_2411_11041_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2411_11041_gb300/build.py "
                              "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
        L.adr_default_opts.argtypes = [C.POINTER(adr_opts)]
        L.adr_default_opts.restype = None
        L.adr_last_error.restype = C.c_char_p
        L.adr_create.argtypes = [C.POINTER(adr_grid), vp, C.c_double, C.c_double, vp, vp, vp,
                                 C.POINTER(adr_opts), vp, C.POINTER(vp)]
        L.adr_solve_stationary.argtypes = [vp, vp, vp, vp, C.POINTER(adr_stats)]
        L.adr_step_parabolic.argtypes = [vp, C.c_double, C.c_int, C.c_int, vp,
                                         C.POINTER(adr_stats)]
        L.adr_destroy.argtypes = [vp]
        L.adr_destroy.restype = None
        L.adr_num_lines.argtypes = [vp, C.c_int]
        L.adr_num_line_nodes.argtypes = [vp, C.c_int]
        L.adr_get_lines.argtypes = [vp, C.c_int, ip, dp, dp, dp]
        L.adr_get_crossings.argtypes = [vp, C.c_int, ip, dp, dp]
        L.adr_get_transfer.argtypes = [vp, C.c_int, ip, dp, dp]
        L.adr_split_step.argtypes = [vp, C.c_double, vp, vp, vp]
        L.adr_paper_u0.argtypes = [vp, vp]
        L.adr_time_kernels.argtypes = [vp, C.c_int, dp]
        L.adr_autotune.argtypes = [vp, C.c_int, ip, ip, dp]
        L.adr_batch_create.argtypes = [C.POINTER(vp), C.c_int, vp, C.POINTER(vp)]
        L.adr_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                      C.POINTER(adr_stats)]
        L.adr_batch_destroy.argtypes = [vp]
        L.adr_batch_destroy.restype = None
        L.adr_batch_autotune.argtypes = [vp, C.c_int, ip, dp]
        L.adr_solve_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(vp), C.POINTER(adr_stats)]
        fp = C.POINTER(C.c_float)
        L.adr_cnn_num_params.argtypes = []
        L.adr_cnn_num_params.restype = C.c_long
        L.adr_cnn_create.argtypes = [C.c_int, fp, vp, C.POINTER(vp)]
        L.adr_cnn_destroy.argtypes = [vp]
        L.adr_cnn_destroy.restype = None
        L.adr_cnn_set_params.argtypes = [vp, fp]
        L.adr_cnn_get_params.argtypes = [vp, fp]
        L.adr_cnn_features.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.adr_cnn_targets.argtypes = [C.c_int, C.c_int, vp, vp, vp, vp, vp]
        L.adr_cnn_forward.argtypes = [vp, C.c_int, vp, vp]
        L.adr_cnn_loss_grad.argtypes = [vp, C.c_int, vp, vp, vp, dp]
        L.adr_cnn_train_step.argtypes = [vp, C.c_int, vp, vp, C.c_float, dp]
        L.adr_cnn_initial_state.argtypes = [vp, vp, vp, vp, vp]
        L.adr_cnn_set_wait_limit.argtypes = [vp, C.c_longlong]
        L.adr_cnn_sync.argtypes = [vp]
        L.adr_set_warm_start.argtypes = [vp, vp]
        _lib = L
    return _lib


EXPORTED = ["adr_default_opts", "adr_create", "adr_solve_stationary", "adr_step_parabolic",
            "adr_destroy", "adr_last_error", "adr_num_lines", "adr_num_line_nodes",
            "adr_get_lines", "adr_get_crossings", "adr_get_transfer", "adr_split_step", "adr_paper_u0",
            "adr_time_kernels", "adr_batch_create", "adr_batch_solve", "adr_batch_destroy",
            "adr_solve_batch", "adr_autotune", "adr_batch_autotune",
            "adr_cnn_num_params", "adr_cnn_create", "adr_cnn_destroy", "adr_cnn_set_params",
            "adr_cnn_get_params", "adr_cnn_features", "adr_cnn_targets", "adr_cnn_forward",
            "adr_cnn_loss_grad", "adr_cnn_train_step", "adr_cnn_initial_state",
            "adr_cnn_set_wait_limit", "adr_cnn_sync", "adr_set_warm_start"]


def tune_key(prob, prec, transfer=0):
    """Cache key of a problem's launch shapes: grid, domain, field kind, precision
    (and the direct transfer, which times other kernels)."""
    b1, b2 = np.asarray(prob.beta1), np.asarray(prob.beta2)
    const = bool(np.all(b1 == b1.flat[0]) and np.all(b2 == b2.flat[0]))
    mask = np.asarray(prob.mask)
    key = f"v2:{prob.nx}x{prob.ny}:{int(mask.sum())}:{'const' if const else 'curved'}:p{int(prec)}"
    return key + (":direct" if transfer else "")


def _tune_path():
    return os.environ.get("ADR_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "adr_gb300", "tune.json"))


def _tune_cache():
    import json
    try:
        with open(_tune_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save_tune_cache(c):
    import json
    path = _tune_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(c, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _check(status, what, allow=()):
    if status != ADR_OK and status not in allow:
        raise AdrError(status, what)
    return status


def default_opts(**kw) -> adr_opts:
    o = adr_opts()
    lib().adr_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ------------------------------------------------------------ C-named calls

def adr_create(grid: adr_grid, mask, mu, sigma, beta1, beta2, f, opts: adr_opts, stream=None):
    h = C.c_void_p()
    st = lib().adr_create(C.byref(grid), _ptr(mask), float(mu), float(sigma), _ptr(beta1),
                          _ptr(beta2), _ptr(f), C.byref(opts), _stream_ptr(stream), C.byref(h))
    _check(st, "adr_create")
    return h


def adr_solve_stationary(h, u_init, u_out, u_iter_out=None):
    s = adr_stats()
    st = lib().adr_solve_stationary(h, _ptr(u_init), _ptr(u_out), _ptr(u_iter_out), C.byref(s))
    _check(st, "adr_solve_stationary", allow=(ADR_ENOCONV,))
    return st, s


def adr_step_parabolic(h, dt, nsteps, mode, u_inout):
    s = adr_stats()
    st = lib().adr_step_parabolic(h, float(dt), int(nsteps), int(mode), _ptr(u_inout), C.byref(s))
    _check(st, "adr_step_parabolic", allow=(ADR_ENOCONV,))
    return st, s


def adr_split_step(h, dt, u, u_half, u_next):
    _check(lib().adr_split_step(h, float(dt), _ptr(u), _ptr(u_half), _ptr(u_next)),
           "adr_split_step")


def adr_paper_u0(h, u0):
    _check(lib().adr_paper_u0(h, _ptr(u0)), "adr_paper_u0")


def adr_time_kernels(h, reps):
    ms = (C.c_double * 6)()
    _check(lib().adr_time_kernels(h, int(reps), ms), "adr_time_kernels")
    return list(ms)


def _ptr_array(items):
    arr = (C.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = None if t is None else (t.value if isinstance(t, C.c_void_p) else t.data_ptr())
    return arr


def adr_batch_create(handles, stream=None):
    b = C.c_void_p()
    _check(lib().adr_batch_create(_ptr_array(handles), len(handles), _stream_ptr(stream),
                                  C.byref(b)), "adr_batch_create")
    return b


def adr_batch_solve(b, u_init, u_out, u_iter_out=None):
    n = len(u_out)
    stats = (adr_stats * n)()
    st = lib().adr_batch_solve(b, None if u_init is None else _ptr_array(u_init), _ptr_array(u_out),
                               None if u_iter_out is None else _ptr_array(u_iter_out), stats)
    _check(st, "adr_batch_solve", allow=(ADR_ENOCONV,))
    return st, [x.as_dict() for x in stats]


def adr_batch_destroy(b):
    lib().adr_batch_destroy(b)


def adr_solve_batch(handles, u_out):
    n = len(handles)
    stats = (adr_stats * n)()
    st = lib().adr_solve_batch(_ptr_array(handles), n, _ptr_array(u_out), stats)
    _check(st, "adr_solve_batch", allow=(ADR_ENOCONV,))
    return st, [x.as_dict() for x in stats]


def adr_destroy(h):
    lib().adr_destroy(h)


# ---------------------------------------------------------- convenience

class Solver:
    """One problem handle on a CUDA device.

    ``prob`` is any object with ``nx, ny, x0, y0, x1, y1, mu, sigma`` and nodal
    arrays ``mask, beta1, beta2, f`` (numpy or torch).  Inputs are copied to
    the device once; the handle owns everything it derives from them.
    """

    def __init__(self, prob, device="cuda:0", stream=None, autotune=False, **opts):
        torch = _torch()
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream
        self.nx, self.ny = int(prob.nx), int(prob.ny)
        key = tune_key(prob, opts.get("prec", ADR_FP64), opts.get("transfer", 0)) if autotune else None
        cached = _tune_cache().get(key) if key else None
        if cached:
            opts.setdefault("rows_per_thread", cached["rows_per_thread"])
            opts.setdefault("map_blocks_per_sm", cached["map_blocks_per_sm"])
        self.opts = default_opts(**opts)
        def dev(a, dt):
            if isinstance(a, torch.Tensor):
                return a.to(device=self.device, dtype=dt).contiguous()
            return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(self.device)
        mask = dev(prob.mask, torch.uint8)
        b1, b2, f = (dev(a, torch.float64) for a in (prob.beta1, prob.beta2, prob.f))
        grid = adr_grid(self.nx, self.ny, prob.x0, prob.y0, prob.x1, prob.y1)
        with torch.cuda.device(self.device):
            self.h = adr_create(grid, mask, prob.mu, prob.sigma, b1, b2, f, self.opts, stream)
        self.tuned = None
        if key and not cached:
            self.tuned = self.autotune()
            c = _tune_cache()
            c[key] = {"rows_per_thread": self.tuned[0], "map_blocks_per_sm": self.tuned[1],
                      "ms_per_step": self.tuned[2]}
            _save_tune_cache(c)

    def autotune(self, reps=10):
        """Measure the launch shapes and keep the fastest (adr_autotune)."""
        r, m, ms = C.c_int(0), C.c_int(0), C.c_double(0)
        _check(lib().adr_autotune(self.h, int(reps), C.byref(r), C.byref(m), C.byref(ms)),
               "adr_autotune")
        return r.value, m.value, ms.value

    def close(self):
        if getattr(self, "h", None):
            adr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _grid(self):
        return self.torch.zeros((self.ny, self.nx), dtype=self.torch.float64, device=self.device)

    def solve_stationary(self, u_init=None, want_iter=False):
        out = self._grid()
        it = self._grid() if want_iter else None
        st, s = adr_solve_stationary(self.h, u_init, out, it)
        return out, it, s.as_dict(), st

    def step_parabolic(self, u, dt, nsteps, mode):
        st, s = adr_step_parabolic(self.h, dt, nsteps, mode, u)
        return s.as_dict(), st

    def split_step(self, u, dt):
        uh, un = self._grid(), self._grid()
        adr_split_step(self.h, dt, u, uh, un)
        return uh, un

    def paper_u0(self):
        out = self._grid()
        adr_paper_u0(self.h, out)  # enqueued on the handle's stream
        if self.stream is not None:
            self.torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out

    def set_warm_start(self, net):
        """Attach a Network (adr_set_warm_start) for init=ADR_INIT_LEARNED; None detaches."""
        _check(lib().adr_set_warm_start(self.h, None if net is None else net.h), "adr_set_warm_start")
        self.net = net  # kept alive while attached

    def time_kernels(self, reps=20):
        """Average device ms per launch of [B gather, B solve, B map, G gather,
        G solve, G map] (0 where a stage has no kernel of its own)."""
        return adr_time_kernels(self.h, reps)

    def line_unknowns(self):
        """Unknowns of one sweep of each family (curve nodes minus the ends)."""
        out = []
        for fam in (0, 1):
            off = self.lines(fam)["off"]
            out.append(int(np.maximum(np.diff(off) - 2, 0).sum()))
        return out

    def lines(self, fam):
        L = lib()
        nl, nn = L.adr_num_lines(self.h, fam), L.adr_num_line_nodes(self.h, fam)
        off = np.zeros(nl + 1, np.int32)
        xi, eta, hh = np.zeros(nn), np.zeros(nn), np.zeros(max(nl, 1))
        _check(L.adr_get_lines(self.h, fam, off.ctypes.data_as(C.POINTER(C.c_int)),
                               xi.ctypes.data_as(C.POINTER(C.c_double)),
                               eta.ctypes.data_as(C.POINTER(C.c_double)),
                               hh.ctypes.data_as(C.POINTER(C.c_double))), "adr_get_lines")
        return dict(off=off, xi=xi, eta=eta, h=hh[:nl])

    def crossings(self, fam):
        n = 4 * self.nx * self.ny
        seg, t, pos = np.zeros(n, np.int32), np.zeros(n), np.zeros(n)
        _check(lib().adr_get_crossings(self.h, fam, seg.ctypes.data_as(C.POINTER(C.c_int)),
                                       t.ctypes.data_as(C.POINTER(C.c_double)),
                                       pos.ctypes.data_as(C.POINTER(C.c_double))),
               "adr_get_crossings")
        s = (self.ny, self.nx, 4)
        return seg.reshape(s), t.reshape(s), pos.reshape(s)

    def transfer_table(self, fam):
        """The direct transfer's crossings of family fam's nodes (adr_get_transfer):
        seg, t, pos of shape [n_nodes, 2] (before / after the node)."""
        nn = lib().adr_num_line_nodes(self.h, fam)
        seg, t, pos = np.zeros(2 * nn, np.int32), np.zeros(2 * nn), np.zeros(2 * nn)
        _check(lib().adr_get_transfer(self.h, fam, seg.ctypes.data_as(C.POINTER(C.c_int)),
                                      t.ctypes.data_as(C.POINTER(C.c_double)),
                                      pos.ctypes.data_as(C.POINTER(C.c_double))),
               "adr_get_transfer")
        return seg.reshape(nn, 2), t.reshape(nn, 2), pos.reshape(nn, 2)


class Batch:
    """Many Solver handles solved together: one persistent launch per sweep
    stage and one CUDA graph for the whole outer loop."""

    def __init__(self, solvers, stream=None):
        self.solvers = list(solvers)
        self.b = adr_batch_create([s.h for s in self.solvers], stream)

    def solve(self, u_init=None, want_iter=False):
        """Returns (u_out grids, stats, status), and the iterates u_{j+1}
        after them when want_iter."""
        outs = [s._grid() for s in self.solvers]
        its = [s._grid() for s in self.solvers] if want_iter else None
        st, stats = adr_batch_solve(self.b, u_init, outs, its)
        if want_iter:
            return outs, stats, st, its
        return outs, stats, st

    def autotune(self, reps=5):
        """Rows per thread of the batch's curve solves by measurement
        (adr_batch_autotune): (rows, ms per batched split step)."""
        r, ms = C.c_int(0), C.c_double(0)
        _check(lib().adr_batch_autotune(self.b, int(reps), C.byref(r), C.byref(ms)),
               "adr_batch_autotune")
        return r.value, ms.value

    def close(self):
        if getattr(self, "b", None):
            adr_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- warm-start network

def adr_cnn_num_params():
    return int(lib().adr_cnn_num_params())


def _cnn_params(params):
    p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
    if p.size != adr_cnn_num_params():
        raise ValueError(f"the network has {adr_cnn_num_params()} parameters, got {p.size}")
    return p


def adr_cnn_create(max_batch, params, stream=None):
    p = _cnn_params(params)
    h = C.c_void_p()
    _check(lib().adr_cnn_create(int(max_batch), p.ctypes.data_as(C.POINTER(C.c_float)),
                                _stream_ptr(stream), C.byref(h)), "adr_cnn_create")
    return h


def adr_cnn_destroy(h):
    lib().adr_cnn_destroy(h)


def adr_cnn_set_params(h, params):
    p = _cnn_params(params)
    _check(lib().adr_cnn_set_params(h, p.ctypes.data_as(C.POINTER(C.c_float))),
           "adr_cnn_set_params")


def adr_cnn_get_params(h):
    p = np.zeros(adr_cnn_num_params(), np.float32)
    _check(lib().adr_cnn_get_params(h, p.ctypes.data_as(C.POINTER(C.c_float))),
           "adr_cnn_get_params")
    return p


def adr_cnn_features(batch, n, f, beta1, beta2, mask, mu, sigma, u0, x, scale, stream=None):
    _check(lib().adr_cnn_features(int(batch), int(n), _ptr(f), _ptr(beta1), _ptr(beta2),
                                  _ptr(mask), _ptr(mu), _ptr(sigma), _ptr(u0), _ptr(x),
                                  _ptr(scale), _stream_ptr(stream)), "adr_cnn_features")


def adr_cnn_targets(batch, n, u, u0, scale, t, stream=None):
    _check(lib().adr_cnn_targets(int(batch), int(n), _ptr(u), _ptr(u0), _ptr(scale), _ptr(t),
                                 _stream_ptr(stream)), "adr_cnn_targets")


def adr_cnn_forward(h, batch, x, y):
    _check(lib().adr_cnn_forward(h, int(batch), _ptr(x), _ptr(y)), "adr_cnn_forward")


def adr_cnn_loss_grad(h, batch, x, t, grad=None):
    loss = C.c_double(0)
    _check(lib().adr_cnn_loss_grad(h, int(batch), _ptr(x), _ptr(t), _ptr(grad), C.byref(loss)),
           "adr_cnn_loss_grad")
    return loss.value


def adr_cnn_train_step(h, batch, x, t, lr, want_loss=True):
    loss = C.c_double(0)
    _check(lib().adr_cnn_train_step(h, int(batch), _ptr(x), _ptr(t), C.c_float(lr),
                                    C.byref(loss) if want_loss else None), "adr_cnn_train_step")
    return loss.value if want_loss else None


def adr_cnn_initial_state(prob_handle, y, u0, scale, u_out):
    _check(lib().adr_cnn_initial_state(prob_handle, _ptr(y), _ptr(u0), _ptr(scale), _ptr(u_out)),
           "adr_cnn_initial_state")


class Network:
    """The warm-start network on a CUDA device (adr_cnn_* calls).

    Inputs are CUDA tensors: features ``x`` bfloat16 [B, 64, 64, 40], targets
    float32 [B, 64, 64], outputs float32 [B, 64, 64, 8] (channel 0 is the
    prediction); parameters are a float32 host vector.  ``u0`` arguments are
    the first initial states the network corrects (normally
    ``Solver.paper_u0()``), stacked [B, 256, 256] float64, or None; ``scale``
    is the per-problem scale features() returns (max |u0|).
    """

    HW = 64

    def __init__(self, max_batch, params=None, device="cuda:0", stream=None, seed=None):
        from . import workloads
        torch = _torch()
        self.torch = torch
        self.device = torch.device(device)
        self.max_batch = int(max_batch)
        if params is None:
            params = workloads.cnn_init_params() if seed is None else \
                workloads.cnn_init_params(seed)
        with torch.cuda.device(self.device):
            self.h = adr_cnn_create(self.max_batch, params, stream)
        self.grad = torch.zeros(adr_cnn_num_params(), dtype=torch.float32, device=self.device)

    @property
    def params(self):
        return adr_cnn_get_params(self.h)

    @params.setter
    def params(self, p):
        adr_cnn_set_params(self.h, p)

    def features(self, f, beta1, beta2, mask, mu, sigma, u0=None):
        """Stacked device problems [B, 256, 256] (float64, mask uint8), mu and
        sigma float64 [B] -> (bfloat16 features [B, 64, 64, 40], scale [B])."""
        B, n = f.shape[0], f.shape[-1]
        x = self.torch.empty((B, self.HW, self.HW, 40), dtype=self.torch.bfloat16,
                             device=self.device)
        scale = self.torch.empty(B, dtype=self.torch.float64, device=self.device)
        adr_cnn_features(B, n, f, beta1, beta2, mask, mu, sigma, u0, x, scale)
        return x, scale

    def targets(self, u, scale, u0=None):
        B, n = u.shape[0], u.shape[-1]
        t = self.torch.empty((B, self.HW, self.HW), dtype=self.torch.float32, device=self.device)
        adr_cnn_targets(B, n, u, u0, scale, t)
        return t

    def forward(self, x):
        y = self.torch.empty((x.shape[0], self.HW, self.HW, 8), dtype=self.torch.float32,
                             device=self.device)
        adr_cnn_forward(self.h, x.shape[0], x, y)
        return y

    def loss_grad(self, x, t):
        loss = adr_cnn_loss_grad(self.h, x.shape[0], x, t, self.grad)
        return loss, self.grad

    def train_step(self, x, t, lr, want_loss=True):
        return adr_cnn_train_step(self.h, x.shape[0], x, t, lr, want_loss)

    def set_wait_limit(self, spins):
        """Bound of the tensor-core kernels' waits in polls (0: the default)."""
        _check(lib().adr_cnn_set_wait_limit(self.h, int(spins)), "adr_cnn_set_wait_limit")

    def sync(self):
        """Wait for the network's stream; the status (ADR_ETIMEOUT if a bounded
        wait gave up since the last report)."""
        return lib().adr_cnn_sync(self.h)

    def initial_state(self, solver, y, u0=None, scale=None):
        """Solver grid initial state u0 + s * bilinear(y[..., 0]) from one
        prediction y [64, 64, 8]; scale: device tensor holding s (or None: 1)."""
        u = solver._grid()
        adr_cnn_initial_state(solver.h, y, u0, scale, u)
        return u

    def close(self):
        if getattr(self, "h", None):
            adr_cnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
