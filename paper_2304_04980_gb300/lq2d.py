"""ctypes binding of the lq2d C-ABI (include/lq2d.h).

Argument marshalling only: every step of the solve runs in the CUDA library.
Loading fails loudly when liblq2d.so has not been built; there is no CPU
fallback.  Device buffers are anything with a ``data_ptr()`` (torch tensors)
or a raw integer address; streams are ``torch.cuda.Stream`` objects, raw
``cudaStream_t`` integers, or None for the legacy default stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "liblq2d.so")

OK, EINVAL, ENOTPD, ENOCONV, EBREAKDOWN, ECUDA, ENOMEM, ETIMEOUT = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOTPD", 3: "ENOCONV", 4: "EBREAKDOWN", 5: "ECUDA",
                6: "ENOMEM", 7: "ETIMEOUT"}
OPT_STOP_MODE, OPT_DRIVER, OPT_TIMING, OPT_MAX_RESTARTS, OPT_PRECONDITIONER, OPT_KAPPA = 1, 2, 3, 4, 5, 6
OPT_SWEEP_THREADS, OPT_SWEEP_STEPS, OPT_TWISTED = 7, 8, 9
BATCH_PERSISTENT, BATCH_THREADS, BATCH_USES_PERSISTENT = 1, 2, 3

EXPORTED = (
    "lq2d_create", "lq2d_create_device", "lq2d_update", "lq2d_update_device", "lq2d_set_affine", "lq2d_solve",
    "lq2d_solve_device", "lq2d_solve_nbjm_device", "lq2d_apply_delta_device", "lq2d_apply_precond_device", "lq2d_apply_delta_static",
    "lq2d_apply_precond_multi_device", "lq2d_solve_multi_device",
    "lq2d_autotune",
    "lq2d_batch_create", "lq2d_batch_solve", "lq2d_batch_destroy", "lq2d_get_solution_device",
    "lq2d_batch_set_option", "lq2d_batch_get_option", "lq2d_batch_autotune", "lq2d_get_option",
    "lq2d_set_option",
    "lq2d_get_stats", "lq2d_set_precision", "lq2d_destroy", "lq2d_last_error",
    "lq2d_wsnet_create", "lq2d_wsnet_param_count", "lq2d_wsnet_set_params", "lq2d_wsnet_get_params",
    "lq2d_wsnet_forward_device", "lq2d_wsnet_loss_grad_device", "lq2d_wsnet_train_step_device",
    "lq2d_wsnet_destroy",
)


class Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("restarts", ctypes.c_int), ("status", ctypes.c_int),
        ("sweep_launches", ctypes.c_int), ("delta_launches", ctypes.c_int), ("sweep_steps", ctypes.c_int),
        ("rel_residual", ctypes.c_double), ("rel_kkt_residual", ctypes.c_double),
        ("kkt_inf", ctypes.c_double), ("cost", ctypes.c_double),
        ("sweep_ms", ctypes.c_double), ("delta_ms", ctypes.c_double),
        ("launches_total", ctypes.c_longlong), ("body_executions", ctypes.c_int),
        ("outer_iterations", ctypes.c_int), ("kappa_estimate", ctypes.c_double),
        ("lambda_min", ctypes.c_double), ("lambda_max", ctypes.c_double),
        ("sweep_threads", ctypes.c_int), ("residual_replacements", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if not name.startswith("pad")}


class LQ2DError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def load() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("liblq2d.so not found at %s: build it with "
                           "`python -m paper_2304_04980_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    i = ctypes.c_int
    d = ctypes.c_double
    pp = ctypes.POINTER(_vp)
    sig = {
        "lq2d_create": (i, [pp, i, i, i, i, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lq2d_create_device": (i, [pp, i, i, i, i, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lq2d_update": (i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lq2d_update_device": (i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lq2d_set_affine": (i, [_vp, _vp]),
        "lq2d_solve": (i, [_vp, d, i, i, i, _vp, _vp, _vp, _vp, _ip, _dp]),
        "lq2d_solve_device": (i, [_vp, d, i, i, i, _vp, _vp, _vp, _vp, _ip, _dp, _vp]),
        "lq2d_solve_nbjm_device": (i, [_vp, d, i, i, _vp, _vp, _vp, _ip, _dp, _vp]),
        "lq2d_apply_delta_device": (i, [_vp, _vp, _vp, _vp]),
        "lq2d_apply_precond_device": (i, [_vp, i, i, _vp, _vp, _vp]),
        "lq2d_apply_precond_multi_device": (i, [_vp, i, i, i, _vp, _vp, _vp]),
        "lq2d_solve_multi_device": (i, [_vp, i, _vp, ctypes.c_double, i, i, i, _vp, _vp, _vp, _ip, _dp, _vp]),
        "lq2d_autotune": (i, [_vp, i, i, i, _ip, _dp, _vp]),
        "lq2d_apply_delta_static": (i, [i, i, i, i, i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "lq2d_batch_create": (i, [pp, i, _vp]),
        "lq2d_batch_solve": (i, [_vp, d, i, i, i, _vp, _vp, _vp, _vp]),
        "lq2d_batch_destroy": (None, [_vp]),
        "lq2d_batch_set_option": (i, [_vp, i, i]),
        "lq2d_batch_get_option": (i, [_vp, i, _ip]),
        "lq2d_batch_autotune": (i, [_vp, i, i, i, _ip, _dp, _vp]),
        "lq2d_get_solution_device": (i, [_vp, _vp, _vp, _vp, _vp]),
        "lq2d_set_option": (i, [_vp, i, d]),
        "lq2d_get_option": (i, [_vp, i, _dp]),
        "lq2d_get_stats": (i, [_vp, ctypes.POINTER(Stats)]),
        "lq2d_set_precision": (i, [_vp, i]),
        "lq2d_destroy": (None, [_vp]),
        "lq2d_last_error": (ctypes.c_char_p, []),
        "lq2d_wsnet_create": (i, [pp, i, i, i, i, i, i, i, d]),
        "lq2d_wsnet_param_count": (i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
        "lq2d_wsnet_set_params": (i, [_vp, _vp]),
        "lq2d_wsnet_get_params": (i, [_vp, _vp]),
        "lq2d_wsnet_forward_device": (i, [_vp, i, _vp, _vp, _vp, _vp]),
        "lq2d_wsnet_loss_grad_device": (i, [_vp, i, _vp, _vp, _vp, _dp, _vp, _vp]),
        "lq2d_wsnet_train_step_device": (i, [_vp, i, _vp, _vp, _vp, d, _dp, _vp]),
        "lq2d_wsnet_destroy": (None, [_vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().lq2d_last_error().decode()


def _check(code: int, allow=()):
    if code != OK and code not in allow:
        raise LQ2DError(code, last_error())
    return code


def _addr(buf):
    """Device or host address of a buffer (None -> NULL)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        if not (buf.dtype == np.float64 and buf.flags.c_contiguous):
            raise ValueError("host arrays must be C-contiguous float64")
        return buf.ctypes.data
    raise TypeError("unsupported buffer type %r" % type(buf))


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def apply_delta_static(K, N, T, n, m, A_self, A_nbr, B, Q, R, Q_T, d_in, d_out, stream=None):
    """y = Delta d from raw device blocks, with no device allocation (see
    lq2d_apply_delta_static in include/lq2d.h)."""
    _check(load().lq2d_apply_delta_static(K, N, T, n, m, *[_addr(a) for a in (A_self, A_nbr, B, Q, R, Q_T)],
                                          _addr(d_in), _addr(d_out), _stream(stream)))


def _host(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """One LQ problem on the GPU (handle of the C library)."""

    def __init__(self, handle, K, N, T, n, m):
        self._h = handle
        self.K, self.N, self.T, self.n, self.m = K, N, T, n, m

    # -- construction -----------------------------------------------------
    @classmethod
    def from_host(cls, K, N, T, n, m, A_self, A_nbr, B, Q, R, Q_T, x0):
        lib = load()
        arrs = [_host(a) for a in (A_self, A_nbr, B, Q, R, Q_T, x0)]
        h = _vp()
        _check(lib.lq2d_create(ctypes.byref(h), K, N, T, n, m, *[a.ctypes.data for a in arrs]))
        return cls(h, K, N, T, n, m)

    @classmethod
    def from_device(cls, K, N, T, n, m, A_self, A_nbr, B, Q, R, Q_T, x0, stream=None):
        lib = load()
        h = _vp()
        _check(lib.lq2d_create_device(ctypes.byref(h), K, N, T, n, m,
                                      *[_addr(a) for a in (A_self, A_nbr, B, Q, R, Q_T, x0)],
                                      _stream(stream)))
        return cls(h, K, N, T, n, m)

    @classmethod
    def from_grid(cls, g):
        """From a synth.GridLQ (host arrays)."""
        return cls.from_host(g.K, g.N, g.T, g.n, g.m, *g.arrays())

    def update(self, A_self, A_nbr, B, Q, R, Q_T, x0):
        """Host arrays (numpy, or pinned host tensors via their address)."""
        args = [a if isinstance(a, int) or hasattr(a, "data_ptr") else _host(a)
                for a in (A_self, A_nbr, B, Q, R, Q_T, x0)]
        _check(load().lq2d_update(self._h, *[_addr(a) for a in args]))

    def update_device(self, A_self, A_nbr, B, Q, R, Q_T, x0, stream=None):
        _check(load().lq2d_update_device(self._h, *[_addr(a) for a in (A_self, A_nbr, B, Q, R, Q_T, x0)],
                                         _stream(stream)))

    def set_affine(self, w):
        self._w = None if w is None else _host(w)
        _check(load().lq2d_set_affine(self._h, None if w is None else self._w.ctypes.data))

    # -- solves -----------------------------------------------------------
    def solve(self, tol=1e-8, S=2, L=2, max_iter=10000, delta0=None, allow=(ENOCONV,), out=None):
        """Host solve; returns dict(x, u, costate, iterations, rel_kkt, status).
        `out` = (x, u, costate) preallocated float64 arrays, else new ones."""
        if out is None:
            x = np.empty((self.T + 1, self.K * self.N, self.n))
            u = np.empty((self.T, self.K * self.N, self.m))
            lam = np.empty_like(x)
        else:
            x, u, lam = out
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        d0 = None if delta0 is None else _host(delta0)
        code = load().lq2d_solve(self._h, tol, S, L, max_iter, None if d0 is None else d0.ctypes.data,
                                 x.ctypes.data, u.ctypes.data, lam.ctypes.data, ctypes.byref(it), ctypes.byref(rel))
        _check(code, allow)
        return dict(x=x, u=u, costate=lam, iterations=it.value, rel_kkt=rel.value, status=code)

    def solve_device(self, tol, S, L, max_iter, delta0=None, x=None, u=None, costate=None, stream=None,
                     allow=(ENOCONV,)):
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        code = load().lq2d_solve_device(self._h, tol, S, L, max_iter, _addr(delta0), _addr(x), _addr(u),
                                        _addr(costate), ctypes.byref(it), ctypes.byref(rel), _stream(stream))
        _check(code, allow)
        return dict(iterations=it.value, rel_kkt=rel.value, status=code)

    def solve_nbjm_device(self, eps, L, max_outer, x=None, u=None, costate=None, stream=None,
                          allow=(ENOCONV,)):
        """Algorithm 2 run to its exit test (the paper's standard NBJM)."""
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        code = load().lq2d_solve_nbjm_device(self._h, eps, L, max_outer, _addr(x), _addr(u), _addr(costate),
                                             ctypes.byref(it), ctypes.byref(rel), _stream(stream))
        _check(code, allow)
        return dict(outer_iterations=it.value, rel_kkt=rel.value, status=code)

    def apply_delta_device(self, d_in, d_out, stream=None):
        _check(load().lq2d_apply_delta_device(self._h, _addr(d_in), _addr(d_out), _stream(stream)))

    def apply_precond_device(self, S, L, d_r, d_q, stream=None):
        _check(load().lq2d_apply_precond_device(self._h, S, L, _addr(d_r), _addr(d_q), _stream(stream)))

    def solve_multi_device(self, nrhs, x0s, tol=1e-8, S=2, L=2, max_iter=10000, x=None, u=None, costate=None,
                           stream=None, allow=(ENOCONV,)):
        """Solves for nrhs <= 32 initial states x0s [nrhs][K*N][n] (device)
        at once; returns per-right-hand-side iterations and true relative
        residuals and the status (tensor-core path, n = 4)."""
        its = (ctypes.c_int * nrhs)()
        rel = (ctypes.c_double * nrhs)()
        code = load().lq2d_solve_multi_device(self._h, nrhs, _addr(x0s), tol, S, L, max_iter, _addr(x), _addr(u),
                                              _addr(costate), its, rel, _stream(stream))
        _check(code, allow)
        return dict(iterations=list(its), rel_residuals=list(rel), status=code)

    def apply_precond_multi_device(self, nrhs, S, L, d_r, d_q, stream=None):
        """q_r = D_S r_r for nrhs <= 32 right-hand sides [nrhs][T+1][K*N][n]
        (tensor-core path, n = 4)."""
        _check(load().lq2d_apply_precond_multi_device(self._h, nrhs, S, L, _addr(d_r), _addr(d_q),
                                                      _stream(stream)))

    def autotune(self, S=2, L=2, reps=5, stream=None):
        """Times the sweep tile widths for this shape and precision mode and
        keeps the fastest; returns (threads, ms per preconditioner apply)."""
        thr, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        _check(load().lq2d_autotune(self._h, S, L, reps, ctypes.byref(thr), ctypes.byref(ms), _stream(stream)))
        return thr.value, ms.value

    def get_solution_device(self, x=None, u=None, costate=None, stream=None):
        _check(load().lq2d_get_solution_device(self._h, _addr(x), _addr(u), _addr(costate), _stream(stream)))

    def set_option(self, option, value):
        _check(load().lq2d_set_option(self._h, option, float(value)))

    def get_option(self, option):
        v = ctypes.c_double(0.0)
        _check(load().lq2d_get_option(self._h, option, ctypes.byref(v)))
        return v.value

    def stats(self) -> dict:
        s = Stats()
        _check(load().lq2d_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def set_precision(self, mode):
        _check(load().lq2d_set_precision(self._h, mode))

    def close(self):
        if self._h is not None and self._h.value:
            load().lq2d_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Problems solved together by one graph launch (lq2d_batch_*)."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (_vp * len(self.problems))(*[p._h.value for p in self.problems])
        self._arr = arr
        h = _vp()
        _check(load().lq2d_batch_create(ctypes.byref(h), len(self.problems), arr))
        self._h = h

    def solve(self, tol=1e-8, S=2, L=2, max_iter=10000, stream=None, allow=(ENOCONV,)):
        n = len(self.problems)
        its = (ctypes.c_int * n)()
        rel = (ctypes.c_double * n)()
        sts = (ctypes.c_int * n)()
        code = load().lq2d_batch_solve(self._h, tol, S, L, max_iter, its, rel, sts, _stream(stream))
        _check(code, allow)
        return dict(iterations=list(its), rel_kkt=list(rel), statuses=list(sts), status=code)

    def set_option(self, option, value):
        _check(load().lq2d_batch_set_option(self._h, option, int(value)))

    def get_option(self, option):
        v = ctypes.c_int(0)
        _check(load().lq2d_batch_get_option(self._h, option, ctypes.byref(v)))
        return v.value

    def autotune(self, S=2, L=2, reps=3, stream=None):
        """Chooses the persistent loop's sweep width by timing; returns
        (threads, ms per D_S of the whole batch)."""
        thr = ctypes.c_int(0)
        ms = ctypes.c_double(0.0)
        _check(load().lq2d_batch_autotune(self._h, S, L, reps, ctypes.byref(thr), ctypes.byref(ms), _stream(stream)))
        return thr.value, ms.value

    def close(self):
        if self._h is not None and self._h.value:
            load().lq2d_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class WarmStartNet:
    """The warm-start network of include/lq2d_warmstart.h: a stack of 3x3
    convolutions over the grid mapping (x0, coupling scale) to delta^(0)."""

    def __init__(self, K, N, T, n, channels=64, layers=6, max_batch=8, sigma=1.0):
        self.K, self.N, self.T, self.n = K, N, T, n
        self.channels, self.layers, self.max_batch, self.sigma = channels, layers, max_batch, sigma
        h = _vp()
        _check(load().lq2d_wsnet_create(ctypes.byref(h), K, N, T, n, channels, layers, max_batch, float(sigma)))
        self._h = h
        cnt = ctypes.c_longlong(0)
        _check(load().lq2d_wsnet_param_count(self._h, ctypes.byref(cnt)))
        self.param_count = cnt.value

    def layer_sizes(self):
        return [self.n + 1] + [self.channels] * (self.layers - 1) + [(self.T + 1) * self.n]

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        if p.size != self.param_count:
            raise ValueError("expected %d parameters, got %d" % (self.param_count, p.size))
        _check(load().lq2d_wsnet_set_params(self._h, p.ctypes.data))

    def get_params(self):
        p = np.empty(self.param_count, dtype=np.float32)
        _check(load().lq2d_wsnet_get_params(self._h, p.ctypes.data))
        return p

    def unflatten(self, flat):
        """[(w [Cout][Cin][3][3], b [Cout]) per layer] from a parameter vector."""
        sizes = self.layer_sizes()
        out, off = [], 0
        for l in range(self.layers):
            ci, co = sizes[l], sizes[l + 1]
            w = np.asarray(flat[off:off + co * ci * 9]).reshape(co, ci, 3, 3)
            off += co * ci * 9
            b = np.asarray(flat[off:off + co])
            off += co
            out.append((w, b))
        return out

    @staticmethod
    def _coupling(c, batch):
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(c, dtype=np.float64), (batch,)))
        return arr

    def forward_device(self, batch, d_x0, coupling, d_delta0, stream=None):
        c = self._coupling(coupling, batch)
        _check(load().lq2d_wsnet_forward_device(self._h, batch, _addr(d_x0), c.ctypes.data, _addr(d_delta0),
                                                _stream(stream)))

    def loss_grad_device(self, batch, d_x0, coupling, d_target, want_grads=True, stream=None):
        c = self._coupling(coupling, batch)
        loss = ctypes.c_double(0.0)
        g = np.empty(self.param_count, dtype=np.float32) if want_grads else None
        _check(load().lq2d_wsnet_loss_grad_device(self._h, batch, _addr(d_x0), c.ctypes.data, _addr(d_target),
                                                  ctypes.byref(loss), None if g is None else g.ctypes.data,
                                                  _stream(stream)))
        return loss.value, g

    def train_step_device(self, batch, d_x0, coupling, d_target, lr, stream=None):
        c = self._coupling(coupling, batch)
        loss = ctypes.c_double(0.0)
        _check(load().lq2d_wsnet_train_step_device(self._h, batch, _addr(d_x0), c.ctypes.data, _addr(d_target),
                                                   float(lr), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def close(self):
        if self._h is not None and self._h.value:
            load().lq2d_wsnet_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
