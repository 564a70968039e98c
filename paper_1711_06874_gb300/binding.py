"""ctypes binding of libtucker_matern (the C-ABI in include/tucker_matern.h).

Argument marshalling only: every step of the decomposition runs in the CUDA
library.  Device buffers are PyTorch CUDA tensors (``data_ptr()``), streams
are ``torch.cuda.Stream`` handles.  The library is loaded on first use; if
it is missing or cannot load, the call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtucker_matern.so")

TK_OK, TK_EINVAL, TK_ENOMEM, TK_ECUDA, TK_ETIMEOUT, TK_EBUSY, TK_ENOTFOUND = range(7)
TK_MATERN, TK_SLATER_P, TK_GAUSSIAN, TK_MATERN_SD = 0, 1, 2, 3
TK_CELL_CENTRED, TK_VERTEX = 0, 1
TK_FP64, TK_SLICED_BF16, TK_BF16X3, TK_TF32X3 = 0, 1, 2, 3
SLICED_AVAILABLE = True  # tensor-core Gram from exact BF16 slices is built
TK_RANK_CAPPED, TK_EPS_UNREACHABLE_AT_PRECISION, TK_SOLVED_AGAIN_IN_FP64 = 1, 2, 4

# every function the header declares, with (restype, argtypes)
_c = ctypes
_vp, _i32, _u32, _dbl = _c.c_void_p, _c.c_int32, _c.c_uint32, _c.c_double


class Kernel(_c.Structure):
    _fields_ = [("kind", _i32), ("nu", _dbl), ("ell", _dbl * 3), ("sigma2", _dbl), ("p", _dbl)]


class Grid(_c.Structure):
    _fields_ = [("n", _i32 * 3), ("b", _dbl * 3), ("kind", _i32)]


class Opts(_c.Structure):
    _fields_ = [("eps", _dbl), ("rmax", _i32 * 3), ("rfix", _i32 * 3), ("precision", _i32),
                ("isotropic_shortcut", _i32), ("reflect_fold", _i32), ("with_error", _i32), ("fused_eval", _i32),
                ("reserved", _i32 * 1)]


class ServeOpts(_c.Structure):
    _fields_ = [("workers", _i32), ("max_batch", _i32), ("mem_fraction", _dbl), ("reserved", _i32 * 4)]


class ServeStats(_c.Structure):
    _fields_ = [(name, _c.c_uint64) for name in ("submitted", "completed", "failed", "batches", "max_batch_seen",
                                                  "bytes_budget", "bytes_peak", "queued", "in_flight_batches")]


SIGNATURES = {
    "tk_strerror": (_c.c_char_p, [_c.c_int]),
    "tk_last_error": (_c.c_char_p, [_vp]),
    "tk_version": (_c.c_char_p, []),
    "tk_create": (_c.c_int, [_c.POINTER(_vp), _c.c_int]),
    "tk_destroy": (None, [_vp]),
    "tk_default_opts": (None, [_c.POINTER(Opts)]),
    "tk_tucker": (_c.c_int, [_vp, _c.POINTER(Kernel), _c.POINTER(Grid), _c.POINTER(Opts),
                             _c.POINTER(_vp), _vp]),
    "tk_ranks": (_c.c_int, [_vp, _c.POINTER(_i32), _c.POINTER(_u32)]),
    "tk_factor": (_c.c_int, [_vp, _c.c_int, _vp, _c.c_int, _vp]),
    "tk_core": (_c.c_int, [_vp, _vp, _c.c_int, _vp]),
    "tk_result_copy": (_c.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "tk_eigenvalues": (_c.c_int, [_vp, _c.c_int, _vp, _c.c_int, _c.POINTER(_c.c_int)]),
    "tk_norm2": (_c.c_int, [_vp, _c.POINTER(_dbl)]),
    "tk_result_rel_error": (_c.c_int, [_vp, _c.POINTER(_dbl)]),
    "tk_reconstruct": (_c.c_int, [_vp, _vp, _vp, _vp]),
    "tk_rel_error": (_c.c_int, [_vp, _vp, _c.POINTER(Kernel), _c.POINTER(Grid), _c.POINTER(_dbl), _vp]),
    "tk_result_free": (None, [_vp]),
    "tk_batch": (_c.c_int, [_vp, _c.c_int, _c.POINTER(Kernel), _c.POINTER(Grid), _c.POINTER(Opts),
                            _c.POINTER(_vp), _vp]),
    "tk_eval": (_c.c_int, [_vp, _c.POINTER(Kernel), _c.POINTER(Grid), _vp, _vp]),
    "tk_gram": (_c.c_int, [_vp, _vp, _c.POINTER(_i32), _c.c_int, _c.c_int, _vp, _vp]),
    "tk_sym_eig": (_c.c_int, [_vp, _vp, _c.c_int, _c.c_int, _vp, _vp, _vp]),
    "tk_ttm_core": (_c.c_int, [_vp, _vp, _c.POINTER(_i32), _vp, _vp, _vp, _c.POINTER(_i32), _c.c_int,
                               _vp, _vp]),
    "tk_gram_noalloc": (_c.c_int, [_vp, _c.POINTER(_i32), _c.c_int, _vp, _vp]),
    "tk_multigrid": (_c.c_int, [_vp, _c.POINTER(Kernel), _c.POINTER(Grid), _c.POINTER(Opts), _c.c_int, _c.c_int,
                                _c.POINTER(_vp), _vp]),
    "tk_als": (_c.c_int, [_vp, _vp, _c.POINTER(_i32), _vp, _vp, _vp, _c.POINTER(_i32), _c.c_int, _vp,
                          _c.POINTER(_dbl), _vp]),
    "tk_c2t": (_c.c_int, [_vp, _c.c_int, _vp, _vp, _vp, _vp, _c.POINTER(_i32), _dbl, _c.POINTER(_i32),
                          _c.POINTER(_i32), _c.c_int, _c.POINTER(_vp), _c.POINTER(_dbl), _vp]),
    "tk_tune": (_c.c_int, [_vp, _c.c_int, _c.c_char_p, _c.POINTER(_c.c_int)]),
    "tk_default_serve_opts": (None, [_c.POINTER(ServeOpts)]),
    "tk_serve_start": (_c.c_int, [_vp, _c.POINTER(ServeOpts)]),
    "tk_serve_stop": (_c.c_int, [_vp]),
    "tk_submit": (_c.c_int, [_vp, _c.POINTER(Kernel), _c.POINTER(Grid), _c.POINTER(Opts),
                             _c.POINTER(_c.c_uint64)]),
    "tk_poll": (_c.c_int, [_vp, _c.c_uint64, _c.POINTER(_vp), _c.POINTER(_dbl), _dbl]),
    "tk_serve_read_stats": (_c.c_int, [_vp, _c.POINTER(ServeStats)]),
    "tk_profile_enable": (_c.c_int, [_vp, _c.c_int]),
    "tk_profile_read": (_c.c_int, [_vp, _c.POINTER(_dbl), _c.POINTER(_c.c_int64)]),
    "tk_kernel_launches": (_c.c_uint64, []),
}

STAGES = ["eval", "norm", "gram", "eig", "rank", "core", "error", "table", "gram_tc", "qr", "jacobi", "start",
          "eig_gemm"]

_lock = threading.Lock()
_lib = None


class TuckerError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it is missing (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libtucker_matern.so not found at {path}; run __graft_entry__.build()")
        lib = _c.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, ctx=None):
    if rc != TK_OK:
        lib = load()
        msg = lib.tk_strerror(rc).decode()
        if ctx is not None and ctx.value:
            detail = lib.tk_last_error(ctx).decode()
            if detail:
                msg += ": " + detail
        raise TuckerError(rc, msg)


def make_kernel(prob: workloads.Problem) -> Kernel:
    return Kernel(prob.kind, prob.nu, (_dbl * 3)(*prob.ell), prob.sigma2, prob.p)


def make_grid(prob: workloads.Problem) -> Grid:
    return Grid((_i32 * 3)(*prob.n), (_dbl * 3)(*prob.b), prob.grid)


_DEFAULT_OPTS = None


def make_opts(prob: workloads.Problem, precision=TK_FP64, rfix=(0, 0, 0), shortcut=True, fold=True,
              with_error=False, fused_eval=True) -> Opts:
    global _DEFAULT_OPTS
    if _DEFAULT_OPTS is None:
        d = Opts()
        load().tk_default_opts(_c.byref(d))
        _DEFAULT_OPTS = d
    o = Opts.from_buffer_copy(_DEFAULT_OPTS)
    o.eps = prob.eps
    o.rmax = (_i32 * 3)(*prob.rmax)
    o.rfix = (_i32 * 3)(*rfix)
    o.precision = precision
    o.isotropic_shortcut = 1 if shortcut else 0
    o.reflect_fold = 1 if fold else 0
    o.with_error = 1 if with_error else 0
    o.fused_eval = 1 if fused_eval else 0
    return o


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class BatchArgs:
    """The C structs of a batch of problems, marshalled once."""

    def __init__(self, probs, precision=TK_FP64, shortcut=True, fold=True, rfixes=None, with_error=False):
        self.probs = list(probs)
        self.count = len(self.probs)
        rfixes = rfixes or [(0, 0, 0)] * self.count
        n = max(self.count, 1)
        self.ks = (Kernel * n)(*[make_kernel(p) for p in self.probs])
        self.gs = (Grid * n)(*[make_grid(p) for p in self.probs])
        self.os = (Opts * n)(*[make_opts(p, precision, rf, shortcut, fold, with_error)
                               for p, rf in zip(self.probs, rfixes)])


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.ptr = _vp()
        _check(self.lib.tk_create(_c.byref(self.ptr), int(device)))
        self.device = device
        self._args = {}  # (problem, options) -> the C structs, built once

    def _structs(self, prob, precision, rfix, shortcut, fold, with_error, fused_eval=True):
        """The C structs of one solve, built once per distinct (problem, options):
        building them costs more than a small solve's launches."""
        key = (prob, precision, tuple(rfix), bool(shortcut), bool(fold), bool(with_error), bool(fused_eval))
        hit = self._args.get(key)
        if hit is None:
            if len(self._args) >= 256:
                self._args.clear()
            hit = (make_kernel(prob), make_grid(prob),
                   make_opts(prob, precision, rfix, shortcut, fold, with_error, fused_eval))
            self._args[key] = hit
        return hit

    def close(self):
        if self.ptr is not None and self.ptr.value:
            self.lib.tk_destroy(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- whole solve -------------------------------------------------------
    def tucker(self, prob: workloads.Problem, precision=TK_FP64, rfix=(0, 0, 0), shortcut=True,
               fold=True, with_error=False, stream=None, fused_eval=True) -> "Result":
        k, g, o = self._structs(prob, precision, rfix, shortcut, fold, with_error, fused_eval)
        out = _vp()
        _check(self.lib.tk_tucker(self.ptr, _c.byref(k), _c.byref(g), _c.byref(o), _c.byref(out),
                                  _stream_ptr(stream)), self.ptr)
        return Result(self, out, prob, k, g)

    def batch(self, probs, precision=TK_FP64, shortcut=True, fold=True, rfixes=None, with_error=False,
              stream=None) -> list:
        """Independent solves in one call (tk_batch); one Result per problem.
        probs: a list of Problems, or BatchArgs built once beforehand.
        rfixes: optional per-problem fixed ranks (tuples of 3, 0 = eps rule)."""
        args = probs if isinstance(probs, BatchArgs) else BatchArgs(probs, precision, shortcut, fold, rfixes,
                                                                    with_error)
        cnt = args.count
        outs = (_vp * max(cnt, 1))()
        _check(self.lib.tk_batch(self.ptr, cnt, args.ks, args.gs, args.os, outs, _stream_ptr(stream)), self.ptr)
        return [Result(self, _vp(outs[i]), args.probs[i]) for i in range(cnt)]

    # ---- serving ----------------------------------------------------------------
    def serve_start(self, workers=2, max_batch=256, mem_fraction=0.8):
        o = ServeOpts()
        self.lib.tk_default_serve_opts(_c.byref(o))
        o.workers, o.max_batch, o.mem_fraction = int(workers), int(max_batch), float(mem_fraction)
        _check(self.lib.tk_serve_start(self.ptr, _c.byref(o)), self.ptr)
        self._tickets = {}

    def serve_stop(self):
        _check(self.lib.tk_serve_stop(self.ptr), self.ptr)

    def submit(self, prob: workloads.Problem, precision=TK_FP64, rfix=(0, 0, 0)) -> int:
        k, g, o = make_kernel(prob), make_grid(prob), make_opts(prob, precision, rfix)
        t = _c.c_uint64(0)
        _check(self.lib.tk_submit(self.ptr, _c.byref(k), _c.byref(g), _c.byref(o), _c.byref(t)), self.ptr)
        self._tickets[t.value] = prob
        return t.value

    def poll(self, ticket: int, wait_s: float = 0.0):
        """(Result, latency seconds) when done, None while running; raises on a failed solve."""
        out = _vp()
        lat = _dbl(0)
        rc = self.lib.tk_poll(self.ptr, _c.c_uint64(ticket), _c.byref(out), _c.byref(lat), float(wait_s))
        if rc == TK_EBUSY:
            return None
        prob = self._tickets.pop(ticket, None)
        _check(rc, self.ptr)
        return Result(self, out, prob), lat.value

    def serve_stats(self) -> dict:
        st = ServeStats()
        _check(self.lib.tk_serve_read_stats(self.ptr, _c.byref(st)), self.ptr)
        return {name: int(getattr(st, name)) for name, _ in ServeStats._fields_}

    # ---- diagnostics ----------------------------------------------------------
    def profile(self, on: bool = True):
        _check(self.lib.tk_profile_enable(self.ptr, 1 if on else 0), self.ptr)

    def profile_read(self) -> dict:
        ms = (_dbl * len(STAGES))()
        calls = (_c.c_int64 * len(STAGES))()
        _check(self.lib.tk_profile_read(self.ptr, ms, calls), self.ptr)
        return {name: (ms[i], int(calls[i])) for i, name in enumerate(STAGES)}

    @staticmethod
    def kernel_launches() -> int:
        return int(load().tk_kernel_launches())

    # ---- stage entry points (device tensors in and out) --------------------
    def eval(self, prob: workloads.Problem, F, stream=None):
        k, g = make_kernel(prob), make_grid(prob)
        _check(self.lib.tk_eval(self.ptr, _c.byref(k), _c.byref(g), F.data_ptr(), _stream_ptr(stream)),
               self.ptr)

    def gram(self, F, mode: int, G, precision=TK_FP64, stream=None):
        n = (_i32 * 3)(*F.shape)
        _check(self.lib.tk_gram(self.ptr, F.data_ptr(), n, int(mode), int(precision), G.data_ptr(),
                                _stream_ptr(stream)), self.ptr)

    def sym_eig(self, G, m: int, lam, V, stream=None):
        _check(self.lib.tk_sym_eig(self.ptr, G.data_ptr(), int(G.shape[0]), int(m), lam.data_ptr(),
                                   V.data_ptr(), _stream_ptr(stream)), self.ptr)

    def ttm_core(self, F, U, B, precision=TK_FP64, stream=None):
        n = (_i32 * 3)(*F.shape)
        r = (_i32 * 3)(*B.shape)
        _check(self.lib.tk_ttm_core(self.ptr, F.data_ptr(), n, U[0].data_ptr(), U[1].data_ptr(),
                                    U[2].data_ptr(), r, int(precision), B.data_ptr(), _stream_ptr(stream)),
               self.ptr)

    def multigrid(self, prob: workloads.Problem, levels: int, sweeps: int, precision=TK_FP64, rfix=(0, 0, 0),
                  shortcut=True, fold=True, stream=None) -> "Result":
        """Multigrid Tucker (tk_multigrid): HOSVD on the grid `levels` dyadic
        coarsenings below prob's, then `sweeps` Tucker-ALS sweeps per grid."""
        k, g, o = self._structs(prob, precision, rfix, shortcut, fold, False)
        out = _vp()
        _check(self.lib.tk_multigrid(self.ptr, _c.byref(k), _c.byref(g), _c.byref(o), int(levels), int(sweeps),
                                     _c.byref(out), _stream_ptr(stream)), self.ptr)
        return Result(self, out, prob, k, g)

    def als(self, F, U, B, sweeps: int, stream=None):
        """Tucker-ALS sweeps on the device tensor F: the device factors U[k]
        (n_k x r_k) are updated in place, B (r1 x r2 x r3) receives the core.
        Returns the core norm^2 after each mode update (numpy, 3 * sweeps)."""
        n = (_i32 * 3)(*F.shape)
        r = (_i32 * 3)(*B.shape)
        hist = (_dbl * max(3 * sweeps, 1))()
        _check(self.lib.tk_als(self.ptr, F.data_ptr(), n, U[0].data_ptr(), U[1].data_ptr(), U[2].data_ptr(), r,
                               int(sweeps), B.data_ptr(), hist, _stream_ptr(stream)), self.ptr)
        return np.array(hist[: 3 * sweeps], dtype=np.float64)

    def tune(self, on: bool = True, cache_path=None) -> int:
        """Autotuning of the sliced Gram's K split (tk_tune); returns the choices held."""
        k = _c.c_int(0)
        path = None if cache_path is None else str(cache_path).encode()
        _check(self.lib.tk_tune(self.ptr, 1 if on else 0, path, _c.byref(k)), self.ptr)
        return int(k.value)

    def c2t(self, c, U, eps: float, sweeps: int, rmax=None, rfix=None, stream=None):
        """Canonical-to-Tucker (tk_c2t) of the device CP tensor (c: R, U[l]:
        n_l x R).  Returns (Result, core norm^2 after each mode update)."""
        R = int(c.shape[0])
        n = (_i32 * 3)(*(int(u.shape[0]) for u in U))
        rm = (_i32 * 3)(*rmax) if rmax is not None else None
        rf = (_i32 * 3)(*rfix) if rfix is not None else None
        hist = (_dbl * max(3 * sweeps, 1))()
        out = _vp()
        _check(self.lib.tk_c2t(self.ptr, R, c.data_ptr(), U[0].data_ptr(), U[1].data_ptr(), U[2].data_ptr(), n,
                               float(eps), rm, rf, int(sweeps), _c.byref(out), hist, _stream_ptr(stream)), self.ptr)
        prob = workloads.problem(n=tuple(int(v) for v in n), eps=eps)
        return Result(self, out, prob), np.array(hist[: 3 * sweeps], dtype=np.float64)


@dataclass
class Result:
    ctx: Context
    ptr: _vp
    prob: workloads.Problem
    kstruct: Kernel = None
    gstruct: Grid = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def free(self):
        if self.ptr is not None and self.ptr.value:
            self.ctx.lib.tk_result_free(self.ptr)
        self.ptr = None

    @property
    def ranks(self):
        r = (_i32 * 3)()
        f = (_u32 * 3)()
        _check(self.ctx.lib.tk_ranks(self.ptr, r, f))
        return [int(v) for v in r], [int(v) for v in f]

    def factor(self, mode: int) -> np.ndarray:
        r, _ = self.ranks
        out = np.empty((self.prob.n[mode], r[mode]), np.float64)
        _check(self.ctx.lib.tk_factor(self.ptr, int(mode), out.ctypes.data, 0, None), self.ctx.ptr)
        return out

    def core(self) -> np.ndarray:
        r, _ = self.ranks
        out = np.empty(tuple(r), np.float64)
        _check(self.ctx.lib.tk_core(self.ptr, out.ctypes.data, 0, None), self.ctx.ptr)
        return out

    def factors_and_core(self, stream=None):
        """(U_1, U_2, U_3, B) on the host through one staged copy (tk_result_copy)."""
        r, _ = self.ranks
        U = [np.empty((self.prob.n[a], r[a]), np.float64) for a in range(3)]
        B = np.empty(tuple(r), np.float64)
        _check(self.ctx.lib.tk_result_copy(self.ptr, U[0].ctypes.data, U[1].ctypes.data, U[2].ctypes.data,
                                           B.ctypes.data, _stream_ptr(stream)), self.ctx.ptr)
        return U[0], U[1], U[2], B

    def eigenvalues(self, mode: int, count: int = 96) -> np.ndarray:
        out = np.empty(count, np.float64)
        w = _c.c_int(0)
        _check(self.ctx.lib.tk_eigenvalues(self.ptr, int(mode), out.ctypes.data, count, _c.byref(w)))
        return out[: w.value].copy()

    @property
    def solve_error(self) -> float:
        """E computed during the solve (with_error=True)."""
        v = _dbl(0)
        _check(self.ctx.lib.tk_result_rel_error(self.ptr, _c.byref(v)))
        return v.value

    @property
    def norm2(self) -> float:
        v = _dbl(0)
        _check(self.ctx.lib.tk_norm2(self.ptr, _c.byref(v)))
        return v.value

    def reconstruct(self, dst, stream=None):
        _check(self.ctx.lib.tk_reconstruct(self.ctx.ptr, self.ptr, dst.data_ptr(), _stream_ptr(stream)),
               self.ctx.ptr)

    def rel_error(self, stream=None) -> float:
        k = self.kstruct if self.kstruct is not None else make_kernel(self.prob)
        g = self.gstruct if self.gstruct is not None else make_grid(self.prob)
        v = _dbl(0)
        _check(self.ctx.lib.tk_rel_error(self.ctx.ptr, self.ptr, _c.byref(k), _c.byref(g), _c.byref(v),
                                         _stream_ptr(stream)), self.ctx.ptr)
        return v.value
