"""Thin ctypes binding of libsgdtucker.so (include/sgd_tucker.h).

Functions keep the C names (std_create, std_sgd_epoch, ...) and only marshal
arguments: numpy arrays are passed as host pointers, torch tensors as their
device pointers (create the context with ptr_kind=1 for those).  Every
computation runs in the library's CUDA kernels; there is no fallback, and
importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

STD_OK = 0
STD_EINVAL = -1
STD_ENOMEM = -2
STD_ECUDA = -3
STD_ETIMEOUT = -4
STD_ENUMERIC = -5
STD_EUNSUPPORTED = -6
STD_MAX_ORDER = 6
STD_MAX_RANK = 32
STD_MAX_CORE = 16384
STD_MAX_MINIBATCH = 16384

_NAMES = {STD_EINVAL: "STD_EINVAL", STD_ENOMEM: "STD_ENOMEM", STD_ECUDA: "STD_ECUDA",
          STD_ETIMEOUT: "STD_ETIMEOUT", STD_ENUMERIC: "STD_ENUMERIC", STD_EUNSUPPORTED: "STD_EUNSUPPORTED"}


class StdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class std_options(ctypes.Structure):
    _fields_ = [
        ("r_core", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("norm_mode", ctypes.c_int32),
        ("init_mode", ctypes.c_int32),
        ("init_mu", ctypes.c_double),
        ("init_sigma", ctypes.c_double),
        ("seed_init", ctypes.c_uint64),
        ("seed_sched", ctypes.c_uint64),
        ("ptr_kind", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("watchdog_ns", ctypes.c_uint64),
        ("hbm_budget_bytes", ctypes.c_uint64),
        ("contraction", ctypes.c_int32),
        ("momentum", ctypes.c_float),
        ("snapshot", ctypes.c_int32),
        ("tile", ctypes.c_int32),
    ]


class std_epoch_stats(ctypes.Structure):
    _fields_ = [
        ("seconds", ctypes.c_double),
        ("sched_seconds", ctypes.c_double),
        ("update_seconds", ctypes.c_double),
        ("nnz_per_s", ctypes.c_double),
        ("nnz", ctypes.c_int64),
        ("batches", ctypes.c_int64),
        ("epoch", ctypes.c_int64),
    ]


class std_batch_stats(ctypes.Structure):
    _fields_ = [
        ("seconds", ctypes.c_double),
        ("update_seconds", ctypes.c_double),
        ("nnz_per_s", ctypes.c_double),
        ("nnz", ctypes.c_int64),
        ("tensors", ctypes.c_int32),
        ("ctas_per_tensor", ctypes.c_int32),
        ("graph_replayed", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class std_probe(ctypes.Structure):
    _fields_ = [
        ("core_V", ctypes.c_void_p),
        ("factor_F", ctypes.c_void_p),
        ("nseg", ctypes.c_void_p),
    ]


_lib = None

# Every symbol the header declares, with its ctypes signature.
_P = ctypes.c_void_p
SIGNATURES = {
    "std_default_options": (None, [_P]),
    "std_create": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "std_destroy": (ctypes.c_int, [_P]),
    "std_sgd_epoch": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_int32, _P]),
    "std_sgd_batches": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P]),
    "std_schedule": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P, _P, _P, _P]),
    "std_predict": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P]),
    "std_rmse": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P]),
    "std_get_params": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "std_set_params": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64]),
    "std_last_error": (ctypes.c_char_p, []),
    "std_rmse_static": (ctypes.c_int, [ctypes.c_int32, _P, _P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P,
                                       _P, _P]),
    "std_batch_create": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32]),
    "std_batch_epoch": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int32, _P]),
    "std_batch_destroy": (ctypes.c_int, [_P]),
    "std_batch_step": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_int32, ctypes.c_int64, _P]),
    "std_progress": (ctypes.c_int, [_P, _P, _P]),
    "std_reserve": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]),
    "std_device_bytes": (ctypes.c_int, [_P, _P]),
    "std_watchdog_probe": (ctypes.c_int, [ctypes.c_uint64, _P]),
    "std_batch_groups": (ctypes.c_int, [_P, _P]),
    "std_batch_tile": (ctypes.c_int, [_P, _P]),
    "std_batch_set_groups": (ctypes.c_int, [_P, _P]),
    "std_predict_many": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P]),
    "std_batch_reset": (ctypes.c_int, [_P, ctypes.c_int32, _P]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libsgdtucker.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(paper_2012_03550_gb300.build.build())")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def std_last_error() -> str:
    return lib().std_last_error().decode()


def _check(rc: int):
    if rc != STD_OK:
        raise StdError(rc, std_last_error())


def _addr(x) -> Optional[int]:
    """Host pointer of a numpy array or device pointer of a torch tensor."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)!r}")


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))(*[_addr(x) for x in items])
    return arr


def std_default_options() -> std_options:
    o = std_options()
    lib().std_default_options(ctypes.byref(o))
    return o


def std_create(order: int, mode_sizes: Sequence[int], ranks: Sequence[int], nnz: int, indices, values,
               opt: Optional[std_options] = None):
    """Returns an opaque context handle (ctypes.c_void_p)."""
    ms = np.ascontiguousarray(mode_sizes, dtype=np.int64)
    rk = np.ascontiguousarray(ranks, dtype=np.int32)
    ctx = ctypes.c_void_p()
    _check(lib().std_create(ctypes.byref(ctx), int(order), ms.ctypes.data, rk.ctypes.data, int(nnz),
                            _addr(indices), _addr(values), ctypes.byref(opt) if opt is not None else None))
    return ctx


def std_destroy(ctx) -> None:
    _check(lib().std_destroy(ctx))


def std_sgd_epoch(ctx, lr_a: float, lr_b: float, lambda_a: float, lambda_b: float, minibatch: int) -> dict:
    st = std_epoch_stats()
    _check(lib().std_sgd_epoch(ctx, lr_a, lr_b, lambda_a, lambda_b, int(minibatch), ctypes.byref(st)))
    return dict(seconds=st.seconds, sched_seconds=st.sched_seconds, update_seconds=st.update_seconds,
                nnz_per_s=st.nnz_per_s, nnz=st.nnz, batches=st.batches, epoch=st.epoch)


def std_sgd_batches(ctx, lr_a, lr_b, lambda_a, lambda_b, minibatch, batch_begin, batch_end, probe=None):
    """probe: None or a dict with numpy arrays 'core_V' [N,R,32], 'factor_F' [N,M,32], 'nseg' [N]."""
    p = None
    if probe is not None:
        p = std_probe(_addr(probe.get("core_V")), _addr(probe.get("factor_F")), _addr(probe.get("nseg")))
    _check(lib().std_sgd_batches(ctx, lr_a, lr_b, lambda_a, lambda_b, int(minibatch), int(batch_begin),
                                 int(batch_end), ctypes.byref(p) if p is not None else None))


def std_schedule(ctx, minibatch, batch_begin, batch_end, sample_ids=None, order=None, seg_start=None,
                 seg_end=None):
    _check(lib().std_schedule(ctx, int(minibatch), int(batch_begin), int(batch_end), _addr(sample_ids),
                              _addr(order), _addr(seg_start), _addr(seg_end)))


def std_predict(ctx, k: int, coords, out) -> None:
    _check(lib().std_predict(ctx, int(k), _addr(coords), _addr(out)))


def std_rmse(ctx, k: int, coords, values):
    r = ctypes.c_double()
    a = ctypes.c_double()
    _check(lib().std_rmse(ctx, int(k), _addr(coords), _addr(values), ctypes.byref(r), ctypes.byref(a)))
    return r.value, a.value


def std_get_params(ctx, A=None, B=None, core=None):
    """Fill the given buffers (lists of arrays / tensors, or None); returns the epoch counter."""
    ep = ctypes.c_int64()
    Ap = _ptr_array(A) if A is not None else None
    Bp = _ptr_array(B) if B is not None else None
    _check(lib().std_get_params(ctx, Ap, Bp, _addr(core), ctypes.byref(ep)))
    return ep.value


def std_set_params(ctx, A=None, B=None, epoch: int = -1) -> None:
    Ap = _ptr_array(A) if A is not None else None
    Bp = _ptr_array(B) if B is not None else None
    _check(lib().std_set_params(ctx, Ap, Bp, int(epoch)))


def check_static_args(order, mode_sizes, ranks, r_core, A, B, k, coords, values, out, current_device=None):
    """Host-side checks of std_rmse_static's arguments, raising ValueError.

    The library receives raw device pointers and cannot tell a host array, a
    tensor on another device, a wrong dtype or a short buffer from a valid
    one; any of those would make its kernels read out of bounds.  So every
    array must be a contiguous CUDA tensor on `current_device` (an index; the
    current device when None): A[n] float32 (I_n, J_n), B[n] float32 (J_n,
    r_core), coords int32 with at least k rows of N columns, values float32
    with at least k entries, out float64 with at least 2 entries."""
    order, r_core, k = int(order), int(r_core), int(k)
    mode_sizes = [int(x) for x in mode_sizes]
    ranks = [int(x) for x in ranks]
    if len(mode_sizes) != order or len(ranks) != order:
        raise ValueError("mode_sizes and ranks need one entry per mode")
    if len(A) != order or len(B) != order:
        raise ValueError("A and B need one matrix per mode")
    if k < 0:
        raise ValueError("k must be >= 0")
    if current_device is None:
        import torch
        if not torch.cuda.is_available():
            raise ValueError("std_rmse_static needs a CUDA device")
        current_device = torch.cuda.current_device()

    def tensor(x, what, dtype_name, shape=None, min_rows=None, min_numel=None):
        if not (hasattr(x, "is_cuda") and hasattr(x, "data_ptr")):
            raise ValueError(f"{what} must be a CUDA torch tensor, got {type(x).__name__}")
        if not x.is_cuda or x.device.index != current_device:
            raise ValueError(f"{what} must live on cuda:{current_device}, not {x.device}")
        if str(x.dtype) != f"torch.{dtype_name}":
            raise ValueError(f"{what} must be {dtype_name}, not {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError(f"{what} has shape {tuple(x.shape)}, expected {tuple(shape)}")
        if min_rows is not None and (x.dim() != 2 or x.shape[0] < min_rows[0] or x.shape[1] != min_rows[1]):
            raise ValueError(f"{what} has shape {tuple(x.shape)}, expected at least ({min_rows[0]}, {min_rows[1]})")
        if min_numel is not None and x.numel() < min_numel:
            raise ValueError(f"{what} has {x.numel()} entries, needs at least {min_numel}")

    for n in range(order):
        tensor(A[n], f"A[{n}]", "float32", shape=(mode_sizes[n], ranks[n]))
        tensor(B[n], f"B[{n}]", "float32", shape=(ranks[n], r_core))
    if k > 0:
        tensor(coords, "coords", "int32", min_rows=(k, order))
        tensor(values, "values", "float32", min_numel=k)
    tensor(out, "out", "float64", min_numel=2)


def std_rmse_static(order, mode_sizes, ranks, r_core, A, B, k, coords, values, out, stream=None) -> None:
    """Allocation-free RMSE/MAE: A, B lists of device tensors, coords/values/out
    device tensors (out: 2 float64); enqueued on `stream` (a cudaStream_t
    handle or None).  Read `out` after synchronising the stream.  The
    arguments are checked on the host first (check_static_args): a bad one
    raises ValueError and nothing is launched."""
    check_static_args(order, mode_sizes, ranks, r_core, A, B, k, coords, values, out)
    ms = np.ascontiguousarray(mode_sizes, dtype=np.int64)
    rk = np.ascontiguousarray(ranks, dtype=np.int32)
    _check(lib().std_rmse_static(int(order), ms.ctypes.data, rk.ctypes.data, int(r_core), _ptr_array(A),
                                 _ptr_array(B), int(k), _addr(coords), _addr(values), _addr(out), stream))


class Tucker:
    """Owning wrapper of one context (host-pointer or device-pointer mode)."""

    def __init__(self, shape, ranks, coords, values, r_core=5, ptr_kind=0, **opts):
        o = std_default_options()
        o.r_core = int(r_core)
        o.ptr_kind = int(ptr_kind)
        for k, v in opts.items():
            setattr(o, k, v)
        self.shape = tuple(int(s) for s in shape)
        self.ranks = tuple(int(j) for j in ranks)
        self.R = int(r_core)
        self.N = len(self.shape)
        self.ptr_kind = int(ptr_kind)
        if ptr_kind == 0:
            coords = np.ascontiguousarray(coords, dtype=np.int32)
            values = np.ascontiguousarray(values, dtype=np.float32)
        self.nnz = int(coords.shape[0])
        self.ctx = std_create(self.N, self.shape, self.ranks, self.nnz, coords, values, o)

    def close(self):
        if self.ctx is not None:
            std_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def epoch(self, lr_a, lr_b, lam_a, lam_b, minibatch):
        return std_sgd_epoch(self.ctx, lr_a, lr_b, lam_a, lam_b, minibatch)

    def batches(self, lr_a, lr_b, lam_a, lam_b, minibatch, b0, b1, probe=False):
        if not probe:
            std_sgd_batches(self.ctx, lr_a, lr_b, lam_a, lam_b, minibatch, b0, b1)
            return None
        pr = dict(core_V=np.zeros((self.N, self.R, STD_MAX_RANK), np.float32),
                  factor_F=np.zeros((self.N, minibatch, STD_MAX_RANK), np.float32),
                  nseg=np.zeros(self.N, np.int64))
        std_sgd_batches(self.ctx, lr_a, lr_b, lam_a, lam_b, minibatch, b0, b1, pr)
        return pr

    def schedule(self, minibatch, b0, b1):
        t0 = b0 * minibatch
        t1 = min(b1 * minibatch, self.nnz)
        cnt = max(0, t1 - t0)
        sid = np.zeros(cnt, np.int32)
        order = np.zeros((self.N, cnt), np.int32)
        s0 = np.zeros((self.N, cnt), np.int32)
        s1 = np.zeros((self.N, cnt), np.int32)
        std_schedule(self.ctx, minibatch, b0, b1, sid, order, s0, s1)
        return sid, order, s0, s1

    def predict(self, coords):
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        out = np.zeros(coords.shape[0], np.float32)
        std_predict(self.ctx, coords.shape[0], coords, out)
        return out

    def rmse(self, coords, values):
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        return std_rmse(self.ctx, coords.shape[0], coords, values)

    def get_params(self):
        A = [np.zeros((I, J), np.float32) for I, J in zip(self.shape, self.ranks)]
        B = [np.zeros((J, self.R), np.float32) for J in self.ranks]
        core = np.zeros(int(np.prod(self.ranks)), np.float32)
        ep = std_get_params(self.ctx, A, B, core)
        return A, B, core, ep

    def progress(self):
        return std_progress(self.ctx)

    def reserve(self, minibatch, ctas_per_tensor, max_query=0):
        std_reserve(self.ctx, minibatch, ctas_per_tensor, max_query)

    def device_bytes(self):
        return std_device_bytes(self.ctx)

    def set_params(self, A=None, B=None, epoch=-1):
        A = [np.ascontiguousarray(a, dtype=np.float32) for a in A] if A is not None else None
        B = [np.ascontiguousarray(b, dtype=np.float32) for b in B] if B is not None else None
        std_set_params(self.ctx, A, B, epoch)


def std_batch_create(ctxs, ctas_per_tensor=0):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    out = ctypes.c_void_p()
    _check(lib().std_batch_create(ctypes.byref(out), len(ctxs), ctypes.cast(arr, ctypes.c_void_p),
                                  int(ctas_per_tensor)))
    return out


def std_batch_epoch(batch, lr_a, lr_b, lambda_a, lambda_b, minibatch):
    st = std_batch_stats()
    _check(lib().std_batch_epoch(batch, lr_a, lr_b, lambda_a, lambda_b, int(minibatch), ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in std_batch_stats._fields_}


def std_batch_step(batch, lr_a, lr_b, lambda_a, lambda_b, minibatch, max_batches):
    st = std_batch_stats()
    _check(lib().std_batch_step(batch, lr_a, lr_b, lambda_a, lambda_b, int(minibatch), int(max_batches),
                                ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in std_batch_stats._fields_}


def std_progress(ctx):
    e = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(lib().std_progress(ctx, ctypes.byref(e), ctypes.byref(b)))
    return e.value, b.value


def std_reserve(ctx, minibatch, ctas_per_tensor, max_query=0):
    _check(lib().std_reserve(ctx, int(minibatch), int(ctas_per_tensor), int(max_query)))


def std_device_bytes(ctx):
    b = ctypes.c_uint64()
    _check(lib().std_device_bytes(ctx, ctypes.byref(b)))
    return b.value


def std_batch_groups(batch, count):
    out = (ctypes.c_int32 * int(count))()
    _check(lib().std_batch_groups(batch, ctypes.cast(out, ctypes.c_void_p)))
    return [int(x) for x in out]


def std_batch_tile(batch):
    out = ctypes.c_int32()
    _check(lib().std_batch_tile(batch, ctypes.byref(out)))
    return int(out.value)


def std_predict_many(ctxs, coords_list, outs):
    n = len(ctxs)
    carr = (ctypes.c_void_p * n)(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    karr = (ctypes.c_int64 * n)(*[int(x.shape[0]) for x in coords_list])
    parr = (ctypes.c_void_p * n)(*[_addr(x) for x in coords_list])
    oarr = (ctypes.c_void_p * n)(*[_addr(x) for x in outs])
    _check(lib().std_predict_many(n, ctypes.cast(carr, ctypes.c_void_p), ctypes.cast(karr, ctypes.c_void_p),
                                  ctypes.cast(parr, ctypes.c_void_p), ctypes.cast(oarr, ctypes.c_void_p)))


def predict_many(tuckers, coords_list):
    """Host numpy coordinates for several Tucker objects; one launch."""
    coords_list = [np.ascontiguousarray(c, dtype=np.int32) for c in coords_list]
    outs = [np.zeros(c.shape[0], np.float32) for c in coords_list]
    std_predict_many([t.ctx for t in tuckers], coords_list, outs)
    return outs


def std_batch_reset(batch, ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    _check(lib().std_batch_reset(batch, len(ctxs), ctypes.cast(arr, ctypes.c_void_p)))


def std_batch_set_groups(batch, sizes):
    arr = (ctypes.c_int32 * len(sizes))(*[int(x) for x in sizes])
    _check(lib().std_batch_set_groups(batch, ctypes.cast(arr, ctypes.c_void_p)))


def std_watchdog_probe(watchdog_ns):
    st = ctypes.c_int32()
    _check(lib().std_watchdog_probe(int(watchdog_ns), ctypes.byref(st)))
    return st.value


def std_batch_destroy(batch):
    _check(lib().std_batch_destroy(batch))


class Batch:
    """Owning wrapper of a batch over existing Tucker objects (which it does not own)."""

    def __init__(self, tuckers, ctas_per_tensor=0):
        self.members = list(tuckers)
        self.ptr = std_batch_create([t.ctx for t in self.members], ctas_per_tensor)

    def epoch(self, lr_a, lr_b, lam_a, lam_b, minibatch):
        return std_batch_epoch(self.ptr, lr_a, lr_b, lam_a, lam_b, minibatch)

    def step(self, lr_a, lr_b, lam_a, lam_b, minibatch, max_batches):
        return std_batch_step(self.ptr, lr_a, lr_b, lam_a, lam_b, minibatch, max_batches)

    def groups(self):
        return std_batch_groups(self.ptr, len(self.members))

    def tile(self):
        return std_batch_tile(self.ptr)

    def set_groups(self, sizes):
        std_batch_set_groups(self.ptr, sizes)

    def reset(self, tuckers):
        std_batch_reset(self.ptr, [t.ctx for t in tuckers])
        self.members = list(tuckers)

    def close(self):
        if self.ptr is not None:
            std_batch_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
