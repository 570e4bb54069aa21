"""ctypes binding of the FP64 SGD_Tucker oracle (sgdt_oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the benchmark's
CPU-baseline / reference legs.  It never imports the CUDA package and never
consumes anything the CUDA path produced.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgdt_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sgdt_oracle.c with the host C compiler into liboracle.so."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_dbl = ctypes.c_double


def _declare(L):
    L.orc_perm.restype = _u64
    L.orc_perm.argtypes = [_u64, _u64, _u64, _u64]
    L.orc_perm_range.restype = None
    L.orc_perm_range.argtypes = [_u64, _u64, _u64, _i64, _i64, _P]
    L.orc_unfold_column.restype = _i64
    L.orc_unfold_column.argtypes = [_int, _P, _int, _P]
    L.orc_unfold_digits_public.restype = None
    L.orc_unfold_digits_public.argtypes = [_int, _P, _int, _i64, _P]
    L.orc_stable_order.restype = _i64
    L.orc_stable_order.argtypes = [_i64, _P, _P, _P]
    common = [_int, _P, _P, _int, _P, _P]
    L.orc_build_core.restype = _int
    L.orc_build_core.argtypes = common + [_P]
    L.orc_predict.restype = _int
    L.orc_predict.argtypes = common + [_P, _i64, _P, _P]
    L.orc_rmse_mae.restype = _int
    L.orc_rmse_mae.argtypes = common + [_P, _i64, _P, _P, _P, _P]
    L.orc_core_gradient.restype = _int
    L.orc_core_gradient.argtypes = common + [_i64, _P, _P, _int, _int, _dbl, _int, _P]
    L.orc_factor_gradient.restype = _int
    L.orc_factor_gradient.argtypes = common + [_P, _i64, _P, _P, _int, ctypes.c_int32, _dbl, _int, _P]
    L.orc_step.restype = _int
    L.orc_step.argtypes = common + [_P, _i64, _P, _P, _dbl, _dbl, _dbl, _dbl, _int, _int, _P, _P, _P]
    L.orc_epoch.restype = _int
    L.orc_epoch.argtypes = common + [_P, _i64, _P, _P, _i64, _u64, _u64, _i64, _i64,
                                     _dbl, _dbl, _dbl, _dbl, _int]
    L.orc_step_momentum.restype = _int
    L.orc_step_momentum.argtypes = common + [_P, _i64, _P, _P, _dbl, _dbl, _dbl, _dbl, _int, _int, _P, _P, _P,
                                             _dbl, _P, _P]
    L.orc_epoch_snapshot.restype = _int
    L.orc_epoch_snapshot.argtypes = common + [_P, _i64, _P, _P, _i64, _u64, _u64, _i64, _i64, _i64,
                                              _dbl, _dbl, _dbl, _dbl, _int]
    L.orc_epoch_momentum.restype = _int
    L.orc_epoch_momentum.argtypes = common + [_P, _i64, _P, _P, _i64, _u64, _u64, _i64, _i64,
                                              _dbl, _dbl, _dbl, _dbl, _int, _dbl, _P, _P]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc):
    if rc != 0:
        raise RuntimeError(f"oracle call failed with code {rc}")


# ---------------------------------------------------------------------------
# Sampler and tiler
# ---------------------------------------------------------------------------

def perm(n: int, seed: int, epoch: int, t: int) -> int:
    return int(lib().orc_perm(n, seed, epoch, t))


def perm_range(n: int, seed: int, epoch: int, t0: int, count: int) -> np.ndarray:
    out = np.empty(max(count, 0), dtype=np.int64)
    if count > 0:
        lib().orc_perm_range(n, seed, epoch, t0, count, _ptr(out))
    return out


def epoch_schedule(n: int, seed: int, epoch: int) -> np.ndarray:
    return perm_range(n, seed, epoch, 0, n)


def unfold_column(dims: Sequence[int], n: int, index: Sequence[int]) -> int:
    """0-based column of entry `index` (0-based) in the mode-n unfolding."""
    d = np.ascontiguousarray(dims, dtype=np.int64)
    i = np.ascontiguousarray(index, dtype=np.int64)
    return int(lib().orc_unfold_column(len(dims), _ptr(d), int(n), _ptr(i)))


def unfold_digits(ranks: Sequence[int], n: int, c: int) -> np.ndarray:
    """Digits (j_k)_{k != n} of column c of a mode-n unfolding (-1 at k = n)."""
    J = np.ascontiguousarray(ranks, dtype=np.int32)
    out = np.empty(len(ranks), dtype=np.int32)
    lib().orc_unfold_digits_public(len(ranks), _ptr(J), int(n), int(c), _ptr(out))
    return out


def stable_order(keys: np.ndarray):
    """Sorted batch positions and segment offsets (U+1) for keys int32[m]."""
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    m = keys.shape[0]
    order = np.empty(m, dtype=np.int32)
    seg = np.empty(m + 1, dtype=np.int32)
    u = lib().orc_stable_order(m, _ptr(keys), _ptr(order), _ptr(seg))
    if u < 0:
        raise MemoryError
    return order, seg[: u + 1].copy()


# ---------------------------------------------------------------------------
# Model
# ---------------------------------------------------------------------------

class Model:
    """FP64 SGD_Tucker state: A_n (I_n x J_n), B_n (J_n x R), G-hat (prod J)."""

    def __init__(self, shape: Sequence[int], ranks: Sequence[int], r_core: int,
                 A: Sequence[np.ndarray], B: Sequence[np.ndarray], momentum: float = 0.0):
        self.N = len(shape)
        self.shape = np.ascontiguousarray(shape, dtype=np.int64)
        self.ranks = np.ascontiguousarray(ranks, dtype=np.int32)
        self.R = int(r_core)
        self.A = [np.ascontiguousarray(a, dtype=np.float64).copy() for a in A]
        self.B = [np.ascontiguousarray(b, dtype=np.float64).copy() for b in B]
        for n in range(self.N):
            assert self.A[n].shape == (int(shape[n]), int(ranks[n]))
            assert self.B[n].shape == (int(ranks[n]), self.R)
        self.G = np.zeros(int(np.prod(self.ranks.astype(np.int64))), dtype=np.float64)
        # heavy-ball momentum: velocities of the factor rows and Kruskal columns
        self.mu = float(momentum)
        self.VA = [np.zeros_like(a) for a in self.A] if self.mu != 0.0 else None
        self.VB = [np.zeros_like(b) for b in self.B] if self.mu != 0.0 else None

    def copy(self) -> "Model":
        return Model(self.shape, self.ranks, self.R, self.A, self.B, self.mu)

    def _vel(self):
        if self.VA is None:
            return [0.0, None, None]
        VAp = (ctypes.c_void_p * self.N)(*[a.ctypes.data for a in self.VA])
        VBp = (ctypes.c_void_p * self.N)(*[b.ctypes.data for b in self.VB])
        self._keepv = (VAp, VBp)
        return [self.mu, ctypes.cast(VAp, ctypes.c_void_p), ctypes.cast(VBp, ctypes.c_void_p)]

    def _args(self):
        Ap = (ctypes.c_void_p * self.N)(*[a.ctypes.data for a in self.A])
        Bp = (ctypes.c_void_p * self.N)(*[b.ctypes.data for b in self.B])
        self._keep = (Ap, Bp)
        return [self.N, _ptr(self.shape), _ptr(self.ranks), self.R,
                ctypes.cast(Ap, ctypes.c_void_p), ctypes.cast(Bp, ctypes.c_void_p)]

    def build_core(self) -> np.ndarray:
        """G-hat from B (Eq. 4), mode-1-fastest vector of length prod J."""
        _check(lib().orc_build_core(*self._args(), _ptr(self.G)))
        return self.G

    def core_tensor(self) -> np.ndarray:
        """G-hat as a numpy array indexed [j1, j2, ..., jN]."""
        g = self.build_core()
        return g.reshape(tuple(int(j) for j in self.ranks), order="F")

    def predict(self, coords: np.ndarray) -> np.ndarray:
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        out = np.empty(coords.shape[0], dtype=np.float64)
        _check(lib().orc_predict(*self._args(), _ptr(self.G), coords.shape[0], _ptr(coords), _ptr(out)))
        return out

    def rmse_mae(self, coords: np.ndarray, values: np.ndarray):
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        r = ctypes.c_double()
        a = ctypes.c_double()
        _check(lib().orc_rmse_mae(*self._args(), _ptr(self.G), coords.shape[0], _ptr(coords),
                                  _ptr(values), ctypes.byref(r), ctypes.byref(a)))
        return r.value, a.value

    def core_gradient(self, coords, values, n, r, lambda_b, literal=False) -> np.ndarray:
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        out = np.empty(int(self.ranks[n]), dtype=np.float64)
        _check(lib().orc_core_gradient(*self._args(), coords.shape[0], _ptr(coords), _ptr(values),
                                       int(n), int(r), float(lambda_b), int(bool(literal)), _ptr(out)))
        return out

    def factor_gradient(self, coords, values, n, row, lambda_a, norm_mode=0) -> np.ndarray:
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        out = np.empty(int(self.ranks[n]), dtype=np.float64)
        _check(lib().orc_factor_gradient(*self._args(), _ptr(self.G), coords.shape[0], _ptr(coords),
                                         _ptr(values), int(n), int(row), float(lambda_a),
                                         int(norm_mode), _ptr(out)))
        return out

    def step(self, coords, values, lr_a, lr_b, lam_a, lam_b, norm_mode=0, literal=False,
             probe=False):
        """One minibatch of Algorithm 1; returns (V, F, nseg) when probe."""
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        m = coords.shape[0]
        jmax = int(self.ranks.max())
        V = F = nseg = None
        pV = pF = pS = None
        if probe:
            V = np.zeros((self.N, self.R, jmax), dtype=np.float64)
            F = np.zeros((self.N, m, jmax), dtype=np.float64)
            nseg = np.zeros(self.N, dtype=np.int64)
            pV, pF, pS = _ptr(V), _ptr(F), _ptr(nseg)
        _check(lib().orc_step_momentum(*self._args(), _ptr(self.G), m, _ptr(coords), _ptr(values),
                                       float(lr_a), float(lr_b), float(lam_a), float(lam_b), int(norm_mode),
                                       int(bool(literal)), pV, pF, pS, *self._vel()))
        if probe:
            return V, F, nseg
        return None

    def epoch(self, coords, values, M, seed, epoch, lr_a, lr_b, lam_a, lam_b, norm_mode=0,
              batch_begin=0, batch_end=None):
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        n = coords.shape[0]
        if batch_end is None:
            batch_end = (n + M - 1) // M
        _check(lib().orc_epoch_momentum(*self._args(), _ptr(self.G), n, _ptr(coords), _ptr(values), int(M),
                                        int(seed), int(epoch), int(batch_begin), int(batch_end),
                                        float(lr_a), float(lr_b), float(lam_a), float(lam_b), int(norm_mode),
                                        *self._vel()))
        self.build_core()

    def epoch_snapshot(self, coords, values, M, seed, epoch, K, lr_a, lr_b, lam_a, lam_b, norm_mode=0,
                       batch_begin=0, batch_end=None):
        """K-snapshot form: minibatches in blocks of K (from batch_begin), each
        minibatch of a block stepping from the block's starting model, their
        changes added to it in minibatch order (orc_epoch_snapshot)."""
        if self.mu != 0.0 and K > 1:
            raise ValueError("momentum is not defined for the K-snapshot form")
        coords = np.ascontiguousarray(coords, dtype=np.int32)
        values = np.ascontiguousarray(values, dtype=np.float32)
        n = coords.shape[0]
        if batch_end is None:
            batch_end = (n + M - 1) // M
        _check(lib().orc_epoch_snapshot(*self._args(), _ptr(self.G), n, _ptr(coords), _ptr(values), int(M),
                                        int(seed), int(epoch), int(batch_begin), int(batch_end), int(K),
                                        float(lr_a), float(lr_b), float(lam_a), float(lam_b), int(norm_mode)))
