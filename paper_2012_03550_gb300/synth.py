"""Seeded synthetic inputs for SGD_Tucker workloads.

This module only manufactures inputs: sparse coordinates, their values, the
train/test split and initial parameter values.  It holds none of the SGD_Tucker
update arithmetic, imports nothing else from this package, and is the single
source of inputs for both the CUDA path and the FP64 oracle, so the two always
see bit-identical arrays.

The paper's datasets (MovieLens, Netflix, Yahoo-music; Sec. 5.1, Table 3) are
not available, so seeded stand-ins with the same shapes are drawn here:

* mode indices are uniform or Zipf(s) distributed (rank r in [1, I] with
  probability proportional to r**-s, drawn by inverse CDF over an FP64 table,
  rank r mapped to index r-1);
* coordinates are distinct: duplicates are rejected and redrawn in draw order
  (vectorised, equivalent to sequential rejection);
* values come from a planted dense Tucker model (Def. 6) with core and factors
  i.i.d. N(0,1)/sqrt(J), plus Gaussian noise; the rating-like workload maps
  them affinely to mean 3 and rounds half-to-even into {1..5} (Table 3 range).

All randomness comes from numpy's PCG64 seeded through SeedSequence, one
independent child stream per purpose, so every array is reproducible on any
machine from (seed, purpose).
"""
from __future__ import annotations

import concurrent.futures
import ctypes
import dataclasses
import math
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

# Purposes of the child streams spawned from the data seed.
_STREAM_COORDS = 0
_STREAM_MODEL = 1
_STREAM_NOISE = 2
_STREAM_SPLIT = 3


@dataclasses.dataclass
class SparseTensor:
    """A sparse N-order tensor in COO form with a train/test split.

    coords: int32 [nnz, N], 0-based; values: float32 [nnz].
    train / test: int64 index arrays into coords (ascending).
    """

    shape: tuple
    coords: np.ndarray
    values: np.ndarray
    train: np.ndarray
    test: np.ndarray
    meta: dict

    @property
    def order(self) -> int:
        return len(self.shape)

    def split(self, which: str):
        idx = self.train if which == "train" else self.test
        return (np.ascontiguousarray(self.coords[idx]),
                np.ascontiguousarray(self.values[idx]))


def _children(seed: int, n: int = 4):
    return np.random.SeedSequence(seed).spawn(n)


def zipf_table(size: int, s: float) -> np.ndarray:
    """FP64 cumulative table of p(r) ~ r**-s over ranks 1..size."""
    w = np.arange(1, size + 1, dtype=np.float64) ** (-float(s))
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def draw_mode_indices(rng: np.random.Generator, count: int, size: int,
                      dist: str = "uniform", s: float = 0.0,
                      table: Optional[np.ndarray] = None) -> np.ndarray:
    """Draw `count` indices in [0, size) uniformly or Zipf(s) by inverse CDF."""
    if dist == "uniform":
        return rng.integers(0, size, size=count, dtype=np.int64)
    if dist == "zipf":
        if table is None:
            table = zipf_table(size, s)
        u = rng.random(count)
        step = 1 << 22
        parts = _parallel(lambda lo: np.searchsorted(table, u[lo:lo + step], side="right"),
                          list(range(0, count, step)))
        r = np.concatenate(parts) if parts else np.empty(0, dtype=np.int64)
        return np.minimum(r, size - 1).astype(np.int64)
    raise ValueError(f"unknown distribution {dist!r}")


_DEDUP_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "synth_dedup.c")
_DEDUP_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsynth_dedup.so")
_dedup = None


def build_native(force: bool = False) -> str:
    """Compile the generator's C helper (first-occurrence hash set)."""
    if (not force and os.path.exists(_DEDUP_LIB)
            and os.path.getmtime(_DEDUP_LIB) >= os.path.getmtime(_DEDUP_SRC)):
        return _DEDUP_LIB
    tmp = _DEDUP_LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _DEDUP_SRC], check=True)
    os.replace(tmp, _DEDUP_LIB)
    return _DEDUP_LIB


def _dedup_lib():
    global _dedup
    if _dedup is None:
        L = ctypes.CDLL(build_native())
        L.synth_first_unique.restype = ctypes.c_int64
        L.synth_first_unique.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_int64]
        _dedup = L
    return _dedup


def _parallel(fn, items, workers=None):
    workers = workers or min(16, os.cpu_count() or 4)
    if len(items) <= 1 or workers <= 1:
        return [fn(x) for x in items]
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


def distinct_coords(rng: np.random.Generator, shape: Sequence[int], nnz: int,
                    dists: Sequence[tuple]) -> np.ndarray:
    """Draw `nnz` distinct coordinates; duplicates are rejected in draw order.

    dists[n] is ("uniform",) or ("zipf", s).  Returns int32 [nnz, N].
    Coordinates are drawn in rounds appended to one stream; a hash set keeps
    the first occurrence of each cell in draw order (the result of drawing one
    coordinate at a time and rejecting repeats).  Round sizes adapt to the
    observed acceptance rate.
    """
    N = len(shape)
    cells = 1
    for d in shape:
        cells *= int(d)
    if nnz > cells:
        raise ValueError("more nonzeros than cells")
    tables = [zipf_table(int(shape[n]), dists[n][1]) if dists[n][0] == "zipf" else None
              for n in range(N)]
    strides = np.ones(N, dtype=np.int64)
    for n in range(1, N):
        strides[n] = strides[n - 1] * int(shape[n - 1])
    cap = 1
    while cap < 2 * nnz + 16:
        cap <<= 1
    table = np.zeros(cap, dtype=np.uint64)
    out = np.empty((nnz, N), dtype=np.int32)
    idx = np.empty(nnz, dtype=np.int64)
    L = _dedup_lib()
    accept_rate = 0.9
    have = 0
    for _ in range(1000):
        need = nnz - have
        if need <= 0:
            break
        draw = int(need / max(accept_rate, 0.02) * 1.05) + 1024
        cols = [draw_mode_indices(rng, draw, int(shape[n]), dists[n][0],
                                  dists[n][1] if len(dists[n]) > 1 else 0.0, tables[n])
                for n in range(N)]
        keys = np.zeros(draw, dtype=np.int64)
        for n in range(N):
            keys += cols[n] * strides[n]
        got = int(L.synth_first_unique(keys.ctypes.data, draw, need, idx.ctypes.data + 8 * have,
                                       table.ctypes.data, cap))
        sel = idx[have:have + got]
        for n in range(N):
            out[have:have + got, n] = cols[n][sel]
        have += got
        accept_rate = max(got / float(draw), 1e-3)
    else:
        raise RuntimeError("coordinate rejection did not converge")
    return out


def planted_tucker(rng: np.random.Generator, shape: Sequence[int], ranks: Sequence[int]):
    """Dense core G (J_1 x ... x J_N, numpy C order [j1, j2, ...]) and factors
    A_n (I_n x J_n), all i.i.d. N(0,1)/sqrt(J) with J = J_n (core: mean rank)."""
    N = len(shape)
    jbar = float(np.mean(ranks))
    core = rng.standard_normal(tuple(int(j) for j in ranks)) / math.sqrt(jbar)
    factors = [rng.standard_normal((int(shape[n]), int(ranks[n]))) / math.sqrt(float(ranks[n]))
               for n in range(N)]
    return core, factors


def planted_values(core: np.ndarray, factors: Sequence[np.ndarray], coords: np.ndarray,
                   chunk: int = 1 << 18) -> np.ndarray:
    """Evaluate the planted dense Tucker model at `coords` in FP64 (numpy
    contractions, chunked): sum over j of core[j] * prod_n factors[n][i_n, j_n].
    The core is contracted with mode 1 by a GEMM, then with the remaining
    modes from the last one inwards."""
    N = coords.shape[1]
    out = np.empty(coords.shape[0], dtype=np.float64)
    J0 = core.shape[0]
    core0 = core.reshape(J0, -1)

    def one(lo):
        hi = min(lo + chunk, coords.shape[0])
        c = coords[lo:hi]
        t = (factors[0][c[:, 0]] @ core0).reshape((hi - lo,) + core.shape[1:])
        for n in range(N - 1, 0, -1):
            a = factors[n][c[:, n]]                     # [m, Jn]
            t = (t * a.reshape((hi - lo,) + (1,) * (n - 1) + (a.shape[1],))).sum(axis=-1)
        out[lo:hi] = t

    _parallel(one, list(range(0, coords.shape[0], chunk)))
    return out


def split_indices(rng: np.random.Generator, nnz: int, test_frac: float):
    n_test = int(round(test_frac * nnz))
    perm = rng.permutation(nnz)
    test = np.sort(perm[:n_test])
    train = np.sort(perm[n_test:])
    return train.astype(np.int64), test.astype(np.int64)


def make_tensor(shape, nnz, dists, ranks, noise_sd, test_frac, seed=0,
                rating=False) -> SparseTensor:
    """Generic planted-Tucker sparse tensor.

    rating=True: y = 3 + z/sd(z) + N(0, noise_sd^2), rounded half-to-even
    and clamped into {1..5}; otherwise y = z + N(0, noise_sd^2).
    """
    ch = _children(seed)
    rc = np.random.Generator(np.random.PCG64(ch[_STREAM_COORDS]))
    rm = np.random.Generator(np.random.PCG64(ch[_STREAM_MODEL]))
    rn = np.random.Generator(np.random.PCG64(ch[_STREAM_NOISE]))
    rs = np.random.Generator(np.random.PCG64(ch[_STREAM_SPLIT]))
    coords = distinct_coords(rc, shape, nnz, dists)
    core, factors = planted_tucker(rm, shape, ranks)
    z = planted_values(core, factors, coords)
    if rating:
        sd = float(np.std(z))
        y = 3.0 + z / (sd if sd > 0 else 1.0) + noise_sd * rn.standard_normal(z.shape[0])
        y = np.clip(np.rint(y), 1.0, 5.0)
    else:
        y = z + noise_sd * rn.standard_normal(z.shape[0])
    train, test = split_indices(rs, coords.shape[0], test_frac)
    meta = dict(shape=tuple(int(s) for s in shape), nnz=int(nnz), dists=[tuple(d) for d in dists],
                ranks=tuple(int(j) for j in ranks), noise_sd=float(noise_sd), rating=bool(rating),
                seed=int(seed), test_frac=float(test_frac))
    return SparseTensor(tuple(int(s) for s in shape), coords, y.astype(np.float32), train, test, meta)


# ---------------------------------------------------------------------------
# The named workloads (shapes from Table 3 of the paper; planted models as the
# workload definitions state).  `scale` < 1 shrinks nnz and mode sizes together
# (same distributions) for oracle-sized parity runs.
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    tensor: SparseTensor
    ranks: tuple
    r_core: int
    minibatch: int
    lr: float
    lam: float
    epochs: int


def _scaled(v, scale, lo=2):
    return max(lo, int(round(v * scale)))


def config1(seed: int = 0) -> Workload:
    """500x400x300, 50,000 distinct uniform coordinates, planted J=(5,5,5),
    noise N(0, 0.01^2), 90/10 split, M=256, lr=lambda=1e-3, 10 epochs, R=5."""
    t = make_tensor((500, 400, 300), 50_000, [("uniform",)] * 3, (5, 5, 5), 0.01, 0.1, seed)
    return Workload("uniform-500x400x300-50k", t, (5, 5, 5), 5, 256, 1e-3, 1e-3, 10)


def config2(scale: float = 1.0, seed: int = 0) -> Workload:
    """Netflix-shaped rating tensor 480,189 x 17,770 x 2,182 with 100M nonzeros;
    Zipf 1.1 (users), Zipf 1.3 (items), uniform (time); planted J=(10,10,10),
    values quantised into {1..5} with N(0, 0.3^2) noise; 99/1 split; J=10, R=5,
    M=4096, lr=0.05, lambda=1e-3, 20 epochs.  The learning rate is not part of
    the workload's definition: with the 1/M normaliser of Eq. 18, lr = 1e-3
    leaves the model at its initial test RMSE, while 0.05 lowers it steadily
    (measured with the FP64 oracle at 0.4% scale: 0.998, 0.990, 0.986, 0.983
    after epochs 1-4 against a spread of 0.995)."""
    shape = (_scaled(480_189, scale), _scaled(17_770, scale), _scaled(2_182, math.sqrt(scale) if scale < 1 else 1.0))
    nnz = _scaled(100_000_000, scale, lo=1000)
    t = make_tensor(shape, nnz, [("zipf", 1.1), ("zipf", 1.3), ("uniform",)], (10, 10, 10),
                    0.3, 0.01, seed, rating=True)
    return Workload(f"netflix-like-{shape[0]}x{shape[1]}x{shape[2]}-{nnz}", t, (10, 10, 10), 5,
                    4096, 0.05, 1e-3, 20)


def config3(scale: float = 1.0, seed: int = 0) -> Workload:
    """4-order 200,000 x 100,000 x 500 x 24 with 50M nonzeros; Zipf 1.2 on the
    first two modes, uniform on the last two; planted J=(8,8,8,8) + N(0,0.05^2);
    M=8192, 90/10 split, R=5, 10 epochs."""
    shape = (_scaled(200_000, scale), _scaled(100_000, scale), _scaled(500, math.sqrt(scale) if scale < 1 else 1.0), 24)
    nnz = _scaled(50_000_000, scale, lo=1000)
    t = make_tensor(shape, nnz, [("zipf", 1.2), ("zipf", 1.2), ("uniform",), ("uniform",)],
                    (8, 8, 8, 8), 0.05, 0.1, seed)
    return Workload(f"4order-{shape[0]}x{shape[1]}x{shape[2]}x{shape[3]}-{nnz}", t, (8, 8, 8, 8), 5,
                    8192, 1e-3, 1e-3, 10)


# The paper's parameter study varies the model ranks on a fixed dataset: J_n
# from 5 to 25 and R_core from 10 to 25.  Sweep points: J_1 in {5..25} with
# J_2 = J_3 = 5 and R_core = 5, then R_core in {10..25} with J = (5, 5, 5).
RANK_SWEEP = [((J, 5, 5), 5) for J in (5, 10, 15, 20, 25)] + [((5, 5, 5), R) for R in (10, 15, 20, 25)]


def ranksweep(scale: float = 0.05, seed: int = 0):
    """The rank-sweep workload: one rating tensor with config 2's shape and
    distributions at `scale` (the data stay fixed across the sweep), and the
    (ranks, R_core) points of RANK_SWEEP.  M = 4096, lr = 0.05, lambda = 1e-3."""
    return config2(scale=scale, seed=seed), list(RANK_SWEEP)


def config4_specs(count: int = 256, seed: int = 0, nnz_scale: float = 1.0):
    """Shapes of the batched workload: `count` independent 3-order tensors with
    mode sizes lognormal(ln 7000, 1) clipped to [1e3, 5e4], nonzeros
    lognormal(ln 1.5e5, 1) clipped to [1e4, 2e6] (capped by 40% of the cells),
    J drawn from {4, 8, 16}, R = min(5, J)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 4])))
    specs = []
    for t in range(count):
        dims = np.clip(np.exp(rng.normal(math.log(7000.0), 1.0, size=3)), 1e3, 5e4).astype(np.int64)
        nnz = float(np.clip(math.exp(rng.normal(math.log(1.5e5), 1.0)), 1e4, 2e6))
        nnz = int(min(nnz * nnz_scale, 0.4 * float(np.prod(dims.astype(np.float64)))))
        J = int(rng.choice([4, 8, 16]))
        specs.append(dict(shape=tuple(int(d) for d in dims), nnz=max(nnz, 64), J=J, R=min(5, J),
                          seed=int(seed * 100003 + t + 1)))
    return specs


def config4_tensor(spec) -> SparseTensor:
    J = spec["J"]
    return make_tensor(spec["shape"], spec["nnz"], [("uniform",)] * 3, (J, J, J), 0.05, 0.1,
                       spec["seed"])


def serve_specs(count: int, seed: int = 0):
    """Job shapes of the serving workload: the batched workload's size
    distribution with order 3 or 4 (even odds).  Mode sizes lognormal(ln 7000,
    1) clipped to [1e3, 5e4], nonzeros lognormal(ln 1.5e5, 1) clipped to
    [1e4, 2e6], J from {4, 8, 16} for order 3 and from {4, 8} for order 4
    (16^4 core entries exceed the library's core limit), R = min(5, J)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 5])))
    specs = []
    for t in range(count):
        order = int(rng.choice([3, 4]))
        dims = np.clip(np.exp(rng.normal(math.log(7000.0), 1.0, size=order)), 1e3, 5e4).astype(np.int64)
        nnz = float(np.clip(math.exp(rng.normal(math.log(1.5e5), 1.0)), 1e4, 2e6))
        nnz = int(min(nnz, 0.4 * float(np.prod(dims.astype(np.float64)))))
        J = int(rng.choice([4, 8, 16] if order == 3 else [4, 8]))
        specs.append(dict(shape=tuple(int(d) for d in dims), nnz=max(nnz, 64), J=J, R=min(5, J),
                          seed=int(seed * 100003 + t + 7)))
    return specs


def serve_tensor(spec) -> SparseTensor:
    J = spec["J"]
    N = len(spec["shape"])
    return make_tensor(spec["shape"], spec["nnz"], [("uniform",)] * N, (J,) * N, 0.05, 0.1, spec["seed"])


# ---------------------------------------------------------------------------
# Initial parameters.  The paper initialises everything from N(0.5, 0.1^2)
# (Sec. 5.1); for zero-mean planted data the default is N(0, 1/J).
# ---------------------------------------------------------------------------

def init_params(shape, ranks, r_core, mode="normal", seed=1, mean_value=None,
                mu=0.5, sigma=0.1):
    """Initial factor matrices A_n (I_n x J_n) and Kruskal matrices B_n (J_n x R),
    float32, row-major.

    mode "normal": A, B i.i.d. N(0, 1/J_n).
    mode "paper":  everything N(mu, sigma^2) (paper: 0.5, 0.1).
    mode "rating": N(m, (m/5)^2) with m = (mean_value/R)^(1/(2N)) / sqrt(J), so
                   that the initial prediction is close to mean_value.
    """
    N = len(shape)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    A, B = [], []
    for n in range(N):
        I, J = int(shape[n]), int(ranks[n])
        if mode == "normal":
            a = rng.standard_normal((I, J)) / math.sqrt(J)
            b = rng.standard_normal((J, r_core)) / math.sqrt(J)
        elif mode == "paper":
            a = mu + sigma * rng.standard_normal((I, J))
            b = mu + sigma * rng.standard_normal((J, r_core))
        elif mode == "rating":
            if mean_value is None:
                raise ValueError("rating init needs mean_value")
            m = (float(mean_value) / r_core) ** (1.0 / (2 * N)) / math.sqrt(J)
            a = m + (m / 5.0) * rng.standard_normal((I, J))
            b = m + (m / 5.0) * rng.standard_normal((J, r_core))
        else:
            raise ValueError(f"unknown init mode {mode!r}")
        A.append(np.ascontiguousarray(a, dtype=np.float32))
        B.append(np.ascontiguousarray(b, dtype=np.float32))
    return A, B


def random_coords(shape, k, seed=5, dist=None) -> np.ndarray:
    """k query coordinates (int32 [k, N]); uniform unless dist gives per-mode
    ("zipf", s) entries."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 11])))
    cols = []
    for n, I in enumerate(shape):
        d = dist[n] if dist is not None else ("uniform",)
        cols.append(draw_mode_indices(rng, k, int(I), d[0], d[1] if len(d) > 1 else 0.0))
    return np.stack(cols, axis=1).astype(np.int32)
