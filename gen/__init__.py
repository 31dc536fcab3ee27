"""Seeded synthetic inputs shaped like the paper's SpMM workloads.

The paper evaluates on SuiteSparse matrices (Section 5.1) and on synthetic
dense-as-CSR and fixed-density matrices (Fig. 1, Fig. 7).  None of those
datasets are used here: every input is drawn from a seed by this module, with
the shapes, row-length distributions and value distributions of the five
workloads the library is measured on:

* ``uniform_rows``  - every row has the same number of nonzeros (uniform
  columns without replacement, sorted), values U[-1, 1].
* ``power_law``     - row lengths from a discrete power law (density exponent
  2.0, minimum 1, mean about 16, capped), plus a fraction of empty rows.
* ``chung_lu_gcn``  - symmetric-normalised adjacency D^-1/2 (S + I) D^-1/2 of a
  Chung-Lu power-law graph (a GNN layer's propagation matrix).
* ``batched_set``   - many independent CSR matrices of log-uniform size with
  Poisson row lengths, each with its own dense right-hand side width.

This module holds none of the SpMM method's arithmetic; it only draws random
numbers and lays them out as CSR arrays.  Both the CPU oracle and the GPU
library consume what it returns.  Bulk arrays are filled by ``csrgen.c``
(counter-based, thread-count independent); small shape decisions use NumPy's
``default_rng``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrgen.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcsrgen.so")
_lock = threading.Lock()
_lib = None

# seeds of the five measured workloads: 1803 + workload number
SEED_BASE = 1803


def build(force: bool = False) -> str:
    """Compile csrgen.c into gen/_build/libcsrgen.so (gcc, OpenMP when available)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            vp = ctypes.c_void_p
            lib.gen_fill_columns.argtypes = [i32, i32, vp, u64, vp]
            lib.gen_fill_columns.restype = ctypes.c_int
            lib.gen_fill_uniform_f32.argtypes = [i64, u64, u64, ctypes.c_float, ctypes.c_float, vp]
            lib.gen_fill_uniform_f32.restype = None
            lib.gen_fill_normal_f32.argtypes = [i64, u64, u64, vp]
            lib.gen_fill_normal_f32.restype = None
            lib.gen_num_threads.argtypes = []
            lib.gen_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values (sort + neighbour mask; faster than np.unique here)."""
    x = np.sort(x)
    if x.size == 0:
        return x
    keep = np.empty(x.size, dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


@dataclasses.dataclass
class CSR:
    """A CSR matrix: 0-based int32 row offsets and column indices, float32 values."""

    m: int
    k: int
    row_ptr: np.ndarray  # int32 [m + 1]
    col_ind: np.ndarray  # int32 [nnz]
    vals: np.ndarray  # float32 [nnz]
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.m > 0 else 0

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


# ----------------------------------------------------------------------------- bulk fills

def uniform_values(count: int, seed: int, stream: int = 1, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    out = np.empty(count, dtype=np.float32)
    if count:
        _load().gen_fill_uniform_f32(count, seed, stream, lo, hi, _ptr(out))
    return out


def normal_matrix(rows: int, cols: int, seed: int, stream: int = 2) -> np.ndarray:
    """Row-major float32 N(0, 1) matrix."""
    out = np.empty((rows, cols), dtype=np.float32)
    if out.size:
        _load().gen_fill_normal_f32(out.size, seed, stream, _ptr(out))
    return out


def csr_from_lengths(lengths: np.ndarray, k: int, seed: int, value_stream: int = 1,
                     col_stream_seed: int | None = None) -> CSR:
    """Build a CSR pattern with the given row lengths, distinct uniform sorted columns
    per row, and U[-1, 1] values."""
    lengths = np.asarray(lengths, dtype=np.int64)
    m = int(lengths.shape[0])
    rp64 = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp64[1:])
    nnz = int(rp64[-1])
    if nnz >= 2**31:
        raise ValueError("nnz must fit in int32")
    col = np.empty(nnz, dtype=np.int32)
    if nnz:
        cs = seed if col_stream_seed is None else col_stream_seed
        if _load().gen_fill_columns(m, k, _ptr(rp64), (cs * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF, _ptr(col)) != 0:
            raise ValueError("a row is longer than k")
    vals = uniform_values(nnz, seed, value_stream)
    return CSR(m, k, rp64.astype(np.int32), col, vals)


# ----------------------------------------------------------------------------- workloads

def uniform_rows(m: int, k: int, per_row: int, seed: int) -> CSR:
    """Every row holds exactly ``per_row`` nonzeros."""
    csr = csr_from_lengths(np.full(m, per_row, dtype=np.int64), k, seed)
    csr.info.update(kind="uniform", per_row=per_row, seed=seed)
    return csr


def power_law_lengths(m: int, k: int, seed: int, exponent: float = 2.0, mean: float = 16.0,
                      cap: int = 100_000, empty_frac: float = 0.01) -> tuple[np.ndarray, dict]:
    """Row lengths floor(x_min / U^(1/(exponent-1))), U ~ U(0, 1], capped at min(cap, k).

    With exponent 2 the length density falls as x^-2 with minimum 1.  x_min is
    calibrated by bisection on the seeded draw so the mean over non-empty rows is
    ``mean``; then a seeded ``empty_frac`` of the rows is emptied.
    """
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(m)  # (0, 1]
    cap = min(cap, k)
    tail = u ** (-1.0 / (exponent - 1.0))

    def lengths_for(x_min: float) -> np.ndarray:
        return np.minimum(cap, np.floor(x_min * tail)).astype(np.int64)

    lo, hi = 1.0, float(max(2.0, mean))
    while lengths_for(hi).mean() < mean and hi < cap:
        hi *= 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if lengths_for(mid).mean() < mean:
            lo = mid
        else:
            hi = mid
    x_min = 0.5 * (lo + hi)
    lengths = np.maximum(lengths_for(x_min), 1)
    n_empty = int(round(empty_frac * m))
    if n_empty:
        lengths[rng.choice(m, size=n_empty, replace=False)] = 0
    return lengths, {"x_min": x_min, "cap": cap, "empty_rows": n_empty,
                     "rows_at_cap": int((lengths == cap).sum()), "max_row": int(lengths.max(initial=0))}


def power_law(m: int, k: int, seed: int, **kw) -> CSR:
    lengths, info = power_law_lengths(m, k, seed, **kw)
    csr = csr_from_lengths(lengths, k, seed)
    csr.info.update(kind="power_law", seed=seed, **info)
    return csr


def chung_lu_gcn(m: int, seed: int, exponent: float = 2.2, mean_degree: float = 20.0) -> CSR:
    """Symmetric-normalised adjacency D^-1/2 (S + I) D^-1/2 of a Chung-Lu graph.

    Weights w_i follow a Pareto law with density exponent ``exponent`` scaled to
    mean ``mean_degree``; sum(w)/2 edges are drawn with both endpoints chosen
    proportionally to w; self-loops and repeated pairs are dropped; the graph is
    symmetrised, the identity is added, and each stored entry (i, j) gets the value
    1/sqrt(d_i d_j) with d the row counts of S + I.
    """
    rng = np.random.default_rng(seed)
    w = (1.0 - rng.random(m)) ** (-1.0 / (exponent - 1.0))
    w *= mean_degree / w.mean()
    n_edges = int(round(w.sum() / 2.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    src = np.minimum(np.searchsorted(cdf, rng.random(n_edges), side="right"), m - 1)
    dst = np.minimum(np.searchsorted(cdf, rng.random(n_edges), side="right"), m - 1)
    keep = src != dst
    a, b = np.minimum(src[keep], dst[keep]).astype(np.int64), np.maximum(src[keep], dst[keep]).astype(np.int64)
    und = _sorted_unique(a * m + b)
    a, b = und // m, und % m
    diag = np.arange(m, dtype=np.int64)
    rows = np.concatenate([a, b, diag])
    cols = np.concatenate([b, a, diag])
    key = _sorted_unique(rows * m + cols)
    rows, cols = key // m, key % m
    deg = np.bincount(rows, minlength=m).astype(np.float64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(deg.astype(np.int64), out=row_ptr[1:])
    vals = (1.0 / np.sqrt(deg[rows] * deg[cols])).astype(np.float32)
    csr = CSR(m, m, row_ptr.astype(np.int32), cols.astype(np.int32), vals)
    csr.info.update(kind="chung_lu_gcn", seed=seed, exponent=exponent, mean_degree_target=mean_degree,
                    mean_degree=float(deg.mean()), max_degree=int(deg.max(initial=0)))
    return csr


@dataclasses.dataclass
class BatchedSet:
    mats: list  # list[CSR]
    ns: list  # list[int], dense width per matrix
    info: dict


def batched_set(count: int, seed: int, m_lo: int = 64, m_hi: int = 65536, lam_lo: float = 4.0,
                lam_hi: float = 64.0, n_choices=(32, 64, 128)) -> BatchedSet:
    """``count`` independent square CSR matrices: m = k = round(exp(U[ln m_lo, ln m_hi])),
    a per-matrix mean row length lambda ~ U[lam_lo, lam_hi], Poisson(lambda) row lengths
    capped at k, uniform sorted columns, U[-1, 1] values; dense width n from n_choices."""
    rng = np.random.default_rng(seed)
    ms = np.rint(np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), count))).astype(np.int64)
    lams = rng.uniform(lam_lo, lam_hi, count)
    ns = rng.choice(np.asarray(n_choices), size=count)
    mats = []
    for i in range(count):
        m = int(ms[i])
        lengths = np.minimum(rng.poisson(lams[i], m), m)
        csr = csr_from_lengths(lengths, m, seed * 7919 + i, value_stream=1000 + i,
                               col_stream_seed=seed * 104729 + i)
        csr.info.update(kind="batched_member", lam=float(lams[i]))
        mats.append(csr)
    total_nnz = int(sum(c.nnz for c in mats))
    return BatchedSet(mats, [int(x) for x in ns], {"count": count, "seed": seed, "total_nnz": total_nnz,
                                                      "total_rows": int(ms.sum())})


# ----------------------------------------------------------------------------- the five workloads

def workload_plain(seed: int = SEED_BASE + 1):
    """4096 x 4096, 16 nonzeros per row, B 4096 x 64 N(0, 1)."""
    a = uniform_rows(4096, 4096, 16, seed)
    return a, normal_matrix(4096, 64, seed)


def workload_power_law(seed: int = SEED_BASE + 2, m: int = 1_000_000):
    """1M x 1M power-law rows (mean about 16, cap 100,000, 1% empty)."""
    return power_law(m, m, seed)


def workload_precision(seed: int = SEED_BASE + 3, m: int = 2_000_000, per_row: int = 32, n: int = 128):
    """2M x 2M, 32 nonzeros per row; B 2M x 128 N(0, 1) in float32 (cast by the caller)."""
    a = uniform_rows(m, m, per_row, seed)
    return a, normal_matrix(m, n, seed)


def workload_gcn(seed: int = SEED_BASE + 4, m: int = 500_000, n: int = 256, mean_degree: float = 20.0):
    a = chung_lu_gcn(m, seed, mean_degree=mean_degree)
    return a, normal_matrix(m, n, seed)


def workload_batched(seed: int = SEED_BASE + 5, count: int = 2048):
    return batched_set(count, seed)


# ----------------------------------------------------------------------------- dtype helpers

def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 to bfloat16 (round-to-nearest-even, via torch's CPU cast) and
    return the 16-bit patterns as uint16."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.view(torch.int16).numpy().view(np.uint16).copy()


def to_f16(x: np.ndarray) -> np.ndarray:
    """Round float32 to IEEE half (NumPy's cast is round-to-nearest-even)."""
    return np.asarray(x, dtype=np.float32).astype(np.float16)


def num_threads() -> int:
    return int(_load().gen_num_threads())


__all__ = [
    "CSR", "BatchedSet", "SEED_BASE", "build", "uniform_values", "normal_matrix", "csr_from_lengths",
    "uniform_rows", "power_law_lengths", "power_law", "chung_lu_gcn", "batched_set", "workload_plain",
    "workload_power_law", "workload_precision", "workload_gcn", "workload_batched", "to_bf16_bits",
    "to_f16", "num_threads",
]

if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
