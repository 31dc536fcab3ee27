"""FP64 CPU oracle for CSR SpMM (arXiv 1803.08601) and the operations around it.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package.  The
CUDA library never calls it, and the two share no code: no kernels, headers,
helpers, tables or pre/post-processing.  The only common dependency is the
seeded input generator in ``gen/``, which holds none of the method's arithmetic.

What each function computes, and where the paper defines it:

* ``spmm`` / ``spmm_rows``   C = A B in float64 (Section 1 problem statement;
  Algorithm 1's output C <- AB).  Plain definition, rows outer, nonzeros, then
  columns.  Pinned in tests against dense float64 GEMM, identity, permutation,
  B = ones (row sums) and exact integer arithmetic.
* ``abs_bound_rows``          D = |A| |B|, the scale of the acceptance metric
  max |C - C_ref| / D.
* ``select_alg``              the Section 5.4 heuristic: merge-based when the
  mean row length nnz / m is below 9.35, row split otherwise.
* ``merge_path_limits``       the merge-path split points of Section 4 item
  2(b) / Fig. 2(c), by walking the merge of row end offsets with nonzero
  indices.  Pinned by the closed-form characterisation of a merge-path
  coordinate, checked exhaustively on small inputs.
* ``spmm_t``                  dB = A^T dC by definition (no transpose formed).
* ``sddmm``                   dvals[p] = <dC[i, :], B[col_ind[p], :]>.
* ``csr_transpose``           stable counting-sort transpose with permutation.
* ``spmm_semiring``           C = A (+).(x) B over (+,x), (min,+), (max,+), (max,x)
  (the GraphBLAS matrix product of Section 1), by definition.

The backward operations (``spmm_t``, ``sddmm``, ``csr_transpose``) are not in the
paper, which names SpMM_T only as future work (Section 6); they are the standard
derivatives of the bilinear map (vals, B) -> A B and are pinned against dense
float64 autograd and central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libspmm_oracle.so")
_lock = threading.Lock()
_lib = None

# Section 5.4: merge-based below this mean row length, row split otherwise.
HEURISTIC_THRESHOLD = 9.35
ALG_ROW_SPLIT = 1
ALG_MERGE = 2


def build(force: bool = False) -> str:
    """Compile spmm_oracle.c (gcc -O2, OpenMP when available) into oracle/_build/."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = f"{_LIB_PATH}.{os.getpid()}.tmp"
    # -ffp-contract=off: every multiply and add is rounded on its own, as written.
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_SIGS = {
    "oracle_spmm_f64": "i64 i64 vp vp vp vp i64 vp i64",
    "oracle_spmm_rows_f64": "i64 vp i64 vp vp vp vp i64 vp",
    "oracle_absbound_rows_f64": "i64 vp i64 vp vp vp vp i64 vp",
    "oracle_spmm_t_f64": "i64 i64 i64 vp vp vp vp i64 vp i64",
    "oracle_sddmm_f64": "i64 i64 vp vp vp i64 vp i64 vp",
    "oracle_sddmm_absbound_f64": "i64 i64 vp vp vp i64 vp i64 vp",
    "oracle_csr_transpose": "i64 i64 vp vp vp vp vp",
    "oracle_merge_path_limits": "i64 vp i64 i64 vp",
    "oracle_spmm_semiring_f64": "i64 i64 int vp vp vp vp i64 vp i64",
    "oracle_set_num_threads": "int",
    "oracle_num_threads": "",
}


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    kinds = {"i64": ctypes.c_int64, "vp": ctypes.c_void_p, "int": ctypes.c_int}
    for name, args in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = [kinds[a] for a in args.split()]
        fn.restype = ctypes.c_int if name == "oracle_num_threads" else None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"], "oracle inputs must be C-contiguous"
    return a.ctypes.data


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    """A bfloat16 value is the float32 whose upper 16 bits are the given pattern
    and whose lower 16 bits are zero; the widening is exact."""
    b = np.ascontiguousarray(bits).view(np.uint16).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def to_f64(x, dtype: str | None = None) -> np.ndarray:
    """Exact float64 copy of float32 / float16 / bfloat16-bit-pattern data."""
    if dtype == "bf16":
        return bf16_bits_to_f64(np.asarray(x))
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def set_threads(t: int) -> None:
    _load().oracle_set_num_threads(int(t))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


# ----------------------------------------------------------------------------- Section 1 / Alg. 1

def spmm(row_ptr, col_ind, vals, B) -> np.ndarray:
    """C = A B in float64 (all rows)."""
    rp, ci = _i32(row_ptr), _i32(col_ind)
    v, b = to_f64(vals), to_f64(B)
    m, n = rp.shape[0] - 1, b.shape[1]
    c = np.empty((m, n), dtype=np.float64)
    if m and n:
        _load().oracle_spmm_f64(m, n, _p(rp), _p(ci), _p(v), _p(b), b.shape[1], _p(c), n)
    elif m:
        c[:] = 0.0
    return c


def spmm_rows(rows, row_ptr, col_ind, vals, B) -> np.ndarray:
    """Rows ``rows`` of C = A B in float64."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rp, ci = _i32(row_ptr), _i32(col_ind)
    v, b = to_f64(vals), to_f64(B)
    n = b.shape[1]
    out = np.zeros((rows.shape[0], n), dtype=np.float64)
    if rows.size and n:
        _load().oracle_spmm_rows_f64(rows.shape[0], _p(rows), n, _p(rp), _p(ci), _p(v), _p(b), b.shape[1], _p(out))
    return out


def abs_bound_rows(rows, row_ptr, col_ind, vals, B) -> np.ndarray:
    """Rows ``rows`` of |A| |B| in float64."""
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rp, ci = _i32(row_ptr), _i32(col_ind)
    v, b = to_f64(vals), to_f64(B)
    n = b.shape[1]
    out = np.zeros((rows.shape[0], n), dtype=np.float64)
    if rows.size and n:
        _load().oracle_absbound_rows_f64(rows.shape[0], _p(rows), n, _p(rp), _p(ci), _p(v), _p(b), b.shape[1], _p(out))
    return out


def abs_bound(row_ptr, col_ind, vals, B) -> np.ndarray:
    m = len(row_ptr) - 1
    return abs_bound_rows(np.arange(m), row_ptr, col_ind, vals, B)


def normalized_error(C, C_ref, D, abs_floor: float = 0.0) -> float:
    """Acceptance metric max |C - C_ref| / D over all elements.  Where D == 0 the
    product has no nonzero terms and C must be exactly zero there; a violation
    returns +inf.  ``abs_floor`` is subtracted from each absolute difference
    first: an output format with subnormals (IEEE binary16 below 2^-14) rounds
    with an absolute error of up to half its subnormal spacing there, which no
    relative bound covers."""
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    D = np.asarray(D, dtype=np.float64)
    if C.size == 0:
        return 0.0
    if not np.all(np.isfinite(C)):
        return float("inf")
    zero = D == 0
    if np.any(C[zero] != 0.0):
        return float("inf")
    err = np.maximum(np.abs(C - C_ref) - abs_floor, 0.0)
    nz = ~zero
    return float((err[nz] / D[nz]).max()) if np.any(nz) else 0.0


# ----------------------------------------------------------------------------- semirings

SEMIRINGS = {"plus_times": 0, "min_plus": 1, "max_plus": 2, "max_times": 3}


def spmm_semiring(row_ptr, col_ind, vals, B, semiring: str) -> np.ndarray:
    """C = A (+).(x) B over the named semiring, in float64 (empty rows: the identity of (+))."""
    rp, ci = _i32(row_ptr), _i32(col_ind)
    v, b = to_f64(vals), to_f64(B)
    m, n = rp.shape[0] - 1, b.shape[1]
    c = np.empty((m, n), dtype=np.float64)
    if m and n:
        _load().oracle_spmm_semiring_f64(m, n, SEMIRINGS[semiring], _p(rp), _p(ci), _p(v), _p(b), b.shape[1], _p(c), n)
    return c


# ----------------------------------------------------------------------------- Section 5.4

def select_alg(m: int, nnz: int, threshold: float = HEURISTIC_THRESHOLD) -> int:
    """Section 5.4: d = mean row length = nnz / m; merge-based iff d < threshold.
    An empty matrix (m == 0) takes row split (nothing to compute)."""
    if m <= 0:
        return ALG_ROW_SPLIT
    return ALG_MERGE if (nnz / m) < threshold else ALG_ROW_SPLIT


# ----------------------------------------------------------------------------- Section 4 merge path

def merge_path_limits(row_ptr, items: int) -> np.ndarray:
    """Split points (rows consumed, nonzeros consumed) of the merge path at
    diagonals t * items, t = 0 .. ceil((m + nnz) / items); shape [tiles + 1, 2]."""
    rp = _i32(row_ptr)
    m = rp.shape[0] - 1
    nnz = int(rp[-1]) if m > 0 else 0
    tiles = (m + nnz + items - 1) // items
    out = np.zeros((tiles + 1, 2), dtype=np.int32)
    _load().oracle_merge_path_limits(m, _p(rp), items, tiles, _p(out))
    return out


# ----------------------------------------------------------------------------- backward operations

def spmm_t(row_ptr, col_ind, vals, dC, k: int) -> np.ndarray:
    """dB = A^T dC in float64, k = number of columns of A."""
    rp, ci = _i32(row_ptr), _i32(col_ind)
    v, g = to_f64(vals), to_f64(dC)
    m, n = rp.shape[0] - 1, g.shape[1]
    out = np.zeros((k, n), dtype=np.float64)
    if m and n and k:
        _load().oracle_spmm_t_f64(m, k, n, _p(rp), _p(ci), _p(v), _p(g), n, _p(out), n)
    return out


def sddmm(row_ptr, col_ind, dC, B) -> np.ndarray:
    """out[p] = sum_j dC[i, j] * B[col_ind[p], j] for each nonzero p of row i."""
    rp, ci = _i32(row_ptr), _i32(col_ind)
    g, b = to_f64(dC), to_f64(B)
    m, n = rp.shape[0] - 1, g.shape[1]
    out = np.zeros(ci.shape[0], dtype=np.float64)
    if m and ci.size:
        _load().oracle_sddmm_f64(m, n, _p(rp), _p(ci), _p(g), n, _p(b), b.shape[1], _p(out))
    return out


def sddmm_abs_bound(row_ptr, col_ind, dC, B) -> np.ndarray:
    rp, ci = _i32(row_ptr), _i32(col_ind)
    g, b = to_f64(dC), to_f64(B)
    m, n = rp.shape[0] - 1, g.shape[1]
    out = np.zeros(ci.shape[0], dtype=np.float64)
    if m and ci.size:
        _load().oracle_sddmm_absbound_f64(m, n, _p(rp), _p(ci), _p(g), n, _p(b), b.shape[1], _p(out))
    return out


def csr_transpose(row_ptr, col_ind, k: int):
    """Stable transpose: returns (row_ptr_t [k+1], col_ind_t [nnz], perm [nnz])."""
    rp, ci = _i32(row_ptr), _i32(col_ind)
    m = rp.shape[0] - 1
    nnz = ci.shape[0]
    rpt = np.zeros(k + 1, dtype=np.int32)
    cit = np.zeros(nnz, dtype=np.int32)
    perm = np.zeros(nnz, dtype=np.int32)
    _load().oracle_csr_transpose(m, k, _p(rp), _p(ci), _p(rpt), _p(cit), _p(perm))
    return rpt, cit, perm


__all__ = [
    "HEURISTIC_THRESHOLD", "ALG_ROW_SPLIT", "ALG_MERGE", "build", "bf16_bits_to_f64", "to_f64",
    "set_threads", "num_threads", "spmm", "spmm_rows", "abs_bound_rows", "abs_bound", "normalized_error",
    "select_alg", "merge_path_limits", "spmm_t", "sddmm", "sddmm_abs_bound", "csr_transpose", "SEMIRINGS",
    "spmm_semiring",
]
