"""GB300 (sm_103a) CSR x dense SpMM: Python binding of ``libspmm_gb300.so``.

The C ABI (``include/spmm.h``) is the boundary; this module only marshals
arguments to it.  Every step of the computation runs in the library's CUDA
kernels: there is no CPU path, and calls fail loudly when the library or a
GPU is missing.

Two layers:

* the C entry points under their C names (``spmm_csr``, ``spmm_csr_ex``,
  ``spmm_csr_workspace_size``, ``spmm_select_alg``, ``spmm_merge_partition``,
  ``spmm_csr_host``, ``spmm_csr_host_async``, ...), taking integers for pointers and streams exactly as
  the C functions do;
* tensor helpers (``spmm``, ``merge_partition``, ``spmm_host``) that take
  torch CUDA tensors, use torch only for device memory and the current stream,
  and raise ``SpMMError`` on a non-zero status.
"""
from __future__ import annotations

import ctypes
import os
import threading

ALG_AUTO, ALG_ROW_SPLIT, ALG_MERGE, ALG_AUTO_GB300, ALG_TILED, ALG_ROW_SPLIT_HYBRID = 0, 1, 2, 3, 4, 5
F32, BF16, F16 = 0, 1, 2
SEMIRING_PLUS_TIMES, SEMIRING_MIN_PLUS, SEMIRING_MAX_PLUS, SEMIRING_MAX_TIMES = 0, 1, 2, 3
SEMIRINGS = {"plus_times": SEMIRING_PLUS_TIMES, "min_plus": SEMIRING_MIN_PLUS, "max_plus": SEMIRING_MAX_PLUS,
             "max_times": SEMIRING_MAX_TIMES}
OK = 0
ERR_INVALID_VALUE, ERR_ALLOC, ERR_LAUNCH, ERR_BAD_CSR, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_CUDA, ERR_WORKSPACE = range(1, 9)
PAPER_THRESHOLD = 9.35  # Section 5.4

_ALG_NAMES = {"auto": ALG_AUTO, "row_split": ALG_ROW_SPLIT, "rowsplit": ALG_ROW_SPLIT, "merge": ALG_MERGE,
              "auto_gb300": ALG_AUTO_GB300, "tiled": ALG_TILED, "hybrid": ALG_ROW_SPLIT_HYBRID,
              "row_split_hybrid": ALG_ROW_SPLIT_HYBRID}
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspmm_gb300.so")
_lock = threading.Lock()
_lib = None


class SpMMError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)}")


class SpmmTuning(ctypes.Structure):
    """Mirror of spmm_tuning_t (zero fields = library's choice)."""

    _fields_ = [("lanes_per_row", ctypes.c_int), ("column_slabs", ctypes.c_int),
                ("items_per_subwarp", ctypes.c_int), ("long_row_len", ctypes.c_int),
                ("merge_threshold", ctypes.c_double), ("max_row_len", ctypes.c_longlong),
                ("block_rows", ctypes.c_int)]


_i, _ll, _vp, _sz, _d = ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_double
_TP = ctypes.POINTER(SpmmTuning)
_SIGNATURES = {
    "spmm_status_string": ([_i], ctypes.c_char_p),
    "spmm_version": ([], _i),
    "spmm_launch_count": ([], _ll),
    "spmm_select_alg": ([_i, _ll, _d], _i),
    "spmm_select_alg_gb300": ([_i, _ll, _ll, _i, _i], _i),
    "spmm_gather_probe": ([_vp, _ll, _i, _vp, _ll, _vp, _vp], _i),
    "spmm_default_column_slabs": ([_i, _i, _i, _i], _i),
    "spmm_tiled_reuse": ([_i, _i, _ll, _i, _i], _d),
    "spmm_csr_max_row_length": ([_i, _vp, ctypes.POINTER(_ll), _vp], _i),
    "spmm_csr": ([_i, _i, _i, _vp, _vp, _vp, _vp, _ll, _vp, _ll, _i, _vp], _i),
    "spmm_csr_ex": ([_i, _i, _i, _ll, _vp, _vp, _vp, _i, _vp, _i, _ll, _vp, _i, _ll, _i, _TP, _vp, _sz, _vp, _vp], _i),
    "spmm_csr_semiring": ([_i, _i, _i, _ll, _vp, _vp, _vp, _vp, _ll, _vp, _ll, _i, _i, _TP, _vp, _sz, _vp, _vp], _i),
    "spmm_csr_workspace_size": ([_i, _i, _i, _ll, _i, _i, _TP], _sz),
    "spmm_merge_partition": ([_i, _ll, _vp, _i, _i, _vp, _vp], _i),
    "spmm_csr_host": ([_i, _i, _i, _vp, _vp, _vp, _i, _vp, _i, _ll, _vp, _i, _ll, _i, _TP, _vp], _i),
    "spmm_csr_host_async": ([_i, _i, _i, _vp, _vp, _vp, _i, _vp, _i, _ll, _vp, _i, _ll, _i, _TP, _vp], _i),
    "spmm_csr_host_multi": ([_i, _i, _vp, _vp, _vp, _i, _i, _vp, _vp, _i, _vp, _vp, _i, _vp, _i, _TP, _vp], _i),
    "spmm_debug_bounded_wait": ([_vp, _ll, _vp], _i),
    "spmm_csr_noalloc": ([_i, _i, _i, _ll, _vp, _vp, _vp, _i, _vp, _i, _ll, _vp, _i, _ll, _i, _TP, _vp, _vp], _i),
    "spmm_csr_static_scratch_bytes": ([], _sz),
    "spmm_csr_transpose_workspace_size": ([_i, _i, _ll], _sz),
    "spmm_csr_transpose": ([_i, _i, _ll, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp], _i),
    "spmm_gather_values": ([_ll, _vp, _vp, _i, _vp, _vp], _i),
    "sddmm_csr": ([_i, _i, _i, _ll, _vp, _vp, _vp, _i, _ll, _vp, _i, _ll, _vp, _i, _vp], _i),
}


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import _build

    return _build.build(force=force)


def load():
    """Load the library (it must have been built; no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1803_08601_gb300.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


# ----------------------------------------------------------------------------- C entry points

def spmm_status_string(status: int) -> str:
    return load().spmm_status_string(status).decode()


status_string = spmm_status_string


def spmm_version() -> int:
    return load().spmm_version()


def spmm_launch_count() -> int:
    return load().spmm_launch_count()


def spmm_select_alg(m: int, nnz: int, threshold: float = 0.0) -> int:
    return load().spmm_select_alg(m, nnz, threshold)


def spmm_select_alg_gb300(m: int, nnz: int, max_row_len: int, n: int, b_type: int = F32) -> int:
    return load().spmm_select_alg_gb300(m, nnz, max_row_len, n, b_type)


def spmm_tiled_reuse(m: int, k: int, nnz: int, n: int, b_type: int = F32) -> float:
    return load().spmm_tiled_reuse(m, k, nnz, n, b_type)


def spmm_csr_max_row_length(m, row_ptr, stream) -> tuple[int, int]:
    """Returns (status, longest row)."""
    out = ctypes.c_longlong(0)
    st = load().spmm_csr_max_row_length(m, row_ptr, ctypes.byref(out), stream)
    return st, out.value


def default_column_slabs(alg: int, k: int, n: int, b_type: int = F32) -> int:
    return load().spmm_default_column_slabs(alg, k, n, b_type)


def gather_probe(B, idx, row_bytes: int, out, stream=None) -> None:
    """spmm_gather_probe on a CUDA tensor B (bytes viewed as rows of row_bytes), int32 CUDA
    indices idx and a one-word int32 CUDA tensor out (XOR of the words read)."""
    _require_cuda(B, idx, out)
    nbytes = B.numel() * B.element_size()
    _check(load().spmm_gather_probe(B.data_ptr(), nbytes // row_bytes, row_bytes, idx.data_ptr(), idx.numel(),
                                    out.data_ptr(), _stream_handle(stream)), "spmm_gather_probe")


def max_row_length(row_ptr, stream=None) -> int:
    _require_cuda(row_ptr)
    st, v = spmm_csr_max_row_length(row_ptr.numel() - 1, row_ptr.data_ptr(), _stream_handle(stream))
    _check(st, "spmm_csr_max_row_length")
    return v


def spmm_csr(m, k, n, row_ptr, col_ind, vals, B, ldb, C, ldc, alg, stream) -> int:
    return load().spmm_csr(m, k, n, row_ptr, col_ind, vals, B, ldb, C, ldc, alg, stream)


def spmm_csr_ex(m, k, n, nnz, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, alg, tuning,
                workspace, workspace_bytes, d_status, stream) -> int:
    return load().spmm_csr_ex(m, k, n, nnz, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, alg,
                              _tuning_ptr(tuning), workspace, workspace_bytes, d_status, stream)


def spmm_csr_workspace_size(m, k, n, nnz, alg, b_type, tuning=None) -> int:
    return load().spmm_csr_workspace_size(m, k, n, nnz, alg, b_type, _tuning_ptr(tuning))


def spmm_merge_partition(m, nnz, row_ptr, items_per_tile, num_tiles, limits, stream) -> int:
    return load().spmm_merge_partition(m, nnz, row_ptr, items_per_tile, num_tiles, limits, stream)


def spmm_csr_host(m, k, n, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, alg, tuning,
                  stream) -> int:
    return load().spmm_csr_host(m, k, n, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, alg,
                                _tuning_ptr(tuning), stream)


def spmm_csr_host_async(m, k, n, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, alg, tuning,
                        stream) -> int:
    return load().spmm_csr_host_async(m, k, n, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc,
                                      alg, _tuning_ptr(tuning), stream)


def spmm_csr_host_multi(m, k, row_ptr, col_ind, vals, vals_type, count, n, B, b_type, ldb, C, c_type, ldc, alg,
                        tuning, stream) -> int:
    """n, B, ldb, C, ldc: addresses of host arrays of count entries (int32, pointers, int64,
    pointers, int64)."""
    return load().spmm_csr_host_multi(m, k, row_ptr, col_ind, vals, vals_type, count, n, B, b_type, ldb, C, c_type,
                                      ldc, alg, _tuning_ptr(tuning), stream)


def spmm_debug_bounded_wait(d_status, limit_ns, stream) -> int:
    return load().spmm_debug_bounded_wait(d_status, limit_ns, stream)


def spmm_csr_noalloc(m, k, n, nnz, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, alg, tuning,
                     d_status, stream) -> int:
    """spmm_csr_ex without a workspace argument, for callers that cannot allocate
    device memory at call time: the merge scratch is a fixed device array of
    spmm_csr_static_scratch_bytes() bytes; larger problems return ERR_WORKSPACE.
    Calls that overlap on the GPU share that array and must be serialised."""
    return load().spmm_csr_noalloc(m, k, n, nnz, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc,
                                   alg, _tuning_ptr(tuning), d_status, stream)


def spmm_csr_semiring(m, k, n, nnz, row_ptr, col_ind, vals, B, ldb, C, ldc, semiring, alg, tuning, workspace,
                      workspace_bytes, d_status, stream) -> int:
    return load().spmm_csr_semiring(m, k, n, nnz, row_ptr, col_ind, vals, B, ldb, C, ldc, semiring, alg,
                                    _tuning_ptr(tuning), workspace, workspace_bytes, d_status, stream)


def spmm_csr_static_scratch_bytes() -> int:
    return load().spmm_csr_static_scratch_bytes()


def spmm_csr_transpose_workspace_size(m, k, nnz) -> int:
    return load().spmm_csr_transpose_workspace_size(m, k, nnz)


def spmm_csr_transpose(m, k, nnz, row_ptr, col_ind, row_ptr_t, col_ind_t, perm, workspace, workspace_bytes,
                       stream) -> int:
    return load().spmm_csr_transpose(m, k, nnz, row_ptr, col_ind, row_ptr_t, col_ind_t, perm, workspace,
                                     workspace_bytes, stream)


def spmm_gather_values(nnz, perm, vals, vals_type, out, stream) -> int:
    return load().spmm_gather_values(nnz, perm, vals, vals_type, out, stream)


def sddmm_csr(m, k, n, nnz, row_ptr, col_ind, dC, dc_type, lddc, B, b_type, ldb, out, out_type, stream) -> int:
    return load().sddmm_csr(m, k, n, nnz, row_ptr, col_ind, dC, dc_type, lddc, B, b_type, ldb, out, out_type, stream)


def _tuning_ptr(t):
    if t is None:
        return None
    if isinstance(t, dict):
        t = SpmmTuning(**t)
    return ctypes.pointer(t)


# ----------------------------------------------------------------------------- tensor helpers

def _torch():
    import torch

    return torch


def dtype_code(dt) -> int:
    torch = _torch()
    m = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
    if dt not in m:
        raise TypeError(f"unsupported dtype {dt}")
    return m[dt]


def alg_code(alg) -> int:
    return _ALG_NAMES[alg] if isinstance(alg, str) else int(alg)


def _check(status: int, where: str):
    if status != OK:
        raise SpMMError(status, where)


def _stream_handle(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("tensors must live on a CUDA device (no CPU path exists)")


def spmm(row_ptr, col_ind, vals, B, alg="auto", out=None, out_dtype=None, nnz=None, tuning=None, workspace=None,
         status=None, stream=None):
    """C = A @ B for a CSR A (row_ptr int32 [m+1], col_ind int32 [nnz], vals) and a
    row-major B [k, n] (row stride B.stride(0)).  Returns C [m, n] (or fills ``out``).

    ``nnz`` (host int) avoids the device read of row_ptr[m] that AUTO needs.
    ``workspace``: optional uint8 CUDA tensor for the merge-based path.
    ``status``: optional int32 CUDA tensor of one element receiving device-side errors.
    """
    torch = _torch()
    _require_cuda(row_ptr, col_ind, vals, B, out)
    if row_ptr.dtype != torch.int32 or col_ind.dtype != torch.int32:
        raise TypeError("row_ptr and col_ind must be int32")
    if B.dim() != 2 or B.stride(1) != 1:
        raise ValueError("B must be a row-major 2-D tensor")
    m = row_ptr.numel() - 1
    k, n = B.shape
    if out is None:
        out = torch.empty((m, n), dtype=out_dtype or B.dtype, device=B.device)
    if out.dim() != 2 or out.shape != (m, n) or out.stride(1) != 1:
        raise ValueError("out must be a row-major [m, n] tensor")
    ws_ptr, ws_bytes = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None else (None, 0)
    st = spmm_csr_ex(m, k, n, -1 if nnz is None else int(nnz), row_ptr.data_ptr(), col_ind.data_ptr(),
                     vals.data_ptr(), dtype_code(vals.dtype), B.data_ptr(), dtype_code(B.dtype), B.stride(0),
                     out.data_ptr(), dtype_code(out.dtype), out.stride(0), alg_code(alg), tuning, ws_ptr, ws_bytes,
                     status.data_ptr() if status is not None else None, _stream_handle(stream))
    _check(st, "spmm_csr_ex")
    return out


def semiring_spmm(row_ptr, col_ind, vals, B, semiring, alg="auto", out=None, nnz=None, tuning=None, workspace=None,
                  status=None, stream=None):
    """C = A (+).(x) B over ``semiring`` (a name of SEMIRINGS or its code), float32
    throughout; arguments as :func:`spmm`.  An empty row of A gives the identity of (+)."""
    torch = _torch()
    _require_cuda(row_ptr, col_ind, vals, B, out)
    for t, name in ((vals, "vals"), (B, "B")):
        if t.dtype != torch.float32:
            raise TypeError(f"{name} must be float32 for a semiring product")
    if row_ptr.dtype != torch.int32 or col_ind.dtype != torch.int32:
        raise TypeError("row_ptr and col_ind must be int32")
    if B.dim() != 2 or B.stride(1) != 1:
        raise ValueError("B must be a row-major 2-D tensor")
    sr = SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)
    m = row_ptr.numel() - 1
    k, n = B.shape
    if out is None:
        out = torch.empty((m, n), dtype=torch.float32, device=B.device)
    if out.dim() != 2 or out.shape != (m, n) or out.stride(1) != 1 or out.dtype != torch.float32:
        raise ValueError("out must be a row-major float32 [m, n] tensor")
    ws_ptr, ws_bytes = (workspace.data_ptr(), workspace.numel() * workspace.element_size()) if workspace is not None else (None, 0)
    st = spmm_csr_semiring(m, k, n, -1 if nnz is None else int(nnz), row_ptr.data_ptr(), col_ind.data_ptr(),
                           vals.data_ptr(), B.data_ptr(), B.stride(0), out.data_ptr(), out.stride(0), sr,
                           alg_code(alg), tuning, ws_ptr, ws_bytes, status.data_ptr() if status is not None else None,
                           _stream_handle(stream))
    _check(st, "spmm_csr_semiring")
    return out


def merge_partition(row_ptr, items_per_tile: int, nnz: int | None = None, stream=None):
    """Merge-path split points of Section 4.2 as an int32 CUDA tensor [tiles + 1, 2]."""
    torch = _torch()
    _require_cuda(row_ptr)
    m = row_ptr.numel() - 1
    if nnz is None:
        nnz = int(row_ptr[-1].item()) if m > 0 else 0
    tiles = (m + nnz + items_per_tile - 1) // items_per_tile
    lim = torch.empty((tiles + 1, 2), dtype=torch.int32, device=row_ptr.device)
    _check(spmm_merge_partition(m, nnz, row_ptr.data_ptr(), items_per_tile, tiles, lim.data_ptr(),
                                _stream_handle(stream)), "spmm_merge_partition")
    return lim


def spmm_host(row_ptr, col_ind, vals, B, C, alg="auto", tuning=None, stream=None, wait=True):
    """C = A @ B with every operand in host memory (CPU tensors, ideally pinned):
    the library copies to the device, computes and copies back.  With
    ``wait=True`` (``spmm_csr_host``) the call returns once C is filled; with
    ``wait=False`` (``spmm_csr_host_async``) it returns once the work is queued,
    and C is filled when ``stream`` (default: torch's current stream) has been
    synchronised; the operands must stay alive and A, B unchanged until then.
    The synchronous call reads its inputs after the work already queued on
    ``stream``; the asynchronous one reads them from call time on (the C of an
    earlier asynchronous call is a valid input only after a synchronisation)."""
    for t in (row_ptr, col_ind, vals, B, C):
        if t.is_cuda:
            raise ValueError("spmm_host takes host tensors")
    m = row_ptr.numel() - 1
    k, n = B.shape
    fn, name = (spmm_csr_host, "spmm_csr_host") if wait else (spmm_csr_host_async, "spmm_csr_host_async")
    st = fn(m, k, n, row_ptr.data_ptr(), col_ind.data_ptr(), vals.data_ptr(), dtype_code(vals.dtype),
            B.data_ptr(), dtype_code(B.dtype), B.stride(0), C.data_ptr(), dtype_code(C.dtype), C.stride(0),
            alg_code(alg), tuning, _stream_handle(stream))
    _check(st, name)
    return C


def spmm_host_multi(row_ptr, col_ind, vals, Bs, Cs, alg="auto", tuning=None, stream=None):
    """C_i = A @ B_i for every pair of host tensors (CPU, ideally pinned) in Bs, Cs, queued through
    ``spmm_csr_host_multi``: A goes up once for all products.  The call returns once the work is
    queued; every C_i is filled when ``stream`` (default: torch's current stream) has been
    synchronised, and the operands must stay alive and A, B_i unchanged until then.  All B_i share
    one dtype, all C_i another."""
    tensors = [row_ptr, col_ind, vals, *Bs, *Cs]
    if any(t.is_cuda for t in tensors):
        raise ValueError("spmm_host_multi takes host tensors")
    if len(Bs) != len(Cs):
        raise ValueError("spmm_host_multi needs one C per B")
    if any(B.dtype != Bs[0].dtype for B in Bs) or any(C.dtype != Cs[0].dtype for C in Cs):
        raise ValueError("spmm_host_multi takes one B dtype and one C dtype")
    count = len(Bs)
    m = row_ptr.numel() - 1
    k = Bs[0].shape[0] if count else 0
    if any(B.shape[0] != k for B in Bs) or any(C.shape[0] != m or C.shape[1] != B.shape[1] for B, C in zip(Bs, Cs)):
        raise ValueError("spmm_host_multi: shapes do not match")
    n = (ctypes.c_int * max(count, 1))(*[B.shape[1] for B in Bs])
    bp = (ctypes.c_void_p * max(count, 1))(*[B.data_ptr() for B in Bs])
    ldb = (ctypes.c_longlong * max(count, 1))(*[B.stride(0) for B in Bs])
    cp = (ctypes.c_void_p * max(count, 1))(*[C.data_ptr() for C in Cs])
    ldc = (ctypes.c_longlong * max(count, 1))(*[C.stride(0) for C in Cs])
    b_type = dtype_code(Bs[0].dtype) if count else F32
    c_type = dtype_code(Cs[0].dtype) if count else F32
    st = spmm_csr_host_multi(m, k, row_ptr.data_ptr(), col_ind.data_ptr(), vals.data_ptr(), dtype_code(vals.dtype),
                             count, ctypes.addressof(n), ctypes.addressof(bp), b_type, ctypes.addressof(ldb),
                             ctypes.addressof(cp), c_type, ctypes.addressof(ldc), alg_code(alg), tuning,
                             _stream_handle(stream))
    _check(st, "spmm_csr_host_multi")
    return Cs


def workspace_size(m, k, n, nnz, alg="auto", b_dtype=None, tuning=None) -> int:
    torch = _torch()
    return spmm_csr_workspace_size(m, k, n, nnz, alg_code(alg), dtype_code(b_dtype or torch.float32), tuning)


def csr_transpose(row_ptr, col_ind, k: int, stream=None):
    """A^T of a CSR A (k = columns of A): returns (row_ptr_t [k+1], col_ind_t, perm) int32 CUDA tensors."""
    torch = _torch()
    _require_cuda(row_ptr, col_ind)
    m, nnz = row_ptr.numel() - 1, col_ind.numel()
    dev = row_ptr.device
    rpt = torch.empty(k + 1, dtype=torch.int32, device=dev)
    cit = torch.empty(nnz, dtype=torch.int32, device=dev)
    perm = torch.empty(nnz, dtype=torch.int32, device=dev)
    _check(spmm_csr_transpose(m, k, nnz, row_ptr.data_ptr(), col_ind.data_ptr(), rpt.data_ptr(), cit.data_ptr(),
                              perm.data_ptr(), None, 0, _stream_handle(stream)), "spmm_csr_transpose")
    return rpt, cit, perm


def gather_values(perm, vals, out=None, stream=None):
    """out[q] = vals[perm[q]] on the device."""
    torch = _torch()
    _require_cuda(perm, vals)
    out = torch.empty_like(vals) if out is None else out
    _check(spmm_gather_values(perm.numel(), perm.data_ptr(), vals.data_ptr(), dtype_code(vals.dtype), out.data_ptr(),
                              _stream_handle(stream)), "spmm_gather_values")
    return out


def sddmm(row_ptr, col_ind, dC, B, out=None, out_dtype=None, stream=None):
    """out[p] = <dC[row(p), :], B[col_ind[p], :]> for every stored entry of the CSR pattern."""
    torch = _torch()
    _require_cuda(row_ptr, col_ind, dC, B, out)
    if dC.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("dC and B must be row-major")
    m, n = dC.shape
    k = B.shape[0]
    nnz = col_ind.numel()
    if out is None:
        out = torch.empty(nnz, dtype=out_dtype or dC.dtype, device=dC.device)
    _check(sddmm_csr(m, k, n, nnz, row_ptr.data_ptr(), col_ind.data_ptr(), dC.data_ptr(), dtype_code(dC.dtype),
                     dC.stride(0), B.data_ptr(), dtype_code(B.dtype), B.stride(0), out.data_ptr(),
                     dtype_code(out.dtype), _stream_handle(stream)), "sddmm_csr")
    return out


from .autograd import CSRMatrix, SpMMFunction, spmm_autograd  # noqa: E402,F401


# ----------------------------------------------------------------------------- batched form

BATCHED_MODEL, BATCHED_AUTOTUNE, BATCHED_ROW_SPLIT, BATCHED_MERGE, BATCHED_ROW_SPLIT_X2 = 0, 1, 2, 3, 4


class SpmmBatchMatrix(ctypes.Structure):
    """Mirror of spmm_batch_matrix_t."""

    _fields_ = [("m", ctypes.c_int), ("k", ctypes.c_int), ("n", ctypes.c_int), ("nnz", ctypes.c_longlong),
                ("row_ptr", ctypes.c_void_p), ("col_ind", ctypes.c_void_p), ("vals", ctypes.c_void_p),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_longlong), ("C", ctypes.c_void_p), ("ldc", ctypes.c_longlong)]


_BSIG = {
    "spmm_batched_plan_create": ([_i, ctypes.POINTER(SpmmBatchMatrix), _i, _vp, ctypes.POINTER(_vp)], _i),
    "spmm_batched_run": ([_vp, _vp], _i),
    "spmm_batched_capture_graph": ([_vp, _vp], _i),
    "spmm_batched_launch_graph": ([_vp, _vp], _i),
    "spmm_batched_run_unfused": ([_vp, _vp], _i),
    "spmm_batched_plan_query": ([_vp, ctypes.POINTER(_i), ctypes.POINTER(_ll), ctypes.POINTER(_i)], _i),
    "spmm_batched_plan_destroy": ([_vp], _i),
    "spmm_autotune_cache_entries": ([], _ll),
    "spmm_autotune_cache_clear": ([], _i),
}
_SIGNATURES.update(_BSIG)


def _bind_batched():
    lib = load()
    for name, (args, res) in _BSIG.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


def spmm_batched_plan_create(count, mats, policy, stream, plan_out) -> int:
    return _bind_batched().spmm_batched_plan_create(count, mats, policy, stream, plan_out)


def spmm_batched_run(plan, stream) -> int:
    return _bind_batched().spmm_batched_run(plan, stream)


def spmm_batched_capture_graph(plan, stream) -> int:
    return _bind_batched().spmm_batched_capture_graph(plan, stream)


def spmm_batched_launch_graph(plan, stream) -> int:
    return _bind_batched().spmm_batched_launch_graph(plan, stream)


def spmm_batched_run_unfused(plan, stream) -> int:
    return _bind_batched().spmm_batched_run_unfused(plan, stream)


def spmm_batched_plan_query(plan, algs, num_items, num_tiles) -> int:
    return _bind_batched().spmm_batched_plan_query(plan, algs, num_items, num_tiles)


def spmm_batched_plan_destroy(plan) -> int:
    return _bind_batched().spmm_batched_plan_destroy(plan)


def spmm_autotune_cache_entries() -> int:
    return _bind_batched().spmm_autotune_cache_entries()


def spmm_autotune_cache_clear() -> int:
    return _bind_batched().spmm_autotune_cache_clear()


class BatchedPlan:
    """A plan over lists of CUDA tensors: row_ptrs, col_inds, vals (float32), Bs [k, n], Cs [m, n].
    The tensors must outlive the plan."""

    def __init__(self, row_ptrs, col_inds, vals, Bs, Cs, policy=BATCHED_MODEL, nnzs=None, stream=None):
        count = len(row_ptrs)
        arr = (SpmmBatchMatrix * max(count, 1))()
        for i in range(count):
            rp, ci, v, B, C = row_ptrs[i], col_inds[i], vals[i], Bs[i], Cs[i]
            _require_cuda(rp, ci, v, B, C)
            m, (k, n) = rp.numel() - 1, B.shape
            nnz = int(nnzs[i]) if nnzs is not None else ci.numel()
            arr[i] = SpmmBatchMatrix(m, k, n, nnz, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), B.data_ptr(),
                                     B.stride(0), C.data_ptr(), C.stride(0))
        self.count = count
        self._keep = (row_ptrs, col_inds, vals, Bs, Cs)
        h = ctypes.c_void_p()
        _check(spmm_batched_plan_create(count, arr, policy, _stream_handle(stream), ctypes.byref(h)),
               "spmm_batched_plan_create")
        self.handle = h
        self.has_graph = False

    def run(self, stream=None):
        _check(spmm_batched_run(self.handle, _stream_handle(stream)), "spmm_batched_run")

    def capture_graph(self, stream=None):
        _check(spmm_batched_capture_graph(self.handle, _stream_handle(stream)), "spmm_batched_capture_graph")
        self.has_graph = True

    def launch_graph(self, stream=None):
        _check(spmm_batched_launch_graph(self.handle, _stream_handle(stream)), "spmm_batched_launch_graph")

    def run_unfused(self, stream=None):
        _check(spmm_batched_run_unfused(self.handle, _stream_handle(stream)), "spmm_batched_run_unfused")

    def query(self):
        algs = (ctypes.c_int * max(self.count, 1))()
        items, tiles = ctypes.c_longlong(0), ctypes.c_int(0)
        _check(spmm_batched_plan_query(self.handle, algs, ctypes.byref(items), ctypes.byref(tiles)),
               "spmm_batched_plan_query")
        return list(algs)[: self.count], items.value, tiles.value

    def close(self):
        if getattr(self, "handle", None):
            spmm_batched_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
