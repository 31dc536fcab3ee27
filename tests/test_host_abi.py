"""The C ABI library loads and exports every declared symbol, and its host-side
logic (heuristic, argument checks, workspace sizing) behaves as documented.
No call here touches a GPU: each returns before any CUDA runtime call."""
import ctypes
import os
import re

import pytest

import oracle
import paper_1803_08601_gb300 as pkg
from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return pkg.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(", txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert "spmm_csr" in decl and "spmm_csr_ex" in decl
    raw = ctypes.CDLL(pkg.LIB_PATH)
    for name in decl:
        assert hasattr(raw, name), f"{name} declared in include/ but not exported"
    assert set(pkg.exported_symbols()) <= set(decl)


def test_status_strings_and_version(lib):
    assert pkg.spmm_status_string(0) == "SPMM_OK"
    for s in range(1, 9):
        assert pkg.spmm_status_string(s).startswith("SPMM_ERR_")
    assert pkg.spmm_version() >= 100


@pytest.mark.parametrize("m,nnz", [(100, 934), (100, 936), (20, 187), (1, 0), (0, 0), (1000, 16000),
                                   (1_000_000, 15_821_532), (7, 65)])
def test_heuristic_matches_oracle(lib, m, nnz):
    """Section 5.4: the library's choice equals the oracle's on both sides of 9.35."""
    assert pkg.spmm_select_alg(m, nnz, 0.0) == oracle.select_alg(m, nnz)
    assert pkg.spmm_select_alg(m, nnz, pkg.PAPER_THRESHOLD) == oracle.select_alg(m, nnz)


def test_gb300_selector(lib):
    F, H = pkg.F32, pkg.BF16
    # Type 1 guard: a very long row sends the matrix to the hybrid row split for rows of B of up
    # to 128 bytes, to merge for wider ones
    assert pkg.spmm_select_alg_gb300(1_000_000, 15_821_532, 100_000, 64, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(1_000_000, 15_821_532, 100_000, 32, F) == pkg.ALG_ROW_SPLIT_HYBRID
    assert pkg.spmm_select_alg_gb300(1_000_000, 15_821_532, 100_000, 8, F) == pkg.ALG_ROW_SPLIT_HYBRID
    assert pkg.spmm_select_alg_gb300(1_000_000, 15_821_532, 100_000, 16, H) == pkg.ALG_ROW_SPLIT_HYBRID
    assert pkg.spmm_select_alg_gb300(1_000_000, 15_821_532, 1_000, 64, F) == pkg.ALG_ROW_SPLIT
    assert pkg.spmm_select_alg_gb300(4096, 65_536, 16, 64, F) == pkg.ALG_ROW_SPLIT
    # the aspect-ratio sweep's boundary: 8192 rows of 2048 (8192 * 2048 = nnz) still go to merge,
    # 16384 rows of 1024 to the row split
    assert pkg.spmm_select_alg_gb300(4096, 1 << 24, 4096, 64, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(8192, 1 << 24, 2048, 64, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(16384, 1 << 24, 1024, 64, F) == pkg.ALG_ROW_SPLIT
    # rows all long (longest under 16 x mean) stay with merge at narrow rows of B too
    assert pkg.spmm_select_alg_gb300(4096, 1 << 24, 4096, 8, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(4096, 1 << 24, 4096, 32, F) == pkg.ALG_MERGE
    # rows of 768 or more nonzeros with rows of B under 256 bytes: merge
    assert pkg.spmm_select_alg_gb300(16384, 1 << 24, 1024, 8, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(16384, 1 << 24, 1024, 32, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(32768, 1 << 24, 512, 32, F) == pkg.ALG_ROW_SPLIT
    # mean-length rules (points of the row-length family sweep, 1M x 1M)
    M = 10**6
    assert pkg.spmm_select_alg_gb300(M, 2 * M, 2, 8, F) == pkg.ALG_ROW_SPLIT          # 32-byte rows
    assert pkg.spmm_select_alg_gb300(M, 2 * M, 2, 32, F) == pkg.ALG_ROW_SPLIT_HYBRID  # d < 3
    assert pkg.spmm_select_alg_gb300(M, 2 * M, 2, 128, F) == pkg.ALG_ROW_SPLIT_HYBRID
    assert pkg.spmm_select_alg_gb300(M, 2 * M, 13, 64, F) == pkg.ALG_ROW_SPLIT_HYBRID  # Poisson-like
    assert pkg.spmm_select_alg_gb300(M, 2 * M, 13, 128, F) == pkg.ALG_MERGE           # uneven, 512 B
    assert pkg.spmm_select_alg_gb300(M, 4 * M, 4, 32, F) == pkg.ALG_ROW_SPLIT         # 128 B: row split
    assert pkg.spmm_select_alg_gb300(M, 4 * M, 16, 32, F) == pkg.ALG_ROW_SPLIT
    assert pkg.spmm_select_alg_gb300(M, 4 * M, 4, 64, F) == pkg.ALG_ROW_SPLIT         # uniform, 256 B: T = 3
    assert pkg.spmm_select_alg_gb300(M, 4 * M, 4, 128, F) == pkg.ALG_MERGE            # uniform, 512 B: T = 5
    assert pkg.spmm_select_alg_gb300(M, 6 * M, 6, 128, F) == pkg.ALG_ROW_SPLIT
    assert pkg.spmm_select_alg_gb300(M, 6 * M, 20, 64, F) == pkg.ALG_MERGE            # uneven: T = 8
    assert pkg.spmm_select_alg_gb300(M, 8 * M, 24, 64, F) == pkg.ALG_ROW_SPLIT
    assert pkg.spmm_select_alg_gb300(M, 6 * M, 20, 128, F) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg_gb300(M, 12 * M, 33, 128, F) == pkg.ALG_ROW_SPLIT
    assert pkg.spmm_select_alg_gb300(M, 32 * M, 61, 128, F) == pkg.ALG_ROW_SPLIT      # longest < 2 x mean
    assert pkg.spmm_select_alg_gb300(0, 0, 0, 64, F) == pkg.ALG_ROW_SPLIT


def test_heuristic_custom_threshold(lib):
    assert pkg.spmm_select_alg(100, 1500, 20.0) == pkg.ALG_MERGE
    assert pkg.spmm_select_alg(100, 1500, 10.0) == pkg.ALG_ROW_SPLIT


def test_argument_checks_return_before_any_device_work(lib):
    F = pkg.F32
    good = dict(m=4, k=4, n=4, nnz=4, row_ptr=8, col_ind=16, vals=32, vals_type=F, B=64, b_type=F, ldb=4, C=128,
                c_type=F, ldc=4, alg=0, tuning=None, workspace=None, workspace_bytes=0, d_status=None, stream=None)

    def call(**kw):
        a = dict(good)
        a.update(kw)
        return pkg.spmm_csr_ex(*a.values())

    assert call(m=-1) == pkg.ERR_INVALID_VALUE
    assert call(n=-3) == pkg.ERR_INVALID_VALUE
    assert call(ldb=3) == pkg.ERR_INVALID_VALUE
    assert call(ldb=1 << 30) == pkg.ERR_INVALID_VALUE  # float32 rows of B 2^32 bytes apart
    assert call(ldb=1 << 31, b_type=pkg.BF16, vals_type=pkg.BF16, c_type=pkg.BF16) == pkg.ERR_INVALID_VALUE
    assert call(ldc=2) == pkg.ERR_INVALID_VALUE
    assert call(alg=7) == pkg.ERR_INVALID_VALUE
    assert call(alg=6) == pkg.ERR_INVALID_VALUE
    assert call(alg=pkg.ALG_TILED, m=0) == pkg.OK
    assert call(row_ptr=None) == pkg.ERR_INVALID_VALUE
    assert call(C=None) == pkg.ERR_INVALID_VALUE
    assert call(col_ind=None) == pkg.ERR_INVALID_VALUE
    assert call(k=0) == pkg.ERR_INVALID_VALUE  # nonzeros need columns
    assert call(nnz=-5) == pkg.ERR_INVALID_VALUE
    assert call(vals_type=pkg.F32, b_type=pkg.BF16) == pkg.ERR_UNSUPPORTED
    assert call(vals_type=9) == pkg.ERR_UNSUPPORTED
    # empty problems are accepted without touching the device
    assert call(m=0) == pkg.OK
    assert call(n=0) == pkg.OK
    assert pkg.spmm_merge_partition(10, 5, 8, 0, 3, 16, None) == pkg.ERR_INVALID_VALUE
    assert pkg.spmm_merge_partition(10, 5, 8, 4, 3, 16, None) == pkg.ERR_INVALID_VALUE  # 3 tiles x 4 < 15 items
    assert pkg.spmm_debug_bounded_wait(None, 1000, None) == pkg.ERR_INVALID_VALUE


def test_host_entries_check_arguments_on_the_host(lib):
    """spmm_csr_host and spmm_csr_host_async read row_ptr[m] on the host and
    reject bad arguments before any CUDA call; empty products return at once."""
    import numpy as np

    rp = np.array([0, 1, 2, 3, 4], dtype=np.int32)
    ci = np.arange(4, dtype=np.int32)
    v = np.ones(4, dtype=np.float32)
    B = np.ones((4, 8), dtype=np.float32)
    C = np.zeros((4, 8), dtype=np.float32)
    F = pkg.F32
    good = dict(m=4, k=4, n=8, row_ptr=rp.ctypes.data, col_ind=ci.ctypes.data, vals=v.ctypes.data, vals_type=F,
                B=B.ctypes.data, b_type=F, ldb=8, C=C.ctypes.data, c_type=F, ldc=8, alg=pkg.ALG_MERGE, tuning=None,
                stream=None)
    for fn in (pkg.spmm_csr_host, pkg.spmm_csr_host_async):
        def call(**kw):
            a = dict(good)
            a.update(kw)
            return fn(*a.values())

        assert call(m=-1) == pkg.ERR_INVALID_VALUE
        assert call(row_ptr=None) == pkg.ERR_INVALID_VALUE
        assert call(ldb=4) == pkg.ERR_INVALID_VALUE
        assert call(ldc=7) == pkg.ERR_INVALID_VALUE
        assert call(alg=9) == pkg.ERR_INVALID_VALUE
        assert call(col_ind=None) == pkg.ERR_INVALID_VALUE
        assert call(vals_type=F, b_type=pkg.F16) == pkg.ERR_UNSUPPORTED
        assert call(m=0) == pkg.OK
        assert call(n=0) == pkg.OK
        assert np.all(C == 0)


def test_host_multi_checks_arguments_on_the_host(lib):
    """spmm_csr_host_multi rejects a bad product (or bad arrays) before any CUDA call, and
    returns at once when there is nothing to compute."""
    import ctypes

    import numpy as np

    rp = np.array([0, 1, 2, 3, 4], dtype=np.int32)
    ci = np.arange(4, dtype=np.int32)
    v = np.ones(4, dtype=np.float32)
    Bs = [np.ones((4, 8), dtype=np.float32), np.ones((4, 4), dtype=np.float32)]
    Cs = [np.zeros((4, 8), dtype=np.float32), np.zeros((4, 4), dtype=np.float32)]
    F = pkg.F32

    def arrays(ns, ldbs, ldcs):
        cnt = len(ns)
        keep = [(ctypes.c_int * cnt)(*ns), (ctypes.c_void_p * cnt)(*[b.ctypes.data for b in Bs[:cnt]]),
                (ctypes.c_longlong * cnt)(*ldbs), (ctypes.c_void_p * cnt)(*[c.ctypes.data for c in Cs[:cnt]]),
                (ctypes.c_longlong * cnt)(*ldcs)]
        return keep, [ctypes.addressof(x) for x in keep]

    def call(ns=(8, 4), ldbs=(8, 4), ldcs=(8, 4), m=4, count=None, alg=pkg.ALG_MERGE, b_type=F, row_ptr=rp.ctypes.data):
        keep, (n, b, ldb, c, ldc) = arrays(list(ns), list(ldbs), list(ldcs))
        return pkg.spmm_csr_host_multi(m, 4, row_ptr, ci.ctypes.data, v.ctypes.data, F,
                                       len(ns) if count is None else count, n, b, b_type, ldb, c, F, ldc, alg, None,
                                       None)

    assert call(m=-1) == pkg.ERR_INVALID_VALUE
    assert call(count=-1) == pkg.ERR_INVALID_VALUE
    assert call(row_ptr=None) == pkg.ERR_INVALID_VALUE
    assert call(ns=(8, -4)) == pkg.ERR_INVALID_VALUE
    assert call(ldbs=(8, 3)) == pkg.ERR_INVALID_VALUE  # the second product's ldb < n
    assert call(ldcs=(4, 4)) == pkg.ERR_INVALID_VALUE
    assert call(alg=9) == pkg.ERR_INVALID_VALUE
    assert call(b_type=pkg.F16) == pkg.ERR_UNSUPPORTED
    assert call(m=0) == pkg.OK
    assert call(ns=(0, 0)) == pkg.OK
    assert pkg.spmm_csr_host_multi(4, 4, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, F, 0, None, None, F, None,
                                   None, F, None, pkg.ALG_MERGE, None, None) == pkg.OK
    assert pkg.spmm_csr_host_multi(4, 4, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, F, 2, None, None, F, None,
                                   None, F, None, pkg.ALG_MERGE, None, None) == pkg.ERR_INVALID_VALUE
    assert all(np.all(C == 0) for C in Cs)


def test_semiring_argument_checks(lib):
    good = dict(m=4, k=4, n=4, nnz=4, row_ptr=8, col_ind=16, vals=32, B=64, ldb=4, C=128, ldc=4,
                semiring=pkg.SEMIRING_MIN_PLUS, alg=0, tuning=None, workspace=None, workspace_bytes=0, d_status=None,
                stream=None)

    def call(**kw):
        a = dict(good)
        a.update(kw)
        return pkg.spmm_csr_semiring(*a.values())

    assert call(semiring=4) == pkg.ERR_INVALID_VALUE
    assert call(semiring=-1) == pkg.ERR_INVALID_VALUE
    assert call(ldc=3) == pkg.ERR_INVALID_VALUE
    assert call(alg=9) == pkg.ERR_INVALID_VALUE
    for sr in pkg.SEMIRINGS.values():
        assert call(semiring=sr, m=0) == pkg.OK
        assert call(semiring=sr, n=0) == pkg.OK
    assert pkg.SEMIRINGS == oracle.SEMIRINGS  # same codes on both sides of the ABI


def test_workspace_size(lib):
    F = pkg.F32
    assert pkg.spmm_csr_workspace_size(1000, 1000, 64, 16000, pkg.ALG_ROW_SPLIT, F) == 0
    assert pkg.spmm_csr_workspace_size(1000, 1000, 64, 16000, pkg.ALG_AUTO, F) == 0  # d = 16: row split
    w = pkg.spmm_csr_workspace_size(1000, 1000, 64, 5000, pkg.ALG_AUTO, F)  # d = 5: merge
    assert w > 0 and w % 256 == 0
    # carries grow with n; the tile count shrinks with more items per lane group
    assert pkg.spmm_csr_workspace_size(10**6, 10**6, 128, 10**7, pkg.ALG_MERGE, F) > \
        pkg.spmm_csr_workspace_size(10**6, 10**6, 8, 10**7, pkg.ALG_MERGE, F)
    small = pkg.spmm_csr_workspace_size(10**6, 10**6, 64, 10**7, pkg.ALG_MERGE, F, dict(items_per_subwarp=512))
    big = pkg.spmm_csr_workspace_size(10**6, 10**6, 64, 10**7, pkg.ALG_MERGE, F, dict(items_per_subwarp=16))
    assert big > small
    assert pkg.spmm_csr_workspace_size(-1, 1, 1, 1, pkg.ALG_MERGE, F) == 0


def test_no_cpu_path():
    torch = pytest.importorskip("torch")
    t = torch.zeros(3, dtype=torch.int32)
    with pytest.raises(ValueError):
        pkg.spmm(t, t[:0], torch.zeros(0), torch.zeros(2, 2))


def test_tiled_needs_no_workspace_and_reuse_formula(lib):
    assert pkg.workspace_size(1000, 1000, 64, 16000, pkg.ALG_TILED) == 0
    # 16 lanes per row at n = 64 float32: 256 / 16 groups x 8 rows = 128 rows per block
    assert abs(pkg.spmm_tiled_reuse(100_000, 100_000, 500_000_000, 64, pkg.F32) - 128 * 0.05) < 1e-9
    # 16-bit B: 8 elements per 16 bytes, n = 64 -> 8 lanes -> 256 rows per block
    assert abs(pkg.spmm_tiled_reuse(1000, 1000, 1000, 64, pkg.BF16) - 256 * 1e-3) < 1e-12
    assert pkg.spmm_tiled_reuse(0, 10, 0, 64, pkg.F32) == 0.0



def test_hybrid_workspace_size(lib):
    """The hybrid row split's queue and partial sums are sized from nnz and n on
    the host: nothing for an empty product, more for wider B and for a lower
    long-row threshold (more rows may be queued)."""
    F = pkg.F32
    H = pkg.ALG_ROW_SPLIT_HYBRID
    assert pkg.spmm_csr_workspace_size(0, 10, 8, 0, H, F) == 0
    assert pkg.spmm_csr_workspace_size(10, 10, 0, 0, H, F) == 0
    w8 = pkg.spmm_csr_workspace_size(1_000_000, 1_000_000, 8, 15_821_532, H, F)
    w128 = pkg.spmm_csr_workspace_size(1_000_000, 1_000_000, 128, 15_821_532, H, F)
    assert 0 < w8 < w128
    t = pkg.SpmmTuning(long_row_len=1)
    low = pkg.spmm_csr_workspace_size(1_000_000, 1_000_000, 8, 15_821_532, H, F, t)
    assert low > w8
    # every queued row needs a 4-byte entry: with rows of 2 nonzeros and a threshold of 1, all 10^6
    # rows may be queued
    assert pkg.spmm_csr_workspace_size(1_000_000, 1_000_000, 8, 2_000_000, H, F, t) >= 4 * 1_000_000
