"""The allocation-free entry point (spmm_csr_noalloc) gives the same C as the
regular entry point (spmm_csr_ex), call after call.

It serves callers that cannot allocate device memory when they call the
library (plugins of a host that owns the device memory, real-time loops that
must not meet allocator latency or failure); its merge scratch is a fixed
device array, so two calls in a row also check that whatever the first call
left in that array does not leak into the second.  This file is collected
last so a stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import FP32_TOL, structure

pytestmark = pytest.mark.gpu


def _noalloc(pkg, torch, d_rp, d_ci, d_v, d_B, nnz, alg):
    m, (k, n) = d_rp.numel() - 1, d_B.shape
    C = torch.full((m, n), float("nan"), device="cuda")
    st = pkg.spmm_csr_noalloc(m, k, n, nnz, d_rp.data_ptr(), d_ci.data_ptr(), d_v.data_ptr(), pkg.F32,
                              d_B.data_ptr(), pkg.F32, d_B.stride(0), C.data_ptr(), pkg.F32, C.stride(0),
                              pkg.alg_code(alg), None, None, torch.cuda.current_stream().cuda_stream)
    assert st == pkg.OK, pkg.spmm_status_string(st)
    return C


@pytest.mark.parametrize("alg", ["merge", "auto"])
def test_noalloc_matches_regular_entry_point_on_consecutive_calls(gpu_lib, alg):
    import torch

    pkg = gpu_lib
    # two different problems back to back: the second call runs on the scratch the first one left
    for call, (name, n) in enumerate([("power_law", 64), ("giant_row", 32), ("power_law", 64)]):
        rp, ci, v, k = structure(name)
        B = gen.normal_matrix(k, n, 50 + call)
        d_rp, d_ci, d_v, d_B = (torch.from_numpy(x).cuda() for x in (rp, ci, v, B))
        nnz = int(rp[-1]) if call != 1 else -1
        C_new = _noalloc(pkg, torch, d_rp, d_ci, d_v, d_B, nnz, alg)
        C_ref = pkg.spmm(d_rp, d_ci, d_v, d_B, alg=alg, nnz=int(rp[-1]))
        torch.cuda.synchronize()
        # the same kernels and tiles: the same bits, whatever the previous call left in the scratch
        assert torch.equal(C_new, C_ref)
        D = oracle.abs_bound(rp, ci, v, B)
        assert oracle.normalized_error(C_new.cpu().numpy(), oracle.spmm(rp, ci, v, B), D) <= FP32_TOL


def test_noalloc_rejects_problems_beyond_its_scratch(gpu_lib):
    pkg = gpu_lib
    cap = pkg.spmm_csr_static_scratch_bytes()
    assert cap == 16 << 20
    m, n, nnz = 4_000_000, 256, 60_000_000
    assert pkg.spmm_csr_workspace_size(m, m, n, nnz, pkg.ALG_MERGE, pkg.F32) > cap
    # sizes are checked before any pointer is touched
    st = pkg.spmm_csr_noalloc(m, m, n, nnz, 256, 512, 768, pkg.F32, 1024, pkg.F32, n, 2048, pkg.F32, n,
                              pkg.ALG_MERGE, None, None, None)
    assert st == pkg.ERR_WORKSPACE


@pytest.mark.parametrize("alg", ["merge", "row_split"])
def test_noalloc_spmv_matches_bitwise(gpu_lib, alg):
    """The SpMV merge kernel keeps its tiles' carries in the same fixed scratch (tiles of 2048
    path items); both SpMV kernels give the regular entry point's bits."""
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("giant_row")
    B = gen.normal_matrix(k, 1, 61)
    d_rp, d_ci, d_v, d_B = (torch.from_numpy(x).cuda() for x in (rp, ci, v, B))
    C_new = _noalloc(pkg, torch, d_rp, d_ci, d_v, d_B, int(rp[-1]), alg)
    C_ref = pkg.spmm(d_rp, d_ci, d_v, d_B, alg=alg, nnz=int(rp[-1]))
    torch.cuda.synchronize()
    assert torch.equal(C_new, C_ref)


def test_noalloc_accepts_only_its_documented_algorithms():
    """AUTO, ROW_SPLIT and MERGE only: AUTO_GB300 would allocate to measure the longest row, and
    neither the A/B tiling nor the hybrid row split (whose queue needs scratch) is offered here;
    they are rejected before any device work."""
    import paper_1803_08601_gb300 as pkg

    for alg in (pkg.ALG_AUTO_GB300, pkg.ALG_TILED, pkg.ALG_ROW_SPLIT_HYBRID):
        st = pkg.spmm_csr_noalloc(4, 4, 4, 4, 8, 16, 32, pkg.F32, 64, pkg.F32, 4, 128, pkg.F32, 4, alg, None, None, None)
        assert st == pkg.ERR_INVALID_VALUE
