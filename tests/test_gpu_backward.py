"""GPU parity of the backward operations (CSR transpose, value gather, SDDMM,
dB = A^T dC, autograd) with the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import FP32_TOL, structure

pytestmark = pytest.mark.gpu

TRANSPOSE_CASES = ["power_law", "giant_row", "duplicates_unsorted", "all_empty", "tall_k1", "identity", "permutation",
                   "empty_runs", "short_rows", "one_nonzero"]


def dev(torch, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


@pytest.mark.parametrize("name", TRANSPOSE_CASES)
def test_transpose_is_bit_exact(gpu_lib, name):
    import torch

    rp, ci, v, k = structure(name)
    d_rp, d_ci, d_v = dev(torch, rp, ci, v)
    rpt, cit, perm = gpu_lib.csr_transpose(d_rp, d_ci, k)
    o_rpt, o_cit, o_perm = oracle.csr_transpose(rp, ci, k)
    assert np.array_equal(rpt.cpu().numpy(), o_rpt)
    assert np.array_equal(cit.cpu().numpy(), o_cit)
    assert np.array_equal(perm.cpu().numpy(), o_perm)
    vt = gpu_lib.gather_values(perm, d_v)
    assert np.array_equal(vt.cpu().numpy(), v[o_perm])
    for dt in (torch.bfloat16, torch.float16):
        vh = d_v.to(dt)
        assert torch.equal(gpu_lib.gather_values(perm, vh), vh[perm.long()])


def test_transpose_large_column_count(gpu_lib):
    """k above 2^16 and 2^24 needs three and four radix passes."""
    import torch

    rng = np.random.default_rng(3)
    for k in (70_000, 20_000_000):
        lens = rng.integers(0, 30, 4000)
        rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
        ci = rng.integers(0, k, int(rp[-1])).astype(np.int32)
        d_rp, d_ci = dev(torch, rp, ci)
        rpt, cit, perm = gpu_lib.csr_transpose(d_rp, d_ci, k)
        o = oracle.csr_transpose(rp, ci, k)
        assert np.array_equal(perm.cpu().numpy(), o[2])
        assert np.array_equal(cit.cpu().numpy(), o[1])
        assert np.array_equal(rpt.cpu().numpy(), o[0])


@pytest.mark.parametrize("name", ["power_law", "giant_row", "duplicates_unsorted", "short_rows", "tall_k1"])
@pytest.mark.parametrize("n", [1, 8, 13, 64, 128, 256, 300, 1024])
def test_sddmm(gpu_lib, name, n):
    import torch

    rp, ci, v, k = structure(name)
    m = len(rp) - 1
    dC = gen.normal_matrix(m, n, 21)
    B = gen.normal_matrix(k, n, 22)
    d_rp, d_ci, d_dC, d_B = dev(torch, rp, ci, dC, B)
    out = gpu_lib.sddmm(d_rp, d_ci, d_dC, d_B)
    torch.cuda.synchronize()
    ref = oracle.sddmm(rp, ci, dC, B)
    D = oracle.sddmm_abs_bound(rp, ci, dC, B)
    assert oracle.normalized_error(out.cpu().numpy(), ref, D) <= FP32_TOL


@pytest.mark.parametrize("n", [64, 256, 1024])
@pytest.mark.parametrize("dt,out_f32", [("bf16", False), ("bf16", True), ("f16", False), ("f16", True)])
def test_sddmm_16bit(gpu_lib, dt, out_f32, n):
    """n = 64 (8 vectors of 16-bit values per row) takes the lane-group kernel; 256 and 1024 the warp
    kernel with dC rows in registers."""
    import torch

    rp, ci, v, k = structure("power_law")
    m = len(rp) - 1
    dC = gen.normal_matrix(m, n, 31)
    B = gen.normal_matrix(k, n, 32)
    tdt = torch.bfloat16 if dt == "bf16" else torch.float16
    d_rp, d_ci = dev(torch, rp, ci)
    d_dC, d_B = torch.from_numpy(dC).cuda().to(tdt), torch.from_numpy(B).cuda().to(tdt)
    out = gpu_lib.sddmm(d_rp, d_ci, d_dC, d_B, out_dtype=torch.float32 if out_f32 else tdt)
    torch.cuda.synchronize()
    got = out.float().cpu().numpy()
    # against the oracle on the rounded inputs: only accumulation (and the output rounding) differ
    dC_r, B_r = d_dC.double().cpu().numpy(), d_B.double().cpu().numpy()
    D = oracle.sddmm_abs_bound(rp, ci, dC_r, B_r)
    tol_rounded = FP32_TOL if out_f32 else (2.0 ** -8 if dt == "bf16" else 2.0 ** -10)
    fl = 2.0 ** -25 if (dt == "f16" and not out_f32) else 0.0  # binary16 subnormal rounding is absolute
    assert oracle.normalized_error(got, oracle.sddmm(rp, ci, dC_r, B_r), D, abs_floor=fl) <= tol_rounded
    # against the oracle on the original float32 inputs: input rounding included
    assert oracle.normalized_error(got, oracle.sddmm(rp, ci, dC, B), oracle.sddmm_abs_bound(rp, ci, dC, B),
                                   abs_floor=fl) <= 1e-2


@pytest.mark.parametrize("name", ["power_law", "giant_row", "duplicates_unsorted", "empty_runs"])
@pytest.mark.parametrize("alg", ["row_split", "merge", "auto_gb300"])
def test_transposed_product(gpu_lib, name, alg):
    import torch

    rp, ci, v, k = structure(name)
    m, n = len(rp) - 1, 64
    dC = gen.normal_matrix(m, n, 41)
    d_rp, d_ci, d_v, d_dC = dev(torch, rp, ci, v, dC)
    A = gpu_lib.CSRMatrix(d_rp, d_ci, (m, k))
    dB = A.spmm_t(d_v, d_dC, alg=gpu_lib.alg_code(alg))
    torch.cuda.synchronize()
    ref = oracle.spmm_t(rp, ci, v, dC, k)
    D = oracle.spmm_t(rp, ci, np.abs(v), np.abs(dC), k)  # |A^T| |dC|
    assert oracle.normalized_error(dB.cpu().numpy(), ref, D) <= FP32_TOL


def test_autograd_central_differences_and_dense_reference(gpu_lib):
    """GCN-shaped m = k = 64 instance: GPU gradients of L = <G, A B> against
    float64 central differences of the oracle and against float64 dense autograd."""
    import torch

    a = gen.chung_lu_gcn(64, 5, mean_degree=6.0)
    n = 16
    rng = np.random.default_rng(9)
    B = rng.standard_normal((a.k, n)).astype(np.float32)
    G = rng.standard_normal((a.m, n)).astype(np.float32)
    d_rp, d_ci = dev(torch, a.row_ptr, a.col_ind)
    A = gpu_lib.CSRMatrix(d_rp, d_ci, (a.m, a.k))
    vals = torch.from_numpy(a.vals).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda().requires_grad_(True)
    C = gpu_lib.spmm_autograd(A, vals, Bt)
    (C * torch.from_numpy(G).cuda()).sum().backward()
    g_vals, g_B = vals.grad.cpu().numpy(), Bt.grad.cpu().numpy()

    v64, B64, G64 = a.vals.astype(np.float64), B.astype(np.float64), G.astype(np.float64)

    def loss(vv, bb):
        return float(np.sum(G64 * oracle.spmm(a.row_ptr, a.col_ind, vv, bb)))

    h = 0.5  # exact for a bilinear form up to rounding
    fd_vals = np.array([(loss(v64 + h * e, B64) - loss(v64 - h * e, B64)) / (2 * h) for e in np.eye(a.nnz)])
    scale_v = oracle.sddmm_abs_bound(a.row_ptr, a.col_ind, np.abs(G64), np.abs(B64))
    assert oracle.normalized_error(g_vals, fd_vals, scale_v) <= FP32_TOL
    idx = [(int(i), int(j)) for i, j in zip(rng.integers(0, a.k, 60), rng.integers(0, n, 60))]
    fd_B = []
    for i, j in idx:
        e = np.zeros_like(B64)
        e[i, j] = h
        fd_B.append((loss(v64, B64 + e) - loss(v64, B64 - e)) / (2 * h))
    scale_B = oracle.spmm_t(a.row_ptr, a.col_ind, np.abs(v64), np.abs(G64), a.k)
    got_B = np.array([g_B[i, j] for i, j in idx])
    assert oracle.normalized_error(got_B, np.array(fd_B), np.array([scale_B[i, j] for i, j in idx])) <= FP32_TOL

    # float64 dense autograd of the same loss
    rows = np.repeat(np.arange(a.m), np.diff(a.row_ptr))
    vt = torch.tensor(v64, requires_grad=True)
    Bd = torch.tensor(B64, requires_grad=True)
    dense = torch.zeros((a.m, a.k), dtype=torch.float64).index_put(
        (torch.from_numpy(rows), torch.from_numpy(a.col_ind.astype(np.int64))), vt, accumulate=True)
    (torch.tensor(G64) * (dense @ Bd)).sum().backward()
    assert oracle.normalized_error(g_vals, vt.grad.numpy(), scale_v) <= FP32_TOL
    assert oracle.normalized_error(g_B, Bd.grad.numpy(), scale_B) <= FP32_TOL


@pytest.mark.slow
def test_gcn_workload_full_size(gpu_lib):
    """500k-node GCN adjacency, n = 256: forward, dX = A^T dY and dvals at full size,
    checked on sampled rows / nonzeros (the transpose bit-exactly, everywhere)."""
    import torch

    a, X = gen.workload_gcn()
    n = X.shape[1]
    dY = gen.normal_matrix(a.m, n, 77)
    d_rp, d_ci, d_v, d_X, d_dY = dev(torch, a.row_ptr, a.col_ind, a.vals, X, dY)
    A = gpu_lib.CSRMatrix(d_rp, d_ci, (a.m, a.k))
    Y = A.spmm(d_v, d_X)
    dX = A.spmm_t(d_v, d_dY)
    dv = gpu_lib.sddmm(d_rp, d_ci, d_dY, d_X)
    torch.cuda.synchronize()
    rpt, cit, perm, _ = A.transpose_pattern()
    o_rpt, o_cit, o_perm = oracle.csr_transpose(a.row_ptr, a.col_ind, a.k)
    assert np.array_equal(perm.cpu().numpy(), o_perm) and np.array_equal(rpt.cpu().numpy(), o_rpt)
    rng = np.random.default_rng(4)
    lens = a.row_lengths()
    rows = np.unique(np.concatenate([rng.choice(a.m, 1500, replace=False), np.argsort(lens)[-10:]]))
    sel = torch.from_numpy(rows).cuda()
    err_y = oracle.normalized_error(Y[sel].cpu().numpy(), oracle.spmm_rows(rows, a.row_ptr, a.col_ind, a.vals, X),
                                    oracle.abs_bound_rows(rows, a.row_ptr, a.col_ind, a.vals, X))
    vt = a.vals[o_perm]
    err_dx = oracle.normalized_error(dX[sel].cpu().numpy(), oracle.spmm_rows(rows, o_rpt, o_cit, vt, dY),
                                     oracle.abs_bound_rows(rows, o_rpt, o_cit, vt, dY))
    # SDDMM on the nonzeros of the sampled rows
    sub_rp = np.concatenate([[0], np.cumsum(lens[rows])]).astype(np.int32)
    pos = np.concatenate([np.arange(a.row_ptr[r], a.row_ptr[r + 1]) for r in rows])
    ref = oracle.sddmm(sub_rp, a.col_ind[pos], dY[rows], X)
    D = oracle.sddmm_abs_bound(sub_rp, a.col_ind[pos], dY[rows], X)
    err_dv = oracle.normalized_error(dv.cpu().numpy()[pos], ref, D)
    assert max(err_y, err_dx, err_dv) <= FP32_TOL, (err_y, err_dx, err_dv)
