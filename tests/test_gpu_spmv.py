"""GPU parity of the SpMV forms (n = 1) of both families with the FP64 oracle,
through the C ABI: the row split with 1 to 32 lanes per row striding over a
row's nonzeros, and the merge-based kernel with 4, 8 and 16 path items per
thread (tiles of 1024 to 4096 items), which also move the merge-path cuts and
so which rows the fix-up finishes."""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import STRUCTURES, check, csr_arrays, structure
from test_gpu_precision import errors, run_case, OUT_TOL, COMBOS

pytestmark = pytest.mark.gpu

LANES = [1, 2, 4, 8, 16, 32]
ITEMS = [4, 8, 16]


def to_dev(torch, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def run(pkg, torch, rp, ci, v, x, alg, **kw):
    d_rp, d_ci, d_v = to_dev(torch, rp, ci, v)
    d_x = x if isinstance(x, torch.Tensor) else to_dev(torch, x)[0]
    y = pkg.spmm(d_rp, d_ci, d_v, d_x, alg=alg, nnz=int(rp[-1]), **kw)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("name", STRUCTURES)
@pytest.mark.parametrize("lanes", LANES)
def test_row_split_lanes(gpu_lib, name, lanes):
    import torch

    rp, ci, v, k = structure(name)
    x = gen.normal_matrix(k, 1, 41)
    check(run(gpu_lib, torch, rp, ci, v, x, "row_split", tuning=dict(lanes_per_row=lanes)), rp, ci, v, x)


@pytest.mark.parametrize("name", STRUCTURES)
@pytest.mark.parametrize("items", ITEMS)
def test_merge_items_per_thread(gpu_lib, name, items):
    import torch

    rp, ci, v, k = structure(name)
    x = gen.normal_matrix(k, 1, 42)
    check(run(gpu_lib, torch, rp, ci, v, x, "merge", tuning=dict(items_per_subwarp=items)), rp, ci, v, x)


@pytest.mark.parametrize("alg,tuning", [("row_split", dict(lanes_per_row=g)) for g in LANES] +
                         [("merge", dict(items_per_subwarp=t)) for t in ITEMS])
def test_integer_spmv_is_bitwise(gpu_lib, alg, tuning):
    """Integer vals and x with rows up to 3 x 10^4 terms: every partial sum is an
    integer below 2^24, so any summation order must give the oracle's value."""
    import torch

    rng = np.random.default_rng(17)
    lens = rng.integers(0, 50, 20_000)
    lens[::997] = 30_000
    lens[5:400] = 0  # a run of empty rows
    rp, ci, v = csr_arrays(lens, 40_000, 9, int_vals=True)
    x = rng.integers(-4, 5, size=(40_000, 1)).astype(np.float32)
    y = run(gpu_lib, torch, rp, ci, v, x, alg, tuning=tuning)
    assert np.array_equal(y, oracle.spmm(rp, ci, v, x).astype(np.float32))


@pytest.mark.parametrize("alg", ["row_split", "merge"])
def test_strided_vector_and_result(gpu_lib, alg):
    """x is column 3 of a 7-wide matrix (ldb = 7) and y a column of a 5-wide
    output (ldc = 5); the other output columns are left untouched."""
    import torch

    rp, ci, v, k = structure("power_law", seed=4)
    X = gen.normal_matrix(k, 7, 43)
    d_rp, d_ci, d_v, d_X = to_dev(torch, rp, ci, v, X)
    Y = torch.full((len(rp) - 1, 5), 7.0, device="cuda")
    gpu_lib.spmm(d_rp, d_ci, d_v, d_X[:, 3:4], alg=alg, out=Y[:, 2:3], nnz=int(rp[-1]))
    torch.cuda.synchronize()
    Y = Y.cpu().numpy()
    check(Y[:, 2:3], rp, ci, v, X[:, 3:4])
    assert np.all(np.delete(Y, 2, axis=1) == 7.0)


@pytest.mark.parametrize("combo", COMBOS)
@pytest.mark.parametrize("alg", ["row_split", "merge"])
def test_16bit_spmv(gpu_lib, combo, alg):
    import torch

    rp, ci, v, k = structure("power_law", seed=5)
    x = gen.normal_matrix(k, 1, 44)
    got, v_r, x_r = run_case(gpu_lib, torch, rp, ci, v, x, combo, alg)
    e_r, e_o = errors(got, rp, ci, v, x, v_r, x_r, out=combo[2])
    assert e_r <= OUT_TOL[combo[2]], e_r
    assert e_o <= 1e-2, e_o


def test_spmv_result_is_deterministic(gpu_lib):
    import torch

    rp, ci, v, k = structure("giant_row")
    x = gen.normal_matrix(k, 1, 45)
    for alg in ("row_split", "merge"):
        first = run(gpu_lib, torch, rp, ci, v, x, alg)
        for _ in range(3):
            assert np.array_equal(run(gpu_lib, torch, rp, ci, v, x, alg), first)


def test_full_size_power_law_sampled(gpu_lib):
    """The 1M x 1M power-law matrix (rows up to 10^5 nonzeros) with the
    selector's pick, compared on 2000 sampled rows including the longest."""
    import torch

    a = gen.workload_power_law()
    x = gen.normal_matrix(a.k, 1, 46)
    lens = np.diff(a.row_ptr)
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([rng.choice(a.m, 2000, replace=False), np.argsort(lens)[-20:]])).astype(np.int64)
    for alg in ("merge", "auto_gb300"):
        y = run(gpu_lib, torch, a.row_ptr, a.col_ind, a.vals, x, alg)
        check(y[rows], a.row_ptr, a.col_ind, a.vals, x, rows=rows)
