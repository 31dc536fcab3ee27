"""GPU parity of the batched form (persistent launches over many CSR
products of uneven sizes, graph replay, autotuned schedule) with the oracle."""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import FP32_TOL

pytestmark = pytest.mark.gpu


def make_batch(torch, count, seed, m_hi=4096, lam_hi=64.0):
    s = gen.batched_set(count, seed, m_hi=m_hi, lam_hi=lam_hi)
    # a few adversarial members: an empty matrix, an all-empty-rows matrix, a heavy row
    mats, ns = list(s.mats), list(s.ns)
    mats[0] = gen.csr_from_lengths(np.zeros(70, dtype=np.int64), 70, 1)
    lens = np.random.default_rng(seed).integers(0, 6, 3000)
    lens[1500] = 2900
    mats[1] = gen.csr_from_lengths(lens, 3000, 2)
    host, dev = [], []
    for i, (a, n) in enumerate(zip(mats, ns)):
        B = gen.normal_matrix(a.k, n, 100 + i)
        host.append((a, B))
        dev.append(tuple(torch.from_numpy(x).cuda() for x in (a.row_ptr, a.col_ind, a.vals, B)) +
                   (torch.full((a.m, n), float("nan"), device="cuda"),))
    return host, dev


def check_all(host, dev):
    for (a, B), d in zip(host, dev):
        C = d[4].cpu().numpy()
        err = oracle.normalized_error(C, oracle.spmm(a.row_ptr, a.col_ind, a.vals, B),
                                      oracle.abs_bound(a.row_ptr, a.col_ind, a.vals, B))
        assert err <= FP32_TOL, err


@pytest.mark.parametrize("policy", ["model", "autotune", "row_split", "merge", "row_split_x2"])
def test_batched_policies(gpu_lib, policy):
    import torch

    pkg = gpu_lib
    host, dev = make_batch(torch, 40, 5)
    pol = {"model": pkg.BATCHED_MODEL, "autotune": pkg.BATCHED_AUTOTUNE, "row_split": pkg.BATCHED_ROW_SPLIT,
           "merge": pkg.BATCHED_MERGE, "row_split_x2": pkg.BATCHED_ROW_SPLIT_X2}[policy]
    plan = pkg.BatchedPlan(*[[d[i] for d in dev] for i in range(5)], policy=pol)
    algs, items, tiles = plan.query()
    assert len(algs) == 40 and items > 0
    if policy == "merge":
        assert set(algs) == {pkg.ALG_MERGE} and tiles > 0
    if policy in ("row_split", "row_split_x2"):
        assert set(algs) == {pkg.ALG_ROW_SPLIT} and tiles == 0
    if policy == "model":
        assert algs[1] == pkg.ALG_MERGE  # heavy row: Type 1 guard
    c0 = pkg.spmm_launch_count()
    plan.run()
    torch.cuda.synchronize()
    # row chunks (one kernel per access width used), merge tiles, fix-up: independent of the batch size
    assert pkg.spmm_launch_count() - c0 <= 4
    check_all(host, dev)
    # graph replay, with new values of B between replays
    plan.capture_graph()
    for d in dev:
        d[4].fill_(float("nan"))
    for (a, B), d in zip(host, dev):
        d[3].mul_(-2.0)
    plan.launch_graph()
    torch.cuda.synchronize()
    check_all([(a, -2.0 * B) for a, B in host], dev)
    # the unfused baseline gives the same products
    for d in dev:
        d[4].fill_(float("nan"))
    plan.run_unfused()
    torch.cuda.synchronize()
    check_all([(a, -2.0 * B) for a, B in host], dev)
    plan.close()
    if policy == "autotune":
        assert pkg.spmm_autotune_cache_entries() > 0


def test_batched_exact_integers(gpu_lib):
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(3)
    host, dev = make_batch(torch, 24, 9)
    for (a, B), d in zip(host, dev):
        a.vals[:] = rng.integers(-2, 3, a.nnz)
        B[:] = rng.integers(-4, 5, B.shape)
        d[2].copy_(torch.from_numpy(a.vals))
        d[3].copy_(torch.from_numpy(B))
    for pol in (pkg.BATCHED_MERGE, pkg.BATCHED_ROW_SPLIT, pkg.BATCHED_ROW_SPLIT_X2):
        plan = pkg.BatchedPlan(*[[d[i] for d in dev] for i in range(5)], policy=pol)
        plan.run()
        torch.cuda.synchronize()
        for (a, B), d in zip(host, dev):
            assert np.array_equal(d[4].cpu().numpy(), oracle.spmm(a.row_ptr, a.col_ind, a.vals, B).astype(np.float32))
        plan.close()


def test_batched_one_and_two_vector_widths_in_one_plan(gpu_lib):
    """Under SPMM_BATCHED_ROW_SPLIT_X2 the widths that are multiples of 8 read two 16-byte vectors
    per lane and the others one: the plan runs one row kernel per width (two launches), and every
    product must equal the oracle bit for bit on integer data."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(17)
    widths = [36, 32, 44, 64, 200, 12, 128, 8]
    host, dev = [], []
    for i, n in enumerate(widths):
        m = int(rng.integers(50, 3000))
        lens = rng.integers(0, 40, m)
        a = gen.csr_from_lengths(lens, m, 200 + i)
        a.vals[:] = rng.integers(-2, 3, a.nnz)
        B = rng.integers(-4, 5, size=(m, n)).astype(np.float32)
        host.append((a, B))
        dev.append(tuple(torch.from_numpy(x).cuda() for x in (a.row_ptr, a.col_ind, a.vals, B)) +
                   (torch.full((m, n), float("nan"), device="cuda"),))
    plan = pkg.BatchedPlan(*[[d[i] for d in dev] for i in range(5)], policy=pkg.BATCHED_ROW_SPLIT_X2)
    c0 = pkg.spmm_launch_count()
    plan.run()
    torch.cuda.synchronize()
    assert pkg.spmm_launch_count() - c0 == 2  # the one-vector and the two-vector row kernels
    for (a, B), d in zip(host, dev):
        assert np.array_equal(d[4].cpu().numpy(), oracle.spmm(a.row_ptr, a.col_ind, a.vals, B).astype(np.float32))
    plan.capture_graph()
    for d in dev:
        d[4].fill_(float("nan"))
    plan.launch_graph()
    torch.cuda.synchronize()
    for (a, B), d in zip(host, dev):
        assert np.array_equal(d[4].cpu().numpy(), oracle.spmm(a.row_ptr, a.col_ind, a.vals, B).astype(np.float32))
    plan.close()


@pytest.mark.slow
def test_batched_workload_full_size_sampled(gpu_lib):
    """2048 matrices (m up to 65,536, Poisson rows with lambda up to 64): graph replay,
    every matrix checked on a few sampled rows."""
    import torch

    pkg = gpu_lib
    s = gen.workload_batched()
    dev = []
    Bs = []
    for i, (a, n) in enumerate(zip(s.mats, s.ns)):
        B = gen.normal_matrix(a.k, n, 5000 + i)
        Bs.append(B)
        dev.append(tuple(torch.from_numpy(x).cuda() for x in (a.row_ptr, a.col_ind, a.vals, B)) +
                   (torch.empty((a.m, n), device="cuda"),))
    plan = pkg.BatchedPlan(*[[d[i] for d in dev] for i in range(5)], policy=pkg.BATCHED_MODEL)
    plan.capture_graph()
    plan.launch_graph()
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    worst = 0.0
    for a, B, d in zip(s.mats, Bs, dev):
        rows = np.unique(rng.integers(0, a.m, 4))
        got = d[4][torch.from_numpy(rows).cuda()].cpu().numpy()
        worst = max(worst, oracle.normalized_error(got, oracle.spmm_rows(rows, a.row_ptr, a.col_ind, a.vals, B),
                                                   oracle.abs_bound_rows(rows, a.row_ptr, a.col_ind, a.vals, B)))
    assert worst <= FP32_TOL
    plan.close()


@pytest.mark.parametrize("policy", ["row_split", "merge", "autotune"])
def test_batched_column_slabs(gpu_lib, policy):
    """Matrices wider than one lane group (n = 256 and 384: 64 and 96 16-byte vectors, so two and
    three column slabs of 32 lanes) next to narrow ones, in one plan: every slab's item writes its
    own columns, and the merge slabs share the matrix's partition and carries."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(17)
    host, dev = [], []
    for i, n in enumerate((256, 32, 384, 64, 256)):
        m = int(rng.integers(500, 3000))
        lens = rng.poisson(12.0, m)
        if i == 2:
            lens[m // 2] = m  # a heavy row: the Type 1 guard sends this matrix to merge under "model"
        a = gen.csr_from_lengths(np.minimum(lens, m), m, 60 + i)
        B = gen.normal_matrix(a.k, n, 70 + i)
        host.append((a, B))
        dev.append(tuple(torch.from_numpy(x).cuda() for x in (a.row_ptr, a.col_ind, a.vals, B)) +
                   (torch.full((a.m, n), float("nan"), device="cuda"),))
    pol = {"row_split": pkg.BATCHED_ROW_SPLIT, "merge": pkg.BATCHED_MERGE, "autotune": pkg.BATCHED_AUTOTUNE}[policy]
    plan = pkg.BatchedPlan(*[[d[i] for d in dev] for i in range(5)], policy=pol)
    plan.run()
    torch.cuda.synchronize()
    check_all(host, dev)
    plan.close()
