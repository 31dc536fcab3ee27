"""GPU parity of the FP32 SpMM paths (row split, merge based, heuristic) with
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import FP32_TOL, STRUCTURES, check, csr_arrays, structure

pytestmark = pytest.mark.gpu

ALGS = ["row_split", "merge", "hybrid", "auto", "auto_gb300"]


def to_dev(torch, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def run(pkg, torch, rp, ci, v, B, alg, **kw):
    d_rp, d_ci, d_v = to_dev(torch, rp, ci, v)
    d_B = B if isinstance(B, torch.Tensor) else to_dev(torch, B)[0]
    C = pkg.spmm(d_rp, d_ci, d_v, d_B, alg=alg, nnz=int(rp[-1]), **kw)
    torch.cuda.synchronize()
    return C


@pytest.mark.parametrize("name", STRUCTURES)
@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("n", [1, 4, 8, 13, 40, 64, 128, 300])
def test_structures(gpu_lib, name, alg, n):
    import torch

    rp, ci, v, k = structure(name)
    B = gen.normal_matrix(k, n, 11 + n)
    C = run(gpu_lib, torch, rp, ci, v, B, alg)
    assert C.shape == (len(rp) - 1, n)
    check(C.cpu().numpy(), rp, ci, v, B)


@pytest.mark.parametrize("alg", ["row_split", "merge", "hybrid"])
@pytest.mark.parametrize("n", [4, 32, 64, 96, 256])
def test_exact_integer_arithmetic_is_bitwise(gpu_lib, alg, n):
    """Integer vals in [-2, 2] and B in [-4, 4] with rows of up to 10^4 terms: every
    partial sum is an integer below 2^24, so float32 must equal the oracle exactly,
    whatever the summation order (this pins the carry-out / fix-up arithmetic)."""
    import torch

    rng = np.random.default_rng(n)
    lens = rng.integers(0, 300, 3000)
    lens[::97] = 10_000
    rp, ci, v = csr_arrays(lens, 12_000, 5, int_vals=True)
    B = rng.integers(-4, 5, size=(12_000, n)).astype(np.float32)
    for ips in (4, 37, 0):
        C = run(gpu_lib, torch, rp, ci, v, B, alg, tuning=dict(items_per_subwarp=ips))
        assert np.array_equal(C.cpu().numpy(), oracle.spmm(rp, ci, v, B).astype(np.float32))


def test_identity_and_permutation_are_exact(gpu_lib):
    import torch

    for name in ("identity", "permutation"):
        rp, ci, v, k = structure(name)
        B = gen.normal_matrix(k, 64, 3)
        for alg in ALGS:
            C = run(gpu_lib, torch, rp, ci, v, B, alg).cpu().numpy()
            assert np.array_equal(C, B[ci])


@pytest.mark.parametrize("alg", ["row_split", "merge", "hybrid"])
@pytest.mark.parametrize("tuning", [dict(lanes_per_row=4), dict(lanes_per_row=32), dict(column_slabs=4),
                                    dict(column_slabs=2, items_per_subwarp=9), dict(items_per_subwarp=4),
                                    dict(items_per_subwarp=700), dict(lanes_per_row=1, items_per_subwarp=5)])
def test_launch_shapes(gpu_lib, alg, tuning):
    import torch

    rp, ci, v, k = structure("power_law", seed=2)
    B = gen.normal_matrix(k, 64, 5)
    C = run(gpu_lib, torch, rp, ci, v, B, alg, tuning=tuning)
    check(C.cpu().numpy(), rp, ci, v, B)


@pytest.mark.parametrize("alg", ALGS)
def test_strides_and_scalar_path(gpu_lib, alg):
    """ldb > n, ldc > n, and a B whose base is not 16-byte aligned (scalar path)."""
    import torch

    rp, ci, v, k = structure("short_rows")
    n = 48
    Bbig = gen.normal_matrix(k, 70, 8)
    d_big = torch.from_numpy(Bbig).cuda()
    out = torch.full((len(rp) - 1, 61), 7.0, device="cuda")
    for Bview, ref_B in ((d_big[:, :n], Bbig[:, :n]), (d_big[:, 1:n + 1], Bbig[:, 1:n + 1])):
        C = run(gpu_lib, torch, rp, ci, v, Bview, alg, out=out[:, 3:3 + n])
        check(C.cpu().numpy(), rp, ci, v, np.ascontiguousarray(ref_B))
        assert torch.all(out[:, :3] == 7.0) and torch.all(out[:, 3 + n:] == 7.0)  # padding untouched


def test_merge_partition_matches_oracle(gpu_lib):
    import torch

    for name in ("power_law", "empty_runs", "giant_row", "all_empty", "single_row"):
        rp, ci, v, k = structure(name)
        d_rp = torch.from_numpy(rp).cuda()
        for items in (1, 7, 64, 2048):
            if (len(rp) - 1 + int(rp[-1])) // items > 2_000_000:
                continue
            lim = gpu_lib.merge_partition(d_rp, items, nnz=int(rp[-1])).cpu().numpy()
            assert np.array_equal(lim, oracle.merge_path_limits(rp, items)), (name, items)


def test_merge_is_deterministic(gpu_lib):
    import torch

    rp, ci, v, k = structure("giant_row")
    B = gen.normal_matrix(k, 64, 9)
    c1 = run(gpu_lib, torch, rp, ci, v, B, "merge").cpu().numpy()
    c2 = run(gpu_lib, torch, rp, ci, v, B, "merge").cpu().numpy()
    assert np.array_equal(c1, c2)


def test_explicit_workspace_and_status(gpu_lib):
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("short_rows")
    B = gen.normal_matrix(k, 32, 2)
    m, nnz = len(rp) - 1, int(rp[-1])
    size = pkg.workspace_size(m, k, 32, nnz, "merge")
    ws = torch.empty(size, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = run(pkg, torch, rp, ci, v, B, "merge", workspace=ws, status=status)
    check(C.cpu().numpy(), rp, ci, v, B)
    assert int(status.item()) == 0
    with pytest.raises(pkg.SpMMError) as e:
        run(pkg, torch, rp, ci, v, B, "merge", workspace=ws[: size // 4])
    assert e.value.status == pkg.ERR_WORKSPACE


def test_gb300_selector_picks_merge_for_heavy_tail(gpu_lib):
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("giant_row")
    d_rp = torch.from_numpy(rp).cuda()
    assert pkg.max_row_length(d_rp) == int(np.diff(rp).max())
    assert pkg.spmm_select_alg_gb300(len(rp) - 1, int(rp[-1]), pkg.max_row_length(d_rp), 64) == pkg.ALG_MERGE
    c0 = pkg.spmm_launch_count()
    B = gen.normal_matrix(k, 64, 3)
    C = run(pkg, torch, rp, ci, v, B, "auto_gb300")  # measures the longest row itself: 1 + 3 launches
    assert pkg.spmm_launch_count() - c0 == 4
    check(C.cpu().numpy(), rp, ci, v, B)


@pytest.mark.parametrize("n,tuning", [(1, dict(items_per_subwarp=4)), (1, None), (13, dict(items_per_subwarp=5)),
                                      (64, dict(items_per_subwarp=4, column_slabs=4)), (128, None)])
def test_rows_crossing_many_tiles_reuse_one_workspace(gpu_lib, n, tuning):
    """Rows that span up to thousands of merge tiles (in every column slab),
    the last of them running to the end of the path, finished by the fix-up.
    Integer values make the result exact in any order; the status word stays
    clear; one workspace reused by back-to-back calls on the stream (each call
    rewrites every entry it reads) gives the same bits every time."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 6, 3000)
    lens[[7, 1500, 2999]] = [40_000, 25_000, 60_000]  # the last row runs to the end of the path
    lens[100:200] = 0
    rp, ci, v = csr_arrays(lens, 70_000, 31, int_vals=True)
    B = rng.integers(-3, 4, size=(70_000, n)).astype(np.float32)
    ref = oracle.spmm(rp, ci, v, B).astype(np.float32)
    d_rp, d_ci, d_v, d_B = to_dev(torch, rp, ci, v, B)
    nnz = int(rp[-1])
    ws = torch.empty(pkg.workspace_size(len(rp) - 1, 70_000, n, nnz, "merge", tuning=tuning), dtype=torch.uint8,
                     device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    outs = [pkg.spmm(d_rp, d_ci, d_v, d_B, alg="merge", nnz=nnz, tuning=tuning, workspace=ws, status=status)
            for _ in range(3)]
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    for C in outs:
        assert np.array_equal(C.cpu().numpy(), ref)


def test_launch_counts(gpu_lib):
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("short_rows")
    B = gen.normal_matrix(k, 32, 2)
    c0 = pkg.spmm_launch_count()
    run(pkg, torch, rp, ci, v, B, "row_split")
    c1 = pkg.spmm_launch_count()
    run(pkg, torch, rp, ci, v, B, "merge")
    c2 = pkg.spmm_launch_count()
    assert c1 - c0 == 1  # one row-split launch
    assert c2 - c1 == 3  # partition, compute, fix-up


def test_bounded_wait_reports_timeout_and_context_survives(gpu_lib):
    """A wait on an mbarrier phase that nothing completes runs out after its limit,
    stores SPMM_ERR_TIMEOUT, and the context keeps working."""
    import torch

    pkg = gpu_lib
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert pkg.spmm_debug_bounded_wait(status.data_ptr(), 2_000_000, torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == pkg.ERR_TIMEOUT
    rp, ci, v, k = structure("uniform16")
    B = gen.normal_matrix(k, 16, 1)
    check(run(pkg, torch, rp, ci, v, B, "merge").cpu().numpy(), rp, ci, v, B)


@pytest.mark.parametrize("n", [8, 13, 64, 128, 300])
def test_host_buffers_entry_point(gpu_lib, n):
    """spmm_csr_host: host arrays in and out, B and C pipelined in column slabs
    over the copy streams (one slab for narrow rows, up to four for wide ones)."""
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("power_law")
    B = gen.normal_matrix(k, n, 4)
    for alg in ALGS:
        C = torch.empty((len(rp) - 1, n), dtype=torch.float32).pin_memory()
        pkg.spmm_host(torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(v), torch.from_numpy(B), C, alg=alg)
        check(C.numpy(), rp, ci, v, B)


def test_host_buffers_strided_and_16bit(gpu_lib):
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("short_rows")
    n = 96
    Bbig = torch.from_numpy(gen.normal_matrix(k, n + 5, 6))
    Cbig = torch.full((len(rp) - 1, n + 7), 3.0)
    pkg.spmm_host(torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(v), Bbig[:, 2:2 + n],
                  Cbig[:, 1:1 + n], alg="merge")
    check(Cbig[:, 1:1 + n].numpy(), rp, ci, v, np.ascontiguousarray(Bbig[:, 2:2 + n].numpy()))
    assert torch.all(Cbig[:, 0] == 3.0) and torch.all(Cbig[:, 1 + n:] == 3.0)
    vb, Bb = torch.from_numpy(v).to(torch.bfloat16), torch.from_numpy(gen.normal_matrix(k, 128, 7)).to(torch.bfloat16)
    Cb = torch.empty((len(rp) - 1, 128), dtype=torch.float32)
    pkg.spmm_host(torch.from_numpy(rp), torch.from_numpy(ci), vb, Bb, Cb, alg="auto_gb300")
    D = oracle.abs_bound(rp, ci, vb.double().numpy(), Bb.double().numpy())
    assert oracle.normalized_error(Cb.numpy(), oracle.spmm(rp, ci, vb.double().numpy(), Bb.double().numpy()), D) <= FP32_TOL


def test_plain_fp32_workload_full(gpu_lib):
    """4096 x 4096, 16 nonzeros per row, n = 64: every element against the oracle."""
    import torch

    a, B = gen.workload_plain()
    for alg in ALGS:
        C = run(gpu_lib, torch, a.row_ptr, a.col_ind, a.vals, B, alg)
        check(C.cpu().numpy(), a.row_ptr, a.col_ind, a.vals, B)


@pytest.mark.slow
@pytest.mark.parametrize("n", [8, 32, 64, 128])
def test_power_law_workload_full_size_sampled(gpu_lib, n):
    """1M x 1M power-law rows at full size, both algorithms and the heuristic;
    checked on a seeded sample of rows that includes the longest ones."""
    import torch

    a = gen.workload_power_law()
    B = gen.normal_matrix(a.k, n, gen.SEED_BASE + 2)
    lens = a.row_lengths()
    rng = np.random.default_rng(n)
    rows = np.unique(np.concatenate([rng.choice(a.m, 3000, replace=False), np.argsort(lens)[-20:],
                                     np.nonzero(lens == 0)[0][:50], [0, a.m - 1]]))
    d_rp, d_ci, d_v = to_dev(torch, a.row_ptr, a.col_ind, a.vals)
    d_B = torch.from_numpy(B).cuda()
    for alg in ALGS:
        C = gpu_lib.spmm(d_rp, d_ci, d_v, d_B, alg=alg, nnz=a.nnz)
        torch.cuda.synchronize()
        check(C[torch.from_numpy(rows).cuda()].cpu().numpy(), a.row_ptr, a.col_ind, a.vals, B, rows=rows)


@pytest.mark.parametrize("name", ["uniform16", "power_law", "short_rows", "alternating_empty", "empty_runs",
                                  "all_empty", "giant_row", "single_row", "one_nonzero", "tall_k1", "identity",
                                  "permutation"])
@pytest.mark.parametrize("n", [8, 13, 64, 128, 300])
def test_tiled_structures(gpu_lib, name, n):
    """A/B tiling on every structure with increasing columns (n = 13 has no
    16-byte path and runs the row split)."""
    import torch

    rp, ci, v, k = structure(name)
    if name == "permutation":  # one entry per row: trivially increasing
        pass
    B = gen.normal_matrix(k, n, 11 + n)
    C = run(gpu_lib, torch, rp, ci, v, B, "tiled")
    check(C.cpu().numpy(), rp, ci, v, B)


@pytest.mark.parametrize("n", [8, 32, 64, 128, 256])
def test_tiled_integer_arithmetic_is_bitwise(gpu_lib, n):
    """Integer data across many k-panels (k = 12,000 spans 23-188 panels): the
    tiled sum must equal the oracle exactly."""
    import torch

    rng = np.random.default_rng(n + 1)
    lens = rng.integers(0, 400, 3000)
    lens[::97] = 8000
    rp, ci, v = csr_arrays(lens, 12_000, 6, int_vals=True)
    B = rng.integers(-4, 5, size=(12_000, n)).astype(np.float32)
    C = run(gpu_lib, torch, rp, ci, v, B, "tiled").cpu().numpy()
    assert np.array_equal(C, oracle.spmm(rp, ci, v, B).astype(np.float32))


def test_tiled_reports_rows_that_go_backwards(gpu_lib):
    """Columns must increase within a row: a row that goes backwards across a
    panel boundary is reported (SPMM_ERR_BAD_CSR) and its late entry skipped;
    every other row is still exact."""
    import torch

    k, n = 4000, 64
    rp = np.array([0, 3, 5, 7], dtype=np.int32)
    ci = np.array([5, 3000, 7, 10, 20, 1, 2], dtype=np.int32)  # row 0: 3000 then 7 (backwards)
    v = np.ones(7, dtype=np.float32)
    B = np.arange(k * n, dtype=np.float32).reshape(k, n) % 7
    d_rp, d_ci, d_v, d_B = to_dev(torch, rp, ci, v, B)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = gpu_lib.spmm(d_rp, d_ci, d_v, d_B, alg="tiled", nnz=7, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == gpu_lib.ERR_BAD_CSR
    C = C.cpu().numpy()
    assert np.array_equal(C[0], B[5] + B[3000])  # the backwards entry (column 7) skipped
    assert np.array_equal(C[1:], oracle.spmm(rp, ci, v, B).astype(np.float32)[1:])


@pytest.mark.parametrize("combo", [("bf16", "bf16", "bf16"), ("bf16", "bf16", "f32"), ("f16", "f16", "f16"),
                                   ("bf16", "f16", "f32")])
def test_tiled_16bit(gpu_lib, combo):
    from test_gpu_precision import OUT_TOL, errors, run_case

    import torch

    rp, ci, v, k = structure("uniform16")
    B = gen.normal_matrix(k, 64, 62)
    got, v_r, B_r = run_case(gpu_lib, torch, rp, ci, v, B, combo, "tiled")
    e_r, e_o = errors(got, rp, ci, v, B, v_r, B_r, out=combo[2])
    assert e_r <= OUT_TOL[combo[2]], e_r
    assert e_o <= 1e-2, e_o


@pytest.mark.parametrize("n", [8, 64, 128])
def test_host_entry_row_chunks(gpu_lib, n):
    """spmm_csr_host splits A into up to four row chunks of at least 8 MB (equal shares of rows +
    nonzeros, each uploaded, rebased and computed on its own): runs of empty rows, a row of
    300,000 nonzeros and short rows, checked on every row against the oracle."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(n)
    lens = rng.integers(0, 48, 200_000)
    lens[50_000:60_000] = 0
    lens[123_456] = 300_000
    lens[-5000:] = 0
    rp, ci, v = csr_arrays(lens, 400_000, 12)
    assert len(rp) * 4 + 8 * int(rp[-1]) >= 32 << 20  # A's bytes: four chunks of at least 8 MB
    B = gen.normal_matrix(400_000, n, 13)
    for alg in ALGS:
        C = torch.full((len(rp) - 1, n), float("nan")).pin_memory()
        pkg.spmm_host(torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(v), torch.from_numpy(B), C, alg=alg)
        check(C.numpy(), rp, ci, v, B)


def test_host_async_back_to_back(gpu_lib):
    """spmm_csr_host_async: products of several widths, families and matrices
    (one large enough for four row chunks of A) queued back to back with no
    synchronisation in between, then one synchronisation of the stream; a copy
    of C queued on the stream after a call sees its result; a second round of
    the same calls (staging memory reused) gives the same bits."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(21)
    lens = rng.integers(0, 48, 200_000)
    lens[77_777] = 250_000
    big = csr_arrays(lens, 300_000, 22)
    assert len(big[0]) * 4 + 8 * int(big[0][-1]) >= 32 << 20  # A's bytes: four chunks of at least 8 MB
    *small, k_small = structure("power_law")
    cases = [(big, 300_000, 8, "merge"), (small, k_small, 64, "row_split"), (big, 300_000, 128, "auto_gb300"),
             (small, k_small, 13, "merge"), (big, 300_000, 32, "row_split")]
    Bs = [torch.from_numpy(gen.normal_matrix(k, n, 23 + i)).pin_memory() for i, (_, k, n, _) in enumerate(cases)]
    As = [tuple(torch.from_numpy(x).pin_memory() for x in a) for a, _, _, _ in cases]
    stream = torch.cuda.current_stream()
    results = []
    for round_ in range(2):
        Cs = [torch.full((len(a[0]) - 1, n), float("nan")).pin_memory() for a, _, n, _ in cases]
        seen = None
        for i, ((a, k, n, alg), (rp, ci, v)) in enumerate(zip(cases, As)):
            pkg.spmm_host(rp, ci, v, Bs[i], Cs[i], alg=alg, wait=False)
            if i == 1:  # queued after the call on the same stream: must see C
                seen = Cs[i].to("cuda", non_blocking=True)
        stream.synchronize()
        if round_ == 0:
            for (a, k, n, alg), B, C in zip(cases, Bs, Cs):
                check(C.numpy(), *a, B.numpy())
        assert torch.equal(seen.cpu(), Cs[1])
        results.append(Cs)
    for c0, c1 in zip(*results):
        assert torch.equal(c0, c1)


@pytest.mark.parametrize("alg", ["auto_gb300", "merge", "hybrid", "row_split"])
def test_host_multi_matches_single_calls(gpu_lib, alg):
    """spmm_csr_host_multi: several widths (one of them 0, one needing the scalar path, one
    large enough for column slabs) against one matrix of four row chunks, A uploaded once.
    Each C_i must equal the oracle and, bit for bit, what spmm_csr_host gives for that width
    alone (same blocks, same kernels); a second call through the same pool gives the same bits."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(31)
    lens = rng.integers(0, 40, 180_000)
    lens[1234] = 150_000
    a = csr_arrays(lens, 200_000, 32)
    k = 200_000
    widths = [8, 0, 13, 64, 128]
    rp, ci, v = (torch.from_numpy(x).pin_memory() for x in a)
    Bs = [torch.from_numpy(gen.normal_matrix(k, n, 40 + i)).pin_memory() for i, n in enumerate(widths)]
    runs = []
    for _ in range(2):
        Cs = [torch.full((len(a[0]) - 1, n), float("nan")).pin_memory() for n in widths]
        pkg.spmm_host_multi(rp, ci, v, Bs, Cs, alg=alg)
        torch.cuda.current_stream().synchronize()
        runs.append(Cs)
    for n, B, C0, C1 in zip(widths, Bs, *runs):
        if n == 0:
            continue
        check(C0.numpy(), *a, B.numpy())
        single = torch.empty_like(C0).pin_memory()
        pkg.spmm_host(rp, ci, v, B, single, alg=alg)
        assert torch.equal(C0, single), n
        assert torch.equal(C0, C1), n


def test_host_multi_16bit_and_empty(gpu_lib):
    """16-bit storage through the multi-product entry, and a call with no products."""
    import torch

    pkg = gpu_lib
    rp, ci, v, k = structure("power_law")
    vb = torch.from_numpy(v).to(torch.bfloat16).pin_memory()
    rpt, cit = torch.from_numpy(rp).pin_memory(), torch.from_numpy(ci).pin_memory()
    Bs = [torch.from_numpy(gen.normal_matrix(k, n, 50 + n)).to(torch.bfloat16).pin_memory() for n in (16, 48)]
    Cs = [torch.empty((len(rp) - 1, B.shape[1]), dtype=torch.bfloat16).pin_memory() for B in Bs]
    pkg.spmm_host_multi(rpt, cit, vb, Bs, Cs, alg="auto_gb300")
    torch.cuda.current_stream().synchronize()
    for B, C in zip(Bs, Cs):
        single = torch.empty_like(C).pin_memory()
        pkg.spmm_host(rpt, cit, vb, B, single, alg="auto_gb300")
        assert torch.equal(C, single)
    assert pkg.spmm_host_multi(rpt, cit, vb, [], []) == []


def test_host_calls_chained_through_host_memory(gpu_lib):
    """The C of an asynchronous host-buffer call is the B of the next call.  The
    synchronous entry orders its uploads after the work already queued on the
    stream, so it reads the finished C with no synchronisation in between (C
    starts as NaN: a stale read would show).  The asynchronous entry reads its
    inputs from call time on, so it is handed C after a synchronisation; both
    chains give the same bits."""
    import torch

    pkg = gpu_lib
    rng = np.random.default_rng(31)
    m1, k1, m2, n = 60_000, 40_000, 30_000, 64
    a1 = csr_arrays(rng.integers(0, 40, m1), k1, 32)
    a2 = csr_arrays(rng.integers(0, 40, m2), m1, 33)
    A1 = tuple(torch.from_numpy(x).pin_memory() for x in a1)
    A2 = tuple(torch.from_numpy(x).pin_memory() for x in a2)
    B1 = torch.from_numpy(gen.normal_matrix(k1, n, 34)).pin_memory()
    stream = torch.cuda.current_stream()
    outs = []
    for chain in ("sync_after_async", "async_after_sync"):
        C1 = torch.full((m1, n), float("nan")).pin_memory()
        C2 = torch.full((m2, n), float("nan")).pin_memory()
        pkg.spmm_host(*A1, B1, C1, alg="auto_gb300", wait=False)
        if chain == "sync_after_async":
            pkg.spmm_host(*A2, C1, C2, alg="auto_gb300", wait=True)
        else:
            stream.synchronize()
            pkg.spmm_host(*A2, C1, C2, alg="auto_gb300", wait=False)
            stream.synchronize()
        check(C1.numpy(), *a1, B1.numpy())
        check(C2.numpy(), *a2, C1.numpy())
        outs.append((C1, C2))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


def test_host_entry_few_long_rows(gpu_lib):
    """Three rows of two million nonzeros: at most as many chunks as rows."""
    import torch

    pkg = gpu_lib
    rp, ci, v = csr_arrays(np.array([2_000_000, 0, 2_000_000, 2_000_000]), 2_500_000, 14)
    B = gen.normal_matrix(2_500_000, 16, 15)
    for alg in ("row_split", "merge", "auto_gb300"):
        C = torch.empty((4, 16)).pin_memory()
        pkg.spmm_host(torch.from_numpy(rp), torch.from_numpy(ci), torch.from_numpy(v), torch.from_numpy(B), C, alg=alg)
        check(C.numpy(), rp, ci, v, B)


@pytest.mark.parametrize("n", [1, 8, 32, 64, 128, 300])
@pytest.mark.parametrize("long_row_len", [1, 7, 64, 1000])
def test_hybrid_integer_rows_across_the_threshold_are_bitwise(gpu_lib, n, long_row_len):
    """Hybrid row split: rows just below, at and above the long-row threshold,
    rows taken by one lane group (at and just above twice the threshold, where
    they move from the front to the back of the queue, and at and just above
    four times it, where they leave it), and rows of many segments (up to 40,000
    nonzeros, so with 512-nonzero segments up to 79 partial sums added by the
    row's last warp) on integer data, with blocks of 1, 37, 128 and 256 rows per
    warp: every partial sum is an exact integer, so the result must equal the
    oracle bit for bit whichever rows the row-block pass keeps and however a
    block's rows are split among its lane groups."""
    import torch

    rng = np.random.default_rng(100 + n)
    lens = rng.integers(0, 80, 6000)
    lens[::211] = long_row_len
    lens[1::211] = long_row_len + 1
    lens[2::211] = 2 * long_row_len
    lens[3::211] = 2 * long_row_len + 1
    lens[4::211] = 4 * long_row_len
    lens[6::211] = 4 * long_row_len + 1
    lens[::997] = 40_000
    lens[5] = 0
    rp, ci, v = csr_arrays(lens, 50_000, 21, int_vals=True)
    B = rng.integers(-4, 5, size=(50_000, n)).astype(np.float32)
    ref = oracle.spmm(rp, ci, v, B).astype(np.float32)
    for tuning in (dict(long_row_len=long_row_len), dict(long_row_len=long_row_len, column_slabs=3),
                   dict(long_row_len=long_row_len, lanes_per_row=1), dict(long_row_len=long_row_len, block_rows=1),
                   dict(long_row_len=long_row_len, block_rows=37, lanes_per_row=2),
                   dict(long_row_len=long_row_len, block_rows=256)):
        C = run(gpu_lib, torch, rp, ci, v, B, "hybrid", tuning=tuning)
        assert np.array_equal(C.cpu().numpy(), ref), tuning


def test_hybrid_is_deterministic_and_reuses_its_workspace(gpu_lib):
    """The partial sums of a row are added in segment order by whichever warp
    finishes last: two runs through one caller workspace give the same bits,
    and the second run is not disturbed by the first run's queue and counters."""
    import torch

    rp, ci, v, k = structure("giant_row")
    B = gen.normal_matrix(k, 64, 9)
    nnz = int(rp[-1])
    ws_bytes = gpu_lib.workspace_size(len(rp) - 1, k, 64, nnz, alg="hybrid")
    assert ws_bytes > 0
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    ws.fill_(0xA5)  # stale contents must not matter
    outs = []
    for _ in range(3):
        C = run(gpu_lib, torch, rp, ci, v, B, "hybrid", workspace=ws)
        outs.append(C.cpu().numpy())
    check(outs[0], rp, ci, v, B)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_hybrid_rejects_a_short_workspace(gpu_lib):
    """The reported size covers every access width the call may pick (it is the
    largest of their layouts); a quarter of it is short for all of them."""
    import torch

    rp, ci, v, k = structure("power_law")
    B = gen.normal_matrix(k, 32, 1)
    need = gpu_lib.workspace_size(len(rp) - 1, k, 32, int(rp[-1]), alg="hybrid")
    ws = torch.empty(need // 4 // 256 * 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(gpu_lib.SpMMError):
        run(gpu_lib, torch, rp, ci, v, B, "hybrid", workspace=ws)


@pytest.mark.parametrize("lanes", [2, 4])
def test_hybrid_reports_an_understated_nonzero_count(gpu_lib, lanes):
    """The hybrid's queues are sized from the nnz the caller passes.  With a
    quarter of the true count, the 800 queued rows of 40 and 100 nonzeros
    overflow the mid queue (capacity nnz / 33 + 1 = 434): with 2-lane groups the
    row-block pass runs past its end; with 4-lane groups the rows of 40 fill it
    from the front and those of 100 from the back, the two ends meet inside it,
    and the segment pass finds that.  Either way the call reports
    SPMM_ERR_BAD_CSR on the status word; every queue write is bounds-checked."""
    import torch

    lens = np.array([40, 100, 3] * 400, dtype=np.int64)
    rp, ci, v = csr_arrays(lens, 5_000, 31)
    B = gen.normal_matrix(5_000, 32, 32)
    d_rp, d_ci, d_v, d_B = to_dev(torch, rp, ci, v, B)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    gpu_lib.spmm(d_rp, d_ci, d_v, d_B, alg="hybrid", nnz=int(rp[-1]) // 4, status=status,
                 tuning={"lanes_per_row": lanes})
    torch.cuda.synchronize()
    assert int(status.item()) == gpu_lib.ERR_BAD_CSR
    # with the true count the same call is exact
    status.zero_()
    C = gpu_lib.spmm(d_rp, d_ci, d_v, d_B, alg="hybrid", nnz=int(rp[-1]), status=status,
                     tuning={"lanes_per_row": lanes})
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    check(C.cpu().numpy(), rp, ci, v, B)
