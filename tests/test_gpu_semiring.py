"""GPU parity of the semiring SpMM C = A (+).(x) B (the GraphBLAS product that
Section 1 names as a use of SpMM) with the FP64 oracle, through the C ABI.

(min,+), (max,+) and (max,x) results are compared bit for bit with the
oracle's result rounded to float32.  That is exact, not a tolerance: each term
val (x) b is one correctly rounded float32 operation on float32 inputs, whose
FP64 value the oracle computes exactly (a product of two floats fits in a
double; the sum of two floats does whenever their exponents differ by less
than 29, which holds for these inputs up to a probability far below one in a
billion per term), and rounding to float32 is monotone, so it commutes with
min and max.  min and max are exact and order-free, so neither the row split
nor the merge-path decomposition and its fix-up may change a single bit.
"""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import FP32_TOL, STRUCTURES, check, csr_arrays, structure

pytestmark = pytest.mark.gpu

SEMIRINGS = ["min_plus", "max_plus", "max_times"]


def to_dev(torch, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrays]


def run(pkg, torch, rp, ci, v, B, semiring, alg, **kw):
    d_rp, d_ci, d_v, d_B = to_dev(torch, rp, ci, v, B)
    C = pkg.semiring_spmm(d_rp, d_ci, d_v, d_B, semiring, alg=alg, nnz=int(rp[-1]), **kw)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def expect_exact(C, rp, ci, v, B, semiring):
    ref = oracle.spmm_semiring(rp, ci, v, B, semiring).astype(np.float32)
    bad = np.argwhere(C != ref)
    assert bad.size == 0, f"{len(bad)} elements differ, first {tuple(bad[0])}: {C[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


@pytest.mark.parametrize("name", STRUCTURES)
@pytest.mark.parametrize("alg", ["row_split", "merge", "hybrid"])
@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("n", [1, 8, 13, 128])
def test_structures_bitwise(gpu_lib, name, alg, semiring, n):
    import torch

    rp, ci, v, k = structure(name)
    B = gen.normal_matrix(k, n, 21 + n)
    expect_exact(run(gpu_lib, torch, rp, ci, v, B, semiring, alg), rp, ci, v, B, semiring)


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("alg", ["auto", "auto_gb300"])
def test_selectors(gpu_lib, semiring, alg):
    import torch

    for name in ("power_law", "short_rows", "uniform16"):
        rp, ci, v, k = structure(name, seed=1)
        B = gen.normal_matrix(k, 64, 2)
        expect_exact(run(gpu_lib, torch, rp, ci, v, B, semiring, alg), rp, ci, v, B, semiring)


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("alg", ["row_split", "merge", "hybrid"])
@pytest.mark.parametrize("tuning", [dict(lanes_per_row=1), dict(lanes_per_row=32), dict(column_slabs=4),
                                    dict(items_per_subwarp=4), dict(items_per_subwarp=37),
                                    dict(items_per_subwarp=700), dict(lanes_per_row=2, items_per_subwarp=5)])
def test_launch_shapes_bitwise(gpu_lib, semiring, alg, tuning):
    """Tiles of 4 to 700 items per lane group move the merge-path cuts, and
    so which rows are split and finished by the fix-up."""
    import torch

    rng = np.random.default_rng(3)
    lens = rng.integers(0, 200, 4000)
    lens[::113] = 20_000
    rp, ci, v = csr_arrays(lens, 25_000, 7)
    B = gen.normal_matrix(25_000, 64, 9)
    expect_exact(run(gpu_lib, torch, rp, ci, v, B, semiring, alg, tuning=tuning), rp, ci, v, B, semiring)


@pytest.mark.parametrize("alg", ["row_split", "merge", "auto"])
def test_plus_times_is_the_ordinary_product(gpu_lib, alg):
    import torch

    rp, ci, v, k = structure("power_law")
    B = gen.normal_matrix(k, 64, 4)
    C = run(gpu_lib, torch, rp, ci, v, B, "plus_times", alg)
    check(C, rp, ci, v, B, tol=FP32_TOL)


def test_empty_rows_give_the_identity(gpu_lib):
    import torch

    rp, ci, v, k = structure("alternating_empty")
    B = gen.normal_matrix(k, 32, 5)
    empty = np.diff(rp) == 0
    for semiring, ident in (("min_plus", np.inf), ("max_plus", -np.inf), ("max_times", -np.inf)):
        for alg in ("row_split", "merge", "hybrid"):
            C = run(gpu_lib, torch, rp, ci, v, B, semiring, alg)
            assert np.all(C[empty] == ident)
            assert np.all(np.isfinite(C[~empty]))


@pytest.mark.parametrize("alg", ["row_split", "merge"])
def test_min_plus_relaxation_gives_shortest_paths(gpu_lib, alg):
    """Repeated (min,+) products D <- A (min.+) D, with A[i][j] the weight of
    edge j -> i and a zero diagonal, converge to single-source shortest-path
    distances for every source column; scipy's Dijkstra is the independent
    check.  Integer weights keep every float32 sum exact."""
    import torch
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")

    rng = np.random.default_rng(11)
    V, E, S = 3000, 24_000, 16
    src, dst = rng.integers(0, V, E), rng.integers(0, V, E)
    w = rng.integers(1, 20, E).astype(np.float64)
    keep = src != dst
    src, dst, w = src[keep], dst[keep], w[keep]
    # parallel edges: keep the lightest (csgraph would sum duplicates)
    order = np.lexsort((w, dst, src))
    src, dst, w = src[order], dst[order], w[order]
    first = np.ones(len(src), dtype=bool)
    first[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
    src, dst, w = src[first], dst[first], w[first]
    W = sp.csr_matrix((w, (src, dst)), shape=(V, V))  # W[s][d]: edge s -> d
    # A: row i lists the edges into i, plus a zero diagonal
    A = sp.csr_matrix((np.concatenate([w, np.zeros(V)]),
                       (np.concatenate([dst, np.arange(V)]), np.concatenate([src, np.arange(V)]))), shape=(V, V))
    A.sort_indices()
    assert A.nnz == len(w) + V
    rp, ci, v = A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float32)
    sources = rng.choice(V, S, replace=False)
    D = np.full((V, S), np.inf, dtype=np.float32)
    D[sources, np.arange(S)] = 0.0
    d_rp, d_ci, d_v = to_dev(torch, rp, ci, v)
    d_D = torch.from_numpy(D).cuda()
    for _ in range(V):
        nxt = gpu_lib.semiring_spmm(d_rp, d_ci, d_v, d_D, "min_plus", alg=alg, nnz=A.nnz)
        if torch.equal(nxt, d_D):
            break
        d_D = nxt
    got = d_D.cpu().numpy()
    ref = csgraph.dijkstra(W, directed=True, indices=sources)  # [S, V]
    assert np.array_equal(got, ref.T.astype(np.float32))


def test_invalid_semiring_is_rejected(gpu_lib):
    import torch

    rp, ci, v, k = structure("uniform16")
    B = gen.normal_matrix(k, 8, 1)
    with pytest.raises(gpu_lib.SpMMError):
        run(gpu_lib, torch, rp, ci, v, B, 7, "merge")
    with pytest.raises(TypeError):
        gpu_lib.semiring_spmm(*to_dev(torch, rp, ci, v), torch.zeros((k, 8), dtype=torch.bfloat16, device="cuda"),
                              "min_plus")
