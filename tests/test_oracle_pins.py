"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it does not share code with:
dense float64 GEMM (a library routine), exact integer arithmetic, closed forms
(identity, permutation, row sums), the paper's printed constants and a
hand-written merge-path walk (tests/golden/), the closed-form characterisation
of a merge-path point, torch float64 autograd, and central finite differences.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from conftest import GOLDEN


# ----------------------------------------------------------------------------- small inputs

def random_csr(rng, m, k, density=0.3, duplicates=False, unsorted=False, empty_every=0, int_vals=False):
    rows_cols, vals = [], []
    row_ptr = [0]
    for i in range(m):
        if empty_every and i % empty_every == 1:
            row_ptr.append(row_ptr[-1])
            continue
        cnt = int(rng.binomial(k, density))
        cols = list(rng.choice(k, size=cnt, replace=False)) if cnt else []
        if duplicates and cols:
            cols += list(rng.choice(cols, size=int(rng.integers(1, 3))))
        if not unsorted:
            cols.sort()
        else:
            rng.shuffle(cols)
        rows_cols += cols
        if int_vals:
            vals += list(rng.integers(-2, 3, size=len(cols)).astype(np.float64))
        else:
            vals += list(rng.uniform(-1, 1, size=len(cols)))
        row_ptr.append(row_ptr[-1] + len(cols))
    return (np.asarray(row_ptr, np.int32), np.asarray(rows_cols, np.int32),
            np.asarray(vals, np.float64))


def to_dense(row_ptr, col_ind, vals, m, k):
    d = np.zeros((m, k))
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    np.add.at(d, (rows, col_ind), vals)  # duplicates summed
    return d


CASES = [
    dict(m=7, k=13, n=5),
    dict(m=16, k=9, n=33, duplicates=True),
    dict(m=31, k=40, n=8, unsorted=True, duplicates=True),
    dict(m=24, k=24, n=1, empty_every=3),
    dict(m=1, k=50, n=17, density=0.9),
    dict(m=40, k=1, n=4, density=0.5),
]


@pytest.mark.parametrize("case", CASES)
def test_spmm_matches_dense_gemm(case):
    rng = np.random.default_rng(hash(str(case)) % 2**32)
    case = dict(case)
    m, k, n = case.pop("m"), case.pop("k"), case.pop("n")
    rp, ci, v = random_csr(rng, m, k, **case)
    B = rng.standard_normal((k, n))
    C = oracle.spmm(rp, ci, v, B)
    ref = to_dense(rp, ci, v, m, k) @ B
    assert C.shape == (m, n)
    np.testing.assert_allclose(C, ref, rtol=1e-12, atol=1e-12)


def test_identity_is_exact():
    m, n = 257, 19
    rng = np.random.default_rng(1)
    B = rng.standard_normal((m, n))
    rp = np.arange(m + 1, dtype=np.int32)
    C = oracle.spmm(rp, np.arange(m, dtype=np.int32), np.ones(m), B)
    assert np.array_equal(C, B)


def test_permutation_is_exact():
    m, n = 300, 7
    rng = np.random.default_rng(2)
    perm = rng.permutation(m).astype(np.int32)
    B = rng.standard_normal((m, n))
    C = oracle.spmm(np.arange(m + 1, dtype=np.int32), perm, np.ones(m), B)
    assert np.array_equal(C, B[perm])
    # A^T of a permutation applies the inverse permutation
    inv = np.argsort(perm)
    assert np.array_equal(oracle.spmm_t(np.arange(m + 1, dtype=np.int32), perm, np.ones(m), B, m), B[inv])


def test_ones_gives_row_sums():
    rng = np.random.default_rng(3)
    m, k, n = 50, 60, 6
    rp, ci, v = random_csr(rng, m, k, duplicates=True, empty_every=4)
    C = oracle.spmm(rp, ci, v, np.ones((k, n)))
    rows = np.repeat(np.arange(m), np.diff(rp))
    sums = np.bincount(rows, weights=v, minlength=m)
    for j in range(n):
        np.testing.assert_allclose(C[:, j], sums, rtol=1e-13, atol=1e-13)


def test_exact_integer_arithmetic():
    rng = np.random.default_rng(4)
    m, k, n = 64, 80, 24
    rp, ci, v = random_csr(rng, m, k, density=0.6, duplicates=True, int_vals=True)
    B = rng.integers(-4, 5, size=(k, n))
    dense = np.zeros((m, k), dtype=np.int64)
    rows = np.repeat(np.arange(m), np.diff(rp))
    np.add.at(dense, (rows, ci), v.astype(np.int64))
    assert np.array_equal(oracle.spmm(rp, ci, v, B.astype(np.float64)), (dense @ B).astype(np.float64))


def test_rows_subset_and_abs_bound():
    rng = np.random.default_rng(5)
    m, k, n = 45, 30, 9
    rp, ci, v = random_csr(rng, m, k, duplicates=True)
    B = rng.standard_normal((k, n))
    rows = np.array([44, 0, 17, 17, 3])
    np.testing.assert_array_equal(oracle.spmm_rows(rows, rp, ci, v, B), oracle.spmm(rp, ci, v, B)[rows])
    D = oracle.abs_bound_rows(rows, rp, ci, v, B)
    # the scale sums |val| over stored entries (duplicates are separate terms of the sum)
    np.testing.assert_allclose(D, (to_dense(rp, ci, np.abs(v), m, k) @ np.abs(B))[rows], rtol=1e-12, atol=1e-12)


def test_normalized_error_semantics():
    D = np.array([[1.0, 0.0], [2.0, 4.0]])
    ref = np.array([[1.0, 0.0], [1.0, -1.0]])
    assert oracle.normalized_error(ref, ref, D) == 0.0
    C = ref + np.array([[1e-3, 0.0], [0.0, 4e-3]])
    assert oracle.normalized_error(C, ref, D) == pytest.approx(1e-3)
    C2 = ref.copy()
    C2[0, 1] = 1e-30  # a nonzero where no term contributes
    assert oracle.normalized_error(C2, ref, D) == float("inf")
    C3 = ref.copy()
    C3[1, 0] = np.nan
    assert oracle.normalized_error(C3, ref, D) == float("inf")
    # an absolute floor forgives differences up to it, and no more
    assert oracle.normalized_error(C, ref, D, abs_floor=1e-3) == pytest.approx(0.75e-3)
    assert oracle.normalized_error(C, ref, D, abs_floor=1.0) == 0.0
    assert oracle.normalized_error(C2, ref, D, abs_floor=1.0) == float("inf")


def test_thread_count_does_not_change_results():
    a = gen.power_law(20_000, 20_000, 11, cap=3000)
    B = gen.normal_matrix(a.k, 16, 11)
    old = oracle.num_threads()
    try:
        oracle.set_threads(1)
        c1 = oracle.spmm(a.row_ptr, a.col_ind, a.vals, B)
        t1 = oracle.spmm_t(a.row_ptr, a.col_ind, a.vals, B[: a.m], a.k)
        oracle.set_threads(4)
        c4 = oracle.spmm(a.row_ptr, a.col_ind, a.vals, B)
        t4 = oracle.spmm_t(a.row_ptr, a.col_ind, a.vals, B[: a.m], a.k)
    finally:
        oracle.set_threads(old)
    assert np.array_equal(c1, c4)
    assert np.array_equal(t1, t4)


# ----------------------------------------------------------------------------- Section 5.4 heuristic

def test_heuristic_threshold_from_paper(paper_constants):
    assert oracle.HEURISTIC_THRESHOLD == paper_constants["heuristic_threshold"]
    # d = nnz / m just below, at, and above 9.35
    assert oracle.select_alg(100, 934) == oracle.ALG_MERGE
    assert oracle.select_alg(100, 936) == oracle.ALG_ROW_SPLIT
    assert oracle.select_alg(20, 187) == oracle.ALG_ROW_SPLIT  # exactly 9.35: not below
    assert oracle.select_alg(1, 0) == oracle.ALG_MERGE
    assert oracle.select_alg(0, 0) == oracle.ALG_ROW_SPLIT
    # the mean row length is nnz / m, not nnz / n: a matrix with long rows but a
    # narrow B still goes to row split
    assert oracle.select_alg(1000, 16_000) == oracle.ALG_ROW_SPLIT


# ----------------------------------------------------------------------------- Section 4 merge path

def read_walk_fixture():
    with open(os.path.join(GOLDEN, "merge_path_example.txt")) as f:
        lines = [l.split() for l in f if l.strip() and not l.startswith("#")]
    row_ptr = np.array([int(x) for x in lines[0][1:]], dtype=np.int32)
    walk = np.array([[int(x) for x in l] for l in lines[1:]])
    return row_ptr, walk


def test_merge_path_hand_walk():
    row_ptr, walk = read_walk_fixture()
    lim = oracle.merge_path_limits(row_ptr, 1)  # a split after every item = the whole walk
    assert np.array_equal(lim, walk[:, 1:])
    assert np.array_equal(walk[:, 0], walk[:, 1] + walk[:, 2])


def on_path(row_ptr, r, z):
    """Closed form: (r, z) lies on the merge path iff the r-th consumed row end is not
    after nonzero z (row_ptr[r] <= z) and nonzero z-1 came before row r's end
    (row_ptr[r+1] >= z)."""
    m = len(row_ptr) - 1
    nnz = row_ptr[-1]
    if not (0 <= r <= m and 0 <= z <= nnz):
        return False
    if r > 0 and row_ptr[r] > z:
        return False
    if r < m and z > 0 and row_ptr[r + 1] < z:
        return False
    return True


@pytest.mark.parametrize("seed", range(6))
def test_merge_path_matches_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(1, 40))
    lengths = rng.integers(0, 6, size=m) * (rng.random(m) < 0.7)
    if seed == 0:
        lengths[:] = 0  # all rows empty
    if seed == 1:
        lengths[m // 2] = 50  # one long row
    row_ptr = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int32)
    nnz = int(row_ptr[-1])
    for items in (1, 2, 3, 7, 32):
        lim = oracle.merge_path_limits(row_ptr, items)
        tiles = -(-(m + nnz) // items)
        assert lim.shape == (tiles + 1, 2)
        assert tuple(lim[-1]) == (m, nnz)
        for t, (r, z) in enumerate(lim):
            d = min(t * items, m + nnz)
            assert r + z == d
            # exactly one point of the diagonal satisfies the closed form, and it is the oracle's
            pts = [rr for rr in range(0, d + 1) if on_path(row_ptr, rr, d - rr)]
            assert pts == [r]
        assert np.all(np.diff(lim[:, 0]) >= 0) and np.all(np.diff(lim[:, 1]) >= 0)
        # every nonzero is covered by exactly one tile; every row end lies in exactly one tile
        assert np.sum(np.diff(lim[:, 1])) == nnz and np.sum(np.diff(lim[:, 0])) == m


def test_merge_path_equal_shares():
    row_ptr = np.concatenate([[0], np.cumsum(np.r_[np.zeros(100, int), [1000], np.ones(50, int)])]).astype(np.int32)
    lim = oracle.merge_path_limits(row_ptr, 64)
    items = lim.sum(axis=1)
    assert np.all(np.diff(items)[:-1] == 64)  # every tile but the last holds exactly 64 items


# ----------------------------------------------------------------------------- backward operations

@pytest.mark.parametrize("case", CASES[:4])
def test_backward_matches_dense_autograd(case):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7 + hash(str(case)) % 1000)
    case = dict(case)
    m, k, n = case.pop("m"), case.pop("k"), case.pop("n")
    rp, ci, v = random_csr(rng, m, k, **case)
    B = rng.standard_normal((k, n))
    G = rng.standard_normal((m, n))
    # dense float64 autograd of L = <G, dense(A) B>
    rows = np.repeat(np.arange(m), np.diff(rp))
    vt = torch.tensor(v, dtype=torch.float64, requires_grad=True)
    Bt = torch.tensor(B, dtype=torch.float64, requires_grad=True)
    dense = torch.zeros((m, k), dtype=torch.float64).index_put(
        (torch.tensor(rows, dtype=torch.long), torch.tensor(ci, dtype=torch.long)), vt, accumulate=True)
    L = (torch.tensor(G) * (dense @ Bt)).sum()
    L.backward()
    np.testing.assert_allclose(oracle.sddmm(rp, ci, G, B), vt.grad.numpy(), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.spmm_t(rp, ci, v, G, k), Bt.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_backward_central_differences():
    a = gen.chung_lu_gcn(64, 5, mean_degree=6.0)
    n = 8
    rng = np.random.default_rng(9)
    B = rng.standard_normal((a.k, n))
    G = rng.standard_normal((a.m, n))
    v = a.vals.astype(np.float64)

    def loss(vals, Bm):
        return float(np.sum(G * oracle.spmm(a.row_ptr, a.col_ind, vals, Bm)))

    h = 0.5  # L is bilinear: the central difference is exact up to rounding for any h
    dv = oracle.sddmm(a.row_ptr, a.col_ind, G, B)
    for p in rng.choice(a.nnz, size=40, replace=False):
        e = np.zeros_like(v)
        e[p] = h
        fd = (loss(v + e, B) - loss(v - e, B)) / (2 * h)
        assert abs(fd - dv[p]) <= 1e-11 * max(1.0, abs(dv[p]))
    dB = oracle.spmm_t(a.row_ptr, a.col_ind, v, G, a.k)
    for _ in range(40):
        i, j = int(rng.integers(a.k)), int(rng.integers(n))
        e = np.zeros_like(B)
        e[i, j] = h
        fd = (loss(v, B + e) - loss(v, B - e)) / (2 * h)
        assert abs(fd - dB[i, j]) <= 1e-11 * max(1.0, abs(dB[i, j]))


def test_sddmm_abs_bound():
    rng = np.random.default_rng(12)
    rp, ci, v = random_csr(rng, 20, 25, duplicates=True)
    B = rng.standard_normal((25, 6))
    G = rng.standard_normal((20, 6))
    rows = np.repeat(np.arange(20), np.diff(rp))
    ref = np.einsum("pj,pj->p", np.abs(G[rows]), np.abs(B[ci]))
    np.testing.assert_allclose(oracle.sddmm_abs_bound(rp, ci, G, B), ref, rtol=1e-12)


@pytest.mark.parametrize("dups", [False, True])
def test_transpose(dups):
    rng = np.random.default_rng(13 + dups)
    m, k = 37, 29
    rp, ci, v = random_csr(rng, m, k, duplicates=dups, empty_every=5)
    rpt, cit, perm = oracle.csr_transpose(rp, ci, k)
    assert rpt.shape == (k + 1,) and rpt[0] == 0 and rpt[-1] == len(ci)
    np.testing.assert_array_equal(to_dense(rpt, cit, v[perm], k, m), to_dense(rp, ci, v, m, k).T)
    # stable: within each row of A^T the original positions increase
    for c in range(k):
        seg = perm[rpt[c]:rpt[c + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(ci[seg] == c)
    # the transpose of the transpose restores A (A's columns are sorted per row)
    rp2, ci2, perm2 = oracle.csr_transpose(rpt, cit, m)
    np.testing.assert_array_equal(rp2, rp)
    np.testing.assert_array_equal(ci2, ci)
    np.testing.assert_array_equal(perm[perm2], np.arange(len(ci)))


# ----------------------------------------------------------------------------- number formats

def test_bf16_widening_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(14)
    x = np.concatenate([rng.standard_normal(5000).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, -2.5, 3.0e38, 1e-40], np.float32)])
    bits = gen.to_bf16_bits(x)
    ref = torch.from_numpy(bits.view(np.int16)).view(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(oracle.bf16_bits_to_f64(bits), ref)
    # the bfloat16 rounding of float32 is to nearest, so the error is at most half a unit in the last place
    rel = np.abs(oracle.bf16_bits_to_f64(bits[:5000]) - x[:5000]) / np.abs(x[:5000])
    assert rel.max() <= 2.0 ** -8


# ----------------------------------------------------------------------------- semirings

def _masked(rp, ci, v, m, k, fill):
    """Dense m x k copy of A with `fill` where nothing is stored (no duplicates)."""
    d = np.full((m, k), fill)
    d[np.repeat(np.arange(m), np.diff(rp)), ci] = v
    return d


def test_semiring_min_plus_against_numpy_broadcast():
    rng = np.random.default_rng(31)
    m, k, n = 17, 23, 9
    rp, ci, v = random_csr(rng, m, k)
    B = rng.standard_normal((k, n))
    ref = np.min(_masked(rp, ci, v, m, k, np.inf)[:, :, None] + B[None, :, :], axis=1)
    np.testing.assert_array_equal(oracle.spmm_semiring(rp, ci, v, B, "min_plus"), ref)
    ref = np.max(_masked(rp, ci, v, m, k, -np.inf)[:, :, None] + B[None, :, :], axis=1)
    np.testing.assert_array_equal(oracle.spmm_semiring(rp, ci, v, B, "max_plus"), ref)
    np.testing.assert_allclose(oracle.spmm_semiring(rp, ci, v, B, "plus_times"), oracle.spmm(rp, ci, v, B), rtol=0,
                               atol=0)


def test_semiring_closed_forms():
    rng = np.random.default_rng(32)
    m, n = 40, 7
    B = rng.standard_normal((m, n))
    ident = np.arange(m + 1, dtype=np.int32)
    # (min,+) with the (min,+) identity matrix (zeros on the diagonal): C = B
    assert np.array_equal(oracle.spmm_semiring(ident, np.arange(m, dtype=np.int32), np.zeros(m), B, "min_plus"), B)
    # (max,x) with B = ones: the row maxima of A; empty rows give -inf
    rp, ci, v = random_csr(rng, m, 30, empty_every=4)
    C = oracle.spmm_semiring(rp, ci, v, np.ones((30, n)), "max_times")
    for i in range(m):
        seg = v[rp[i]:rp[i + 1]]
        assert np.all(C[i] == (seg.max() if seg.size else -np.inf))
    # one relaxation step of shortest paths on a path graph 0 -> 1 -> 2 -> 3 (edge weight 1):
    # D1 = A (min,+) D0 with D0 the distances from node 3 reached in at most 0 hops
    rp = np.array([0, 1, 2, 3, 3], np.int32)
    ci = np.array([1, 2, 3], np.int32)
    w = np.ones(3)
    D0 = np.array([[np.inf], [np.inf], [np.inf], [0.0]])
    D1 = np.minimum(D0, oracle.spmm_semiring(rp, ci, w, D0, "min_plus"))
    D2 = np.minimum(D1, oracle.spmm_semiring(rp, ci, w, D1, "min_plus"))
    D3 = np.minimum(D2, oracle.spmm_semiring(rp, ci, w, D2, "min_plus"))
    assert D3[:, 0].tolist() == [3.0, 2.0, 1.0, 0.0]
