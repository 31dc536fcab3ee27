"""The seeded generators produce the workload shapes they promise."""
import numpy as np

import gen


def _rows_sorted_distinct(a):
    rows = np.repeat(np.arange(a.m, dtype=np.int64), a.row_lengths())
    key = rows * a.k + a.col_ind
    return bool(np.all(np.diff(key) > 0)) and a.col_ind.min(initial=0) >= 0 and a.col_ind.max(initial=0) < a.k


def test_uniform_rows():
    a = gen.uniform_rows(1000, 500, 16, 3)
    assert a.nnz == 16_000 and np.all(a.row_lengths() == 16)
    assert _rows_sorted_distinct(a)
    assert a.vals.dtype == np.float32 and a.vals.min() >= -1 and a.vals.max() < 1
    # dense rows use the selection sampler
    d = gen.uniform_rows(10, 20, 20, 4)
    assert np.array_equal(d.col_ind.reshape(10, 20), np.tile(np.arange(20), (10, 1)))


def test_deterministic():
    a1, a2 = gen.uniform_rows(300, 300, 9, 7), gen.uniform_rows(300, 300, 9, 7)
    assert np.array_equal(a1.col_ind, a2.col_ind) and np.array_equal(a1.vals, a2.vals)
    assert np.array_equal(gen.normal_matrix(33, 5, 1), gen.normal_matrix(33, 5, 1))
    assert not np.array_equal(gen.normal_matrix(33, 5, 1), gen.normal_matrix(33, 5, 2))


def test_power_law_shape():
    a = gen.power_law(200_000, 200_000, 5, cap=20_000)
    lengths = a.row_lengths()
    nonempty = lengths[lengths > 0]
    assert abs(nonempty.mean() - 16.0) < 0.5
    assert (lengths == 0).sum() == 2000
    assert lengths.max() <= 20_000 and nonempty.min() >= 1
    assert _rows_sorted_distinct(a)
    # heavy tail: the longest rows are orders of magnitude above the mean
    assert lengths.max() > 100 * 16


def test_normal_moments():
    b = gen.normal_matrix(1000, 100, 9)
    assert abs(b.mean()) < 0.01 and abs(b.std() - 1.0) < 0.01


def test_chung_lu_gcn():
    a = gen.chung_lu_gcn(2000, 6, mean_degree=10.0)
    assert _rows_sorted_distinct(a)
    rows = np.repeat(np.arange(a.m), a.row_lengths())
    key = set(zip(rows.tolist(), a.col_ind.tolist()))
    assert all((j, i) in key for i, j in key)  # symmetric pattern
    assert all((i, i) in key for i in range(a.m))  # identity added
    deg = a.row_lengths().astype(np.float64)
    np.testing.assert_allclose(a.vals, 1.0 / np.sqrt(deg[rows] * deg[a.col_ind]), rtol=1e-6)


def test_batched_set_small():
    s = gen.batched_set(20, 3, m_hi=2000)
    assert len(s.mats) == 20 and len(s.ns) == 20
    assert set(s.ns) <= {32, 64, 128}
    for a in s.mats:
        assert 64 <= a.m <= 2000 and a.m == a.k
        assert _rows_sorted_distinct(a)
