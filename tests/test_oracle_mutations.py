"""Mistakes planted in a copy of the oracle are caught by its pins.

Each case compiles spmm_oracle.c with one plausible mistake (a dropped term,
a flipped sign, a wrong operand, a flipped merge tie rule, an unstable
transpose, ...), swaps it in for the real oracle library, and checks that at
least one of the independent pin checks below fails.  Everything runs on the
CPU; no mutant reads out of bounds.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "spmm_oracle.c")


def _in_function(src, func, old, new):
    """Replace the first `old` after the definition of `func`."""
    i = src.index(func)
    j = src.index(old, i)
    return src[:j] + new + src[j + len(old):]


MUTANTS = {
    "spmm drops each row's last term": ("void oracle_spmm_f64(", "p < row_ptr[i + 1]; ++p", "p < row_ptr[i + 1] - 1; ++p"),
    "spmm subtracts": ("void oracle_spmm_f64(", "c[j] += a * b[j]", "c[j] -= a * b[j]"),
    "spmm gathers row i of B instead of row col_ind[p]": (
        "void oracle_spmm_f64(", "B + (int64_t)col_ind[p] * ldb", "B + (int64_t)(i % 1) * ldb"),
    "spmm_rows ignores the value": ("void oracle_spmm_rows_f64(", "c[j] += a * b[j]", "c[j] += b[j]"),
    "abs bound keeps the sign of the value": ("void oracle_absbound_rows_f64(", "fabs(val[p])", "(val[p])"),
    "spmm_t drops the value": ("void oracle_spmm_t_f64(", "d[j] += a * g[j]", "d[j] += g[j]"),
    "sddmm squares dC": ("void oracle_sddmm_f64(", "s += g[j] * b[j]", "s += g[j] * g[j]"),
    "transpose walks rows backwards (unstable)": (
        "void oracle_csr_transpose(", "for (int64_t i = 0; i < m; ++i)", "for (int64_t i = m - 1; i >= 0; --i)"),
    "merge walk takes the nonzero first on ties": (
        "void oracle_merge_path_limits(", "row_ptr[r + 1] <= z", "row_ptr[r + 1] < z"),
    "(min,+) starts from 0 instead of +inf": (
        "void oracle_spmm_semiring_f64(", "semiring == 1 ? INFINITY", "semiring == 1 ? 0.0"),
    "(max,x) multiplies into a sum": ("void oracle_spmm_semiring_f64(", "c[j] = fmax(c[j], a * b[j])", "c[j] += a * b[j]"),
}


def _build_mutant(tmp, name, func, old, new):
    src = open(SRC).read()
    mutated = _in_function(src, func, old, new)
    assert mutated != src, name
    path_c = os.path.join(tmp, "mutant.c")
    with open(path_c, "w") as f:
        f.write(mutated)
    path_so = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", path_c, "-o", path_so, "-lm"], check=True,
                   capture_output=True)
    return oracle._bind(ctypes.CDLL(path_so))


# ----------------------------------------------------------------------------- pin checks (no oracle code)

def _random_csr(rng, m, k, dup=True):
    """Random small CSR with empty rows and (optionally) one repeated column per row."""
    cols, vals, row_ptr = [], [], [0]
    for L in rng.integers(0, 6, m):
        c = sorted(rng.choice(k, size=min(int(L), k), replace=False).tolist())
        if dup and c:
            c.append(c[-1])
        cols += c
        vals += list(rng.uniform(-1, 1, len(c)))
        row_ptr.append(len(cols))
    return np.array(row_ptr, np.int32), np.array(cols, np.int32), np.array(vals)


def _dense(rp, ci, v, m, k):
    d = np.zeros((m, k))
    np.add.at(d, (np.repeat(np.arange(m), np.diff(rp)), ci), v)
    return d


def check_products(rng):
    m, k, n = 23, 17, 6
    rp, ci, v = _random_csr(rng, m, k)
    B = rng.standard_normal((k, n))
    G = rng.standard_normal((m, n))
    dense = _dense(rp, ci, v, m, k)
    np.testing.assert_allclose(oracle.spmm(rp, ci, v, B), dense @ B, atol=1e-12)
    rows = np.arange(m)
    np.testing.assert_allclose(oracle.spmm_rows(rows, rp, ci, v, B), dense @ B, atol=1e-12)
    np.testing.assert_allclose(oracle.abs_bound_rows(rows, rp, ci, v, B), _dense(rp, ci, np.abs(v), m, k) @ np.abs(B),
                               atol=1e-12)
    np.testing.assert_allclose(oracle.spmm_t(rp, ci, v, G, k), dense.T @ G, atol=1e-12)
    r = np.repeat(np.arange(m), np.diff(rp))
    np.testing.assert_allclose(oracle.sddmm(rp, ci, G, B), np.einsum("pj,pj->p", G[r], B[ci]), atol=1e-12)


def check_transpose(rng):
    m, k = 19, 11
    rp, ci, v = _random_csr(rng, m, k)
    rpt, cit, perm = oracle.csr_transpose(rp, ci, k)
    np.testing.assert_allclose(_dense(rpt, cit, v[perm], k, m), _dense(rp, ci, v, m, k).T, atol=0)
    for c in range(k):
        assert np.all(np.diff(perm[rpt[c]:rpt[c + 1]]) > 0)


def check_merge_path(rng):
    lens = rng.integers(0, 4, 15)
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    m, nnz = 15, int(rp[-1])
    lim = oracle.merge_path_limits(rp, 1)
    for r, z in lim:
        assert (r == 0 or rp[r] <= z) and (r == m or z == 0 or rp[r + 1] >= z)


def check_semirings(rng):
    m, k, n = 13, 9, 4
    rp, ci, v = _random_csr(rng, m, k, dup=False)
    B = rng.standard_normal((k, n))
    full = np.full((m, k), np.inf)
    full[np.repeat(np.arange(m), np.diff(rp)), ci] = v
    np.testing.assert_array_equal(oracle.spmm_semiring(rp, ci, v, B, "min_plus"),
                                  np.min(full[:, :, None] + B[None], axis=1))
    C = oracle.spmm_semiring(rp, ci, v, np.ones((k, n)), "max_times")
    for i in range(m):
        seg = v[rp[i]:rp[i + 1]]
        assert np.all(C[i] == (seg.max() if seg.size else -np.inf))


CHECKS = [check_products, check_transpose, check_merge_path, check_semirings]


def test_real_oracle_passes_every_check():
    rng = np.random.default_rng(0)
    for chk in CHECKS:
        chk(rng)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc missing")
    mutant = _build_mutant(str(tmp_path), name, *MUTANTS[name])
    saved = oracle._lib
    oracle._lib = mutant
    caught = []
    try:
        for chk in CHECKS:
            try:
                chk(np.random.default_rng(0))
            except AssertionError:
                caught.append(chk.__name__)
    finally:
        oracle._lib = saved
    assert caught, f"no pin caught the planted mistake: {name}"
