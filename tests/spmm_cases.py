"""Shared helpers of the GPU parity tests: seeded CSR structures and the
comparison of a library result with the FP64 oracle."""
import numpy as np

import gen
import oracle

FP32_TOL = 1e-5  # max |C - C_ref| / (|A||B|) for float32 storage (acceptance bound)


def csr_arrays(row_lengths, k, seed, int_vals=False, unsorted=False, duplicates=False):
    """CSR with the given row lengths; distinct sorted columns unless asked otherwise."""
    a = gen.csr_from_lengths(np.asarray(row_lengths, dtype=np.int64), k, seed)
    rp, ci, v = a.row_ptr, a.col_ind.copy(), a.vals.copy()
    rng = np.random.default_rng(seed)
    if duplicates and len(ci) > 1:
        # repeat the previous column at some positions of long-enough rows
        lens = np.diff(rp)
        for i in np.nonzero(lens >= 2)[0][::3]:
            ci[rp[i] + 1] = ci[rp[i]]
    if unsorted:
        for i in range(len(rp) - 1):
            seg = ci[rp[i]:rp[i + 1]]
            rng.shuffle(seg)
    if int_vals:
        v = rng.integers(-2, 3, size=len(ci)).astype(np.float32)
    return rp, ci, v


def structure(name, seed=0):
    """(row_ptr, col_ind, vals, k) of a named edge-case structure."""
    rng = np.random.default_rng(1000 + seed)
    if name == "uniform16":
        return (*csr_arrays(np.full(3000, 16), 2500, seed), 2500)
    if name == "power_law":
        lens, _ = gen.power_law_lengths(20_000, 20_000, seed + 3, cap=6000)
        return (*csr_arrays(lens, 20_000, seed), 20_000)
    if name == "short_rows":  # mean 3: the heuristic's merge side
        return (*csr_arrays(rng.poisson(3.0, 30_000), 30_000, seed), 30_000)
    if name == "alternating_empty":
        lens = np.where(np.arange(5000) % 2 == 0, 0, rng.integers(1, 40, 5000))
        return (*csr_arrays(lens, 4000, seed), 4000)
    if name == "empty_runs":  # long runs of empty rows between a few full ones
        lens = np.zeros(40_000, dtype=np.int64)
        lens[rng.choice(40_000, 300, replace=False)] = rng.integers(1, 200, 300)
        return (*csr_arrays(lens, 3000, seed), 3000)
    if name == "all_empty":
        return (*csr_arrays(np.zeros(777, dtype=np.int64), 50, seed), 50)
    if name == "giant_row":  # one row spanning many merge tiles
        lens = rng.integers(0, 5, 60)
        lens[30] = 100_000
        return (*csr_arrays(lens, 150_000, seed), 150_000)
    if name == "single_row":
        return (*csr_arrays(np.array([5000]), 9000, seed), 9000)
    if name == "one_nonzero":
        return (*csr_arrays(np.array([1]), 1, seed), 1)
    if name == "tall_k1":
        return (*csr_arrays(rng.integers(0, 2, 5000), 1, seed), 1)
    if name == "duplicates_unsorted":
        rp, ci, v = csr_arrays(rng.integers(0, 60, 4000), 3000, seed, unsorted=True, duplicates=True)
        return rp, ci, v, 3000
    if name == "identity":
        m = 4099
        return np.arange(m + 1, dtype=np.int32), np.arange(m, dtype=np.int32), np.ones(m, np.float32), m
    if name == "permutation":
        m = 3001
        return (np.arange(m + 1, dtype=np.int32), rng.permutation(m).astype(np.int32), np.ones(m, np.float32), m)
    raise KeyError(name)


STRUCTURES = ["uniform16", "power_law", "short_rows", "alternating_empty", "empty_runs", "all_empty", "giant_row",
              "single_row", "one_nonzero", "tall_k1", "duplicates_unsorted", "identity", "permutation"]


def check(C, rp, ci, v, B, tol=FP32_TOL, rows=None, vals_f64=None, B_f64=None):
    """Normalised error of C (numpy, [m or len(rows), n]) against the oracle."""
    vv = v if vals_f64 is None else vals_f64
    bb = B if B_f64 is None else B_f64
    if rows is None:
        ref = oracle.spmm(rp, ci, vv, bb)
        D = oracle.abs_bound(rp, ci, vv, bb)
    else:
        ref = oracle.spmm_rows(rows, rp, ci, vv, bb)
        D = oracle.abs_bound_rows(rows, rp, ci, vv, bb)
    err = oracle.normalized_error(C, ref, D)
    assert err <= tol, f"normalised error {err:.3e} > {tol:.1e}"
    return err
