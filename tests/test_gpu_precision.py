"""GPU parity of the 16-bit storage forms (vals, B and C in bf16 / f16,
float32 accumulation) with the FP64 oracle.

Two checks per result:
* against the oracle on the ROUNDED inputs (the exact 16-bit values widened to
  float64): only accumulation order and the one output rounding differ, so the
  bound is 1e-5 for float32 output and one unit of the output's last place
  (2^-8 bf16, 2^-10 f16, relative to |A||B|) for 16-bit output;
* against the oracle on the ORIGINAL float32 data: adds the input rounding of
  vals and B (2^-9 each for bf16), bounded by 1e-2 (the acceptance bound).
"""
import numpy as np
import pytest

import gen
import oracle
from spmm_cases import FP32_TOL, structure

pytestmark = pytest.mark.gpu

COMBOS = [("bf16", "bf16", "bf16"), ("bf16", "bf16", "f32"), ("bf16", "f16", "f16"), ("bf16", "f16", "f32"),
          ("f16", "f16", "f16"), ("f16", "f16", "f32")]
OUT_TOL = {"f32": FP32_TOL, "bf16": 2.0 ** -8, "f16": 2.0 ** -10}
# binary16 outputs below 2^-14 are subnormal: their rounding error is absolute, up to
# half the subnormal spacing 2^-24 (bfloat16 and float32 subnormals are far below any result here)
ABS_FLOOR = {"f32": 0.0, "bf16": 0.0, "f16": 2.0 ** -25}


def tdtype(torch, name):
    return {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[name]


def run_case(pkg, torch, rp, ci, v, B, combo, alg, rows=None, tuning=None):
    tv, tb, tc = (tdtype(torch, x) for x in combo)
    d_rp = torch.from_numpy(rp).cuda()
    d_ci = torch.from_numpy(ci).cuda()
    d_v = torch.from_numpy(v).cuda().to(tv)
    d_B = torch.from_numpy(B).cuda().to(tb)
    C = pkg.spmm(d_rp, d_ci, d_v, d_B, alg=alg, out_dtype=tc, nnz=int(rp[-1]), tuning=tuning)
    torch.cuda.synchronize()
    if rows is not None:
        C = C[torch.from_numpy(rows).cuda()]
    got = C.float().cpu().numpy()
    v_r, B_r = d_v.double().cpu().numpy(), d_B.double().cpu().numpy()
    return got, v_r, B_r


def errors(got, rp, ci, v, B, v_r, B_r, rows=None, out="f32"):
    if rows is None:
        rows = np.arange(len(rp) - 1)
    fl = ABS_FLOOR[out]
    e_rounded = oracle.normalized_error(got, oracle.spmm_rows(rows, rp, ci, v_r, B_r),
                                        oracle.abs_bound_rows(rows, rp, ci, v_r, B_r), abs_floor=fl)
    e_orig = oracle.normalized_error(got, oracle.spmm_rows(rows, rp, ci, v, B), oracle.abs_bound_rows(rows, rp, ci, v, B),
                                     abs_floor=fl)
    return e_rounded, e_orig


@pytest.mark.parametrize("combo", COMBOS)
@pytest.mark.parametrize("alg", ["row_split", "merge", "hybrid"])
@pytest.mark.parametrize("name,n", [("power_law", 64), ("giant_row", 128), ("short_rows", 8), ("uniform16", 24),
                                    ("duplicates_unsorted", 13)])
def test_precision_forms(gpu_lib, combo, alg, name, n):
    import torch

    rp, ci, v, k = structure(name)
    B = gen.normal_matrix(k, n, 61)
    got, v_r, B_r = run_case(gpu_lib, torch, rp, ci, v, B, combo, alg)
    e_r, e_o = errors(got, rp, ci, v, B, v_r, B_r, out=combo[2])
    assert e_r <= OUT_TOL[combo[2]], e_r
    assert e_o <= 1e-2, e_o


def test_f32_output_of_16bit_inputs_is_accumulation_exact_on_integers(gpu_lib):
    """Small integers are exact in bf16 and f16: with float32 output the result is
    bit-exact for every algorithm."""
    import torch

    rng = np.random.default_rng(8)
    rp, ci, _, k = structure("power_law")
    v = rng.integers(-2, 3, len(ci)).astype(np.float32)
    B = rng.integers(-4, 5, (k, 64)).astype(np.float32)
    ref = oracle.spmm(rp, ci, v, B)
    if np.abs(ref).max() < 2 ** 24:
        for combo in (("bf16", "bf16", "f32"), ("f16", "f16", "f32"), ("bf16", "f16", "f32")):
            for alg in ("row_split", "merge"):
                got, _, _ = run_case(gpu_lib, torch, rp, ci, v, B, combo, alg)
                assert np.array_equal(got, ref.astype(np.float32))


@pytest.mark.slow
@pytest.mark.parametrize("combo", [("bf16", "bf16", "bf16"), ("bf16", "bf16", "f32"), ("bf16", "f16", "f32")])
def test_precision_workload_full_size_sampled(gpu_lib, combo):
    """2M x 2M, 32 nonzeros per row, n = 128 at full size; sampled rows."""
    import torch

    a, B = gen.workload_precision()
    rng = np.random.default_rng(5)
    rows = np.sort(rng.choice(a.m, 2000, replace=False))
    for alg in ("row_split", "merge"):
        got, v_r, B_r = run_case(gpu_lib, torch, a.row_ptr, a.col_ind, a.vals, B, combo, alg, rows=rows)
        e_r, e_o = errors(got, a.row_ptr, a.col_ind, a.vals, B, v_r, B_r, rows=rows, out=combo[2])
        assert e_r <= OUT_TOL[combo[2]] and e_o <= 1e-2, (alg, e_r, e_o)
