// Instantiation of the SpMM launchers for (vals, B, C) = (__nv_bfloat16, __half, __half).
#include "launch.cuh"

SPMM_DEFINE_LAUNCHERS(launchers_bf16_f16_f16, __nv_bfloat16, __half, __half)
