// Instantiation of the SpMM launchers for (vals, B, C) = (__nv_bfloat16, __nv_bfloat16, __nv_bfloat16).
#include "launch.cuh"

SPMM_DEFINE_LAUNCHERS(launchers_bf16_bf16_bf16, __nv_bfloat16, __nv_bfloat16, __nv_bfloat16)
