// Instantiation of the SpMM launchers for (vals, B, C) = (__half, __half, __half).
#include "launch.cuh"

SPMM_DEFINE_LAUNCHERS(launchers_f16_f16_f16, __half, __half, __half)
