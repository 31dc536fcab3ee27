// Instantiation of the SpMM launchers for (vals, B, C) = (float, float, float).
#include "launch.cuh"

SPMM_DEFINE_LAUNCHERS(launchers_f32_f32_f32, float, float, float)
