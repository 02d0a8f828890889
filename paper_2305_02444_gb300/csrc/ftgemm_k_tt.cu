// Single-problem FP64 kernels for op(A) = t, op(B) = t (one translation unit per layout).
#include "ftgemm_launch.cuh"

FTG_LAYOUT_LAUNCHERS(tt, true, true)
