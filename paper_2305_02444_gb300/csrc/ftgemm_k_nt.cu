// Single-problem FP64 kernels for op(A) = n, op(B) = t (one translation unit per layout).
#include "ftgemm_launch.cuh"

FTG_LAYOUT_LAUNCHERS(nt, false, true)
