// Single-problem FP64 kernels for op(A) = n, op(B) = n (one translation unit per layout).
#include "ftgemm_launch.cuh"

FTG_LAYOUT_LAUNCHERS(nn, false, false)
