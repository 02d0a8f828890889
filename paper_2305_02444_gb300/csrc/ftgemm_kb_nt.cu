// Batched FP64 kernel for op(A) = n, op(B) = t (one translation unit per layout).
#include "ftgemm_launch.cuh"

FTG_LAYOUT_BATCHED_LAUNCHERS(nt, false, true)
