// Batched FP64 kernel for op(A) = t, op(B) = t (one translation unit per layout).
#include "ftgemm_launch.cuh"

FTG_LAYOUT_BATCHED_LAUNCHERS(tt, true, true)
