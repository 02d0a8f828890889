// Batched FP64 kernel for op(A) = t, op(B) = n (one translation unit per layout).
#include "ftgemm_launch.cuh"

FTG_LAYOUT_BATCHED_LAUNCHERS(tn, true, false)
