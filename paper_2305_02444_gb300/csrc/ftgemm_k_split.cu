// Split-precision kernel instantiations (all operand layouts, with and without
// the fault tolerance) and the slicing kernels' launchers.
#include <cuda_bf16.h>

#include "ftgemm_split.cuh"

namespace ftg {

template <bool TA, bool TB, int CK>
static cudaError_t launch_split_variant(const CUtensorMap &a, const CUtensorMap &b, const SplitParams &p,
                                        cudaStream_t s) {
  auto k = ftsplit_kernel<TA, TB, CK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SP_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)p.nI * (unsigned)p.nJ, 256, SP_SMEM_BYTES, s>>>(a, b, p);
  return cudaGetLastError();
}

template <int CK>
static cudaError_t launch_split_ck(bool ta, bool tb, const CUtensorMap &a, const CUtensorMap &b,
                                   const SplitParams &p, cudaStream_t s) {
  if (!ta && !tb) return launch_split_variant<false, false, CK>(a, b, p, s);
  if (!ta && tb) return launch_split_variant<false, true, CK>(a, b, p, s);
  if (ta && !tb) return launch_split_variant<true, false, CK>(a, b, p, s);
  return launch_split_variant<true, true, CK>(a, b, p, s);
}

cudaError_t launch_split(bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &b,
                         const SplitParams &p, cudaStream_t s) {
  if (ck == 1) return launch_split_ck<1>(ta, tb, a, b, p, s);
  if (ck == 2) return launch_split_ck<2>(ta, tb, a, b, p, s);
  return launch_split_ck<0>(ta, tb, a, b, p, s);
}

cudaError_t launch_slicing(const double *X, long long ld, int trans, long long R, long long K, long long Kp, int *e,
                           int S, int w, int plain, void *out, cudaStream_t s) {
  if (!plain) {
    if (trans) split_rowexp_kernel<<<(unsigned)((R + 7) / 8), 256, 0, s>>>(X, ld, trans, R, K, e);
    else split_rowexp_kernel<<<(unsigned)((R + 255) / 256), 256, 0, s>>>(X, ld, trans, R, K, e);
  }
  dim3 grid((unsigned)((Kp + 63) / 64), (unsigned)((R + 63) / 64));
  split_slice_kernel<<<grid, 256, 0, s>>>(X, ld, trans, R, K, Kp, e, S, w, plain, (__nv_bfloat16 *)out);
  return cudaGetLastError();
}

}  // namespace ftg
