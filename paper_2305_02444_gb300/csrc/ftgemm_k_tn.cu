// Main-kernel instantiations for op(A) = t, op(B) = n: the unprotected kernel,
// the fault-tolerant kernel, and the fault-tolerant kernel with the injector.
#include "ftgemm_kernel.cuh"

namespace ftg {

template <bool FT, bool INJ>
static cudaError_t launch_variant_tn(const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                                      const Params &p, cudaStream_t s) {
  auto k = ftdgemm_kernel<true, false, FT, INJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)p.nI * (unsigned)p.nJ, NTHREADS, SMEM_BYTES, s>>>(a, b, c, p);
  return cudaGetLastError();
}

cudaError_t launch_main_tn(bool ft, bool inj, const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                           const Params &p, cudaStream_t s) {
  if (!ft) return launch_variant_tn<false, false>(a, b, c, p, s);
  if (inj) return launch_variant_tn<true, true>(a, b, c, p, s);
  return launch_variant_tn<true, false>(a, b, c, p, s);
}

}  // namespace ftg
