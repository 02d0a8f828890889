// Main-kernel instantiations for op(A) = n, op(B) = t: the unprotected kernel,
// the fault-tolerant kernel, and the fault-tolerant kernel with the injector.
#include "ftgemm_kernel.cuh"

namespace ftg {

template <bool FT, bool INJ>
static cudaError_t launch_variant_nt(const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                                      const Params &p, cudaStream_t s) {
  auto k = ftdgemm_kernel<false, true, FT, INJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)p.nI * (unsigned)p.nJ, NTHREADS, SMEM_BYTES, s>>>(a, b, c, p);
  return cudaGetLastError();
}

cudaError_t launch_main_nt(bool ft, bool inj, const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                           const Params &p, cudaStream_t s) {
  if (!ft) return launch_variant_nt<false, false>(a, b, c, p, s);
  if (inj) return launch_variant_nt<true, true>(a, b, c, p, s);
  return launch_variant_nt<true, false>(a, b, c, p, s);
}

}  // namespace ftg
