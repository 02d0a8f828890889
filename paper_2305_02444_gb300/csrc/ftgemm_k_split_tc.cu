// Instantiations of the tcgen05 split-precision kernel (all operand layouts;
// without checks and with the FP64 checksums).
#include "ftgemm_split_tc.cuh"

namespace ftg {

template <bool TA, bool TB, int CK>
static cudaError_t launch_split_tc_variant(const CUtensorMap &a, const CUtensorMap &b, const SplitParams &p,
                                           cudaStream_t s) {
  auto k = ftsplit_tc_kernel<TA, TB, CK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)p.nI * (unsigned)p.nJ, 256, TC_SMEM_BYTES, s>>>(a, b, p);
  return cudaGetLastError();
}

template <int CK>
static cudaError_t launch_split_tc_ck(bool ta, bool tb, const CUtensorMap &a, const CUtensorMap &b,
                                      const SplitParams &p, cudaStream_t s) {
  if (!ta && !tb) return launch_split_tc_variant<false, false, CK>(a, b, p, s);
  if (!ta && tb) return launch_split_tc_variant<false, true, CK>(a, b, p, s);
  if (ta && !tb) return launch_split_tc_variant<true, false, CK>(a, b, p, s);
  return launch_split_tc_variant<true, true, CK>(a, b, p, s);
}

// ck: 0 no checks, 2 FP64 checksums (FP32 checksums run on the mma.sync kernel);
// a, b: slice maps with 128-row boxes; one CTA per tile.
cudaError_t launch_split_tc(bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &b,
                            const SplitParams &p, cudaStream_t s) {
  if (ck != 0 && ck != 2) return cudaErrorInvalidValue;
  return ck ? launch_split_tc_ck<2>(ta, tb, a, b, p, s) : launch_split_tc_ck<0>(ta, tb, a, b, p, s);
}

}  // namespace ftg
