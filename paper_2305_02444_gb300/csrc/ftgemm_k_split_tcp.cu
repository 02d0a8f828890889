// Instantiations of the persistent tcgen05 split-precision kernel (all operand
// layouts; without checks and with the FP64 checksums).
#include "ftgemm_split_tcp.cuh"

namespace ftg {

template <bool TA, bool TB, int CK>
static cudaError_t launch_split_tcp_variant(const CUtensorMap &a, const CUtensorMap &b, const SplitParams &p,
                                            int nctas, cudaStream_t s) {
  auto k = ftsplit_tcp_kernel<TA, TB, CK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)nctas, 256, TCP_SMEM_BYTES, s>>>(a, b, p);
  return cudaGetLastError();
}

template <int CK>
static cudaError_t launch_split_tcp_ck(bool ta, bool tb, const CUtensorMap &a, const CUtensorMap &b,
                                       const SplitParams &p, int nctas, cudaStream_t s) {
  if (!ta && !tb) return launch_split_tcp_variant<false, false, CK>(a, b, p, nctas, s);
  if (!ta && tb) return launch_split_tcp_variant<false, true, CK>(a, b, p, nctas, s);
  if (ta && !tb) return launch_split_tcp_variant<true, false, CK>(a, b, p, nctas, s);
  return launch_split_tcp_variant<true, true, CK>(a, b, p, nctas, s);
}

// ck: 0 no checks, 2 FP64 checksums; a, b: slice maps with 128-row boxes;
// nctas: CTAs of the persistent grid (at most one per SM, at most the tile
// count); with ck 2, p.tscratch holds nctas 128 x 128 FP64 tiles.
cudaError_t launch_split_tcp(bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &b,
                             const SplitParams &p, int nctas, cudaStream_t s) {
  if ((ck != 0 && ck != 2) || nctas < 1 || (ck == 2 && !p.tscratch)) return cudaErrorInvalidValue;
  return ck ? launch_split_tcp_ck<2>(ta, tb, a, b, p, nctas, s) : launch_split_tcp_ck<0>(ta, tb, a, b, p, nctas, s);
}

}  // namespace ftg
