// Instantiations of the persistent tcgen05 split-precision kernel (all operand
// layouts; without checks and with the FP64 checksums).
#include <algorithm>

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

template <bool TA, bool TB, int CK>
static cudaError_t launch_split_tcp2_variant(const CUtensorMap &a, const CUtensorMap &bh, const SplitParams &p,
                                             int max_pairs, cudaStream_t s) {
  auto k = ftsplit_tcp2_kernel<TA, TB, CK>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TCP2_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = TCP2_SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // every pair of the persistent grid must be resident at once: as many
  // clusters as the device holds together (a GPC with an odd SM count
  // leaves one SM out), at most one per pair tile
  cfg.gridDim = dim3(2);
  int fit = 0;
  e = cudaOccupancyMaxActiveClusters(&fit, k, &cfg);
  if (e != cudaSuccess) return e;
  const long long npt = (long long)((p.nI + 1) / 2) * p.nJ;
  const int ncl = (int)std::max(1LL, std::min<long long>({npt, (long long)fit, (long long)max_pairs}));
  cfg.gridDim = dim3((unsigned)(2 * ncl));
  return cudaLaunchKernelEx(&cfg, k, a, bh, p);
}

template <int CK>
static cudaError_t launch_split_tcp2_ck(bool ta, bool tb, const CUtensorMap &a, const CUtensorMap &bh,
                                        const SplitParams &p, int max_pairs, cudaStream_t s) {
  if (!ta && !tb) return launch_split_tcp2_variant<false, false, CK>(a, bh, p, max_pairs, s);
  if (!ta && tb) return launch_split_tcp2_variant<false, true, CK>(a, bh, p, max_pairs, s);
  if (ta && !tb) return launch_split_tcp2_variant<true, false, CK>(a, bh, p, max_pairs, s);
  return launch_split_tcp2_variant<true, true, CK>(a, bh, p, max_pairs, s);
}

// Pair form: a with 128-row boxes, bh with 64-row boxes; at most max_pairs
// clusters of 2 CTAs (with ck 2, p.tscratch holds 2 max_pairs tiles).
cudaError_t launch_split_tcp2(bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &bh,
                              const SplitParams &p, int max_pairs, cudaStream_t s) {
  if ((ck != 0 && ck != 2) || max_pairs < 1 || (ck == 2 && !p.tscratch)) return cudaErrorInvalidValue;
  return ck ? launch_split_tcp2_ck<2>(ta, tb, a, bh, p, max_pairs, s)
            : launch_split_tcp2_ck<0>(ta, tb, a, bh, p, max_pairs, s);
}

}  // namespace ftg
