// Instantiations of the tcgen05 split-precision kernel (all operand layouts;
// without checks and with the FP64 checksums).
#include "ftgemm_split_tc.cuh"

namespace ftg {

template <bool TA, bool TB, int CK, int CL>
static cudaError_t launch_split_tc_variant(const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &b2,
                                           const SplitParams &p, cudaStream_t s) {
  auto k = ftsplit_tc_kernel<TA, TB, CK, CL>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  if (CL == 1) {
    k<<<(unsigned)p.nI * (unsigned)p.nJ, 256, TC_SMEM_BYTES, s>>>(a, b, b2, p);
    return cudaGetLastError();
  }
  // 1 x 2 or 2 x 2 clusters over the tile grid padded to even counts
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = CL == 2 ? dim3((unsigned)(p.nI * ((p.nJ + 1) / 2) * 2))
                        : dim3((unsigned)(((p.nI + 1) / 2) * ((p.nJ + 1) / 2) * 4));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = TC_SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, a, b, b2, p);
}

template <int CK, int CL>
static cudaError_t launch_split_tc_ck(bool ta, bool tb, const CUtensorMap &a, const CUtensorMap &b,
                                      const CUtensorMap &b2, const SplitParams &p, cudaStream_t s) {
  if (!ta && !tb) return launch_split_tc_variant<false, false, CK, CL>(a, b, b2, p, s);
  if (!ta && tb) return launch_split_tc_variant<false, true, CK, CL>(a, b, b2, p, s);
  if (ta && !tb) return launch_split_tc_variant<true, false, CK, CL>(a, b, b2, p, s);
  return launch_split_tc_variant<true, true, CK, CL>(a, b, b2, p, s);
}

// ck: 0 no checks, 2 FP64 checksums (FP32 checksums run on the mma.sync kernel).
// cluster 1: a, b with 128-row boxes; 2: a with 64-row boxes, b2 with 128-row
// boxes; 4: a, b with 64-row boxes.
cudaError_t launch_split_tc(bool ta, bool tb, int ck, int cluster, const CUtensorMap &a, const CUtensorMap &b,
                            const CUtensorMap &b2, const SplitParams &p, cudaStream_t s) {
  if (ck != 0 && ck != 2) return cudaErrorInvalidValue;
  if (cluster == 4)
    return ck ? launch_split_tc_ck<2, 4>(ta, tb, a, b, b2, p, s) : launch_split_tc_ck<0, 4>(ta, tb, a, b, b2, p, s);
  if (cluster == 2)
    return ck ? launch_split_tc_ck<2, 2>(ta, tb, a, b, b2, p, s) : launch_split_tc_ck<0, 2>(ta, tb, a, b, b2, p, s);
  if (cluster == 1)
    return ck ? launch_split_tc_ck<2, 1>(ta, tb, a, b, b2, p, s) : launch_split_tc_ck<0, 1>(ta, tb, a, b, b2, p, s);
  return cudaErrorInvalidValue;
}

}  // namespace ftg
