// Main-kernel instantiations for op(A) = n, op(B) = n: the unprotected kernel,
// the fault-tolerant kernel and the fault-tolerant kernel with the injector, for
// whole tiles (mode 0), split-K partials (mode 1) and reductions (mode 2), the
// verify-only pass (mode 3), and the persistent batched kernel.
#include "ftgemm_kernel.cuh"

namespace ftg {

template <bool FT, bool INJ, int MODE>
static cudaError_t launch_variant_nn(const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                                      const CUtensorMap &w, const Params &p, cudaStream_t s) {
  auto k = ftdgemm_kernel<false, false, FT, INJ, MODE>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const unsigned count = p.tile_count ? (unsigned)p.tile_count : (unsigned)p.nI * (unsigned)p.nJ;
  const unsigned grid = count * (MODE == 1 ? (unsigned)p.nsplit : 1u);
  k<<<grid, NTHREADS, SMEM_BYTES, s>>>(a, b, c, w, p);
  return cudaGetLastError();
}

cudaError_t launch_gemm_nn(bool ft, bool inj, int mode, const CUtensorMap &a, const CUtensorMap &b,
                           const CUtensorMap &c, const CUtensorMap &w, const Params &p, cudaStream_t s) {
  if (mode == 1) {
    if (!ft) return launch_variant_nn<false, false, 1>(a, b, c, w, p, s);
    if (inj) return launch_variant_nn<true, true, 1>(a, b, c, w, p, s);
    return launch_variant_nn<true, false, 1>(a, b, c, w, p, s);
  }
  if (mode == 3) return launch_variant_nn<true, false, 3>(a, b, c, w, p, s);
  if (mode == 2) {
    if (!ft) return launch_variant_nn<false, false, 2>(a, b, c, w, p, s);
    return launch_variant_nn<true, false, 2>(a, b, c, w, p, s);
  }
  if (!ft) return launch_variant_nn<false, false, 0>(a, b, c, w, p, s);
  if (inj) return launch_variant_nn<true, true, 0>(a, b, c, w, p, s);
  return launch_variant_nn<true, false, 0>(a, b, c, w, p, s);
}

cudaError_t launch_main_nn(bool ft, bool inj, const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                           const Params &p, cudaStream_t s) {
  return launch_gemm_nn(ft, inj, 0, a, b, c, c, p, s);
}

template <bool FT, bool INJ>
static cudaError_t launch_batched_variant_nn(const BatchProblem *probs, const int *order, const int *tile_prob,
                                              const int *tile_local, int total, int chunk, int *counter, int *gerr,
                                              int grid, cudaStream_t s) {
  auto k = ftdgemm_batched_kernel<false, false, FT, INJ>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<grid, NTHREADS, SMEM_BYTES, s>>>(probs, order, tile_prob, tile_local, total, chunk, counter, gerr);
  return cudaGetLastError();
}

cudaError_t launch_batched_nn(bool ft, bool inj, const BatchProblem *probs, const int *order,
                               const int *tile_prob, const int *tile_local, int total, int chunk, int *counter,
                               int *gerr, int grid, cudaStream_t s) {
  if (!ft) return launch_batched_variant_nn<false, false>(probs, order, tile_prob, tile_local, total, chunk,
                                                            counter, gerr, grid, s);
  if (inj) return launch_batched_variant_nn<true, true>(probs, order, tile_prob, tile_local, total, chunk,
                                                          counter, gerr, grid, s);
  return launch_batched_variant_nn<true, false>(probs, order, tile_prob, tile_local, total, chunk, counter,
                                                  gerr, grid, s);
}

// fault-tolerant whole-tile kernel with the per-k-panel verification
cudaError_t launch_panel_nn(bool inj, const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c,
                             const Params &p, cudaStream_t s) {
  auto k = inj ? ftdgemm_kernel<false, false, true, true, 0, true> : ftdgemm_kernel<false, false, true, false, 0, true>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)p.nI * (unsigned)p.nJ, NTHREADS, SMEM_BYTES, s>>>(a, b, c, c, p);
  return cudaGetLastError();
}

}  // namespace ftg
