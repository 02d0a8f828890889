// Launchers of the FP64 kernels for one operand layout (op(A) = A or A^T,
// op(B) = B or B^T): the unprotected kernel, the fault-tolerant kernel and
// the fault-tolerant kernel with the injector, for whole tiles (mode 0),
// split-K partials (mode 1) and reductions (mode 2), each of the first two
// with or without the per-k-panel verification; the verify-only pass (mode
// 3); and the persistent batched kernel.  Each ftgemm_k_<layout>.cu and
// ftgemm_kb_<layout>.cu instantiates them for its layout, so that the layouts
// compile in parallel.
#pragma once

#include "ftgemm_kernel.cuh"

namespace ftg {

template <bool TA, bool TB>
struct LayoutLaunch {
  template <bool FT, bool INJ, int MODE, bool PANEL>
  static cudaError_t variant(const CUtensorMap &a, const CUtensorMap &b, const CUtensorMap &c, const CUtensorMap &w,
                             const Params &p, cudaStream_t s) {
    auto k = ftdgemm_kernel<TA, TB, FT, INJ, MODE, PANEL>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const unsigned count = p.tile_count ? (unsigned)p.tile_count : (unsigned)p.nI * (unsigned)p.nJ;
    const unsigned grid = count * (MODE == 1 ? (unsigned)p.nsplit : 1u);
    k<<<grid, NTHREADS, SMEM_BYTES, s>>>(a, b, c, w, p);
    return cudaGetLastError();
  }

  // modes 0 and 1 with the k-loop: unprotected, FT, FT + injection, each FT
  // one also with the per-k-panel checks
  template <int MODE>
  static cudaError_t kloop(bool ft, bool inj, bool panel, const CUtensorMap &a, const CUtensorMap &b,
                           const CUtensorMap &c, const CUtensorMap &w, const Params &p, cudaStream_t s) {
    if (!ft) return variant<false, false, MODE, false>(a, b, c, w, p, s);
    if (panel)
      return inj ? variant<true, true, MODE, true>(a, b, c, w, p, s) : variant<true, false, MODE, true>(a, b, c, w, p, s);
    return inj ? variant<true, true, MODE, false>(a, b, c, w, p, s) : variant<true, false, MODE, false>(a, b, c, w, p, s);
  }

  static cudaError_t gemm(bool ft, bool inj, int mode, bool panel, const CUtensorMap &a, const CUtensorMap &b,
                          const CUtensorMap &c, const CUtensorMap &w, const Params &p, cudaStream_t s) {
    if (mode == 1) return kloop<1>(ft, inj, panel, a, b, c, w, p, s);
    if (mode == 3) return variant<true, false, 3, false>(a, b, c, w, p, s);
    if (mode == 2) return ft ? variant<true, false, 2, false>(a, b, c, w, p, s) : variant<false, false, 2, false>(a, b, c, w, p, s);
    return kloop<0>(ft, inj, panel, a, b, c, w, p, s);
  }

  template <bool FT, bool INJ>
  static cudaError_t batched_variant(const BatchProblem *probs, const int *order, const int *tile_prob,
                                     const int *tile_local, int total, int chunk, int *counter, int *gerr, int grid,
                                     cudaStream_t s) {
    auto k = ftdgemm_batched_kernel<TA, TB, FT, INJ>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    k<<<grid, NTHREADS, SMEM_BYTES, s>>>(probs, order, tile_prob, tile_local, total, chunk, counter, gerr);
    return cudaGetLastError();
  }

  static cudaError_t batched(bool ft, bool inj, const BatchProblem *probs, const int *order, const int *tile_prob,
                             const int *tile_local, int total, int chunk, int *counter, int *gerr, int grid,
                             cudaStream_t s) {
    if (!ft) return batched_variant<false, false>(probs, order, tile_prob, tile_local, total, chunk, counter, gerr, grid, s);
    if (inj) return batched_variant<true, true>(probs, order, tile_prob, tile_local, total, chunk, counter, gerr, grid, s);
    return batched_variant<true, false>(probs, order, tile_prob, tile_local, total, chunk, counter, gerr, grid, s);
  }
};

}  // namespace ftg

// The entry points of one layout XX (nn, nt, tn, tt) for the host code: the
// single-problem kernels (ftgemm_k_<layout>.cu) and the batched kernel
// (ftgemm_kb_<layout>.cu), in separate translation units so that they
// compile in parallel.
#define FTG_LAYOUT_LAUNCHERS(XX, TA, TB)                                                                          \
  namespace ftg {                                                                                                 \
  cudaError_t launch_gemm_##XX(bool ft, bool inj, int mode, bool panel, const CUtensorMap &a, const CUtensorMap &b, \
                               const CUtensorMap &c, const CUtensorMap &w, const Params &p, cudaStream_t s) {     \
    return LayoutLaunch<TA, TB>::gemm(ft, inj, mode, panel, a, b, c, w, p, s);                                    \
  }                                                                                                               \
  }

#define FTG_LAYOUT_BATCHED_LAUNCHERS(XX, TA, TB)                                                                  \
  namespace ftg {                                                                                                 \
  cudaError_t launch_batched_##XX(bool ft, bool inj, const BatchProblem *probs, const int *order,                 \
                                  const int *tile_prob, const int *tile_local, int total, int chunk, int *counter, \
                                  int *gerr, int grid, cudaStream_t s) {                                          \
    return LayoutLaunch<TA, TB>::batched(ft, inj, probs, order, tile_prob, tile_local, total, chunk, counter,     \
                                         gerr, grid, s);                                                          \
  }                                                                                                               \
  }
