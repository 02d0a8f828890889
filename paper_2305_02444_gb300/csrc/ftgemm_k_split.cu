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

// ---------------------------------------------------------------- slicing

// Row exponent: e with max_k |x(r, k)| < 2^e (0 for an all-zero row).
// X is op(X) given by (ptr, ld, trans): element (r, k) = trans ? X[k + r*ld] : X[r + k*ld].
__global__ void split_rowexp_kernel(const double *__restrict__ X, long long ld, int trans, long long R,
                                    long long K, int *__restrict__ e) {
  // one warp per row for trans (k contiguous); one thread per row otherwise (r contiguous)
  if (trans) {
    const long long r = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    double m = 0.0;
    for (long long k = lane; k < K; k += 32) m = fmax(m, fabs(X[k + r * ld]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[r] = (m > 0.0) ? ilogb(m) + 1 : 0;
  } else {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double m = 0.0;
    for (long long k = 0; k < K; ++k) m = fmax(m, fabs(X[r + k * ld]));
    e[r] = (m > 0.0) ? ilogb(m) + 1 : 0;
  }
}

// Slices: out[s][r][k] (bf16, row length Kp, zero padded), 64 x 64 tiles through
// shared memory so that both the read and the write are coalesced.
__global__ void __launch_bounds__(256) split_slice_kernel(const double *__restrict__ X, long long ld, int trans,
                                                          long long R, long long K, long long Kp,
                                                          const int *__restrict__ e, int S, int w, int plain,
                                                          __nv_bfloat16 *__restrict__ out) {
  __shared__ double t[64][65];
  const long long r0 = (long long)blockIdx.y * 64, k0 = (long long)blockIdx.x * 64;
  for (int q = threadIdx.x; q < 64 * 64; q += 256) {
    int rr, kk;
    if (trans) { kk = q & 63; rr = q >> 6; } else { rr = q & 63; kk = q >> 6; }
    const long long r = r0 + rr, k = k0 + kk;
    double v = 0.0;
    if (r < R && k < K) v = trans ? X[k + r * ld] : X[r + k * ld];
    t[rr][kk] = v;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 64 * 64; q += 256) {
    const int kk = q & 63, rr = q >> 6;
    const long long r = r0 + rr, k = k0 + kk;
    if (r >= R || k >= Kp) continue;
    double x = t[rr][kk];
    if (plain) {
      out[r * Kp + k] = __double2bfloat16(x);
      continue;
    }
    x = ldexp(x, -e[r]);  // |x| < 1, exact
    for (int s = 0; s < S; ++s) {
      const double v = ldexp(x, w);
      const double n = trunc(v);
      out[((long long)s * R + r) * Kp + k] = __double2bfloat16(n);  // |n| < 2^w <= 256: exact
      x = v - n;                                                      // exact
    }
  }
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
