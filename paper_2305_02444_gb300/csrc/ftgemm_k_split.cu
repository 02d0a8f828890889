// Split-precision mma.sync kernel instantiations (all operand layouts, with
// and without the fault tolerance), and the slicing kernels with their
// launcher.
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
// Integer arithmetic on the bits of the FP64 entries throughout: the FP64
// pipe is the scarce unit of this GPU.

// |x| as ordered bits (the order of non-negative doubles is that of their bit
// patterns); non-finite entries count as 0 for the row exponent.
__device__ __forceinline__ unsigned long long abs_bits_finite(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  return b < 0x7FF0000000000000ull ? b : 0ull;
}

// e with |x| < 2^e for the largest |x| given by its bits (0 for zero).
__device__ __forceinline__ int exponent_above(unsigned long long mb) {
  if (mb == 0) return 0;
  const int E = (int)(mb >> 52);
  const int ilog = E ? E - 1023 : (63 - __clzll((long long)mb)) - 1074;  // subnormal: leading bit
  return ilog + 1;
}

// Row exponent: e(r) with max_k |x(r, k)| < 2^e(r) over the finite entries.
// X is op(X) given by (ptr, ld, trans): element (r, k) = trans ? X[k + r*ld] : X[r + k*ld].
__global__ void __launch_bounds__(256) split_rowexp_kernel(const double *__restrict__ X, long long ld, int trans,
                                                           long long R, long long K, int *__restrict__ e) {
  if (trans) {  // k contiguous: one warp per row
    const long long r = (long long)blockIdx.x * 8 + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    unsigned long long m = 0;
    for (long long k = lane; k < K; k += 32) m = max(m, abs_bits_finite(X[k + r * ld]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[r] = exponent_above(m);
  } else {  // r contiguous: 32 rows x 8 k-groups per block
    __shared__ unsigned long long part[8][32];
    const int rl = threadIdx.x & 31, g = threadIdx.x >> 5;
    const long long r = (long long)blockIdx.x * 32 + rl;
    unsigned long long m = 0;
    if (r < R) {
#pragma unroll 4
      for (long long k = g; k < K; k += 8) m = max(m, abs_bits_finite(X[r + k * ld]));
    }
    part[g][rl] = m;
    __syncthreads();
    if (g == 0 && r < R) {
      for (int q = 1; q < 8; ++q) m = max(m, part[q][rl]);
      e[r] = exponent_above(m);
    }
  }
}

// Slice s of x: sign(x) * (floor(|x| 2^(w(s+1) - eR)) mod 2^w), exact, from
// the bits of x (|x| = m 2^(E' - 1075) with the 53-bit integer m).  This is
// the error-free splitting x 2^-eR = sum_s n_s 2^-w(s+1) + r, |n_s| < 2^w.
__device__ __forceinline__ int slice_of(unsigned long long m, int base, int w, int s) {
  const int t = base + w * (s + 1);
  unsigned long long q;
  if (t >= 0) q = (t >= w) ? 0ull : (m << t);
  else q = (t <= -64) ? 0ull : (m >> (-t));
  return (int)(q & ((1ull << w) - 1ull));
}

// Slices: out[s][r][k] (bf16, row length Kp, zero padded), 64 x 64 tiles through
// shared memory so that both the read and the write are coalesced.  A
// non-finite entry is carried by slice 0 (the product is then not finite).
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
    const double x = t[rr][kk];
    if (plain) {
      out[r * Kp + k] = __double2bfloat16(x);
      continue;
    }
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    const bool neg = (b >> 63) != 0;
    if (E == 0x7FF) {  // Inf / NaN
      out[r * Kp + k] = __double2bfloat16(x);
      for (int s = 1; s < S; ++s) out[((long long)s * R + r) * Kp + k] = __float2bfloat16(0.0f);
      continue;
    }
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
    const int base = (E ? E : 1) - 1075 - e[r];
    for (int s = 0; s < S; ++s) {
      const int n = slice_of(m, base, w, s);                           // 0 <= n < 2^w <= 256
      out[((long long)s * R + r) * Kp + k] = __float2bfloat16_rn((float)(neg ? -n : n));  // exact
    }
  }
}

cudaError_t launch_slicing(const double *X, long long ld, int trans, long long R, long long K, long long Kp, int *e,
                           int S, int w, int plain, void *out, cudaStream_t s) {
  if (!plain) {
    if (trans) split_rowexp_kernel<<<(unsigned)((R + 7) / 8), 256, 0, s>>>(X, ld, trans, R, K, e);
    else split_rowexp_kernel<<<(unsigned)((R + 31) / 32), 256, 0, s>>>(X, ld, trans, R, K, e);
  }
  dim3 grid((unsigned)((Kp + 63) / 64), (unsigned)((R + 63) / 64));
  split_slice_kernel<<<grid, 256, 0, s>>>(X, ld, trans, R, K, Kp, e, S, w, plain, (__nv_bfloat16 *)out);
  return cudaGetLastError();
}

}  // namespace ftg
