// Split-precision mma.sync kernel instantiations (all operand layouts, with
// and without the fault tolerance), and the slicing kernels with their
// launcher.
#include <algorithm>

#include <cuda_bf16.h>

#include "ftgemm_split.cuh"

namespace ftg {

template <bool TA, bool TB, int CK, bool I8>
static cudaError_t launch_split_variant(const CUtensorMap &a, const CUtensorMap &b, const SplitParams &p,
                                        cudaStream_t s) {
  auto k = ftsplit_kernel<TA, TB, CK, I8>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SP_SMEM_BYTES);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)p.nI * (unsigned)p.nJ, 256, SP_SMEM_BYTES, s>>>(a, b, p);
  return cudaGetLastError();
}

template <int CK, bool I8 = false>
static cudaError_t launch_split_ck(bool ta, bool tb, const CUtensorMap &a, const CUtensorMap &b,
                                   const SplitParams &p, cudaStream_t s) {
  if (!ta && !tb) return launch_split_variant<false, false, CK, I8>(a, b, p, s);
  if (!ta && tb) return launch_split_variant<false, true, CK, I8>(a, b, p, s);
  if (ta && !tb) return launch_split_variant<true, false, CK, I8>(a, b, p, s);
  return launch_split_variant<true, true, CK, I8>(a, b, p, s);
}

// ck: 0 no checks, 1 FP32 checksums in the kernel, 2 FP64 checksums computed
// before it; i8: INT8 slices (ck 0 or 2)
cudaError_t launch_split(bool ta, bool tb, int ck, bool i8, const CUtensorMap &a, const CUtensorMap &b,
                         const SplitParams &p, cudaStream_t s) {
  if (i8) {
    if (ck == 1) return cudaErrorInvalidValue;
    return ck == 2 ? launch_split_ck<2, true>(ta, tb, a, b, p, s) : launch_split_ck<0, true>(ta, tb, a, b, p, s);
  }
  if (ck == 1) return launch_split_ck<1>(ta, tb, a, b, p, s);
  if (ck == 2) return launch_split_ck<2>(ta, tb, a, b, p, s);
  return launch_split_ck<0>(ta, tb, a, b, p, s);
}

// ---------------------------------------------------------------- slicing
// Integer arithmetic on the bits of the FP64 entries throughout: the FP64
// pipe is the scarce unit of this GPU.

// |x| as ordered bits (the order of non-negative doubles is that of their bit
// patterns); non-finite entries count as 0 for the row exponent.  Built from
// the two 32-bit halves: a mask of the 64-bit pattern reads as fabs and would
// take the FP64 pipe.
__device__ __forceinline__ unsigned long long abs_bits_finite(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x) & 0x7FFFFFFFu, lo = (uint32_t)__double2loint(x);
  return hi < 0x7FF00000u ? ((unsigned long long)hi << 32 | lo) : 0ull;
}

// e with |x| < 2^e for the largest |x| given by its bits (0 for zero).
__device__ __forceinline__ int exponent_above(unsigned long long mb) {
  if (mb == 0) return 0;
  const int E = (int)(mb >> 52);
  const int ilog = E ? E - 1023 : (63 - __clzll((long long)mb)) - 1074;  // subnormal: leading bit
  return ilog + 1;
}

// Row maxima of |op(X)| over the finite entries, as ordered bits, combined
// across the k-splits of the grid (blockIdx.y) by atomicMax into mb (zeroed
// before).  op(X)(r, k) = trans ? X[k + r*ld] : X[r + k*ld].  trans = 0 (r
// contiguous): a thread per row, a warp reads 32 consecutive rows per k;
// trans = 1 (k contiguous): a warp per row, lanes along k.  Eight loads in
// flight per thread.
__global__ void __launch_bounds__(256) split_rowmax_kernel(const double *__restrict__ X, long long ld, int trans,
                                                           long long R, long long K, long long kper,
                                                           unsigned long long *__restrict__ mb,
                                                           unsigned int *__restrict__ nf) {
  const long long k0 = (long long)blockIdx.y * kper, k1 = min(K, k0 + kper);
  unsigned long long m = 0;
  bool bad = false;  // a non-finite entry in this part of the row
  long long r;
  if (!trans) {
    r = (long long)blockIdx.x * 256 + threadIdx.x;
    if (r >= R) return;
    const double *x = X + r;
    long long k = k0;
    for (; k + 8 <= k1; k += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = x[(k + u) * ld];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        m = max(m, abs_bits_finite(v[u]));
        bad = bad || !isfinite(v[u]);
      }
    }
    for (; k < k1; ++k) {
      m = max(m, abs_bits_finite(x[k * ld]));
      bad = bad || !isfinite(x[k * ld]);
    }
  } else {
    r = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    const double *x = X + r * ld;
    long long k = k0 + lane;
    for (; k + 7 * 32 < k1; k += 8 * 32) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = x[k + 32 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        m = max(m, abs_bits_finite(v[u]));
        bad = bad || !isfinite(v[u]);
      }
    }
    for (; k < k1; k += 32) {
      m = max(m, abs_bits_finite(x[k]));
      bad = bad || !isfinite(x[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, (unsigned long long)__shfl_xor_sync(0xffffffffu, m, o));
    bad = __any_sync(0xffffffffu, bad);
    if (lane != 0) return;
  }
  if (m) atomicMax(mb + r, m);
  if (bad && nf) atomicOr(nf + r, 1u);
}

// floor(m 2^t) mod 2^64 for the 53-bit integer m and any t.
__device__ __forceinline__ unsigned long long shift_trunc(unsigned long long m, int t) {
  if (t >= 0) return t >= 64 ? 0ull : (m << t);
  return t <= -64 ? 0ull : (m >> (-t));
}

// The error-free splitting x 2^-e(r) = sum_s n_s 2^-w(s+1) + r with
// |n_s| < 2^w: slice s of x is sign(x) (floor(|x| 2^(w(s+1) - e(r))) mod 2^w),
// taken exactly from the bits of x.
// One entry prepared for slicing.  With |x| 2^-e(r) = m 2^base (m the 53-bit
// integer of x), slice s is n_s = floor(m 2^(base + w(s+1))) mod 2^w.  The
// first S1 = floor(64 / w) slices come from f1 = floor(m 2^(base + w S1)) (an
// integer below 2^(w S1), as |x| 2^-e(r) < 1), the others from the low 64
// bits f2 of floor(m 2^(base + w S)); then n_s is a field of f1 or f2 at a
// shift that is the same for every entry.  nfb: the bf16 bits of a
// non-finite entry (carried by slice 0), else 0.
struct SliceIn {
  unsigned long long f1, f2;
  uint32_t sg, nfb;
};

__device__ __forceinline__ SliceIn slice_prep(double x, int er, int w, int S, int S1) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  SliceIn q;
  q.sg = (uint32_t)(b >> 48) & 0x8000u;
  q.nfb = E == 0x7FF ? (uint32_t)__bfloat16_as_ushort(__double2bfloat16(x)) : 0u;
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
  const int base = (E ? E : 1) - 1075 - er;
  q.f1 = shift_trunc(m, base + w * S1);
  q.f2 = S > S1 ? shift_trunc(m, base + w * S) : 0ull;
  return q;
}

// bf16 bits of slice s: the w-bit field, converted exactly (n < 2^8 as the
// FP32 (2^23 + n) - 2^23, whose low 16 bits are zero), with the entry's sign.
__device__ __forceinline__ uint32_t slice_bits(const SliceIn &q, int w, int S, int S1, int s) {
  if (q.nfb) return s == 0 ? q.nfb : 0u;
  const unsigned long long f = s < S1 ? q.f1 : q.f2;
  const int c = s < S1 ? w * (S1 - 1 - s) : w * (S - 1 - s);
  const uint32_t n = (uint32_t)(f >> c) & ((1u << w) - 1u);
  if (!n) return 0u;
  return q.sg | (__float_as_uint(__fsub_rn(__uint_as_float(0x4B000000u | n), 8388608.0f)) >> 16);
}

// INT8 form of slice s: the w-bit field (w <= 7) with the entry's sign, as a
// two's-complement byte; a non-finite entry gives 0 (its row is recomputed
// in FP64 by the product kernel, which INT8 slices cannot carry Inf / NaN to).
__device__ __forceinline__ uint32_t slice_i8(const SliceIn &q, int w, int S, int S1, int s) {
  if (q.nfb) return 0u;
  const unsigned long long f = s < S1 ? q.f1 : q.f2;
  const int c = s < S1 ? w * (S1 - 1 - s) : w * (S - 1 - s);
  const int n = (int)((uint32_t)(f >> c) & ((1u << w) - 1u));
  return (uint32_t)(uint8_t)(int8_t)(q.sg ? -n : n);
}

// Slices: out[s][r][k] (bf16, row length Kp, zero padded past K); plain: the
// bf16 rounding of each entry.  The row exponent e(r) (max |op(X)(r, :)| <
// 2^e(r), 0 for a zero row) comes from the row maxima mb and is written to e
// by the threads of k-block 0.
//   trans = 1 (k contiguous): a warp per row; each lane takes two consecutive
//     k of each of four 64-k spans (bf16x2 stores);
//   trans = 0 (r contiguous): a thread per row and 8 consecutive k (a 16-byte
//     store per slice), a warp reads 32 consecutive rows per k; the 8 warps
//     take the 8 8-k groups of a 64-k block.
// Eight loads in flight per thread.
// I8: INT8 slices (bytes) instead of bf16, and e[r] = SPLIT_NONFINITE_ROW
// for a row with a non-finite entry (nf, from the row-maxima pass).
template <int trans, int plain, bool I8 = false>
__global__ void __launch_bounds__(256) split_slice_kernel(const double *__restrict__ X, long long ld, long long R,
                                                          long long K, long long Kp,
                                                          const unsigned long long *__restrict__ mb,
                                                          const unsigned int *__restrict__ nf,
                                                          int *__restrict__ e, int S, int w,
                                                          __nv_bfloat16 *__restrict__ out) {
  uint16_t *o16 = reinterpret_cast<uint16_t *>(out);
  uint8_t *o8 = reinterpret_cast<uint8_t *>(out);
  const long long RK = R * Kp;
  const int ns = plain ? 1 : S;
  if constexpr (trans != 0) {
    const long long r = (long long)blockIdx.y * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    const int er = plain ? 0 : exponent_above(mb[r]);
    if (!plain && blockIdx.x == 0 && lane == 0) e[r] = (I8 && nf[r]) ? SPLIT_NONFINITE_ROW : er;
    const long long kb = (long long)blockIdx.x * 256 + 2 * lane;  // k of span u: kb + 64 u
    const double *x = X + r * ld;
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long k = kb + 64 * (u >> 1) + (u & 1);
      v[u] = k < K ? x[k] : 0.0;
    }
    if constexpr (plain != 0) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long k = kb + 64 * u;
        if (k < Kp)
          *reinterpret_cast<uint32_t *>(o16 + r * Kp + k) =
              bf16_rn_bits(v[2 * u]) | (bf16_rn_bits(v[2 * u + 1]) << 16);
      }
    } else {
      const int S1 = min(S, 64 / w);
      SliceIn q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q[u] = slice_prep(v[u], er, w, S, S1);
      for (int s = 0; s < ns; ++s) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const long long k = kb + 64 * u;
          if (k >= Kp) continue;
          if constexpr (I8)
            *reinterpret_cast<uint16_t *>(o8 + s * RK + r * Kp + k) =
                (uint16_t)(slice_i8(q[2 * u], w, S, S1, s) | (slice_i8(q[2 * u + 1], w, S, S1, s) << 8));
          else
            *reinterpret_cast<uint32_t *>(o16 + s * RK + r * Kp + k) =
                slice_bits(q[2 * u], w, S, S1, s) | (slice_bits(q[2 * u + 1], w, S, S1, s) << 16);
        }
      }
    }
  } else {
    const long long r = (long long)blockIdx.y * 32 + (threadIdx.x & 31);
    const int g = threadIdx.x >> 5;
    if (r >= R) return;
    const int er = plain ? 0 : exponent_above(mb[r]);
    if (!plain && blockIdx.x == 0 && g == 0) e[r] = (I8 && nf[r]) ? SPLIT_NONFINITE_ROW : er;
    const long long k0 = (long long)blockIdx.x * 64 + 8 * g;
    const double *x = X + r;
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = k0 + u < K ? x[(k0 + u) * ld] : 0.0;
    uint4 *dst = reinterpret_cast<uint4 *>(o16 + r * Kp + k0);  // 16-byte aligned (Kp is a multiple of 64)
    if constexpr (plain != 0) {
      uint32_t h[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) h[u] = bf16_rn_bits(v[2 * u]) | (bf16_rn_bits(v[2 * u + 1]) << 16);
      *dst = make_uint4(h[0], h[1], h[2], h[3]);
    } else {
      const int S1 = min(S, 64 / w);
      SliceIn q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) q[u] = slice_prep(v[u], er, w, S, S1);
      for (int s = 0; s < ns; ++s) {
        if constexpr (I8) {
          uint32_t h[2];
#pragma unroll
          for (int u = 0; u < 2; ++u)
            h[u] = slice_i8(q[4 * u], w, S, S1, s) | (slice_i8(q[4 * u + 1], w, S, S1, s) << 8) |
                   (slice_i8(q[4 * u + 2], w, S, S1, s) << 16) | (slice_i8(q[4 * u + 3], w, S, S1, s) << 24);
          *reinterpret_cast<uint2 *>(o8 + s * RK + r * Kp + k0) = make_uint2(h[0], h[1]);  // 8-byte aligned
        } else {
          uint32_t h[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            h[u] = slice_bits(q[2 * u], w, S, S1, s) | (slice_bits(q[2 * u + 1], w, S, S1, s) << 16);
          dst[s * (RK / 8)] = make_uint4(h[0], h[1], h[2], h[3]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------- checksum vectors of the plain form
// From the bf16 operand X (R rows of Kp entries, k contiguous; rows of op(A)
// or columns of op(B)) and its groups of 128 rows g:
//   pieces[g][k] and pieces[nG + g][k]: the two bf16 pieces hi = bf16(s),
//     lo = bf16(s - hi) of s = fl32(sum_{r in g} X[r][k]) (rows in order);
//   part_row[c][r] = sum over chunk c's k of |X[r][k]|, FP32 rounded up;
//   part_gmax[c][g] = max over chunk c's k of sum_{r in g} |X[r][k]|, FP32
//     rounded up.
// Block (g, c): the 128 rows of g and k-chunk c of BF16CS_KC entries, a thread
// per two consecutive k (32-bit loads; 128 bytes per warp and row).  FP32
// adds only: the FP64 pipe is this GPU's scarcest unit.
constexpr int BF16CS_KC = 512;

__global__ void __launch_bounds__(256) bf16_checksum_kernel(const uint16_t *__restrict__ X, long long R,
                                                            long long Kp, uint16_t *__restrict__ pieces,
                                                            float *__restrict__ part_row,
                                                            float *__restrict__ part_gmax, int nG) {
  __shared__ float rowp[8][128];
  __shared__ float colmax[8];
  const int g = blockIdx.x, c = blockIdx.y, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const long long r0 = (long long)g * 128, nrows = min(128LL, R - r0);
  const long long k = (long long)c * BF16CS_KC + 2 * t;
  const bool kin = k < Kp;                       // Kp is even: both entries of the pair are in range
  float s0 = 0.f, s1 = 0.f, a0 = 0.f, a1 = 0.f;
  const uint32_t *x = reinterpret_cast<const uint32_t *>(X + r0 * Kp + (kin ? k : 0));
  const long long stride = Kp / 2;               // in 32-bit words
#pragma unroll 1
  for (int r = 0; r < nrows; r += 8) {
    uint32_t v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (kin && r + u < nrows) ? __ldg(x + (long long)(r + u) * stride) : 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float x0 = __uint_as_float(v[u] << 16), x1 = __uint_as_float(v[u] & 0xFFFF0000u);
      s0 = __fadd_rn(s0, x0);
      s1 = __fadd_rn(s1, x1);
      a0 = __fadd_ru(a0, fabsf(x0));
      a1 = __fadd_ru(a1, fabsf(x1));
      float ra = __fadd_ru(fabsf(x0), fabsf(x1));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ra = __fadd_ru(ra, __shfl_xor_sync(0xffffffffu, ra, o));
      if (lane == 0 && r + u < 128) rowp[w][r + u] = ra;
    }
  }
  if (kin) {
    const float h0 = __bfloat162float(__float2bfloat16_rn(s0)), h1 = __bfloat162float(__float2bfloat16_rn(s1));
    const float l0 = __fsub_rn(s0, h0), l1 = __fsub_rn(s1, h1);   // exact
    const uint32_t hi = (__float_as_uint(h0) >> 16) | (__float_as_uint(h1) & 0xFFFF0000u);
    const uint32_t lo = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(l0)) |
                        ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(l1)) << 16);
    *reinterpret_cast<uint32_t *>(pieces + (long long)g * Kp + k) = hi;
    *reinterpret_cast<uint32_t *>(pieces + (long long)(nG + g) * Kp + k) = lo;
  }
  float m = fmaxf(a0, a1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) colmax[w] = m;
  __syncthreads();
  if (t < nrows) {
    float ra = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) ra = __fadd_ru(ra, rowp[q][t]);
    part_row[(long long)c * R + r0 + t] = ra;
  }
  if (t == 0) {
    float mm = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) mm = fmaxf(mm, colmax[q]);
    part_gmax[(long long)c * nG + g] = mm;
  }
}

// rowabs[r] = sum over chunks of part_row (rounded up, chunk order), gmax[g]
// = max over chunks of part_gmax; as doubles (exact).
__global__ void __launch_bounds__(256) bf16_checksum_finish_kernel(const float *__restrict__ part_row,
                                                                   const float *__restrict__ part_gmax,
                                                                   long long R, int nG, int nch,
                                                                   double *__restrict__ rowabs,
                                                                   double *__restrict__ gmax) {
  const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
  if (i < R) {
    float s = 0.f;
    for (int c = 0; c < nch; ++c) s = __fadd_ru(s, part_row[(long long)c * R + i]);
    rowabs[i] = (double)s;
  } else if (i < R + nG) {
    const int g = (int)(i - R);
    float m = 0.f;
    for (int c = 0; c < nch; ++c) m = fmaxf(m, part_gmax[(long long)c * nG + g]);
    gmax[g] = (double)m;
  }
}

// The checksum vectors and absolute sums of the plain form for one bf16
// operand X (R x Kp): pieces (2 ceil(R/128) rows of Kp bf16), rowabs (R),
// gmax (ceil(R/128)); part: device scratch of bf16_checksum_scratch floats.
long long bf16_checksum_scratch(long long R, long long Kp) {
  const long long nG = (R + 127) / 128, nch = (Kp + BF16CS_KC - 1) / BF16CS_KC;
  return nch * (R + nG);
}

cudaError_t launch_bf16_checksums(const void *X, long long R, long long Kp, void *pieces, double *rowabs,
                                  double *gmax, float *part, cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  const int nG = (int)((R + 127) / 128), nch = (int)((Kp + BF16CS_KC - 1) / BF16CS_KC);
  float *part_row = part, *part_gmax = part + (long long)nch * R;
  bf16_checksum_kernel<<<dim3((unsigned)nG, (unsigned)nch), 256, 0, s>>>(
      (const uint16_t *)X, R, Kp, (uint16_t *)pieces, part_row, part_gmax, nG);
  bf16_checksum_finish_kernel<<<(unsigned)((R + nG + 255) / 256), 256, 0, s>>>(part_row, part_gmax, R, nG, nch,
                                                                              rowabs, gmax);
  return cudaGetLastError();
}

// Row exponents (unless plain) and slices of op(X) (R x K, padded to Kp);
// i8: INT8 slices (Kp a multiple of 128) with non-finite rows marked in e.
// mb: device scratch of 12 R bytes (the row maxima, then the rows' non-finite
// flags); nsm: the SM count (sizes the k-split of the maxima pass).
cudaError_t launch_slicing(const double *X, long long ld, int trans, long long R, long long K, long long Kp, int *e,
                           int S, int w, int plain, int i8, void *out, unsigned long long *mb, int nsm,
                           cudaStream_t s) {
  if (R <= 0) return cudaSuccess;
  unsigned int *nf = reinterpret_cast<unsigned int *>(mb + R);
  if (!plain) {
    cudaError_t err = cudaMemsetAsync(mb, 0, (sizeof(unsigned long long) + sizeof(unsigned int)) * (size_t)R, s);
    if (err != cudaSuccess) return err;
    // enough warps to cover every SM several times over, k-ranges of at least 64
    const long long rows_per_block = trans ? 8 : 256, bx = (R + rows_per_block - 1) / rows_per_block;
    const long long want = (long long)nsm * 8, ksplit = std::max(1LL, std::min((K + 63) / 64, (want + bx - 1) / bx));
    const long long kper = (K + ksplit - 1) / ksplit;
    split_rowmax_kernel<<<dim3((unsigned)bx, (unsigned)((K + kper - 1) / kper)), 256, 0, s>>>(X, ld, trans, R, K,
                                                                                             kper, mb, nf);
  }
  __nv_bfloat16 *o = (__nv_bfloat16 *)out;
  if (trans) {
    dim3 grid((unsigned)((Kp + 255) / 256), (unsigned)((R + 7) / 8));
    if (plain) split_slice_kernel<1, 1><<<grid, 256, 0, s>>>(X, ld, R, K, Kp, mb, nf, e, S, w, o);
    else if (i8) split_slice_kernel<1, 0, true><<<grid, 256, 0, s>>>(X, ld, R, K, Kp, mb, nf, e, S, w, o);
    else split_slice_kernel<1, 0><<<grid, 256, 0, s>>>(X, ld, R, K, Kp, mb, nf, e, S, w, o);
  } else {
    dim3 grid((unsigned)(Kp / 64), (unsigned)((R + 31) / 32));
    if (plain) split_slice_kernel<0, 1><<<grid, 256, 0, s>>>(X, ld, R, K, Kp, mb, nf, e, S, w, o);
    else if (i8) split_slice_kernel<0, 0, true><<<grid, 256, 0, s>>>(X, ld, R, K, Kp, mb, nf, e, S, w, o);
    else split_slice_kernel<0, 0><<<grid, 256, 0, s>>>(X, ld, R, K, Kp, mb, nf, e, S, w, o);
  }
  return cudaGetLastError();
}

}  // namespace ftg
