// Integer shortcuts of the kernels against the CUDA conversions and FP64
// operations they stand in for, bit for bit, on 2^26 seeded inputs:
//   f32_ru_abs(x)        vs __double2float_ru(fabs(x))
//   bf16_rn_bits(x)      vs __double2bfloat16(x)
//   scale_pow2_int(x, e) vs scale_pow2(x, e)
//   f32_bits_to_f64(f)   vs (double)f (FP32 subnormals included)
//   f32_rn(x)            vs __double2float_rn(x)
//   scaled_exact_f32(f, sh) vs the FP64 product 2^-sh * f, for integer-valued
//                        f with |f| < 2^24 (the exact FP32 pair products) and
//                        0 <= sh < 800
// Inputs come from a counter-based hash (splitmix64) in eight families: raw
// 64-bit patterns, the FP32 exponent range, exact bf16 and FP32 halfway cases, values
// exact in FP32, values near the FP32 maximum and minimum, zeros / Inf / NaN /
// FP64 subnormals, raw FP32 patterns, integer pair products.  Prints one JSON
// line: the mismatch count of each check and the first mismatching input.
#include <cstdio>
#include <cstdint>

#include "ftgemm_split_tcp.cuh"

using namespace ftg;

constexpr int NCHECK = 6;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

__device__ void record(unsigned long long *bad, unsigned long long *first, int k, unsigned long long in) {
  atomicAdd(&bad[k], 1ull);
  atomicCAS(&first[k], 0ull, in | 1ull);
}

__global__ void check(unsigned long long n, unsigned long long *bad, unsigned long long *first) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long h = mix64(i), g = mix64(i ^ 0xA5A5A5A5A5A5A5A5ull);
    const unsigned long long mant = h & 0xFFFFFFFFFFFFFull, sign = h & 0x8000000000000000ull;
    unsigned long long b;
    switch (i & 7) {
      case 0: b = h; break;
      case 1: b = sign | ((unsigned long long)(866 + g % 316) << 52) | mant; break;  // around the FP32 range
      case 2:
        b = (g & 2) ? sign | ((unsigned long long)(850 + g % 310) << 52) | (mant & ~((1ull << 45) - 1)) | (1ull << 44)
                    : sign | ((unsigned long long)(850 + g % 310) << 52) | (mant & ~((1ull << 29) - 1)) | (1ull << 28);
        break;  // exact bf16 / FP32 halfway
      case 3: b = sign | ((unsigned long long)(896 + g % 254) << 52) | (mant & ~((1ull << 29) - 1)) | (g & 1); break;
      case 4: b = sign | ((unsigned long long)((g & 1) ? 1150 : 897) << 52) | mant; break;  // FP32 max / min
      case 5: {
        const unsigned long long sp[8] = {0ull, 0x8000000000000000ull, 0x7FF0000000000000ull, 0xFFF0000000000000ull,
                                          0x7FF8000000000001ull, 1ull, 0x000FFFFFFFFFFFFFull, 0x0010000000000000ull};
        b = (g & 8) ? (sign | (mant >> (g % 52))) : sp[g & 7];  // FP64 subnormals, specials
        break;
      }
      default: b = sign | ((unsigned long long)(g % 2048) << 52) | mant; break;
    }
    const double x = __longlong_as_double((long long)b);
    // 0: |x| rounded up to FP32
    const float u1 = f32_ru_abs(x), u2 = __double2float_ru(fabs(x));
    if (__float_as_uint(u1) != __float_as_uint(u2) && !(isnan(u1) && isnan(u2))) record(bad, first, 0, b);
    // 1: bf16 rounding
    if (bf16_rn_bits(x) != (uint32_t)__bfloat16_as_ushort(__double2bfloat16(x))) record(bad, first, 1, b);
    // 2: power-of-two scaling
    const int e = (int)(g % 2200) - 1100;
    const double s1 = scale_pow2_int(x, e), s2 = scale_pow2(x, e);
    if (dbits(s1) != dbits(s2) && !(isnan(s1) && isnan(s2))) record(bad, first, 2, b);
    // 3: FP32 -> FP64
    const uint32_t fb = (i & 3) == 3 ? ((uint32_t)h & 0x807FFFFFu) : (i & 1) ? (uint32_t)h : __float_as_uint((float)x);
    const double c1 = f32_bits_to_f64(fb), c2 = (double)__uint_as_float(fb);
    if (dbits(c1) != dbits(c2) && !(isnan(c1) && isnan(c2))) record(bad, first, 3, fb);
    // 4: 2^-sh * f for an integer-valued f, |f| < 2^24
    const float f = (float)((long long)(h % (1ull << 25)) - (1ll << 24) + 1);
    const int sh = (int)(g % 800);
    const double p1 = scaled_exact_f32(__float_as_uint(f), sh), p2 = (double)f * ldexp(1.0, -sh);
    if (dbits(p1) != dbits(p2)) record(bad, first, 4, __float_as_uint(f) | ((unsigned long long)sh << 32));
    // 5: FP32 rounding to nearest
    const float r1 = f32_rn(x), r2 = __double2float_rn(x);
    if (__float_as_uint(r1) != __float_as_uint(r2) && !(isnan(r1) && isnan(r2))) record(bad, first, 5, b);
  }
}

int main() {
  const unsigned long long n = 1ull << 26;
  unsigned long long *bad = nullptr, *first = nullptr;
  if (cudaMalloc(&bad, 2 * NCHECK * sizeof(unsigned long long)) != cudaSuccess) return 1;
  first = bad + NCHECK;
  cudaMemset(bad, 0, 2 * NCHECK * sizeof(unsigned long long));
  check<<<1024, 256>>>(n, bad, first);
  unsigned long long h[2 * NCHECK];
  if (cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
  cudaFree(bad);
  printf("{\"inputs\": %llu, \"mismatch\": {\"f32_ru_abs\": %llu, \"bf16_rn_bits\": %llu, \"scale_pow2_int\": %llu, "
         "\"f32_bits_to_f64\": %llu, \"scaled_exact_f32\": %llu, \"f32_rn\": %llu}, \"first\": [\"%llx\", \"%llx\", "
         "\"%llx\", \"%llx\", \"%llx\", \"%llx\"]}\n",
         n, h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7], h[8], h[9], h[10], h[11]);
  return 0;
}
