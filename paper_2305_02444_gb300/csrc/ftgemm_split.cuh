// Split-precision FT-GEMM on the BF16 tensor cores (mma.sync m16n8k16, FP32
// accumulation), for C = alpha * op(A) * op(B) + beta * C with FP64 inputs
// and output.
//
// Two forms share one kernel:
//  - emulated FP64 (Ozaki, Ogita, Oishi and Rump's error-free splitting): each
//    row of op(A) is scaled by a power of two sigma_i so that |x| < 1, and
//    split into S integer slices of w bits, x = sum_s n_s 2^{-w(s+1)} + r,
//    |n_s| < 2^w (exact in bf16 for w <= 8); op(B)'s columns likewise.  Every
//    kept slice pair (s, t), s + t < S, is one integer product whose FP32
//    accumulation is exact while K_chunk * (2^w - 1)^2 < 2^24; the pair's
//    FP32 tile is folded into FP64 accumulators with the pair's power-of-two
//    weight 2^{-w(s+t+2)}; out = alpha * sigma_i tau_j acc64 + beta * C.
//  - plain BF16: op(A), op(B) rounded to bf16, one pair, FP32 accumulation
//    over the whole K (the usual BF16-in / FP32-accumulate GEMM).
//
// Fault tolerance of this kernel (ft = 1): the predicted checksums are
// carried in FP32 (each slab's column sums of the A slice and row sums of the
// B slice are taken on the CUDA cores from the staged tiles, then multiplied
// into the other operand's slab), folded into FP64 with the same weights; the
// reference sums of the FP64 accumulators, the verification and the
// correction (an FP64 dot product of the original FP64 operands, or of the
// bf16 operands in the plain form) stay in FP64.  The threshold is the FP32
// rounding bound of the predicted checksums (accumulated alongside as an
// absolute-value checksum) plus the FP64 folding bound, and in the plain form
// the tensor core's FP32 accumulation bound.  The tile epilogue below
// (split_tile_finish, split_check, split_tile_recompute) also serves the
// tcgen05 kernels, which verify against checksum products computed before the
// product (CK 2).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "ftgemm_common.cuh"

namespace ftg {

// ---------------------------------------------------------------- GEMM kernel

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// The INT8 form: m16n8k32 with INT32 accumulators.  Its A and B fragments
// hold the same bytes of a 128-byte slab row as the bf16 m16n8k16 ones (32 k
// of int8 where bf16 has 16), so the same ldmatrix addresses load them.
__device__ __forceinline__ void mma_s8(int (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                       uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma_acc(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1) {
  mma_bf16(d, a0, a1, a2, a3, b0, b1);
}
__device__ __forceinline__ void mma_acc(int (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1) {
  mma_s8(d, a0, a1, a2, a3, b0, b1);
}

// bf16 element (row, k) of a [128][64] slab written by TMA with 128-byte swizzle.
__device__ __forceinline__ float slab_at(const unsigned char *slab, int row, int k) {
  const __nv_bfloat16 *p = reinterpret_cast<const __nv_bfloat16 *>(
      slab + row * 128 + ((((k >> 3) ^ (row & 7)) << 4) | ((k & 7) << 1)));
  return __bfloat162float(*p);
}

template <bool TA, bool TB>
__device__ __forceinline__ double sp_glob_a(const SplitParams &p, long long i, long long k) {
  return TA ? p.A[k + i * p.lda] : p.A[i + k * p.lda];
}
template <bool TA, bool TB>
__device__ __forceinline__ double sp_glob_b(const SplitParams &p, long long k, long long j) {
  return TB ? p.B[j + k * p.ldb] : p.B[k + j * p.ldb];
}

// x * 2^e, exactly as ldexp (one correctly rounded multiply when 2^e is a
// normal double, ldexp otherwise).
__device__ __forceinline__ double scale_pow2(double x, int e) {
  if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(x, e);
}
__device__ __forceinline__ double pow2_or_ldexp(int e) { return scale_pow2(1.0, e); }

__device__ __forceinline__ float warp_sum_ru(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_ru(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}


// FP32 accumulation bound of the plain BF16 form: the tensor core's FP32 sum
// of K exact bf16 products differs from the exact sum by at most e32(K)
// times the sum of their magnitudes.  The order and rounding inside one MMA
// are not documented; the bound assumes only blocks of two or more inputs,
// each aligned to its largest with 24 bits kept and rounded or truncated
// once, which errs by at most 2 K 2^-23 of the magnitudes (16 products of
// slack for ragged blocks).
__device__ __forceinline__ double plain_acc_bound(long long K) { return (double)(K + 16) * 0x1p-22; }

__device__ __forceinline__ double bf16_bits_to_f64(uint16_t h) {
  return (double)__uint_as_float((uint32_t)h << 16);
}

// Recompute the flagged elements of a tile: the flagged row x column
// intersections (or, with one side empty or more than 64 of them, the whole
// flagged row and column segments).  The emulated forms recompute from the
// original FP64 operands; the plain BF16 form from the bf16 operands its
// product used (p.Ab / p.Bb), in FP64, so that a corrected element is the
// form's own product without its FP32 accumulation error.  buf holds the
// tile's output (column-major 128 x 128, shared or global memory) and takes
// the recomputed values; a value that differs by more than the element bound
// counts as detected (cnt[2]) with a location record.  Warp `wid` of `nw`
// warps takes every nw-th candidate; the caller synchronises.
template <bool TA, bool TB>
__device__ __forceinline__ void split_tile_recompute(const SplitParams &p, double *buf, const int *s_fr,
                                                     const int *s_fc, int *cnt, int tile, int I, int J, int wid,
                                                     int nw, int lane) {
  const int i0 = I * SP_BM, j0 = J * SP_BN;
  const int mI = (int)min((long long)SP_BM, p.M - i0), nJt = (int)min((long long)SP_BN, p.N - j0);
  const bool use_c = p.beta != 0.0;
  const int nr = cnt[0], nc = cnt[1];
  const bool inter = nr > 0 && nc > 0 && nr * nc <= MAX_INTERSECT;
  const int ncand = inter ? nr * nc : (nr + nc > 0) ? (nr * nJt + nc * mI) : 0;
  for (int e = wid; e < ncand; e += nw) {
    int il, jl;
    if (inter) { il = s_fr[e / nc]; jl = s_fc[e % nc]; }
    else if (e < nr * nJt) { il = s_fr[e / nJt]; jl = e % nJt; }
    else { il = (e - nr * nJt) % mI; jl = s_fc[(e - nr * nJt) / mI]; }
    const long long gi = i0 + il, gj = j0 + jl;
    const bool bf = p.S == 0 && p.Ab != nullptr;
    double dot = 0.0, ab = 0.0;
    for (long long k = lane; k < p.K; k += 32) {
      const double av = bf ? bf16_bits_to_f64(p.Ab[gi * p.ldk + k]) : sp_glob_a<TA, TB>(p, gi, k);
      const double bv = bf ? bf16_bits_to_f64(p.Bb[gj * p.ldk + k]) : sp_glob_b<TA, TB>(p, k, gj);
      dot = fma(av, bv, dot);
      ab = fma(fabs(av), fabs(bv), ab);
    }
    dot = warp_sum(dot);
    ab = warp_sum(ab);
    if (lane == 0) {
      const double c = use_c ? p.C[gi + gj * p.ldc] : 0.0;
      const double nv = use_c ? fma(p.alpha, dot, p.beta * c) : p.alpha * dot;
      // the emulated value may differ from the FP64 one by the splitting error
      // (plain BF16: the input rounding) plus FP64 roundings
      double te;
      if (bf) {
        // the plain form's FP32 accumulation against the FP64 recomputation
        // from the same bf16 operands (products below the FP32 normal range
        // may be flushed: the last term)
        te = fabs(p.alpha) * ab * 1.01 * plain_acc_bound(p.K) +
             2.01 * (p.K + 4) * 0x1p-53 * (fabs(p.alpha) * ab + (use_c ? fabs(p.beta * c) : 0.0)) +
             fabs(p.alpha) * (double)(p.K + 16) * 0x1p-124;
      } else {
        const double sc = ldexp(1.0, p.eA[gi] + p.eB[gj]);
        const double split_err = (p.S > 0) ? (double)p.K * (p.S + 4) * ldexp(1.0, -p.w * p.S) * sc
                                           : 0x1p-7 * ab + 2.01 * (p.K + 2) * 0x1p-24 * ab;
        te = fabs(p.alpha) * split_err +
             2.01 * (p.K + p.npairs + 3) * 0x1p-53 * (fabs(p.alpha) * ab + (use_c ? fabs(p.beta * c) : 0.0));
      }
      const double old = buf[jl * SP_BM + il];
      if ((!isfinite(old) && isfinite(nv)) || fabs(old - nv) > te) {
        atomicAdd(&cnt[2], 1);
        const unsigned long long q = atomicAdd(&p.rep->n_loc, 1ull);
        if ((long long)q < p.loc_cap) {
          DevLoc L;
          L.row = gi; L.col = gj; L.tile = tile; L.kind = 0; L.delta = old - nv;
          p.loc[q] = L;
        }
      }
      buf[jl * SP_BM + il] = nv;
    }
  }
}

// Add a tile's counters (cnt[0] flagged rows, [1] columns, [2] detected,
// [4] unverifiable) to the call's report; one thread.
__device__ __forceinline__ void split_tile_report(const SplitParams &p, const int *cnt) {
  DevReport *r = p.rep;
  if (cnt[0]) atomicAdd(&r->flagged_rows, (unsigned long long)cnt[0]);
  if (cnt[1]) atomicAdd(&r->flagged_cols, (unsigned long long)cnt[1]);
  if (cnt[2]) {
    atomicAdd(&r->detected, (unsigned long long)cnt[2]);
    atomicAdd(&r->corrected, (unsigned long long)cnt[2]);
  }
  if (cnt[4]) atomicAdd(&r->unverifiable, (unsigned long long)cnt[4]);
}

// The threshold test of one row or column checksum: ref, the sum of the
// output; cs / ca, the sums of C and of |C| (FP32 rounded up); P, the
// predicted checksum of the product; gmax * vsum, the Hoelder bound of the
// absolute product checksum (for a column check of tile (I, J):
// max_k sum_{i in I} |a_ik| and sum_k |b_kj|); sig, the splitting-error
// scale of the emulated forms.  Returns 0 verified, 1 flagged, 2
// unverifiable.
//  - Emulated forms: FP64 roundings of the folded pair sums and the
//    epilogue, plus the splitting error of the reference (and of P when it
//    is an emulated product too, in sig).
//  - Plain BF16 form (S == 0), checksums carried in FP32: the reference's
//    FP32 accumulation errors (at most e32 H), the predicted checksum's
//    (the FP32 group sums of the bf16 operands over at most 128 rows, their
//    two-piece bf16 split within 2^-16, the FP32 accumulation of the piece
//    products; the sum of C in FP32, within (L + 1) 2^-24 of the sum of
//    |C|), the FP64 roundings, and results below the FP32 normal range
//    (flushed products; checksum pieces that lose bits there, at most 2^-134
//    per entry times the other operand).
__device__ __forceinline__ int split_check(const SplitParams &p, double ref, double cs, double ca, double P,
                                           double gmax, double vsum, double sig) {
  const bool use_c = p.beta != 0.0;
  const double pred = use_c ? fma(p.alpha, P, p.beta * cs) : p.alpha * P;
  const double S64 = gmax * vsum;
  double tau;
  if (p.S == 0) {
    const double e32 = plain_acc_bound(p.K), L = (double)SP_BM;
    tau = fabs(p.alpha) * S64 * (2.04 * e32 + 1.01 * (L + 1.0) * 0x1p-24 + 1.01 * 0x1p-16) +
          (use_c ? fabs(p.beta) * ca * 1.01 * (L + 1.0) * 0x1p-24 : 0.0) +
          2.01 * (L + 40.0) * 0x1p-53 * (fabs(p.alpha) * S64 * (1.0 + e32) + (use_c ? fabs(p.beta) * ca : 0.0)) +
          fabs(p.alpha) * ((L + 2.0) * (double)(p.K + 16) * 0x1p-124 + vsum * 0x1p-130) + (L + 40.0) * 0x1p-1021;
  } else {
    const double n = (double)(p.K + SP_BM + 3 + 32 + p.npairs);
    const double split_err = fabs(p.alpha) * sig * (double)p.K * (p.S + 4) * ldexp(1.0, -p.w * p.S);
    tau = 2.01 * n * 0x1p-53 * (fabs(p.alpha) * S64 + (use_c ? fabs(p.beta) * ca : 0.0)) + split_err +
          n * 0x1p-1021;
  }
  if (!isfinite(pred) || !isfinite(tau)) return 2;
  return fabs(ref - pred) <= tau ? 0 : 1;
}

// The predicted checksums of the product: column j of tile row I (P1) and
// row i of tile column J (P2), each the sum of two pieces in the plain
// BF16 form.
__device__ __forceinline__ double split_p1(const SplitParams &p, int I, long long gj) {
  const double *q = p.P1 + (long long)I + gj * p.ldp1;
  return p.p1_lo ? q[0] + q[p.p1_lo] : q[0];
}
__device__ __forceinline__ double split_p2(const SplitParams &p, long long gi, int J) {
  const double *q = p.P2 + gi + (long long)J * p.ldp2;
  return p.p2_lo ? q[0] + q[p.p2_lo] : q[0];
}

// The end of a tile shared by the split kernels, run by 256 threads: sC holds
// the tile's unscaled FP64 accumulators (column-major, 128 x 128); scale to
// the output, verify with the FP64 checksums (CK 2), recompute the flagged
// elements from the original operands (CK >= 1; s_fr / s_fc / cnt[0..1] hold
// the rows / columns flagged so far), report, store.  `red` is shared-memory
// scratch of SP_RED_DOUBLES doubles.  Thread t scales row t mod 128 over the
// columns of parity t / 128 (C read coalesced); with CK 2 it also takes that
// row's partial sums (output, C, |C|) and, by warp reductions, its warp's
// 32-row partial sums of each column it visits.
template <bool TA, bool TB, int CK>
__device__ __forceinline__ void split_tile_finish(const SplitParams &p, double *sC, double *red, int *s_fr,
                                                  int *s_fc, int *cnt, int tile, int I, int J) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = I * SP_BM, j0 = J * SP_BN;
  const int mI = (int)min((long long)SP_BM, p.M - i0), nJt = (int)min((long long)SP_BN, p.N - j0);
  // out = alpha * 2^(eA_i + eB_j) * acc + beta * C  (C read only if beta != 0)
  const bool use_c = p.beta != 0.0;
  const int il = tid & 127, h = tid >> 7, wq = warp & 3;
  double *colp = red;                 // [4 row quarters][128 columns][3]: output, C, |C| (FP32 ru)
  double *rowp = red + 4 * 128 * 3;   // [2 column halves][128 rows][3]
  double *sigp = rowp + 2 * 128 * 3;  // [0..3] sum of 2^eA over a row quarter, [4..5] of 2^eB over a column half
  double rref = 0.0, rcs = 0.0, sb = 0.0;
  float rca = 0.0f;
  const int eAi = il < mI ? p.eA[i0 + il] : 0;
  for (int jl = h; jl < SP_BN; jl += 2) {
    double out = 0.0, c = 0.0;
    if (il < mI && jl < nJt) {
      const long long gi = i0 + il, gj = j0 + jl;
      const int eBj = p.eB[gj];
      double v = scale_pow2(sC[jl * SP_BM + il], eAi + eBj);
      if (p.i8 && (eAi == SPLIT_NONFINITE_ROW || eBj == SPLIT_NONFINITE_ROW)) {
        // INT8 slices cannot carry Inf / NaN: a row or column with a
        // non-finite entry is multiplied in FP64 (IEEE results)
        v = 0.0;
        for (long long k = 0; k < p.K; ++k) v = fma(sp_glob_a<TA, TB>(p, gi, k), sp_glob_b<TA, TB>(p, k, gj), v);
      }
      if (use_c) c = p.C[gi + gj * p.ldc];
      out = use_c ? fma(p.alpha, v, p.beta * c) : p.alpha * v;
      sC[jl * SP_BM + il] = out;
    }
    if (CK == 2) {
      rref += out;
      rcs += c;
      const float fa = f32_ru_abs(c);
      rca = __fadd_ru(rca, fa);
      if (il == 0 && jl < nJt) sb += pow2_or_ldexp(p.eB[j0 + jl]);  // lane 0 of quarter 0: the half's 2^eB sum
      const double wr = warp_sum(out), wc = warp_sum(c);
      const float wa = warp_sum_ru(fa);
      if (lane == 0) {
        double *q = colp + (wq * 128 + jl) * 3;
        q[0] = wr;
        q[1] = wc;
        q[2] = (double)wa;
      }
    }
  }
  if (CK == 2) {
    double *q = rowp + (h * 128 + il) * 3;
    q[0] = rref;
    q[1] = rcs;
    q[2] = (double)rca;
    const double sa = warp_sum(il < mI ? pow2_or_ldexp(eAi) : 0.0);
    if (lane == 0 && h == 0) sigp[wq] = sa;
    if (il == 0) sigp[4 + h] = sb;
  }
  __syncthreads();
  if (CK == 2) {
    // FP64 checksums: reference sums of the scaled output tile against
    // alpha * (acs x op(B) or op(A) x bcs) + beta * (sums of C_in)
    const int idx = tid & 127;
    const bool col = tid < 128;
    const bool valid = col ? (idx < nJt) : (idx < mI);
    if (valid) {
      double ref, cs, ca, sig;
      if (col) {
        const double *q = colp + idx * 3;
        ref = (q[0] + q[384]) + (q[768] + q[1152]);
        cs = (q[1] + q[385]) + (q[769] + q[1153]);
        ca = (double)__fadd_ru(__fadd_ru((float)q[2], (float)q[386]), __fadd_ru((float)q[770], (float)q[1154]));
        sig = ((sigp[0] + sigp[1]) + (sigp[2] + sigp[3])) * pow2_or_ldexp(p.eB[j0 + idx]);
      } else {
        const double *q = rowp + idx * 3;
        ref = q[0] + q[384];
        cs = q[1] + q[385];
        ca = (double)__fadd_ru((float)q[2], (float)q[386]);
        sig = (sigp[4] + sigp[5]) * pow2_or_ldexp(p.eA[i0 + idx]);
      }
      const double P = col ? split_p1(p, I, j0 + idx) : split_p2(p, i0 + idx, J);
      const double gmax = col ? p.aabsmax[I] : p.babsmax[J];
      const double vsum = col ? p.bcolabs[j0 + idx] : p.arowabs[i0 + idx];
      // splitting error of the reference sum, plus that of the predicted
      // checksum when it is an emulated product as well
      if (p.ePA) sig += col ? ldexp(1.0, p.ePA[I] + p.eB[j0 + idx]) : ldexp(1.0, p.eA[i0 + idx] + p.ePB[J]);
      const int r = split_check(p, ref, cs, ca, P, gmax, vsum, sig);
      if (r == 2) atomicAdd(&cnt[4], 1);
      else if (r == 1) {
        if (col) s_fc[atomicAdd(&cnt[1], 1)] = idx;
        else s_fr[atomicAdd(&cnt[0], 1)] = idx;
      }
    }
    __syncthreads();
  }
  if (CK >= 1) {
    split_tile_recompute<TA, TB>(p, sC, s_fr, s_fc, cnt, tile, I, J, warp, 8, lane);
    __syncthreads();
    if (tid == 0) split_tile_report(p, cnt);
  }
  // store (plain coalesced stores: rows of the tile are contiguous in C)
  for (int e = tid; e < SP_BM * SP_BN; e += 256) {
    const int il = e & 127, jl = e >> 7;
    if (il < mI && jl < nJt) p.C[(long long)(i0 + il) + (long long)(j0 + jl) * p.ldc] = sC[e];
  }
}

// One CTA per 128 x 128 tile; 8 warps as 2 (rows) x 4 (columns), warp tile
// 64 x 32 = 4 x 4 mma tiles.  tmA / tmB: 3-D maps {Kp, R, S} of the slices.
// CK 0: no checks; 1: FP32 predicted checksums from the staged slices;
// 2: FP64 predicted checksums from the original operands (two skinny FP64
// GEMMs before the kernel), verified against the scaled FP64 result.
// I8: INT8 slices (w = 7; m16n8k32 s8 MMAs with exact INT32 accumulation
// over k-chunks of up to 133 120 products), 128 k per slab; CK 0 or 2.
template <bool TA, bool TB, int CK, bool I8 = false>
__global__ void __launch_bounds__(256, 1)
    ftsplit_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ SplitParams p) {
  static_assert(!I8 || CK != 1, "INT8 slices: no checks or FP64 checksums");
  constexpr int SBK = I8 ? SP_BK_I8 : SP_BK;  // k per slab (128 bytes per row either way)
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float *s_csA = reinterpret_cast<float *>(smem + SP_STAGES * SP_STAGE_BYTES);  // [2][64]: sum and abs sum
  float *s_csB = s_csA + 2 * SP_BK;
  double *s_r = reinterpret_cast<double *>(s_csB + 2 * SP_BK);  // [4][128]: reference/predicted scratch
  int *s_fr = reinterpret_cast<int *>(s_r + 4 * 128);
  int *s_fc = s_fr + 128;
  int *cnt = s_fc + 128;  // [0] nr [1] nc [2] det [3] abort [4] unverifiable
  uint64_t *bars = reinterpret_cast<uint64_t *>(cnt + 64);
  double *s_red = reinterpret_cast<double *>(bars + 2 * SP_STAGES);  // epilogue scratch
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + SP_STAGES);

  constexpr bool FT = CK == 1;  // FP32 checksum work in the mainloop
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x, I = tile % p.nI, J = tile / p.nI;
  const int i0 = I * SP_BM, j0 = J * SP_BN;
  const int mI = (int)min((long long)SP_BM, p.M - i0), nJt = (int)min((long long)SP_BN, p.N - j0);
  const int wm = warp >> 2, wn = warp & 3;  // warp tile rows wm*64.., cols wn*32..
  const int g = lane >> 2, t4 = lane & 3;
  int *err = &p.rep->err;
  const unsigned long long limit = p.wait_limit_ns;

  if (tid == 0) {
    for (int c = 0; c < 8; ++c) cnt[c] = 0;
    for (int s = 0; s < SP_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 8);
    }
    fence_mbar_init();
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  __syncthreads();

  // work list: (pair q, k-chunk c, slab b) in the order pairs x chunks x slabs
  const int nslab_total = (int)(p.Kp / SBK);
  const int chunk_slabs = max(1, p.kchunk / SBK);
  const int nchunks = (nslab_total + chunk_slabs - 1) / chunk_slabs;
  const int nsteps = p.npairs * nslab_total;  // every pair sweeps all slabs once
  auto step_coords = [&](int step, int &pq, int &slab) {
    pq = step / nslab_total;
    slab = step % nslab_total;
  };
  auto issue = [&](int step) {
    int pq, slab;
    step_coords(step, pq, slab);
    const int st = step % SP_STAGES;
    const uint32_t sb = smem_u32(smem + st * SP_STAGE_BYTES);
    const uint32_t fb = full0 + 8 * st;
    mbar_arrive_expect_tx(fb, SP_STAGE_BYTES);
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(sb),
        "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(fb), "r"(slab * SBK), "r"(i0), "r"(p.pair_s[pq])
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(sb + SP_A_BYTES),
        "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(fb), "r"(slab * SBK), "r"(j0), "r"(p.pair_t[pq])
        : "memory");
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < SP_STAGES && issued < nsteps; ++issued) issue(issued);

  using Acc = typename std::conditional<I8, int, float>::type;  // exact pair sums: INT32 or FP32
  Acc acc32[4][4][4];
  double acc64[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) { acc32[a][b][c] = 0; acc64[a][b][c] = 0.0; }
  float cs32 = 0.f, ca32 = 0.f;     // FT: this pair-chunk's predicted checksum (t < 128: column, else row)
  double cs64 = 0.0, ca64 = 0.0;    // folded predicted checksum and its absolute bound
  int fptr = 0, fend = 0;
  if (CK >= 1 && p.inj) { fptr = p.tile_off[tile]; fend = p.tile_off[tile + 1]; }

  bool ok = true;
  for (int step = 0; step < nsteps; ++step) {
    int pq, slab;
    step_coords(step, pq, slab);
    const int st = step % SP_STAGES;
    if (ok && !mbar_wait_bounded(full0 + 8 * st, (step / SP_STAGES) & 1, limit, err)) ok = false;
    if (ok) {
      const unsigned char *sA = smem + st * SP_STAGE_BYTES, *sB = sA + SP_A_BYTES;
      const uint32_t aA = smem_u32(sA), aB = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < SP_BK / 16; ++kk) {
        uint32_t af[4][4], bf[4][2];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
          const int r = wm * 64 + mt * 16 + (lane & 15), c = kk * 2 + (lane >> 4);
          ldsm_x4(aA + r * 128 + ((c ^ (r & 7)) << 4), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
        }
#pragma unroll
        for (int np = 0; np < 2; ++np) {
          const int q = lane >> 3;
          const int r = wn * 32 + np * 16 + (q >> 1) * 8 + (lane & 7), c = kk * 2 + (q & 1);
          ldsm_x4(aB + r * 128 + ((c ^ (r & 7)) << 4), bf[2 * np][0], bf[2 * np][1], bf[2 * np + 1][0],
                  bf[2 * np + 1][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
            mma_acc(acc32[mt][nt], af[mt][0], af[mt][1], af[mt][2], af[mt][3], bf[nt][0], bf[nt][1]);
      }
    }  // ok
    if (FT) {
      // slab checksums of the staged slices on the CUDA cores: column sums of
      // the A slice over the tile's rows and row sums of the B slice over the
      // tile's columns (signed and absolute, exact in FP32), then the predicted
      // checksum FMAs.  The barriers run in every thread, stalled or not.
      const unsigned char *sA = smem + st * SP_STAGE_BYTES, *sB = sA + SP_A_BYTES;
      float *tmp = reinterpret_cast<float *>(s_r);  // [4 parts][4 kinds][64]
      const int k = tid & 63, part = tid >> 6;
      if (ok) {
        float sa = 0.f, saa = 0.f, sb = 0.f, sba = 0.f;
        for (int r = part * 32; r < part * 32 + 32; ++r) {
          const float av = slab_at(sA, r, k), bv = slab_at(sB, r, k);
          sa += av; saa += fabsf(av);
          sb += bv; sba += fabsf(bv);
        }
        tmp[(part * 4 + 0) * 64 + k] = sa;
        tmp[(part * 4 + 1) * 64 + k] = saa;
        tmp[(part * 4 + 2) * 64 + k] = sb;
        tmp[(part * 4 + 3) * 64 + k] = sba;
      }
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (ok && tid < 4 * SP_BK) {
        const int kind = tid >> 6;  // 0 A sum, 1 A abs, 2 B sum, 3 B abs
        const float v = (tmp[(0 * 4 + kind) * 64 + k] + tmp[(1 * 4 + kind) * 64 + k]) +
                        (tmp[(2 * 4 + kind) * 64 + k] + tmp[(3 * 4 + kind) * 64 + k]);
        if (kind < 2) s_csA[kind * SP_BK + k] = v; else s_csB[(kind - 2) * SP_BK + k] = v;
      }
      asm volatile("bar.sync 2, 256;" ::: "memory");
      if (ok) {
        if (tid < 128) {
#pragma unroll 8
          for (int kk = 0; kk < SP_BK; ++kk) {
            const float bv = slab_at(sB, tid, kk);
            cs32 = fmaf(s_csA[kk], bv, cs32);
            ca32 = fmaf(s_csA[SP_BK + kk], fabsf(bv), ca32);
          }
        } else {
#pragma unroll 8
          for (int kk = 0; kk < SP_BK; ++kk) {
            const float av = slab_at(sA, tid - 128, kk);
            cs32 = fmaf(av, s_csB[kk], cs32);
            ca32 = fmaf(fabsf(av), s_csB[SP_BK + kk], ca32);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0 && ok) mbar_arrive(empty0 + 8 * st);
    if (tid == 0 && ok && step >= 1 && issued < nsteps) {
      const int sp = step - 1;
      if (!mbar_wait_bounded(empty0 + 8 * (sp % SP_STAGES), (sp / SP_STAGES) & 1, limit, err)) ok = false;
      else issue(issued++);
    }
    // end of a k-chunk (or of the pair): fold the exact FP32 tile into FP64
    const bool chunk_end = ((slab + 1) % chunk_slabs == 0) || (slab + 1 == nslab_total);
    if (chunk_end) {
      const double wgt = ldexp(1.0, -p.w * (p.pair_s[pq] + p.pair_t[pq] + 2));
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            acc64[a][b][c] = fma(wgt, (double)acc32[a][b][c], acc64[a][b][c]);
            acc32[a][b][c] = 0;
          }
      if (FT) {
        cs64 = fma(wgt, (double)cs32, cs64);
        ca64 = fma(wgt, (double)ca32, ca64);
        cs32 = 0.f;
        ca32 = 0.f;
      }
      if (CK >= 1 && p.inj && slab + 1 == nslab_total) {
        // injection point: after pair pq has been folded in (kstep = pair index)
        while (fptr < fend) {
          DevFlip *f = p.flips + fptr;
          if (f->kstep != pq) break;
          const int il = (int)(f->row - i0), jl = (int)(f->col - j0);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int ri = wm * 64 + a * 16 + g + ((c >> 1) << 3), cj = wn * 32 + b * 8 + 2 * t4 + (c & 1);
                if (ri == il && cj == jl) {
                  const double before = acc64[a][b][c];
                  acc64[a][b][c] = flip_bit(before, f->bit);
                  f->before = before;
                  f->after = acc64[a][b][c];
                  f->applied = 1;
                  f->kfirst = 0;
                }
              }
          ++fptr;
        }
      }
    }
  }
  (void)nchunks;
  if (!ok) {
    atomicExch(&cnt[3], 1);
    if (tid == 0)
      for (int s = issued > SP_STAGES ? issued - SP_STAGES : 0; s < issued; ++s)
        mbar_wait_bounded(full0 + 8 * (s % SP_STAGES), (s / SP_STAGES) & 1, limit, err);
  }
  __syncthreads();
  if (cnt[3]) return;

  // ------------------------------------------------------------- epilogue
  // acc64 (unscaled: sum of the kept pairs) -> staged tile sC (column-major [128][128] doubles)
  double *sC = reinterpret_cast<double *>(smem);  // 128 KiB: the ring is free
  fence_proxy_async_smem();
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ri = wm * 64 + a * 16 + g + ((c >> 1) << 3), cj = wn * 32 + b * 8 + 2 * t4 + (c & 1);
        sC[cj * SP_BM + ri] = acc64[a][b][c];
      }
  __syncthreads();
  if (FT) {
    // reference sums of the accumulators, one per thread: column (tid < 128) or row
    double ref = 0.0;
    if (tid < 128) {
      for (int i = 0; i < SP_BM; ++i) ref += sC[tid * SP_BM + i];
    } else {
      for (int j = 0; j < SP_BN; ++j) ref += sC[j * SP_BM + tid - 128];
    }
    // the predicted checksum carries the FP32 rounding of up to kchunk products
    // per pair-chunk (CUDA-core FMAs, rounded to nearest); the accumulators
    // carry one FP64 rounding per fold, and in the plain BF16 form also the
    // tensor core's FP32 accumulation over the whole K (plain_acc_bound)
    const double u32 = 0x1p-24, u64 = 0x1p-53;
    const double n32 = (double)(min((long long)p.kchunk, p.Kp) + 128 + 2);
    const double nfold = (double)(p.npairs * ((p.Kp + p.kchunk - 1) / p.kchunk) + 128 + 2);
    const double ref32 = p.S == 0 ? 1.01 * plain_acc_bound(p.K) : 2.01 * n32 * u32;
    const double tau = (2.01 * n32 * u32 + ref32) * ca64 + 2.01 * nfold * u64 * ca64 + 0x1p-1000;
    const int idx = tid & 127;
    const bool valid = (tid < 128) ? (idx < nJt) : (idx < mI);
    if (valid) {
      if (!isfinite(cs64) || !isfinite(tau)) atomicAdd(&cnt[4], 1);
      else if (!(fabs(ref - cs64) <= tau)) {
        if (tid < 128) s_fc[atomicAdd(&cnt[1], 1)] = idx;
        else s_fr[atomicAdd(&cnt[0], 1)] = idx;
      }
    }
  }
  __syncthreads();
  split_tile_finish<TA, TB, CK>(p, sC, s_red, s_fr, s_fc, cnt, tile, I, J);
}

}  // namespace ftg
