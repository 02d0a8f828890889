// Persistent form of the tcgen05 split-precision kernel: one CTA per SM walks
// a sequence of output tiles, so that the loads and MMAs of the next tile run
// while the current one is being finished, and a tile is finished from
// tensor memory instead of being staged in shared memory.
//
// Roles as in ftsplit_tc_kernel (warp 0 TMA producer, warp 1 MMA issuer,
// warp 2 tensor-memory allocation, warp 3 waiter, warps 4-7 folders).  Every
// role walks the same sequence of (tile, pair, k-chunk, slab) with running
// step and item counters, so the ring and the two FP32 accumulators pass from
// one tile to the next without a pause.  The folders fold each pair into the
// FP64 accumulators (tensor-memory columns 256..511) and then finish the tile
// themselves, thread = tile row (a warp's 32 lanes are 32 consecutive rows of
// one column of C: coalesced):
//   CK 0: out = alpha 2^(eA_i + eB_j) acc + beta C, stored in one pass;
//   CK 2: pass 1 computes out with the row and column sums of out and C,
//         writing out back into the FP64 accumulator columns; the sums are
//         verified against the predicted checksums; pass 2 stores out.  A
//         tile with flagged rows or columns goes through the CTA's slice of
//         a global scratch buffer instead, where its flagged elements are
//         recomputed before the copy to C.
// The column sums use a transposing butterfly over the warp (15 shuffled adds
// per 16 columns, then one more: each lane ends with one column's sum), not a
// full shuffle reduction per column (5 adds per column): GB300's FP64 pipe
// (2 DFMA per clock per SM) is its scarcest unit, and for the same reason the
// scaling by 2^(eA_i + eB_j) adds to the exponent field with integer
// operations whenever the result is a normal number (exact, the same bits as
// the multiply).
// The plain BF16 form (one pair, one k-chunk) skips the fold and finishes the
// tile from its FP32 accumulator.
// Output bits equal those of ftsplit_tc_kernel and ftsplit_kernel: the same
// fold order and FP64 operations per element; only the order of the checksum
// sums differs, which the rounding bound of the verification covers.
// Every wait is bounded; the folders agree on each accumulator wait through a
// barrier that carries the OR of their timeouts, so that they stop together.
#pragma once

#include "ftgemm_split_tc.cuh"

namespace ftg {

#ifndef FTG_TCP_STAGES
#define FTG_TCP_STAGES 6  // ring depth: 6 x 32 KiB leaves room for the column sums
#endif
constexpr int TCP_STAGES = FTG_TCP_STAGES;
constexpr int TCP_FOLD_BAR = 4;  // named barrier of the four folder warps
// after the ring: column sums of out and C per row quarter ([4][128] doubles
// each), of |C| ([4][128] floats), sums of 2^eA and 2^eB per quarter (8
// doubles), flagged rows and columns, counters, barriers, the tensor-memory
// address
constexpr int TCP_SMEM_BYTES = TCP_STAGES * SP_STAGE_BYTES + 2 * 4 * 128 * 8 + 4 * 128 * 4 + 8 * 8 +
                               2 * 128 * 4 + 64 * 4 + (2 * TCP_STAGES + 5) * 8 + 16 + 1024;
static_assert(TCP_SMEM_BYTES <= 232448, "shared memory per CTA");

// x * 2^e with the same result as scale_pow2: an add to the exponent field
// when x and the result are normal numbers, the multiply otherwise.
__device__ __forceinline__ double scale_pow2_int(double x, int e) {
  const uint32_t hi = tc_hi(x);
  const int ex = (int)((hi >> 20) & 0x7FFu);
  if (ex != 0 && ex != 0x7FF && ex + e >= 1 && ex + e <= 2046) return tc_pack_f64(tc_lo(x), hi + ((uint32_t)e << 20));
  return scale_pow2(x, e);
}

// The FP64 value of an FP32 number: field moves for normal numbers, the
// conversion otherwise.
__device__ __forceinline__ double f32_bits_to_f64(uint32_t fb) {
  const uint32_t ef = (fb >> 23) & 0xFFu;
  if (ef != 0 && ef != 0xFF) return scaled_exact_f32(fb, 0);
  return (double)__uint_as_float(fb);
}

// The same for FP32 values, rounded to nearest (the plain form's C sums).
__device__ __forceinline__ float colsum16_rn(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o], keep = up ? v[i + o] : v[i];
      v[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
    }
  }
  return __fadd_rn(v[0], __shfl_xor_sync(0xffffffffu, v[0], 16));
}

// The same with FP32 adds rounded upward (the |C| sums of the threshold).
__device__ __forceinline__ float colsum16_ru(float (&v)[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o], keep = up ? v[i + o] : v[i];
      v[i] = __fadd_ru(keep, __shfl_xor_sync(0xffffffffu, send, o));
    }
  }
  return __fadd_ru(v[0], __shfl_xor_sync(0xffffffffu, v[0], 16));
}

// The folder warps' work on one tile (4 warps, thread = tile row fw*32 +
// lane): fold each pair (k-chunk) of the tile into the FP64 accumulators as
// the MMAs finish it, inject, then finish the tile (see the file comment).
// `item` is the running accumulator-item counter; acce0 is the address of
// the accumulator-release barriers.  Returns false when a wait gave up; the
// four folder warps agree on it.
template <bool TA, bool TB, int CK>
__device__ __forceinline__ bool tcp_folder_tile(const SplitParams &p, int I, int J, int &item, uint32_t tbase,
                                                uint32_t accf0, uint32_t acce0, double *s_co, double *s_cc,
                                                float *s_ca, double *s_sig, int *s_fr, int *s_fc, int *cnt,
                                                int nchunks, int fw, int lane) {
  const int il = fw * 32 + lane;
  const uint32_t trow = tbase + ((uint32_t)(fw * 32) << 16);
  const uint32_t t64 = trow + TC_ACC64_COL;
  const bool use_c = p.beta != 0.0;
  const bool direct = p.S == 0;  // plain BF16: one pair, one chunk, no fold
  int *err = &p.rep->err;
  const unsigned long long limit = p.wait_limit_ns;
  bool ok = true;
  const int tile = I + J * p.nI;  // injection and location records number tiles column-major
  const int i0 = I * SP_BM, j0 = J * SP_BN;
  const int mI = (int)min((long long)SP_BM, p.M - i0), nJt = (int)min((long long)SP_BN, p.N - j0);
  int fptr = 0, fend = 0;
  if (CK >= 1 && p.inj) { fptr = p.tile_off[tile]; fend = p.tile_off[tile + 1]; }
  int blast = 0;
  for (int pq = 0; pq < p.npairs && ok; ++pq) {
    const int sh = p.w * (p.pair_s[pq] + p.pair_t[pq] + 2);  // the pair's weight is 2^-sh
    for (int c = 0; c < nchunks; ++c, ++item) {
      const int b = item & 1;
      blast = b;
      int got = 1;
      if (lane == 0) got = mbar_wait_bounded(accf0 + 8 * b, (item >> 1) & 1, limit, err) ? 1 : 0;
      got = __shfl_sync(0xffffffffu, got, 0);
      if (bar_red_or(TCP_FOLD_BAR, 128, got == 0)) { ok = false; break; }
      tc_fence_after();
      if (direct) continue;  // finished from the FP32 accumulator below
      const bool first = pq == 0 && c == 0;
#pragma unroll 1
      for (int ch = 0; ch < SP_BN / 32; ++ch) {
        uint32_t f[32], d[64];
        tmem_ld_x32(trow + (uint32_t)(b * SP_BN + ch * 32), f);
        if (first) {
#pragma unroll
          for (int j = 0; j < 64; ++j) d[j] = 0u;
        } else {
          tmem_ld_x64(t64 + (uint32_t)(ch * 64), d);
        }
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const double a = tc_pack_f64(d[2 * j], d[2 * j + 1]) + scaled_exact_f32(f[j], sh);
          d[2 * j] = tc_lo(a);
          d[2 * j + 1] = tc_hi(a);
        }
        tmem_st_x64(t64 + (uint32_t)(ch * 64), d);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * b);
    }
    if (!ok) break;
    if (CK >= 1 && p.inj && !direct) {
      // injection point: after pair pq has been folded in (kstep = pair index)
      while (fptr < fend) {
        DevFlip *f = p.flips + fptr;
        if (f->kstep != pq) break;
        const int fr = (int)(f->row - i0), fc = (int)(f->col - j0);
        if ((fr >> 5) == fw) {
          uint32_t v[2];
          tmem_ld_x2(t64 + (uint32_t)(2 * fc), v);
          if (lane == (fr & 31)) {
            const double before = tc_pack_f64(v[0], v[1]);
            const double after = flip_bit(before, f->bit);
            v[0] = tc_lo(after);
            v[1] = tc_hi(after);
            f->before = before;
            f->after = after;
            f->applied = 1;
            f->kfirst = 0;
          }
          tmem_st_x2(t64 + (uint32_t)(2 * fc), v);
        }
        ++fptr;
      }
    }
  }
  if (!ok) return false;

  // ------------------------------------------------------------ end of the tile
  const bool rowok = il < mI;
  const long long gi = i0 + il;
  const int eAi = rowok ? p.eA[gi] : 0;
  double *crow = p.C + gi;  // C(gi, j0 + col) = crow[(j0 + col) * ldc]
  // CK 2: the verification's inputs (predicted checksums of this thread's
  // column il and row il, in one or two pieces, and the absolute sums of
  // their thresholds), loaded now so that their latency passes under pass 1
  double v_p1a = 0.0, v_p1b = 0.0, v_p2a = 0.0, v_p2b = 0.0, v_amax = 0.0, v_bsum = 0.0, v_bmax = 0.0,
         v_asum = 0.0;
  if (CK == 2) {
    if (il < nJt) {
      const double *q = p.P1 + (long long)I + (long long)(j0 + il) * p.ldp1;
      v_p1a = q[0];
      if (p.p1_lo) v_p1b = q[p.p1_lo];
      v_amax = p.aabsmax[I];
      v_bsum = p.bcolabs[j0 + il];
    }
    if (rowok) {
      const double *q = p.P2 + gi + (long long)J * p.ldp2;
      v_p2a = q[0];
      if (p.p2_lo) v_p2b = q[p.p2_lo];
      v_bmax = p.babsmax[J];
      v_asum = p.arowabs[gi];
    }
  }
  if (CK == 0) {
#pragma unroll 1
    for (int ch = 0; ch < SP_BN / 32; ++ch) {
      double acc[32], cv[32];
      if (direct) {
        uint32_t f[32];
        tmem_ld_x32(trow + (uint32_t)(blast * SP_BN + ch * 32), f);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = f32_bits_to_f64(f[j]);
      } else {
        uint32_t d[64];
        tmem_ld_x64(t64 + (uint32_t)(ch * 64), d);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = tc_pack_f64(d[2 * j], d[2 * j + 1]);
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = ch * 32 + j;
        cv[j] = (use_c && rowok && col < nJt) ? crow[(long long)(j0 + col) * p.ldc] : 0.0;
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = ch * 32 + j;
        if (rowok && col < nJt) {
          const double v = direct ? acc[j] : scale_pow2_int(acc[j], eAi + __ldg(p.eB + j0 + col));
          crow[(long long)(j0 + col) * p.ldc] = use_c ? fma(p.alpha, v, p.beta * cv[j]) : p.alpha * v;
        }
      }
    }
    if (direct) {
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * blast);
    }
    return true;
  }

  // CK 2, pass 1: out, written back over the FP64 accumulators, and the sums.
  // The plain BF16 form reads its FP32 accumulator instead (converted
  // exactly; an injected fault flips a bit of that FP64 value, its only pair
  // being k-step 0), writes out into the unused FP64 columns and then
  // releases the accumulator to the next tile's MMAs; its C-side sums are
  // FP32 like the rest of its predicted checksums (the reference sums of out
  // stay FP64).  The next chunk's C is loaded while the current one is
  // summed.
  double rs0 = 0.0, rs1 = 0.0, rc0 = 0.0, rc1 = 0.0;  // row sums of out and C over even / odd columns
  float rf0 = 0.0f, rf1 = 0.0f;                       // plain form: row sums of C in FP32
  float ra0 = 0.0f, ra1 = 0.0f;                       // and of |C| (rounded up)
  const bool tile_faults = direct && CK >= 1 && p.inj && fptr < fend;
  const bool beta1 = p.beta == 1.0;
  double cn[16];
  auto load_c = [&](int ch, double (&dst)[16]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = ch * 16 + j;
      dst[j] = (use_c && rowok && col < nJt) ? crow[(long long)(j0 + col) * p.ldc] : 0.0;
    }
  };
  load_c(0, cn);
#pragma unroll 1
  for (int ch = 0; ch < SP_BN / 16; ++ch) {
    double cv[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) cv[j] = cn[j];
    if (ch + 1 < SP_BN / 16) load_c(ch + 1, cn);
    uint32_t d[32];
    if (direct) {
      uint32_t f[16];
      tmem_ld_x16(trow + (uint32_t)(blast * SP_BN + ch * 16), f);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const double v = f32_bits_to_f64(f[j]);
        d[2 * j] = tc_lo(v);
        d[2 * j + 1] = tc_hi(v);
      }
      if (tile_faults) {
        for (int q = fptr; q < fend; ++q) {
          DevFlip *fl = p.flips + q;
          const int fc = (int)(fl->col - j0) - ch * 16;
          if ((int)(fl->row - i0) != il || fc < 0 || fc >= 16) continue;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j == fc) {
              const double before = tc_pack_f64(d[2 * j], d[2 * j + 1]);
              const double after = flip_bit(before, fl->bit);
              d[2 * j] = tc_lo(after);
              d[2 * j + 1] = tc_hi(after);
              fl->before = before;
              fl->after = after;
              fl->applied = 1;
              fl->kfirst = 0;
            }
        }
      }
    } else {
      tmem_ld_x32(t64 + (uint32_t)(ch * 32), d);
    }
    double bc[16], ov[16];  // beta C (C itself when beta is 1: the same values)
    if (beta1) {
#pragma unroll
      for (int j = 0; j < 16; ++j) bc[j] = cv[j];
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) bc[j] = p.beta * cv[j];
    }
    float av[16], cf[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = ch * 16 + j;
      double o = 0.0;
      if (rowok && col < nJt) {
        const double a = tc_pack_f64(d[2 * j], d[2 * j + 1]);
        const double v = direct ? a : scale_pow2_int(a, eAi + __ldg(p.eB + j0 + col));
        o = use_c ? fma(p.alpha, v, bc[j]) : p.alpha * v;
      }
      ov[j] = o;
      d[2 * j] = tc_lo(o);
      d[2 * j + 1] = tc_hi(o);
      av[j] = f32_ru_abs(cv[j]);
      if (j & 1) { rs1 += o; ra1 = __fadd_ru(ra1, av[j]); }
      else { rs0 += o; ra0 = __fadd_ru(ra0, av[j]); }
    }
    if (direct) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        cf[j] = f32_rn(cv[j]);
        if (j & 1) rf1 = __fadd_rn(rf1, cf[j]);
        else rf0 = __fadd_rn(rf0, cf[j]);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j & 1) rc1 += cv[j];
        else rc0 += cv[j];
      }
    }
    tmem_st_x32(t64 + (uint32_t)(ch * 32), d);
    if (direct && ch + 1 == SP_BN / 16) {  // the FP32 accumulator is read: the next tile's MMAs may reuse it
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(acce0 + 8 * blast);
    }
    const double so = colsum16(ov, lane);
    const double sc = direct ? (double)colsum16_rn(cf, lane) : colsum16(cv, lane);
    const float sa = colsum16_ru(av, lane);
    if (lane < 16) {
      s_co[fw * 128 + ch * 16 + lane] = so;
      s_cc[fw * 128 + ch * 16 + lane] = sc;
      s_ca[fw * 128 + ch * 16 + lane] = sa;
    }
  }
  if (direct) {
    rc0 = (double)rf0;
    rc1 = (double)rf1;
  } else {  // the splitting-error scales of the emulated forms
    const double sa = warp_sum(rowok ? pow2_or_ldexp(eAi) : 0.0);
    const double sb = warp_sum(il < nJt ? pow2_or_ldexp(p.eB[j0 + il]) : 0.0);
    if (lane == 0) { s_sig[fw] = sa; s_sig[4 + fw] = sb; }
  }
  asm volatile("bar.sync %0, 128;" ::"r"(TCP_FOLD_BAR) : "memory");
  // verification: thread il takes column il and row il
  if (il < nJt) {
    const long long gj = j0 + il;
    const double ref = (s_co[il] + s_co[128 + il]) + (s_co[256 + il] + s_co[384 + il]);
    const double cs = (s_cc[il] + s_cc[128 + il]) + (s_cc[256 + il] + s_cc[384 + il]);
    const double ca = (double)__fadd_ru(__fadd_ru(s_ca[il], s_ca[128 + il]), __fadd_ru(s_ca[256 + il], s_ca[384 + il]));
    double sig = direct ? 0.0 : ((s_sig[0] + s_sig[1]) + (s_sig[2] + s_sig[3])) * pow2_or_ldexp(p.eB[gj]);
    if (p.ePA) sig += ldexp(1.0, p.ePA[I] + p.eB[gj]);
    const int r = split_check(p, ref, cs, ca, p.p1_lo ? v_p1a + v_p1b : v_p1a, v_amax, v_bsum, sig);
    if (r == 2) atomicAdd(&cnt[4], 1);
    else if (r == 1) s_fc[atomicAdd(&cnt[1], 1)] = il;
  }
  if (rowok) {
    double sig = direct ? 0.0 : ((s_sig[4] + s_sig[5]) + (s_sig[6] + s_sig[7])) * pow2_or_ldexp(eAi);
    if (p.ePA) sig += ldexp(1.0, eAi + p.ePB[J]);
    const int r = split_check(p, rs0 + rs1, rc0 + rc1, (double)__fadd_ru(ra0, ra1),
                              p.p2_lo ? v_p2a + v_p2b : v_p2a, v_bmax, v_asum, sig);
    if (r == 2) atomicAdd(&cnt[4], 1);
    else if (r == 1) s_fr[atomicAdd(&cnt[0], 1)] = il;
  }
  asm volatile("bar.sync %0, 128;" ::"r"(TCP_FOLD_BAR) : "memory");
  if (cnt[0] + cnt[1] == 0) {
    // pass 2: store
#pragma unroll 1
    for (int ch = 0; ch < SP_BN / 32; ++ch) {
      uint32_t d[64];
      tmem_ld_x64(t64 + (uint32_t)(ch * 64), d);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = ch * 32 + j;
        if (rowok && col < nJt) crow[(long long)(j0 + col) * p.ldc] = tc_pack_f64(d[2 * j], d[2 * j + 1]);
      }
    }
  } else {
    // flagged rows or columns: recompute in the CTA's scratch tile, then copy
    double *buf = p.tscratch + (size_t)blockIdx.x * (SP_BM * SP_BN);
#pragma unroll 1
    for (int ch = 0; ch < SP_BN / 32; ++ch) {
      uint32_t d[64];
      tmem_ld_x64(t64 + (uint32_t)(ch * 64), d);
#pragma unroll
      for (int j = 0; j < 32; ++j) buf[(ch * 32 + j) * SP_BM + il] = tc_pack_f64(d[2 * j], d[2 * j + 1]);
    }
    asm volatile("bar.sync %0, 128;" ::"r"(TCP_FOLD_BAR) : "memory");
    split_tile_recompute<TA, TB>(p, buf, s_fr, s_fc, cnt, tile, I, J, fw, 4, lane);
    asm volatile("bar.sync %0, 128;" ::"r"(TCP_FOLD_BAR) : "memory");
    if (rowok)
      for (int col = 0; col < nJt; ++col) crow[(long long)(j0 + col) * p.ldc] = buf[col * SP_BM + il];
  }
  asm volatile("bar.sync %0, 128;" ::"r"(TCP_FOLD_BAR) : "memory");
  if (il == 0) {
    split_tile_report(p, cnt);
    cnt[0] = cnt[1] = cnt[2] = cnt[4] = 0;
  }
  return true;
}

template <bool TA, bool TB, int CK>
__global__ void __launch_bounds__(256, 1)
    ftsplit_tcp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ SplitParams p) {
  static_assert(CK == 0 || CK == 2, "no checks, or checks against the checksum products P1 / P2");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  double *s_co = reinterpret_cast<double *>(smem + TCP_STAGES * SP_STAGE_BYTES);  // [4][128] column sums of out
  double *s_cc = s_co + 4 * 128;                                                 // [4][128] of C
  float *s_ca = reinterpret_cast<float *>(s_cc + 4 * 128);                       // [4][128] of |C|
  double *s_sig = reinterpret_cast<double *>(s_ca + 4 * 128);  // [0..3] 2^eA, [4..7] 2^eB per quarter
  int *s_fr = reinterpret_cast<int *>(s_sig + 8);
  int *s_fc = s_fr + 128;
  int *cnt = s_fc + 128;  // [0] nr [1] nc [2] det [3] abort [4] unverifiable
  uint64_t *bars = reinterpret_cast<uint64_t *>(cnt + 64);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 2 * TCP_STAGES + 5);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * TCP_STAGES;
  const uint32_t accf0 = empty0 + 8 * TCP_STAGES, acce0 = accf0 + 16, done_bar = acce0 + 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = p.nI * p.nJ;
  // tile n of the grouped rasterization (the order of ftsplit_tc_kernel's CTAs)
  auto tile_coords = [&](int n, int &I, int &J) {
    const int per = TC_GROUP * p.nJ, g = n / per, r = n % per;
    const int rows = min(TC_GROUP, p.nI - g * TC_GROUP);
    I = g * TC_GROUP + r % rows;
    J = r / rows;
  };
  int *err = &p.rep->err;
  const unsigned long long limit = p.wait_limit_ns;

  if (tid == 0) {
    for (int c = 0; c < 8; ++c) cnt[c] = 0;
    for (int s = 0; s < TCP_STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);
    }
    mbar_init(done_bar, 1);
    fence_mbar_init();
    prefetch_tmap(&tmA);
    prefetch_tmap(&tmB);
  }
  if (warp == 2) {
    tmem_alloc(smem_u32(s_tmem), TC_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *s_tmem;

  const int nslab = (int)(p.Kp / SP_BK);
  const int chunk_slabs = max(1, p.kchunk / SP_BK);
  const int nchunks = (nslab + chunk_slabs - 1) / chunk_slabs;
  const int nsteps = p.npairs * nslab;  // per tile

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      bool ok = true;
      int step = 0;
      for (int n = blockIdx.x; n < ntiles && ok; n += gridDim.x) {
        int I, J;
        tile_coords(n, I, J);
        const int i0 = I * SP_BM, j0 = J * SP_BN;
        for (int s = 0; s < nsteps; ++s, ++step) {
          const int pq = s / nslab, slab = s % nslab, st = step % TCP_STAGES;
          if (step >= TCP_STAGES &&
              !mbar_wait_bounded(empty0 + 8 * st, ((step / TCP_STAGES) - 1) & 1, limit, err)) {
            ok = false;
            break;
          }
          if (*(volatile int *)&cnt[3]) { ok = false; break; }
          const uint32_t sb = smem_u32(smem + st * SP_STAGE_BYTES), fb = full0 + 8 * st;
          mbar_arrive_expect_tx(fb, SP_STAGE_BYTES);
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(sb),
              "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(fb), "r"(slab * SP_BK), "r"(i0), "r"(p.pair_s[pq])
              : "memory");
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
              " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(sb + SP_A_BYTES),
              "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(fb), "r"(slab * SP_BK), "r"(j0), "r"(p.pair_t[pq])
              : "memory");
        }
      }
      if (!ok) atomicExch(&cnt[3], 1);
      // the last loads in flight land before the CTA may leave (bounded)
      for (int n = step > TCP_STAGES ? step - TCP_STAGES : 0; n < step; ++n)
        mbar_wait_bounded(full0 + 8 * (n % TCP_STAGES), (n / TCP_STAGES) & 1, limit, err);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    int step = 0, item = 0;
    bool stop = false;
    for (int n = blockIdx.x; n < ntiles && !stop; n += gridDim.x) {
      for (int pq = 0; pq < p.npairs && !stop; ++pq) {
        for (int c = 0; c < nchunks && !stop; ++c, ++item) {
          const int b = item & 1;
          const uint32_t dt = tbase + (uint32_t)(b * SP_BN);
          const int s0 = c * chunk_slabs, s1 = min(nslab, s0 + chunk_slabs);
          for (int slab = s0; slab < s1; ++slab, ++step) {
            if (bar_red_or(TC_HANDOFF_BAR, 64, false)) { stop = true; break; }
            tc_fence_after();
            const int st = step % TCP_STAGES;
            if (elect_one()) {
              const uint32_t a0 = smem_u32(smem + st * SP_STAGE_BYTES), b0 = a0 + SP_A_BYTES;
#pragma unroll
              for (int kk = 0; kk < SP_BK / 16; ++kk)
                tc_mma_bf16(dt, tc_desc_k128(a0 + 32 * kk), tc_desc_k128(b0 + 32 * kk), TC_IDESC,
                            (slab > s0 || kk > 0) ? 1u : 0u);
              tc_commit(empty0 + 8 * st);
              if (slab + 1 == s1) tc_commit(accf0 + 8 * b);
            }
            __syncwarp();
          }
        }
      }
    }
    // every MMA issued above has completed before the tensor memory is freed
    if (elect_one()) tc_commit(done_bar);
    __syncwarp();
    if (lane == 0) {
      if (stop) atomicExch(&cnt[3], 1);
      mbar_wait_bounded(done_bar, 0, limit, err);
    }
  } else if (warp == 3) {
    // ---------------------------------------------------------------- waiter
    int step = 0, item = 0;
    bool bad = false;
    for (int n = blockIdx.x; n < ntiles && !bad; n += gridDim.x) {
      for (int pq = 0; pq < p.npairs && !bad; ++pq) {
        for (int c = 0; c < nchunks && !bad; ++c, ++item) {
          const int b = item & 1;
          const int s0 = c * chunk_slabs, s1 = min(nslab, s0 + chunk_slabs);
          for (int slab = s0; slab < s1; ++slab, ++step) {
            int fail = 0;
            if (lane == 0) {
              if (slab == s0 && item >= 2 &&
                  !mbar_wait_bounded(acce0 + 8 * b, ((item >> 1) - 1) & 1, limit, err))
                fail = 1;
              const int st = step % TCP_STAGES;
              if (!fail && !mbar_wait_bounded(full0 + 8 * st, (step / TCP_STAGES) & 1, limit, err)) fail = 1;
            }
            fail = __shfl_sync(0xffffffffu, fail, 0);
            if (bar_red_or(TC_HANDOFF_BAR, 64, fail != 0)) { bad = true; break; }
          }
        }
      }
    }
  } else if (warp >= 4) {
    // ---------------------------------------------------------------- folders
    const int fw = warp - 4;  // tensor-memory lane quadrant fw: tile rows fw*32 + lane
    int item = 0;
    bool ok = true;
    for (int n = blockIdx.x; n < ntiles && ok; n += gridDim.x) {
      int I, J;
      tile_coords(n, I, J);
      ok = tcp_folder_tile<TA, TB, CK>(p, I, J, item, tbase, accf0, acce0, s_co, s_cc, s_ca, s_sig, s_fr, s_fc,
                                       cnt, nchunks, fw, lane);
    }
    if (!ok && lane == 0) atomicExch(&cnt[3], 1);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tbase, TC_TMEM_COLS);
  }
}

}  // namespace ftg
