// The FT-DGEMM kernel for sm_103a.
//
// One CTA computes one BM x BN tile of C = alpha*op(A)*op(B) + beta*C:
//  - thread 0 streams BK-deep slabs of op(A) and op(B) into a ring of
//    shared-memory stages with TMA (cp.async.bulk.tensor), together with the
//    matching BK-slabs of the operand checksum vectors (bulk copies); a
//    separate producer warp would cap the 9-warp CTA at 168 registers/thread;
//  - 8 compute warps accumulate an 8x8 register tile per thread with DFMA
//    (on GB300, DFMA is the fastest FP64 path: FP64 mma.sync shares its pipe
//    and issues fewer flops) and, while the slab is staged, fold it into the
//    predicted checksums: column j gets sum_k acs_I[k] * B(k,j), row i gets
//    sum_k A(i,k) * bcs_J[k] (the reuse of each staged operand load for the
//    checksum updates of FT-GEMM §2.2);
//  - the epilogue reads beta*C once (TMA), forms out = alpha*acc + beta*C,
//    adds beta * (row/column sums of C) to the predicted checksums (the
//    encoding of C^c and C^r fused with C = beta*C, §2.2), sums the reference
//    checksums of out before it leaves the chip (§2.2), compares, and on a
//    mismatch recomputes the flagged elements (readings: per-tile
//    verification, a-priori rounding threshold, intersection recompute with
//    a segment fallback), then stores the tile with one TMA store.
// FT = false compiles the same kernel without any checksum work (the
// unprotected baseline); INJ adds the source-level fault injector (§3.2).
#pragma once

#include "ftgemm_common.cuh"

namespace ftg {

// op(A)(i,k) of the staged slab: 'N' slabs are [BK][BM] (i contiguous),
// 'T' slabs are [BM][BK] swizzled.
template <bool TA>
__device__ __forceinline__ double stage_a(const unsigned char *sA, int i, int k) {
  if (TA) return *reinterpret_cast<const double *>(sA + swz_off(i, k));
  return reinterpret_cast<const double *>(sA)[k * BM + i];
}
// op(B)(k,j): 'N' slabs are [BN][BK] swizzled, 'T' slabs are [BK][BN].
template <bool TB>
__device__ __forceinline__ double stage_b(const unsigned char *sB, int k, int j) {
  if (TB) return reinterpret_cast<const double *>(sB)[k * BN + j];
  return *reinterpret_cast<const double *>(sB + swz_off(j, k));
}

template <bool TA, bool TB>
__device__ __forceinline__ double glob_a(const Params &p, long long i, long long k) {
  return TA ? p.A[k + i * p.lda] : p.A[i + k * p.lda];
}
template <bool TA, bool TB>
__device__ __forceinline__ double glob_b(const Params &p, long long k, long long j) {
  return TB ? p.B[j + k * p.ldb] : p.B[k + j * p.ldb];
}

// counters in shared memory
enum { C_NR = 0, C_NC, C_DET, C_CSONLY, C_UNVER, C_RECOMP, C_ABORT, C_FAIL, C_PNR, C_PNC, C_PDET, C_SUBFAIL, C_NCNT };

// Recompute element (il, jl) of the tile from the original operands with one
// warp (lanes split k), compare with the staged value and rewrite it.
template <bool TA, bool TB>
__device__ __forceinline__ void recompute_elem(const Params &p, double *sC, int *cnt, int tile,
                                               long long i0, long long j0, int il, int jl,
                                               int kind, bool use_c, int lane) {
  const long long gi = i0 + il, gj = j0 + jl;
  double dot = 0.0, ab = 0.0;
  for (long long k = lane; k < p.K; k += 32) {
    const double a = glob_a<TA, TB>(p, gi, k), b = glob_b<TA, TB>(p, k, gj);
    dot = fma(a, b, dot);
    ab = fma(fabs(a), fabs(b), ab);
  }
  dot = warp_sum(dot);
  ab = warp_sum(ab);
  if (lane == 0) {
    const double c = use_c ? p.C[gi + gj * p.ldc] : 0.0;
    const double nv = use_c ? fma(p.alpha, dot, p.beta * c) : p.alpha * dot;
    const double E = fabs(p.alpha) * ab + (use_c ? fabs(p.beta) * fabs(c) : 0.0);
    const double n = (double)(p.K + 3);
    const double te = 2.01 * n * 0x1p-53 * E + n * 0x1p-1021;
    const double old = sC[jl * BM + il];
    const bool wrong = (!isfinite(old) && isfinite(nv)) || fabs(old - nv) > te;
    atomicAdd(&cnt[C_RECOMP], 1);
    if (wrong) {
      atomicAdd(&cnt[C_DET], 1);
      const unsigned long long q = atomicAdd(&p.rep->n_loc, 1ull);
      if ((long long)q < p.loc_cap) {
        DevLoc L;
        L.row = gi; L.col = gj; L.tile = tile; L.kind = kind; L.delta = old - nv;
        p.loc[q] = L;
      }
    }
    sC[jl * BM + il] = nv;
  }
}

// One k-slab of the tile product for this thread's PP x QQ accumulator
// blocks (rows tx + 16 pp, columns ty + 16 qq).
template <bool TA, bool TB, int PP, int QQ>
__device__ __forceinline__ void slab_fma(double (&acc)[8][8], const unsigned char *sA, const unsigned char *sB,
                                         int tx, int ty) {
#pragma unroll
  for (int k = 0; k < BK; ++k) {
    double a[PP], b[QQ];
#pragma unroll
    for (int pp = 0; pp < PP; ++pp) a[pp] = stage_a<TA>(sA, tx + 16 * pp, k);
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq) b[qq] = stage_b<TB>(sB, k, ty + 16 * qq);
#pragma unroll
    for (int pp = 0; pp < PP; ++pp)
#pragma unroll
      for (int qq = 0; qq < QQ; ++qq) acc[pp][qq] = fma(a[pp], b[qq], acc[pp][qq]);
  }
}

// One k-slab for the accumulator blocks P0 .. P0+PP-1 (rows) x Q0 .. Q0+QQ-1
// (columns) of this thread: the same FMAs, in the same k order, as those
// blocks get in slab_fma.  KT: only the first kv k's of the slab (the last
// slab of a problem whose K is not a multiple of BK; the rest are TMA zero
// fill, whose FMAs would leave the accumulators as they are), in a loop that
// is not unrolled.
template <bool TA, bool TB, int P0, int PP, int Q0, int QQ, bool KT = false>
__device__ __forceinline__ void slab_fma_part(double (&acc)[8][8], const unsigned char *sA, const unsigned char *sB,
                                              int tx, int ty, int kv = BK) {
#pragma unroll(KT ? 1 : BK)
  for (int k = 0; k < (KT ? kv : BK); ++k) {
    double a[PP], b[QQ];
#pragma unroll
    for (int pp = 0; pp < PP; ++pp) a[pp] = stage_a<TA>(sA, tx + 16 * (P0 + pp), k);
#pragma unroll
    for (int qq = 0; qq < QQ; ++qq) b[qq] = stage_b<TB>(sB, k, ty + 16 * (Q0 + qq));
#pragma unroll
    for (int pp = 0; pp < PP; ++pp)
#pragma unroll
      for (int qq = 0; qq < QQ; ++qq) acc[P0 + pp][Q0 + qq] = fma(a[pp], b[qq], acc[P0 + pp][Q0 + qq]);
  }
}

// The column blocks 0 .. cblk-1 (cblk in 1..8) for the row blocks P0 ..
// P0+PP-1: all 8 in one pass, else in binary pieces (4, 2, 1), one pass each.
template <bool TA, bool TB, int P0, int PP, bool KT>
__device__ __forceinline__ void slab_fma_rowpiece(int cblk, double (&acc)[8][8], const unsigned char *sA,
                                                  const unsigned char *sB, int tx, int ty, int kv) {
  if (cblk == 8) {
    slab_fma_part<TA, TB, P0, PP, 0, 8, KT>(acc, sA, sB, tx, ty, kv);
    return;
  }
  if (cblk & 4) slab_fma_part<TA, TB, P0, PP, 0, 4, KT>(acc, sA, sB, tx, ty, kv);
  if (cblk & 2) {
    if (cblk & 4) slab_fma_part<TA, TB, P0, PP, 4, 2, KT>(acc, sA, sB, tx, ty, kv);
    else slab_fma_part<TA, TB, P0, PP, 0, 2, KT>(acc, sA, sB, tx, ty, kv);
  }
  if (cblk & 1) {
    switch (cblk & 6) {
      case 0: slab_fma_part<TA, TB, P0, PP, 0, 1, KT>(acc, sA, sB, tx, ty, kv); break;
      case 2: slab_fma_part<TA, TB, P0, PP, 2, 1, KT>(acc, sA, sB, tx, ty, kv); break;
      case 4: slab_fma_part<TA, TB, P0, PP, 4, 1, KT>(acc, sA, sB, tx, ty, kv); break;
      default: slab_fma_part<TA, TB, P0, PP, 6, 1, KT>(acc, sA, sB, tx, ty, kv); break;
    }
  }
}

// slab_fma for rblk x cblk accumulator blocks.  Without FINE each count is 2,
// 4 or 8 and the blocks take one fused pass.  With FINE (the batched kernel,
// whose small problems often end in partly filled tiles) each count is any of
// 1..8, so a tile computes its valid rows and columns rounded up to 16 only:
// the row and column blocks split into binary pieces and each pair of pieces
// takes one pass over the slab.  Every accumulator gets the same FMAs in the
// same order either way (the same bits); the extra passes re-read operands
// from shared memory, which is cheap beside the FP64 pipe.
template <bool TA, bool TB, bool FINE, bool KT = false>
__device__ __forceinline__ void slab_fma_blocks(int rblk, int cblk, double (&acc)[8][8], const unsigned char *sA,
                                                const unsigned char *sB, int tx, int ty, int kv = BK) {
  if constexpr (!FINE) {
    if (rblk == 8 && cblk == 8) slab_fma<TA, TB, 8, 8>(acc, sA, sB, tx, ty);
    else if (rblk == 8 && cblk == 4) slab_fma<TA, TB, 8, 4>(acc, sA, sB, tx, ty);
    else if (rblk == 8) slab_fma<TA, TB, 8, 2>(acc, sA, sB, tx, ty);
    else if (rblk == 4 && cblk == 8) slab_fma<TA, TB, 4, 8>(acc, sA, sB, tx, ty);
    else if (rblk == 4 && cblk == 4) slab_fma<TA, TB, 4, 4>(acc, sA, sB, tx, ty);
    else if (rblk == 4) slab_fma<TA, TB, 4, 2>(acc, sA, sB, tx, ty);
    else if (cblk == 8) slab_fma<TA, TB, 2, 8>(acc, sA, sB, tx, ty);
    else if (cblk == 4) slab_fma<TA, TB, 2, 4>(acc, sA, sB, tx, ty);
    else slab_fma<TA, TB, 2, 2>(acc, sA, sB, tx, ty);
  } else {
    if (rblk == 8) {
      slab_fma_rowpiece<TA, TB, 0, 8, KT>(cblk, acc, sA, sB, tx, ty, kv);
      return;
    }
    if (rblk & 4) slab_fma_rowpiece<TA, TB, 0, 4, KT>(cblk, acc, sA, sB, tx, ty, kv);
    if (rblk & 2) {
      if (rblk & 4) slab_fma_rowpiece<TA, TB, 4, 2, KT>(cblk, acc, sA, sB, tx, ty, kv);
      else slab_fma_rowpiece<TA, TB, 0, 2, KT>(cblk, acc, sA, sB, tx, ty, kv);
    }
    if (rblk & 1) {
      switch (rblk & 6) {
        case 0: slab_fma_rowpiece<TA, TB, 0, 1, KT>(cblk, acc, sA, sB, tx, ty, kv); break;
        case 2: slab_fma_rowpiece<TA, TB, 2, 1, KT>(cblk, acc, sA, sB, tx, ty, kv); break;
        case 4: slab_fma_rowpiece<TA, TB, 4, 1, KT>(cblk, acc, sA, sB, tx, ty, kv); break;
        default: slab_fma_rowpiece<TA, TB, 6, 1, KT>(cblk, acc, sA, sB, tx, ty, kv); break;
      }
    }
  }
}

// MODE 0: the whole tile (mainloop + epilogue).
// MODE 1: split-K partial: one k-range of a tile; stores the raw partial
//         product and its predicted-checksum partials for MODE 2.
// MODE 2: split-K reduction: sums the partials of a tile, then runs the same
//         epilogue as MODE 0 (beta*C encode, verify, locate, correct, store).
// MODE 3: verify-only pass of the unfused ablation: the tile of a finished
//         GEMM, predicted checksums and C sums computed by separate passes.
template <bool TA, bool TB, bool FT, bool INJ, int MODE, bool PANEL = false, bool FINE = false>
__device__ __forceinline__ void ftd_tile(const CUtensorMap *tmA, const CUtensorMap *tmB, const CUtensorMap *tmC,
                                         const CUtensorMap *tmW, const Params &p, const int tile, const int split,
                                         unsigned char *smem) {
  double *epi = reinterpret_cast<double *>(smem + TILE_REGION);
  double *s_rc = epi, *s_rca = epi + 128, *s_cc = epi + 256, *s_cca = epi + 384;
  double *s_ro = epi + 512, *s_co = epi + 640, *s_pr = epi + 768, *s_pc = epi + 896;
  double *s_tr = epi + 1024, *s_tc = epi + 1152;
  int *s_fr = reinterpret_cast<int *>(epi + 1280);
  int *s_fc = s_fr + 128, *s_rfail = s_fc + 128, *s_cfail = s_rfail + 128;
  int *cnt = s_cfail + 128;
  double *s_abv = epi + 1568;  // the verify's absolute sums: columns, rows, then the two maxima
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + TILE_REGION + EPI_BYTES);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), cbar = smem_u32(bars + 2 * STAGES);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wcount = p.tile_count ? p.tile_count : p.nI * p.nJ;          // split-K partial slots per split
  const int s_begin = (MODE == 1) ? split * p.ks_slabs : 0;              // first k-slab (global)
  const int s_end = (MODE == 1) ? min(p.nks, s_begin + p.ks_slabs) : p.nks;
  const int I = tile % p.nI, J = tile / p.nI;
  const int i0 = I * BM, j0 = J * BN;
  const int mI = (int)min((long long)BM, p.M - i0), nJt = (int)min((long long)BN, p.N - j0);
  const int nks = (MODE >= 2) ? 0 : s_end - s_begin;  // k-slabs this CTA accumulates
  const unsigned long long limit = p.wait_limit_ns;
  int *err = &p.rep->err;
  double *sC = reinterpret_cast<double *>(smem);  // output tile, column-major [BN][BM]

  if (tid == 0) {
    for (int c = 0; c < C_NCNT; ++c) cnt[c] = 0;
    cnt[C_ABORT] = (*reinterpret_cast<volatile int *>(err) != 0);
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, NCOMPUTE / 32);
    }
    mbar_init(cbar, 1);
    fence_mbar_init();
  }
  if (tid == 32) {
    if (MODE != 2) {
      prefetch_tmap(tmA);
      prefetch_tmap(tmB);
    }
    prefetch_tmap(MODE == 1 || MODE == 2 ? tmW : tmC);
  }
  if (tid < 128) { s_rfail[tid] = 0; s_cfail[tid] = 0; }
  // a previous tile of a persistent CTA read and wrote the ring with generic
  // accesses: order them before this tile's TMA writes into it
  fence_proxy_async_smem();
  __syncthreads();
  if (cnt[C_ABORT]) return;  // an earlier tile hit a timeout: skip the work

  // ------------------------------------------------------------------ compute
  // Thread 0 is also the producer: it fills the first STAGES slabs, then after
  // each slab refills the stage that the previous slab freed.
  const uint32_t tx_bytes = FT ? A_BYTES + B_BYTES + 2 * CS_BYTES : A_BYTES + B_BYTES;
  auto issue = [&](int s) {
    const int st = s % STAGES;
    const uint32_t sb = smem_u32(smem + st * STAGE_BYTES);
    const uint32_t fb = full0 + 8 * st;
    mbar_arrive_expect_tx(fb, tx_bytes);
    const int k0 = (s_begin + s) * BK;
    if (TA) tma_load_2d(sb, tmA, fb, k0, i0); else tma_load_2d(sb, tmA, fb, i0, k0);
    if (TB) tma_load_2d(sb + A_BYTES, tmB, fb, j0, k0); else tma_load_2d(sb + A_BYTES, tmB, fb, k0, j0);
    if (FT) {
      bulk_load(sb + A_BYTES + B_BYTES, p.acs + (long long)I * p.Kp + k0, CS_BYTES, fb);
      bulk_load(sb + A_BYTES + B_BYTES + CS_BYTES, p.bcs + (long long)J * p.Kp + k0, CS_BYTES, fb);
    }
  };
  int issued = 0;
  if (tid == 0) {
    for (; issued < STAGES && issued < nks; ++issued) issue(issued);
  }
  if (FT && MODE != 1) {  // fetched while the first slabs are in flight
    if (tid < 128) s_abv[tid] = tid < nJt ? p.bcolabs[j0 + tid] : 0.0;
    else s_abv[tid] = tid - 128 < mI ? p.arowabs[i0 + tid - 128] : 0.0;
    if (tid == 32) {
      s_abv[256] = p.aabsmax[I];
      s_abv[257] = p.babsmax[J];
    }
  }

  const int tx = tid & 15, ty = tid >> 4;  // rows tx + 16*pp, columns ty + 16*qq
  // accumulator blocks (16 rows / columns each) that hold valid rows / columns:
  // 2, 4 or 8, and any of 1..8 in the batched kernel (FINE)
  auto blocks = [](int v) { return FINE ? (v + 15) >> 4 : v <= 32 ? 2 : v <= 64 ? 4 : 8; };
  const int rblk = blocks(mI), cblk = blocks(nJt);
  double acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
  double csacc = 0.0;  // FT: predicted column (tid < 128) or row (tid >= 128) checksum
  int fptr = 0, fend = 0;
  if (INJ) {
    fptr = p.tile_off[tile];
    fend = p.tile_off[tile + 1];
    while (fptr < fend && p.flips[fptr].kstep < s_begin) ++fptr;  // earlier k-splits' faults
  }

  // A thread whose bounded wait expired stops waiting and computing but keeps
  // iterating, so that every thread reaches the same CTA-wide barriers of the
  // panel checks; the abort is acted on after the loop.
  bool ok = true;
  for (int s = 0; s < nks; ++s) {
    const int st = s % STAGES;
    if (ok && !mbar_wait_bounded(full0 + 8 * st, (s / STAGES) & 1, limit, err)) ok = false;
    if (ok) {
    const unsigned char *sA = smem + st * STAGE_BYTES;
    const unsigned char *sB = sA + A_BYTES;
    // rows tx + 16 pp >= mI and columns ty + 16 qq >= nJt hold zeros (TMA
    // zero fill): a tile whose valid rows or columns end before the last
    // blocks skips those blocks' FMAs, leaving the same bits
    if (FINE && s_begin + s == p.nks - 1 && p.K < (long long)p.nks * BK)
      slab_fma_blocks<TA, TB, FINE, true>(rblk, cblk, acc, sA, sB, tx, ty, (int)(p.K - (long long)(p.nks - 1) * BK));
    else
      slab_fma_blocks<TA, TB, FINE>(rblk, cblk, acc, sA, sB, tx, ty);
    if (FT) {
      const double *scs = reinterpret_cast<const double *>(sA + A_BYTES + B_BYTES);
      if (tid < 128) {
#pragma unroll
        for (int k = 0; k < BK; ++k) csacc = fma(scs[k], stage_b<TB>(sB, k, tid), csacc);
      } else {
#pragma unroll
        for (int k = 0; k < BK; ++k) csacc = fma(stage_a<TA>(sA, tid - 128, k), scs[BK + k], csacc);
      }
    }
    if (INJ) {
      while (fptr < fend) {
        DevFlip *f = p.flips + fptr;
        if (f->kstep != s_begin + s) break;
        const int il = (int)(f->row - i0), jl = (int)(f->col - j0);
        if ((il & 15) == tx && (jl & 15) == ty) {
          const int pq = (il >> 4) * 8 + (jl >> 4);
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b)
              if (a * 8 + b == pq) {
                const double before = acc[a][b];
                acc[a][b] = flip_bit(before, f->bit);
                f->before = before;
                f->after = acc[a][b];
                f->applied = 1;
                f->kfirst = (long long)s_begin * BK;
              }
        }
        ++fptr;
      }
    }
    }  // ok
    __syncwarp();
    if (lane == 0 && ok) mbar_arrive(empty0 + 8 * st);
    if (tid == 0 && ok && s >= 1 && issued < nks) {
      // refill the stage of slab s-1 once every warp has released it
      const int sp = s - 1;
      if (!mbar_wait_bounded(empty0 + 8 * (sp % STAGES), (sp / STAGES) & 1, limit, err)) ok = false;
      else issue(issued++);
    }
    if (PANEL && p.panel_slabs > 0 && (s + 1) % p.panel_slabs == 0 && s + 1 < nks &&
        __syncthreads_or(!ok) == 0) {
      // ---- verification of the accumulators after this k-panel -------------
      const long long kbeg = (long long)s_begin * BK;
      const long long kdone = min(p.K, (long long)(s_begin + s + 1) * BK);
      double rsum[8], csum[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        rsum[a] = 0.0;
        csum[a] = 0.0;
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          rsum[a] += acc[a][b];
          csum[b] += acc[a][b];
        }
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        rsum[a] += __shfl_xor_sync(0xffffffffu, rsum[a], 16);  // lanes l, l^16: same rows
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) csum[a] += __shfl_xor_sync(0xffffffffu, csum[a], o);  // same columns
      }
      double *s_rpart = epi, *s_csum = epi + 1024, *s_rsum = epi + 1152, *s_val = epi;
      if (lane < 16) {
#pragma unroll
        for (int a = 0; a < 8; ++a) s_rpart[warp * 128 + tx + 16 * a] = rsum[a];
      }
      if (tx == 0) {
#pragma unroll
        for (int b = 0; b < 8; ++b) s_csum[ty + 16 * b] = csum[b];
      }
      compute_sync();
      if (tid < 128) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += s_rpart[w * 128 + tid];
        s_rsum[tid] = t;
      }
      compute_sync();
      {
        const double u = 0x1p-53;
        if (tid < 128) {
          const int j = tid;
          if (j < nJt) {
            const double n = (double)(kdone - kbeg + mI + 3);
            const double tau = 2.01 * n * u * (p.bcolabs[j0 + j] * p.aabsmax[I]) + n * 0x1p-1021;
            if (isfinite(csacc) && isfinite(tau) && !(fabs(s_csum[j] - csacc) <= tau))
              s_fc[atomicAdd(&cnt[C_PNC], 1)] = j;
          }
        } else {
          const int i = tid - 128;
          if (i < mI) {
            const double n = (double)(kdone - kbeg + nJt + 3);
            const double tau = 2.01 * n * u * (p.arowabs[i0 + i] * p.babsmax[J]) + n * 0x1p-1021;
            if (isfinite(csacc) && isfinite(tau) && !(fabs(s_rsum[i] - csacc) <= tau))
              s_fr[atomicAdd(&cnt[C_PNR], 1)] = i;
          }
        }
      }
      compute_sync();
      const int pnr = cnt[C_PNR], pnc = cnt[C_PNC];
      if (pnr > 0 && pnc > 0 && pnr * pnc <= MAX_INTERSECT) {
        // recompute each flagged intersection over the products done so far
        for (int e = warp; e < pnr * pnc; e += NCOMPUTE / 32) {
          const long long gi = i0 + s_fr[e / pnc], gj = j0 + s_fc[e % pnc];
          double dot = 0.0, ab = 0.0;
          for (long long k = kbeg + lane; k < kdone; k += 32) {
            const double av = glob_a<TA, TB>(p, gi, k), bv = glob_b<TA, TB>(p, k, gj);
            dot = fma(av, bv, dot);
            ab = fma(fabs(av), fabs(bv), ab);
          }
          dot = warp_sum(dot);
          ab = warp_sum(ab);
          if (lane == 0) { s_val[2 * e] = dot; s_val[2 * e + 1] = ab; }
        }
        compute_sync();
        // the owning thread replaces its accumulator
        for (int e = 0; e < pnr * pnc; ++e) {
          const int il = s_fr[e / pnc], jl = s_fc[e % pnc];
          if ((il & 15) == tx && (jl & 15) == ty) {
            const int pq = (il >> 4) * 8 + (jl >> 4);
            const double nv = s_val[2 * e];
            const double n = (double)(kdone - kbeg + 3);
            const double te = 2.01 * n * 0x1p-53 * s_val[2 * e + 1] + n * 0x1p-1021;
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
              for (int b = 0; b < 8; ++b)
                if (a * 8 + b == pq) {
                  const double old = acc[a][b];
                  if ((!isfinite(old) && isfinite(nv)) || fabs(old - nv) > te) {
                    atomicAdd(&cnt[C_PDET], 1);
                    const unsigned long long q = atomicAdd(&p.rep->n_loc, 1ull);
                    if ((long long)q < p.loc_cap) {
                      DevLoc L;
                      L.row = i0 + il; L.col = j0 + jl; L.tile = tile; L.kind = 2; L.delta = old - nv;
                      p.loc[q] = L;
                    }
                  }
                  acc[a][b] = nv;
                }
          }
        }
      }
      compute_sync();
      if (tid == 0) { cnt[C_PNR] = 0; cnt[C_PNC] = 0; }
      compute_sync();
    }
  }
  if (!ok) {
    atomicExch(&cnt[C_ABORT], 1);
    if (tid == 0)  // give the copies already in flight a bounded chance to land
      for (int s = issued > STAGES ? issued - STAGES : 0; s < issued; ++s)
        mbar_wait_bounded(full0 + 8 * (s % STAGES), (s / STAGES) & 1, limit, err);
  }
  fence_proxy_async_smem();  // generic reads of the ring precede the async C load
  compute_sync();
  if (*reinterpret_cast<volatile int *>(&cnt[C_ABORT])) return;

  if (MODE == 1) {
    // split-K partial: raw accumulators and predicted-checksum partials
#pragma unroll
    for (int pp = 0; pp < 8; ++pp)
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) sC[(ty + 16 * qq) * BM + tx + 16 * pp] = acc[pp][qq];
    if (FT) {
      if (tid < 128) {
        if (tid < nJt) p.wpc[((long long)split * p.nI + I) * p.N + j0 + tid] = csacc;
      } else if (tid - 128 < mI) {
        p.wpr[((long long)split * p.nJ + J) * p.M + i0 + tid - 128] = csacc;
      }
    }
    fence_proxy_async_smem();
    compute_sync();
    if (tid == 0) {
      tma_store_3d(tmW, smem_u32(sC), 0, 0, split * wcount + (tile - p.tile_base));
      if (PANEL && cnt[C_PDET]) {  // faults this split's panel checks corrected
        DevReport *r = p.rep;
        atomicAdd(&r->detected, (unsigned long long)cnt[C_PDET]);
        atomicAdd(&r->corrected, (unsigned long long)cnt[C_PDET]);
        atomicAdd(&r->panel_detected, (unsigned long long)cnt[C_PDET]);
      }
      bulk_commit();
      bulk_wait_all();
    }
    return;
  }
  if (MODE == 2) {
    // split-K reduction: acc = sum over splits of the partial tiles (ascending
    // split).  Each partial tile comes in as one TMA bulk load into the staged
    // tile buffer (the ring is idle: no k-slabs here), then is summed from
    // shared memory; the rows / columns outside the matrix load as zeros.
    // With p.presummed, slot 0 already holds that sum (splitk_sum_kernel, the
    // same additions in the same order): one load, the checksum partials of
    // every split still added here.
    if (FT) {
      // the predicted-checksum partials of every split, added in ascending
      // split order; their loads do not depend on one another, so they go out
      // four at a time, ahead of the partial tiles' loads
      const bool col = tid < 128;
      const int idx = col ? tid : tid - 128;
      if (col ? idx < nJt : idx < mI) {
        const double *base = col ? p.wpc + (long long)I * p.N + j0 + idx : p.wpr + (long long)J * p.M + i0 + idx;
        const long long stride = col ? (long long)p.nI * p.N : (long long)p.nJ * p.M;
        int sp = 0;
        for (; sp + 4 <= p.nsplit; sp += 4) {
          const double v0 = base[sp * stride], v1 = base[(sp + 1) * stride];
          const double v2 = base[(sp + 2) * stride], v3 = base[(sp + 3) * stride];
          csacc += v0;
          csacc += v1;
          csacc += v2;
          csacc += v3;
        }
        for (; sp < p.nsplit; ++sp) csacc += base[sp * stride];
      }
    }
    for (int sp = 0; sp < p.nsplit; ++sp) {
      if (!p.presummed || sp == 0) {
      if (tid == 0) {
        mbar_arrive_expect_tx(full0, CTILE_BYTES);
        tma_load_3d(smem_u32(sC), tmW, full0, 0, 0, sp * wcount + (tile - p.tile_base));
      }
      if (!mbar_wait_bounded(full0, sp & 1, limit, err)) atomicExch(&cnt[C_ABORT], 1);
      compute_sync();  // every thread leaves together if a partial never landed
      if (*reinterpret_cast<volatile int *>(&cnt[C_ABORT])) return;
#pragma unroll
      for (int pp = 0; pp < 8; ++pp)
#pragma unroll
        for (int qq = 0; qq < 8; ++qq) acc[pp][qq] += sC[(ty + 16 * qq) * BM + tx + 16 * pp];
      fence_proxy_async_smem();  // these generic reads precede the next async write (next partial or C)
      compute_sync();
      }
    }
  }

  if (MODE == 3) {
    // predicted checksums without alpha/beta, from the separate skinny GEMMs
    if (tid < 128) {
      if (tid < nJt) csacc = p.P1[(long long)I + (long long)(j0 + tid) * p.ldp1];
    } else if (tid - 128 < mI) {
      csacc = p.P2[(long long)(i0 + tid - 128) + (long long)J * p.ldp2];
    }
  }

  // ----------------------------------------------------------------- epilogue
  const bool use_c = (p.beta != 0.0);
  // rounding terms of the threshold: K products, L sums, the epilogue, and
  // (split-K) one addition per partial
  // (split-K) one addition per partial; MODE 3's predicted checksums come from
  // a separate GEMM that may itself have split K (at most 32 partials)
  const long long nextra = 3 + ((MODE == 2) ? p.nsplit : 0) + ((MODE == 3) ? 32 : 0);
  if (use_c || MODE == 3) {  // MODE 3 loads the finished output tile instead
    if (tid == 0) {
      mbar_arrive_expect_tx(cbar, CTILE_BYTES);
      tma_load_2d(smem_u32(sC), tmC, cbar, i0, j0);
    }
    if (!mbar_wait_bounded(cbar, 0, limit, err)) atomicExch(&cnt[C_ABORT], 1);
    compute_sync();  // every thread leaves together if the C tile never landed
    if (*reinterpret_cast<volatile int *>(&cnt[C_ABORT])) return;
  }

  // Row and column sums of a staged 128x128 tile by all 256 threads: thread t
  // takes row (t mod 128) over half of the columns and column (t mod 128) over
  // half of the rows (rows visited in a rotated order so a warp's loads hit
  // distinct banks); the two halves are combined through shared memory.  The
  // absolute sums, needed only for the threshold's upper bound, run on the
  // FP32 pipe with upward rounding (each partial sum stays an upper bound).
  const int r = tid & 127, h = tid >> 7;
  // beta-side sums of C for the predicted checksums and the thresholds
  if ((MODE == 3 || (MODE == 2 && FT && p.csums)) && use_c) {
    // from the separate pass over C (the same sums, same order)
    if (tid < 128) {
      s_cc[tid] = tid < nJt ? p.ccs[(long long)I * p.N + j0 + tid] : 0.0;
      s_cca[tid] = tid < nJt ? p.ccsa[(long long)I * p.N + j0 + tid] : 0.0;
    } else {
      const int i = tid - 128;
      s_rc[i] = i < mI ? p.crs[(long long)J * p.M + i0 + i] : 0.0;
      s_rca[i] = i < mI ? p.crsa[(long long)J * p.M + i0 + i] : 0.0;
    }
  } else if (FT && use_c) {
    double rs = 0.0, cs = 0.0;
    float ra = 0.0f, ca = 0.0f;
    if constexpr (FINE) {
      // the batched kernel sums the valid rows and columns only: half h of
      // row r has xc valid columns, half h of column r xr valid rows (visited
      // in the rotated order modulo xr)
      const int xc = min(max(nJt - 64 * h, 0), 64), xr = min(max(mI - 64 * h, 0), 64);
      if (r < mI) {
        for (int q = 0; q < xc; ++q) {
          const double v = sC[(64 * h + q) * BM + r];
          rs += v;
          ra = __fadd_ru(ra, f32_ru_abs(v));
        }
      }
      if (r < nJt && xr > 0) {
        int x = r % xr;
        for (int q = 0; q < xr; ++q) {
          const double v = sC[r * BM + 64 * h + x];
          cs += v;
          ca = __fadd_ru(ca, f32_ru_abs(v));
          x = (x + 1 == xr) ? 0 : x + 1;
        }
      }
    } else {
#pragma unroll 8
      for (int q = 0; q < 64; ++q) {
        const double vr = sC[(64 * h + q) * BM + r];
        const double vc = sC[r * BM + 64 * h + ((q + r) & 63)];
        rs += vr;
        cs += vc;
        ra = __fadd_ru(ra, f32_ru_abs(vr));
        ca = __fadd_ru(ca, f32_ru_abs(vc));
      }
    }
    if (h) { s_ro[r] = rs; s_co[r] = cs; s_pr[r] = (double)ra; s_pc[r] = (double)ca; }
    compute_sync();
    if (!h) {
      s_rc[r] = rs + s_ro[r];
      s_cc[r] = cs + s_co[r];
      s_rca[r] = (double)__fadd_ru(ra, (float)s_pr[r]);
      s_cca[r] = (double)__fadd_ru(ca, (float)s_pc[r]);
    }
  }
  if (FT) compute_sync();

  // out = alpha*acc + beta*C, written over the staged C tile (the batched
  // kernel writes the computed blocks only; the rest of the tile lies outside
  // C, and no later step reads it)
  if (MODE != 3) {
#pragma unroll
    for (int pp = 0; pp < 8; ++pp)
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) {
        if (FINE && (pp >= rblk || qq >= cblk)) continue;
        const int idx = (ty + 16 * qq) * BM + tx + 16 * pp;
        sC[idx] = use_c ? fma(p.alpha, acc[pp][qq], p.beta * sC[idx]) : p.alpha * acc[pp][qq];
      }
    compute_sync();
  }

  if (FT) {
    // reference checksums of the computed tile (the batched kernel: over the
    // valid rows and columns, as the C sums above)
    {
      double rs = 0.0, cs = 0.0;
      if constexpr (FINE) {
        const int xc = min(max(nJt - 64 * h, 0), 64), xr = min(max(mI - 64 * h, 0), 64);
        if (r < mI)
          for (int q = 0; q < xc; ++q) rs += sC[(64 * h + q) * BM + r];
        if (r < nJt && xr > 0) {
          int x = r % xr;
          for (int q = 0; q < xr; ++q) {
            cs += sC[r * BM + 64 * h + x];
            x = (x + 1 == xr) ? 0 : x + 1;
          }
        }
      } else {
#pragma unroll 8
        for (int q = 0; q < 64; ++q) {
          rs += sC[(64 * h + q) * BM + r];
          cs += sC[r * BM + 64 * h + ((q + r) & 63)];
        }
      }
      if (h) { s_pr[r] = rs; s_pc[r] = cs; }
      compute_sync();
      if (!h) { s_ro[r] = rs + s_pr[r]; s_co[r] = cs + s_pc[r]; }
    }
    compute_sync();
    // verify: predicted vs reference, per column (tid < 128) and per row
    {
      const double u = 0x1p-53;
      if (tid < 128) {
        const int j = tid;
        if (j < nJt) {
          const double pc = use_c ? fma(p.alpha, csacc, p.beta * s_cc[j]) : p.alpha * csacc;
          const double S = fabs(p.alpha) * s_abv[j] * s_abv[256] + (use_c ? fabs(p.beta) * s_cca[j] : 0.0);
          const double n = (double)(p.K + mI + nextra);
          const double tau = 2.01 * n * u * S + n * 0x1p-1021;
          s_pc[j] = pc;
          s_tc[j] = tau;
          if (!isfinite(pc) || !isfinite(tau)) atomicAdd(&cnt[C_UNVER], 1);
          else if (!(fabs(s_co[j] - pc) <= tau)) s_fc[atomicAdd(&cnt[C_NC], 1)] = j;
        }
      } else {
        const int i = tid - 128;
        if (i < mI) {
          const double pr = use_c ? fma(p.alpha, csacc, p.beta * s_rc[i]) : p.alpha * csacc;
          const double S = fabs(p.alpha) * s_abv[128 + i] * s_abv[257] + (use_c ? fabs(p.beta) * s_rca[i] : 0.0);
          const double n = (double)(p.K + nJt + nextra);
          const double tau = 2.01 * n * u * S + n * 0x1p-1021;
          s_pr[i] = pr;
          s_tr[i] = tau;
          if (!isfinite(pr) || !isfinite(tau)) atomicAdd(&cnt[C_UNVER], 1);
          else if (!(fabs(s_ro[i] - pr) <= tau)) s_fr[atomicAdd(&cnt[C_NR], 1)] = i;
        }
      }
    }
    compute_sync();
    const int nr = cnt[C_NR], nc = cnt[C_NC];
    if (nr + nc > 0) {
      // locate and correct: flagged row x flagged column intersections
      if (p.correct_mode == 1 && nr == 1 && nc == 1) {
        // FT-BLAS style: subtract the column's checksum residual from the one
        // located element, when it is finite and agrees with the row's
        // residual within the row threshold (one fault explains both); else
        // the element is recomputed.  The subtraction carries the rounding
        // of the 128-term sums; a huge fault cancels badly and fails the
        // agreement test.
        if (tid == 0) {
          const int il = s_fr[0], jl = s_fc[0];
          const double old = sC[jl * BM + il], dlt = s_co[jl] - s_pc[jl], nv = old - dlt;
          const double drow = s_ro[il] - s_pr[il];
          if (isfinite(dlt) && isfinite(nv) && fabs(drow - dlt) <= s_tr[il]) {
            sC[jl * BM + il] = nv;
            cnt[C_DET] += 1;
            const unsigned long long q = atomicAdd(&p.rep->n_loc, 1ull);
            if ((long long)q < p.loc_cap) {
              DevLoc L;
              L.row = i0 + il; L.col = j0 + jl; L.tile = tile; L.kind = 3; L.delta = dlt;
              p.loc[q] = L;
            }
          } else {
            cnt[C_SUBFAIL] = 1;
          }
        }
        compute_sync();
        if (cnt[C_SUBFAIL] && warp == 0)
          recompute_elem<TA, TB>(p, sC, cnt, tile, i0, j0, s_fr[0], s_fc[0], 0, use_c, lane);
      } else if (nr > 0 && nc > 0 && nr * nc <= MAX_INTERSECT) {
        for (int e = warp; e < nr * nc; e += NCOMPUTE / 32)
          recompute_elem<TA, TB>(p, sC, cnt, tile, i0, j0, s_fr[e / nc], s_fc[e % nc], 0, use_c, lane);
      }
      compute_sync();
      // re-verify the flagged rows and columns
      for (int e = warp; e < nr + nc; e += NCOMPUTE / 32) {
        double s = 0.0;
        if (e < nr) {
          const int i = s_fr[e];
          for (int j = lane; j < nJt; j += 32) s += sC[j * BM + i];
          s = warp_sum(s);
          if (lane == 0 && !(fabs(s - s_pr[i]) <= s_tr[i])) { s_rfail[i] = 1; atomicAdd(&cnt[C_FAIL], 1); }
        } else {
          const int j = s_fc[e - nr];
          for (int i = lane; i < mI; i += 32) s += sC[j * BM + i];
          s = warp_sum(s);
          if (lane == 0 && !(fabs(s - s_pc[j]) <= s_tc[j])) { s_cfail[j] = 1; atomicAdd(&cnt[C_FAIL], 1); }
        }
      }
      compute_sync();
      if (cnt[C_FAIL] > 0) {
        // fallback: recompute the whole tile segments of rows/columns still failing
        for (int e = warp; e < mI * nJt; e += NCOMPUTE / 32) {
          const int il = e % mI, jl = e / mI;
          if (s_rfail[il] || s_cfail[jl]) recompute_elem<TA, TB>(p, sC, cnt, tile, i0, j0, il, jl, 1, use_c, lane);
        }
        compute_sync();
        for (int e = warp; e < BM + BN; e += NCOMPUTE / 32) {
          double s = 0.0;
          if (e < BM) {
            if (!s_rfail[e]) continue;
            for (int j = lane; j < nJt; j += 32) s += sC[j * BM + e];
            s = warp_sum(s);
            if (lane == 0 && !(fabs(s - s_pr[e]) <= s_tr[e])) atomicAdd(&cnt[C_CSONLY], 1);
          } else {
            const int j = e - BM;
            if (!s_cfail[j]) continue;
            for (int i = lane; i < mI; i += 32) s += sC[j * BM + i];
            s = warp_sum(s);
            if (lane == 0 && !(fabs(s - s_pc[j]) <= s_tc[j])) atomicAdd(&cnt[C_CSONLY], 1);
          }
        }
        compute_sync();
      }
    }
  }

  // Store the tile.  TMA clips the tile at the edges of C, but in the inner
  // (row) dimension it writes whole 16-byte chunks, so a tile ending on an odd
  // row would also write the first padding row: such tiles use plain stores.
  const bool tma_store = !((p.M & 1) && (i0 + BM > p.M));
  if (MODE == 3 && cnt[C_NR] + cnt[C_NC] == 0) {
    // verify-only pass: nothing was corrected, the output is already in place
    if (tid == 0) {
      DevReport *r = p.rep;
      if (cnt[C_UNVER]) atomicAdd(&r->unverifiable, (unsigned long long)cnt[C_UNVER]);
    }
    return;
  }
  double *Cst = (MODE == 3) ? p.Cout : p.C;
  const long long ldst = (MODE == 3) ? p.ldcout : p.ldc;
  if (tma_store) {
    fence_proxy_async_smem();
    compute_sync();
  } else {
    compute_sync();
    for (int e = tid; e < mI * nJt; e += NCOMPUTE) {
      const int il = e % mI, jl = e / mI;
      Cst[(long long)(i0 + il) + (long long)(j0 + jl) * ldst] = sC[jl * BM + il];
    }
  }
  if (tid == 0) {
    if (tma_store) {
      tma_store_2d(tmC, smem_u32(sC), i0, j0);
      bulk_commit();
    }
    if (FT) {
      DevReport *r = p.rep;
      if (cnt[C_NR]) atomicAdd(&r->flagged_rows, (unsigned long long)cnt[C_NR]);
      if (cnt[C_NC]) atomicAdd(&r->flagged_cols, (unsigned long long)cnt[C_NC]);
      if (cnt[C_DET]) {
        atomicAdd(&r->detected, (unsigned long long)cnt[C_DET]);
        atomicAdd(&r->corrected, (unsigned long long)cnt[C_DET]);
      }
      if (cnt[C_CSONLY]) atomicAdd(&r->checksum_only, (unsigned long long)cnt[C_CSONLY]);
      if (cnt[C_UNVER]) atomicAdd(&r->unverifiable, (unsigned long long)cnt[C_UNVER]);
      if (cnt[C_RECOMP]) atomicAdd(&r->recomputed, (unsigned long long)cnt[C_RECOMP]);
      if (PANEL && cnt[C_PDET]) {
        atomicAdd(&r->detected, (unsigned long long)cnt[C_PDET]);
        atomicAdd(&r->corrected, (unsigned long long)cnt[C_PDET]);
        atomicAdd(&r->panel_detected, (unsigned long long)cnt[C_PDET]);
      }
    }
    if (tma_store) bulk_wait_all();
  }
}

// One CTA per tile (MODE 0, 2, 3) or per tile and k-split (MODE 1).
template <bool TA, bool TB, bool FT, bool INJ, int MODE, bool PANEL = false>
__global__ void __launch_bounds__(NTHREADS, 1)
    ftdgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmW,
                   const Params p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int count = p.tile_count ? p.tile_count : p.nI * p.nJ;
  const int tile = p.tile_base + ((MODE == 1) ? (int)(blockIdx.x % count) : (int)blockIdx.x);
  const int split = (MODE == 1) ? (int)(blockIdx.x / count) : 0;
  ftd_tile<TA, TB, FT, INJ, MODE, PANEL>(&tmA, &tmB, &tmC, &tmW, p, tile, split, smem);
}

// Persistent batched kernel: one CTA per SM takes `chunk` work items at a time
// from a global counter; item q is tile tile_local[order[q]] of problem
// tile_prob[order[q]] (the order is the schedule the host chose).  A bounded
// wait that expires in any tile stops every CTA before its next tile.
template <bool TA, bool TB, bool FT, bool INJ>
__global__ void __launch_bounds__(NTHREADS, 1)
    ftdgemm_batched_kernel(const BatchProblem *__restrict__ probs, const int *__restrict__ order,
                           const int *__restrict__ tile_prob, const int *__restrict__ tile_local, int total,
                           int chunk, int *counter, int *gerr) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ int s_next, s_stop;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_stop = *reinterpret_cast<volatile int *>(gerr) != 0;
      s_next = s_stop ? total : atomicAdd(counter, chunk);
    }
    __syncthreads();
    const int base = s_next;
    if (base >= total) break;
    for (int c = 0; c < chunk && base + c < total; ++c) {
      const int g = order[base + c];
      const BatchProblem *bp = probs + tile_prob[g];
      ftd_tile<TA, TB, FT, INJ, 0, false, true>(&bp->tmA, &bp->tmB, &bp->tmC, &bp->tmC, bp->p, tile_local[g], 0,
                                                smem);
      __syncthreads();
      if (threadIdx.x == 0 && *reinterpret_cast<volatile int *>(&bp->p.rep->err) != 0) atomicExch(gerr, ERR_TIMEOUT);
    }
  }
}

}  // namespace ftg
