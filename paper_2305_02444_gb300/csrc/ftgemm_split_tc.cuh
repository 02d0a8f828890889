// Split-precision GEMM on the tcgen05 tensor cores: the slice-pair products
// of the error-free splitting (Ozaki, Ogita, Oishi and Rump) and the plain
// BF16 form, with FP32 accumulators in tensor memory and the FP64 fold of
// every pair also held in tensor memory.
//
// One CTA per 128 x 128 output tile, 256 threads in fixed roles:
//   warp 0   TMA producer: the A slice slab (128 rows x 64 k, bf16) and the
//            B slice slab of the current pair into a TC_STAGES-deep ring;
//   warp 1   MMA issuer: 4 tcgen05.mma (M 128, N 128, K 16) per slab into
//            one of two FP32 accumulators (tensor-memory columns 0..255),
//            a commit per slab frees the ring stage, a commit per pair (or
//            k-chunk) hands the accumulator to the folders.  It never polls
//            memory (a poll waits behind its queued MMAs and drains the
//            tensor pipe: measured 64 -> ~130 cycles per MMA);
//   warp 2   allocates / frees the 512 tensor-memory columns;
//   warp 3   waiter: polls the ring's full barriers and the accumulators'
//            release, and hands each slab to warp 1 at a named barrier;
//   warps 4-7 folders: thread = tile row; acc64 += 2^-w(s+t+2) * acc32 with
//            the FP64 accumulators in columns 256..511 (two 32-bit columns
//            per element), overlapped with the next pair's MMAs; the scaled
//            FP32 value is built with integer operations, so that a fold
//            costs one FP64 add per element.
// The fold order, weights and FP64 arithmetic are those of the mma.sync
// kernel (the pair products are exact integers in FP32), so both kernels
// produce the same bits for the emulated forms.  The end of the tile (scale,
// FP64-checksum verification, recomputation, store) is split_tile_finish.
// Every wait is bounded: a wait that gives up records ERR_TIMEOUT, the roles
// stop issuing, the loads and MMAs already issued are waited for (bounded),
// the tensor memory is freed and the CTA returns.
#pragma once

#include "ftgemm_split.cuh"
#include "ftgemm_tc.cuh"

namespace ftg {

#ifndef FTG_TC_STAGES
#define FTG_TC_STAGES 7  // ring depth (a build-time tuning knob; 7 x 32 KiB is what fits)
#endif
#ifndef FTG_TC_GROUP
#define FTG_TC_GROUP 8  // tile rows per rasterization group
#endif
constexpr int TC_STAGES = FTG_TC_STAGES;
constexpr int TC_GROUP = FTG_TC_GROUP;
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_ACC64_COL = 256;
constexpr int TC_HANDOFF_BAR = 3;  // named barrier of the waiter -> MMA-issuer handoff (warps 1 and 3)
constexpr uint32_t TC_IDESC = tc_idesc_bf16_f32(SP_BM, SP_BN);
constexpr int TC_SMEM_BYTES = TC_STAGES * SP_STAGE_BYTES + 2 * 128 * 4 + 64 * 4 + (2 * TC_STAGES + 5) * 8 + 16 +
                              1024;
static_assert(TC_STAGES * SP_STAGE_BYTES >= SP_BM * SP_BN * 8 + SP_RED_DOUBLES * 8,
              "the ring holds the FP64 tile and the epilogue scratch at the end");

// 2^-sh * f as a double, for f an integer-valued float (the exact FP32 result
// of a slice-pair product) and 0 <= sh < 800: f's sign, exponent - sh and
// mantissa moved into the FP64 fields with integer operations (exact, and
// off the FP64 pipe).
__device__ __forceinline__ double scaled_exact_f32(uint32_t fb, int sh) {
  const uint32_t ef = (fb >> 23) & 0xFFu;
  const uint32_t keep = ef ? 0xFFFFFFFFu : 0u;  // +-0 stays +-0
  const uint32_t hi = (fb & 0x80000000u) | (keep & (((ef + (1023u - 127u) - (uint32_t)sh) << 20) |
                                                    ((fb & 0x7FFFFFu) >> 3)));
  return tc_pack_f64((fb & 7u) << 29, hi);
}

// One CTA per tile, each loading its own slabs (tmA / tmB: slice maps with
// 128-row boxes).
template <bool TA, bool TB, int CK>
__global__ void __launch_bounds__(256, 1)
    ftsplit_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ SplitParams p) {
  static_assert(CK == 0 || CK == 2, "no checks, or checks against the checksum products P1 / P2");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *smem =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  int *s_fr = reinterpret_cast<int *>(smem + TC_STAGES * SP_STAGE_BYTES);
  int *s_fc = s_fr + 128;
  int *cnt = s_fc + 128;  // [0] nr [1] nc [2] det [3] abort [4] unverifiable
  uint64_t *bars = reinterpret_cast<uint64_t *>(cnt + 64);
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(bars + 2 * TC_STAGES + 5);
  const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * TC_STAGES;
  const uint32_t accf0 = empty0 + 8 * TC_STAGES, acce0 = accf0 + 16, done_bar = acce0 + 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // grouped rasterization: consecutive CTAs sweep TC_GROUP tile rows column
  // by column, so that the CTAs resident at one time cover a compact block of
  // tiles and share the slices' slabs in L2
  int I, J;
  {
    const int b = blockIdx.x, per = TC_GROUP * p.nJ, g = b / per, r = b % per;
    const int rows = min(TC_GROUP, p.nI - g * TC_GROUP);
    I = g * TC_GROUP + r % rows;
    J = r / rows;
  }
  const int tile = I + J * p.nI;  // injection and location records number tiles column-major
  const int i0 = I * SP_BM, j0 = J * SP_BN;
  int *err = &p.rep->err;
  const unsigned long long limit = p.wait_limit_ns;

  if (tid == 0) {
    for (int c = 0; c < 8; ++c) cnt[c] = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
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
  const int nsteps = p.npairs * nslab;
  bool ok = true;

  if (warp == 0) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      int issued = 0;
      for (int step = 0; step < nsteps; ++step) {
        const int pq = step / nslab, slab = step % nslab, st = step % TC_STAGES;
        if (step >= TC_STAGES &&
            !mbar_wait_bounded(empty0 + 8 * st, ((step / TC_STAGES) - 1) & 1, limit, err)) {
          ok = false;
          break;
        }
        if (*(volatile int *)&cnt[3]) break;
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
        issued = step + 1;
      }
      if (!ok) atomicExch(&cnt[3], 1);
      // the last loads in flight land before the CTA may leave (bounded)
      for (int n = issued > TC_STAGES ? issued - TC_STAGES : 0; n < issued; ++n)
        mbar_wait_bounded(full0 + 8 * (n % TC_STAGES), (n / TC_STAGES) & 1, limit, err);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    // never waits on memory: every slab starts with the rendezvous with the
    // waiter warp, which carries "stop" after a wait that gave up
    int step = 0, item = 0;
    bool stop = false;
    for (int pq = 0; pq < p.npairs && !stop; ++pq) {
      for (int c = 0; c < nchunks && !stop; ++c, ++item) {
        const int b = item & 1;
        const uint32_t dt = tbase + (uint32_t)(b * SP_BN);
        const int s0 = c * chunk_slabs, s1 = min(nslab, s0 + chunk_slabs);
        for (int slab = s0; slab < s1; ++slab, ++step) {
          if (bar_red_or(TC_HANDOFF_BAR, 64, false)) { stop = true; break; }
          tc_fence_after();
          const int st = step % TC_STAGES;
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
    // every MMA issued above has completed before the tensor memory is freed
    if (elect_one()) tc_commit(done_bar);
    __syncwarp();
    if (lane == 0) {
      if (stop) atomicExch(&cnt[3], 1);
      mbar_wait_bounded(done_bar, 0, limit, err);
    }
  } else if (warp == 3) {
    // ---------------------------------------------------------------- waiter
    // waits (bounded) for each slab's data and, at an item's first slab, for
    // the folders to have released the accumulator, then hands over
    int step = 0, item = 0;
    bool bad = false;
    for (int pq = 0; pq < p.npairs && !bad; ++pq) {
      for (int c = 0; c < nchunks && !bad; ++c, ++item) {
        const int b = item & 1;
        const int s0 = c * chunk_slabs, s1 = min(nslab, s0 + chunk_slabs);
        for (int slab = s0; slab < s1; ++slab, ++step) {
          int fail = 0;
          if (lane == 0) {
            if (slab == s0 && item >= 2 && !mbar_wait_bounded(acce0 + 8 * b, ((item >> 1) - 1) & 1, limit, err))
              fail = 1;
            const int st = step % TC_STAGES;
            if (!fail && !mbar_wait_bounded(full0 + 8 * st, (step / TC_STAGES) & 1, limit, err)) fail = 1;
          }
          fail = __shfl_sync(0xffffffffu, fail, 0);
          if (bar_red_or(TC_HANDOFF_BAR, 64, fail != 0)) { bad = true; break; }
        }
      }
    }
  } else if (warp >= 4) {
    // ---------------------------------------------------------------- folders
    const int fw = warp - 4;  // lane quadrant of the tensor memory: tile rows fw*32 + lane
    const uint32_t trow = tbase + ((uint32_t)(fw * 32) << 16);
    const uint32_t t64 = trow + TC_ACC64_COL;
    int fptr = 0, fend = 0;
    if (CK >= 1 && p.inj) { fptr = p.tile_off[tile]; fend = p.tile_off[tile + 1]; }
    int item = 0;
    const bool plain = p.S == 0;
    for (int pq = 0; pq < p.npairs && ok; ++pq) {
      const int sh = p.w * (p.pair_s[pq] + p.pair_t[pq] + 2);  // the pair's weight is 2^-sh
      for (int c = 0; c < nchunks; ++c, ++item) {
        const int b = item & 1;
        int got = 1;
        if (lane == 0) got = mbar_wait_bounded(accf0 + 8 * b, (item >> 1) & 1, limit, err) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) { ok = false; break; }
        tc_fence_after();
#pragma unroll 1
        for (int ch = 0; ch < SP_BN / 32; ++ch) {
          uint32_t f[32], d[64];
          tmem_ld_x32(trow + (uint32_t)(b * SP_BN + ch * 32), f);
          if (item == 0) {
#pragma unroll
            for (int j = 0; j < 64; ++j) d[j] = 0u;
          } else {
            tmem_ld_x64(t64 + (uint32_t)(ch * 64), d);
          }
          // acc64 += 2^-sh * acc32: one FP64 add (the same rounding as an FMA
          // with the exact product); the plain BF16 form converts its FP32 sum
          if (plain) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const double a = tc_pack_f64(d[2 * j], d[2 * j + 1]) + (double)__uint_as_float(f[j]);
              d[2 * j] = tc_lo(a);
              d[2 * j + 1] = tc_hi(a);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const double a = tc_pack_f64(d[2 * j], d[2 * j + 1]) + scaled_exact_f32(f[j], sh);
              d[2 * j] = tc_lo(a);
              d[2 * j + 1] = tc_hi(a);
            }
          }
          tmem_st_x64(t64 + (uint32_t)(ch * 64), d);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * b);
      }
      if (!ok) break;
      if (CK >= 1 && p.inj) {
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
    if (!ok && lane == 0) atomicExch(&cnt[3], 1);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (cnt[3]) {
    if (warp == 2) tmem_dealloc(tbase, TC_TMEM_COLS);
    return;
  }
  // the ring is free: stage the FP64 accumulators as a column-major tile
  double *sC = reinterpret_cast<double *>(smem);
  fence_proxy_async_smem();
  if (warp >= 4) {
    const int fw = warp - 4, il = fw * 32 + lane;
    const uint32_t t64 = tbase + ((uint32_t)(fw * 32) << 16) + TC_ACC64_COL;
#pragma unroll 1
    for (int ch = 0; ch < SP_BN / 32; ++ch) {
      uint32_t d[64];
      tmem_ld_x64(t64 + (uint32_t)(ch * 64), d);
#pragma unroll
      for (int j = 0; j < 32; ++j) sC[(ch * 32 + j) * SP_BM + il] = tc_pack_f64(d[2 * j], d[2 * j + 1]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tbase, TC_TMEM_COLS);
  }
  split_tile_finish<TA, TB, CK>(p, sC, reinterpret_cast<double *>(smem + SP_BM * SP_BN * 8), s_fr, s_fc, cnt,
                                tile, I, J);
}

}  // namespace ftg
