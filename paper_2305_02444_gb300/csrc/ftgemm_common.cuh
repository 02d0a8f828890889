// Shared device definitions of libftgemm: tile shape, parameter block,
// device report layout, and inline-PTX helpers for mbarriers and the tensor
// memory accelerator (TMA) on sm_103a.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ftg {

// Output tile BM x BN per CTA, k-slab BK (the injection k-step), ring depth.
constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 16;
constexpr int STAGES = 4;
constexpr int NCOMPUTE = 256;  // 8 compute warps, 8x8 accumulators each
constexpr int NTHREADS = 256;  // thread 0 also issues the TMA loads
constexpr int A_BYTES = BM * BK * 8;  // 16 KiB
constexpr int B_BYTES = BN * BK * 8;  // 16 KiB
constexpr int CS_BYTES = BK * 8;      // one k-slab of a checksum vector
constexpr int STAGE_BYTES = 33 * 1024;  // A | B | acs | bcs, 1 KiB aligned
constexpr int RING_BYTES = STAGES * STAGE_BYTES;
constexpr int CTILE_BYTES = BM * BN * 8;  // output tile staged for verify/store
constexpr int TILE_REGION = RING_BYTES > CTILE_BYTES ? RING_BYTES : CTILE_BYTES;
// epilogue arrays: 10 x 128 doubles + 4 x 128 ints + counters
constexpr int EPI_BYTES = 10 * 128 * 8 + 4 * 128 * 4 + 256 + 264 * 8;
constexpr int BAR_BYTES = 2 * STAGES * 8 + 8 + 8;
constexpr int SMEM_BYTES = TILE_REGION + EPI_BYTES + BAR_BYTES + 1024;
constexpr int MAX_INTERSECT = 64;  // flagged row x column intersections per tile

// Device copy of the fault report (zeroed by the host before each call).
struct DevReport {
  unsigned long long detected, corrected, checksum_only, unverifiable;
  unsigned long long flagged_rows, flagged_cols, recomputed, n_loc, panel_detected;
  int err;  // FTGEMM_ERR_TIMEOUT when a bounded wait expired
  int pad;
};

struct DevLoc {
  long long row, col;
  int tile, kind;
  double delta;
};

// One injected fault, sorted by (tile, kstep); before/after written by the kernel.
struct DevFlip {
  long long row, col, kstep;
  int bit, applied;
  double before, after;
  long long kfirst;  // first product index held by the flipped accumulator (split-K)
};

struct Params {
  long long M, N, K;
  double alpha, beta;
  const double *A, *B;
  double *C;
  long long lda, ldb, ldc;
  int nI, nJ, nks;
  long long Kp;                  // row stride of acs / bcs (K rounded up to BK)
  const double *acs, *bcs;       // (nI x Kp), (nJ x Kp) operand checksum vectors
  const double *arowabs, *aabsmax, *bcolabs, *babsmax;
  DevReport *rep;
  DevLoc *loc;
  long long loc_cap;
  DevFlip *flips;                // injection table (INJ kernels only)
  const int *tile_off;           // ntiles + 1 offsets into flips
  unsigned long long wait_limit_ns;
  // grids over a range of tiles: CTA b takes tile tile_base + b (MODE 1:
  // tile_base + b mod tile_count, split b / tile_count); tile_count 0 means
  // all nI x nJ tiles
  int tile_base, tile_count;
  // split-K (MODE 1 / 2 kernels)
  int nsplit, ks_slabs;          // number of k-splits, k-slabs per split
  int presummed;                 // MODE 2: slot 0 of each tile already holds the sum of its partial tiles
  int csums;                     // MODE 2: the beta-side sums of C come from ccs .. crsa (enc_c_kernel)
  double *W;                     // partial tiles, 128 x 128 each, slot split * tile_count + (tile - tile_base)
  double *wpc, *wpr;             // predicted-checksum partials [split][nI][N], [split][nJ][M]
  // unfused ablation (MODE 3): predicted checksums and C sums from separate passes
  const double *P1, *P2;         // nI x N (ld ldp1) and M x nJ (ld ldp2), column-major
  long long ldp1, ldp2;
  const double *ccs, *ccsa, *crs, *crsa;  // [I][N] column sums, [J][M] row sums of C (and |C|)
  int panel_slabs;               // PANEL kernels: verify the accumulators every panel_slabs k-slabs
  int correct_mode;              // 0: recompute located elements; 1: subtract the checksum residual
  double *Cout;                  // where the verified tile lives (p.C is the copy of C_in)
  long long ldcout;
};

// ---------------------------------------------------------------- split precision
constexpr int SP_BM = 128, SP_BN = 128, SP_BK = 64;  // bf16 k-slab of 128 bytes per row
constexpr int SP_STAGES = 4;
constexpr int SP_A_BYTES = SP_BM * SP_BK * 2, SP_B_BYTES = SP_BN * SP_BK * 2;  // 16 KiB each
constexpr int SP_STAGE_BYTES = SP_A_BYTES + SP_B_BYTES;
constexpr int SP_MAX_PAIRS = 128;
// INT8 slices: the row exponent of a row (column) of op(A) (op(B)) that
// holds a non-finite entry, whose products the kernel recomputes in FP64
constexpr int SPLIT_NONFINITE_ROW = -(1 << 20);
constexpr int SP_BK_I8 = 128;  // INT8 k-slab: 128 bytes per row, like the bf16 slab
constexpr int SP_RED_DOUBLES = (4 + 2) * 3 * 128 + 8;  // epilogue scratch of the split kernels
constexpr int SP_SMEM_BYTES = SP_STAGES * SP_STAGE_BYTES + 4 * SP_BK * 4 + 4 * 128 * 8 + 2 * 128 * 4 + 256 +
                              2 * SP_STAGES * 8 + SP_RED_DOUBLES * 8 + 1024;

struct SplitParams {
  long long M, N, K, Kp;        // Kp: K rounded up to SP_BK (slices are zero padded)
  double alpha, beta;
  int S, w, npairs, kchunk;     // slices, bits per slice, kept pairs, products per exact FP32 chunk
  int pair_s[SP_MAX_PAIRS], pair_t[SP_MAX_PAIRS];
  const int *eA, *eB;           // row exponents of op(A), column exponents of op(B)
  const double *A, *B;          // original operands (recomputation)
  long long lda, ldb;
  bool ta, tb;
  double *C;
  long long ldc;
  int nI, nJ;
  DevReport *rep;
  DevLoc *loc;
  long long loc_cap;
  unsigned long long wait_limit_ns;
  int verify;                   // 1: fault tolerant
  // injection: flips of the FP64 accumulator of (row, col) after pair `kstep` is folded in
  DevFlip *flips;
  const int *tile_off;
  int inj;
  // CK 2: FP64 predicted checksums (skinny GEMMs) and the absolute sums
  const double *P1, *P2;        // nI x N (ld ldp1), M x nJ (ld ldp2)
  long long ldp1, ldp2;
  const double *arowabs, *aabsmax, *bcolabs, *babsmax;
  // P1 / P2 computed by the same emulated product (else null): the
  // power-of-two scales of the checksum operands' rows (tile rows I of the
  // column sums of op(A), tile columns J of the row sums of op(B))
  const int *ePA, *ePB;
  // persistent kernel: one 128 x 128 FP64 tile per CTA, where the flagged
  // elements of a tile are recomputed before the tile is copied to C
  double *tscratch;
  // plain BF16 form (S == 0) with checks: the bf16 operands the product used
  // (rows of op(A) and columns of op(B), k contiguous, rows of ldk entries),
  // from which flagged elements are recomputed; and the predicted checksums
  // as sums of two pieces, the second at element offset p1_lo of P1 and
  // p2_lo of P2 (0: a single value)
  const uint16_t *Ab, *Bb;
  long long ldk;
  long long p1_lo, p2_lo;
  // INT8 slices (mma.sync s8): rows / columns marked SPLIT_NONFINITE_ROW in
  // eA / eB are recomputed in FP64
  int i8;
};


// One problem of a batch: its TMA descriptors (global memory, 128-byte
// aligned like every CUtensorMap) and its parameters (rep/loc/flips point at
// the problem's own slices).
struct __align__(128) BatchProblem {
  CUtensorMap tmA, tmB, tmC;
  Params p;
};
static_assert(alignof(BatchProblem) == 128 && alignof(CUtensorMap) == 128, "descriptor alignment");

constexpr int ERR_TIMEOUT = 2;

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of an mbarrier.  Gives up after limit_ns
// nanoseconds of %globaltimer (or 2^28 polls, whichever comes first), records
// ERR_TIMEOUT in the device report and returns false; never traps.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long limit_ns, int *err) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = globaltimer_ns();
  for (uint32_t it = 1; it < (1u << 28); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0 && globaltimer_ns() - t0 > limit_ns) break;
  }
  atomicExch(err, ERR_TIMEOUT);
  return false;
}

// Byte offset of element (row, k) of a [rows][16] fp64 tile written by TMA with
// 128-byte swizzle: the 16-byte chunk index is XORed with row % 8.
__device__ __forceinline__ int swz_off(int row, int k) {
  return row * 128 + ((((k >> 1) ^ (row & 7)) << 4) | ((k & 1) << 3));
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1,
                                            int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int c0, int c1) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(c0), "r"(c1)
               : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, uint32_t src, int c0, int c1, int c2) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(src), "r"(c0), "r"(c1), "r"(c2)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Untiled bulk copy global -> shared (16-byte aligned addresses, size % 16 == 0).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Named barrier over the 256 compute threads (barrier 0 is __syncthreads).
__device__ __forceinline__ void compute_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// v[0..15]: this lane's values of 16 columns.  Returns in lane l the sum of
// column l mod 16 over the warp's 32 lanes (v is overwritten).
__device__ __forceinline__ double colsum16(double (&v)[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const double send = up ? v[i] : v[i + o], keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// x rounded to bf16, to nearest with ties to even (the result of
// __double2bfloat16): the fields are rounded with integer operations when the
// result is a normal bf16 number or overflows, the conversion handles zeros,
// subnormal results, Inf and NaN.
__device__ __forceinline__ uint32_t bf16_rn_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF), eb = E - 1023 + 127;
  if (E != 0x7FF && eb >= 1 && eb <= 254) {
    const unsigned long long rest = b & ((1ull << 45) - 1ull), half = 1ull << 44;
    uint32_t v = ((uint32_t)eb << 7) | (uint32_t)((b >> 45) & 0x7Fu);
    v += (rest > half || (rest == half && (v & 1u))) ? 1u : 0u;  // a carry moves into the exponent (or to Inf)
    return ((uint32_t)(b >> 48) & 0x8000u) | v;
  }
  return (uint32_t)__bfloat16_as_ushort(__double2bfloat16(x));
}

// |x| rounded upward to FP32 (the result of __double2float_ru(fabs(x)), a NaN
// for a NaN), with integer operations only, on the two 32-bit halves of x (a
// mask of the 64-bit pattern reads as fabs and would take the FP64 pipe): the
// absolute sums of the detection thresholds run over every element of the
// operands and of partly filled tiles (zeros included), and the FP64 pipe is
// this GPU's scarcest unit.
__device__ __forceinline__ float f32_ru_abs(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x) & 0x7FFFFFFFu, lo = (uint32_t)__double2loint(x);
  const int E = (int)(hi >> 20), ef = E - 1023 + 127;
  if (ef >= 1 && ef <= 254) {  // a normal FP32 result (or, by the carry, Inf)
    uint32_t v = ((uint32_t)ef << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    v += (lo & 0x1FFFFFFFu) ? 1u : 0u;  // a carry moves into the exponent (or to Inf)
    return __uint_as_float(v);
  }
  if (ef > 254)  // NaN; Inf
    return __uint_as_float((hi > 0x7FF00000u || (hi == 0x7FF00000u && lo != 0u)) ? 0x7FFFFFFFu : 0x7F800000u);
  if ((hi | lo) == 0u) return 0.0f;
  // below FP32's normal range: |x| = m 2^(max(E,1) - 1075), that is m 2^-sh in
  // units of FP32's smallest subnormal 2^-149 (sh >= 30), rounded up; q <= 2^23
  // (2^23 is the bit pattern of the smallest normal number)
  const unsigned long long m = ((unsigned long long)(hi & 0xFFFFFu) << 32 | lo) | (E ? (1ull << 52) : 0ull);
  const int sh = 926 - (E ? E : 1);
  const uint32_t q = sh >= 64 ? 1u : (uint32_t)(m >> sh) + ((m & ((1ull << sh) - 1ull)) ? 1u : 0u);
  return __uint_as_float(q);
}

// x rounded to FP32, to nearest with ties to even (the result of
// __double2float_rn): the fields are rounded with integer operations when the
// result is a normal FP32 number or overflows, the conversion handles zeros,
// subnormal results, Inf and NaN.  Keeps the C-side checksum sums of the
// plain BF16 form off the FP64 pipe.
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF), ef = E - 1023 + 127;
  if (E != 0x7FF && ef >= 1 && ef <= 254) {
    const unsigned long long rest = b & ((1ull << 29) - 1ull), half = 1ull << 28;
    uint32_t v = ((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu);
    v += (rest > half || (rest == half && (v & 1u))) ? 1u : 0u;  // a carry moves into the exponent (or to Inf)
    return __uint_as_float(((uint32_t)(b >> 32) & 0x80000000u) | v);
  }
  return __double2float_rn(x);
}

__device__ __forceinline__ double flip_bit(double x, int bit) {
  return __longlong_as_double(__double_as_longlong(x) ^ (1ll << bit));
}

}  // namespace ftg
