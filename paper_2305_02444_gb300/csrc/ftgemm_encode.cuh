// Operand checksum pass: per-tile checksum vectors of op(A) and op(B) and the
// absolute sums the detection threshold uses (the A and B checksums of
// FT-GEMM §2.2/§2.3).  One read of each operand; deterministic (fixed
// reduction order; the partials of a group's chunks are combined by the
// block that completes the group last).
//
// Both operands reduce to the same two shapes on a column-major X (R x S):
//  SEG: groups of 128 consecutive rows; gsum[G][s] = sum_{r in G} X[r,s],
//       gmax[G] = max_s sum_{r in G} |X[r,s]|, rabs[r] = sum_s |X[r,s]|.
//       (op(A) with 'N': rows i, columns k.  op(B) with 'T': rows j, columns k.)
//  STR: groups of 128 consecutive columns; gsum[G][r] = sum_{s in G} X[r,s],
//       gmax[G] = max_r sum_{s in G} |X[r,s]|, cabs[s] = sum_r |X[r,s]|.
//       (op(A) with 'T': rows k, columns i.  op(B) with 'N': rows k, columns j.)
#pragma once

#include "ftgemm_common.cuh"

namespace ftg {

constexpr int ENC_CHUNK = 64;  // unit of the chunked dimension; a block takes 1, 2 or 4 units

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The absolute sums, which only bound the rounding in the detection
// thresholds, in FP64 (ABS32 = false: the exact sums ftgemm_encode_operands
// returns) or on the FP32 pipe with every operation rounded upward (each
// partial stays an upper bound of the FP64 sum; the FP64 pipe is this GPU's
// scarcest unit).  Where FP32's range makes an absolute sum overflow or
// leaves it tiny (below 2^-90, where terms under FP32's normal range were
// rounded up to its smallest numbers), it is taken again in FP64.
template <bool ABS32> struct AbsAcc;
template <> struct AbsAcc<false> {
  using T = double;
  static __device__ __forceinline__ double of(double v) { return fabs(v); }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double mx(double a, double b) { return fmax(a, b); }
};
template <> struct AbsAcc<true> {
  using T = float;
  static __device__ __forceinline__ float of(double v) { return f32_ru_abs(v); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_ru(a, b); }
  static __device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
};

// An FP32 absolute sum that does not stand for the FP64 one (see above).  A
// NaN (from a NaN operand) stands: the FP64 sum is NaN as well.
__device__ __forceinline__ bool abs32_loose(float s) { return isinf(s) || (s > 0.0f && s < 0x1p-90f); }

// colsum16 for the absolute sums: FP64, or FP32 with every addition rounded
// upward.
__device__ __forceinline__ double colsum16_abs(double (&v)[16], int lane) { return colsum16(v, lane); }
__device__ __forceinline__ float colsum16_abs(float (&v)[16], int lane) {
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

// The transposing butterfly for 8 columns: lane l's v[c] is its part of
// column c; the result in lane l is the whole warp's sum of column l mod 8
// (3 levels exchange half of the columns each, 2 more add across lane bits 3
// and 4).  RU: FP32 with every addition rounded upward.
template <typename T, bool RU>
__device__ __forceinline__ T colsum8(T (&v)[8], int lane) {
  auto add = [](T x, T y) -> T {
    if constexpr (RU) return __fadd_ru(x, y);
    else return x + y;
  };
#pragma unroll
  for (int o = 4; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const T send = up ? v[i] : v[i + o], keep = up ? v[i + o] : v[i];
      v[i] = add(keep, __shfl_xor_sync(0xffffffffu, send, o));
    }
  }
  T t = add(v[0], __shfl_xor_sync(0xffffffffu, v[0], 8));
  return add(t, __shfl_xor_sync(0xffffffffu, t, 16));
}

// The FP64 absolute sums of one 128-wide group, from global memory (the rare
// path behind the FP32 ones), by the whole block: X(x, k) = X[k + x ld] when
// kfirst, else X[x + k ld]; x0 .. x0 + xv - 1 the group's x, L the k extent;
// absv[x] = sum over k of |X(x, k)|, *gmax = max over k of sum over the
// group's x of |X(x, k)|.  s_md: 8 doubles of shared memory.
__device__ __forceinline__ void enc_abs64_group(const double *X, long long ld, bool kfirst, long long x0, int xv,
                                                long long L, double *absv, double *gmax, double *s_md) {
  auto at = [&](long long x, long long k) { return kfirst ? X[k + x * ld] : X[x + k * ld]; };
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  if (tid < xv) {
    double a = 0.0;
    for (long long k = 0; k < L; ++k) a += fabs(at(x0 + tid, k));
    absv[x0 + tid] = a;
  }
  double md = 0.0;
  for (long long k = tid; k < L; k += blockDim.x) {
    double a = 0.0;
    for (int xx = 0; xx < xv; ++xx) a += fabs(at(x0 + xx, k));
    md = fmax(md, a);
  }
  md = warp_max(md);
  if (lane == 0) s_md[w] = md;
  __syncthreads();
  if (tid == 0) {
    double g = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) g = fmax(g, s_md[q]);
    *gmax = g;
  }
}

// The finish of a group of the pass, run by the block that completes the
// group last (the others' partials are visible: each block fences its
// partials before counting itself done): abs_out[x] = sum over the chunks c
// of part_abs[c * L + x] for the group's 128 entries x0 .. (ascending c: a
// fixed order), gmax[G] = max over c of part_max[c * nG + G].  With ABS32 the
// partials are FP32 upper bounds (summed rounded upward), and a group with a
// loose one takes its absolute sums again in FP64 (X, ld, kfirst, Lk: the
// operand, as enc_abs64_group takes it).  The counter goes back to zero for
// the next pass.
template <bool ABS32>
__device__ __forceinline__ void enc_group_finish(unsigned int *cnt, int G, int nG, int nch, long long x0,
                                                 long long L, const double *part_abs, const double *part_max,
                                                 double *abs_out, double *gmax, const double *X, long long ld,
                                                 bool kfirst, long long Lk) {
  using A = AbsAcc<ABS32>;
  using T = typename A::T;
  __shared__ int s_last;
  __shared__ double s_md[8];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cnt[G], 1u) == (unsigned)(nch - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  T t = (T)0, m = (T)0;
  bool loose = false;
  const long long x = x0 + threadIdx.x;
  const bool mine = threadIdx.x < 128 && x < L;
  if (mine) {
    for (int c = 0; c < nch; ++c) t = A::add(t, (T)__ldcg(part_abs + (long long)c * L + x));
    if constexpr (ABS32) loose = abs32_loose(t);
  }
  if (threadIdx.x == 0) {
    for (int c = 0; c < nch; ++c) m = A::mx(m, (T)__ldcg(part_max + (long long)c * nG + G));
    if constexpr (ABS32) loose = loose || abs32_loose(m);
  }
  bool redo = false;
  if constexpr (ABS32) redo = __syncthreads_or(loose) != 0;
  if (!redo) {
    if (mine) abs_out[x] = (double)t;
    if (threadIdx.x == 0) gmax[G] = (double)m;
  } else {
    enc_abs64_group(X, ld, kfirst, x0, (int)min(128LL, L - x0), Lk, abs_out, gmax + G, s_md);
  }
  if (threadIdx.x == 0) cnt[G] = 0u;
}

// grid (nG, ceil(S / cw)), 256 threads; block (G, c) covers columns c*cw ..
// c*cw + cw - 1 of the 128-row group G.  Warp w takes batches of 8 columns
// (8w, 8w + 64, ...), lane l the rows l + 32q (q < 4) of each column; a
// column's sum and absolute sum are the lanes' 4-row partials reduced by the
// transposing butterfly (9 shuffled adds per 8 columns, not 5 per column: the
// FP64 pipe is GB300's scarcest unit).
template <bool ABS32>
__global__ void __launch_bounds__(256) enc_seg_kernel(const double *__restrict__ X, long long R, long long S,
                                                      long long ld, double *__restrict__ gsum, long long gstride,
                                                      double *__restrict__ part_rabs, double *__restrict__ part_max,
                                                      int cw, unsigned int *__restrict__ cnt,
                                                      double *__restrict__ rabs_out, double *__restrict__ gmax) {
  using A = AbsAcc<ABS32>;
  using T = typename A::T;
  __shared__ T sh[8][128];
  __shared__ T smx[8];
  const int G = blockIdx.x, c = blockIdx.y, nG = gridDim.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)G * 128;
  T rabs[4] = {(T)0, (T)0, (T)0, (T)0};
  T mx = (T)0;
  const long long c0 = (long long)c * cw, s1 = min(S, c0 + cw);
  for (long long sb = c0 + 8 * w; sb < s1; sb += 64) {
    // the batch's 32 loads first: the absolute values' branches would
    // otherwise hold each load back until the previous value was used
    double v[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long s = sb + j, r = r0 + lane + 32 * q;
        v[j][q] = (s < s1 && r < R) ? X[r + s * ld] : 0.0;
      }
    double ps[8];
    T pa[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      T a[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = A::of(v[j][q]);
        rabs[q] = A::add(rabs[q], a[q]);
      }
      ps[j] = (v[j][0] + v[j][1]) + (v[j][2] + v[j][3]);
      pa[j] = A::add(A::add(a[0], a[1]), A::add(a[2], a[3]));
    }
    const double sum = colsum8<double, false>(ps, lane);
    const T ab = colsum8<T, ABS32>(pa, lane);
    const long long s = sb + (lane & 7);
    if (lane < 8 && s < s1) {
      gsum[(long long)G * gstride + s] = sum;
      mx = A::mx(mx, ab);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[w][lane + 32 * q] = rabs[q];
  mx = warp_max(mx);
  if (lane == 0) smx[w] = mx;
  __syncthreads();
  if (threadIdx.x < 128) {
    T t = (T)0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t = A::add(t, sh[q][threadIdx.x]);
    const long long r = r0 + threadIdx.x;
    if (r < R) part_rabs[(long long)c * R + r] = (double)t;
  }
  if (threadIdx.x == 0) {
    T m = (T)0;
    for (int q = 0; q < 8; ++q) m = A::mx(m, smx[q]);
    part_max[(long long)c * nG + G] = (double)m;
  }
  enc_group_finish<ABS32>(cnt, G, nG, (int)gridDim.y, r0, R, part_rabs, part_max, rabs_out, gmax, X, ld, false, S);
}

// grid (nG, ceil(R / (64 nsub))), 256 threads: a block covers nsub chunks of
// 64 rows of one 128-column group; warp w takes the group's columns
// 16w..16w+15, lane l the rows l and l + 32 of a chunk.  A column's absolute
// sum is kept per lane over the block's rows and reduced once at the end (the
// transposing butterfly over the warp's 16 columns).
template <bool ABS32>
__global__ void __launch_bounds__(256) enc_str_kernel(const double *__restrict__ X, long long R, long long S,
                                                      long long ld, double *__restrict__ gsum, long long gstride,
                                                      double *__restrict__ part_cabs, double *__restrict__ part_max,
                                                      int nsub, unsigned int *__restrict__ cnt,
                                                      double *__restrict__ cabs_out, double *__restrict__ gmax) {
  static_assert(ENC_CHUNK == 64, "two rows per lane");
  using A = AbsAcc<ABS32>;
  using T = typename A::T;
  __shared__ double srs[8][64];
  __shared__ T sra[8][64];
  __shared__ T smx[2];
  const int G = blockIdx.x, c = blockIdx.y, nG = gridDim.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = (long long)G * 128;
  const int ns = (int)min(128LL, S - s0);
  T cab[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) cab[q] = (T)0;
  T mloc = (T)0;  // largest row absolute sum seen by this thread (threads < 64)
  for (int sub = 0; sub < nsub; ++sub) {
    const long long r0 = ((long long)c * nsub + sub) * 64, ra = r0 + lane, rb = ra + 32;
    if (r0 >= R) break;
    double rs_a = 0.0, rs_b = 0.0;
    T ab_a = (T)0, ab_b = (T)0;
    // the chunk's 32 loads first (see enc_seg_kernel)
    double vs[16][2];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int sl = w * 16 + q;
      const double *col = X + (s0 + min(sl, ns - 1)) * ld;
      vs[q][0] = (sl < ns && ra < R) ? col[ra] : 0.0;
      vs[q][1] = (sl < ns && rb < R) ? col[rb] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double va = vs[q][0], vb = vs[q][1];
      rs_a += va;
      rs_b += vb;
      const T fa = A::of(va), fb = A::of(vb);
      ab_a = A::add(ab_a, fa);
      ab_b = A::add(ab_b, fb);
      cab[q] = A::add(cab[q], A::add(fa, fb));
    }
    srs[w][lane] = rs_a;
    srs[w][lane + 32] = rs_b;
    sra[w][lane] = ab_a;
    sra[w][lane + 32] = ab_b;
    __syncthreads();
    if (threadIdx.x < 64) {
      const long long r = r0 + threadIdx.x;
      double t = 0.0;
      T ta = (T)0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        t += srs[q][threadIdx.x];
        ta = A::add(ta, sra[q][threadIdx.x]);
      }
      if (r < R) {
        gsum[(long long)G * gstride + r] = t;
        mloc = A::mx(mloc, ta);
      }
    }
    __syncthreads();
  }
  const T cs = colsum16_abs(cab, lane);
  if (lane < 16 && w * 16 + lane < ns) part_cabs[(long long)c * S + s0 + w * 16 + lane] = (double)cs;
  if (threadIdx.x < 64) {
    const T m = warp_max(mloc);
    if (lane == 0) smx[w] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) part_max[(long long)c * nG + G] = (double)A::mx(smx[0], smx[1]);
  enc_group_finish<ABS32>(cnt, G, nG, (int)gridDim.y, s0, S, part_cabs, part_max, cabs_out, gmax, X, ld, true, R);
}

// Batched checksum pass: one item per operand of each problem of a batch;
// one block per 128-wide group of an item (the x dimension: rows i of op(A),
// columns j of op(B)), over the item's whole k dimension.  Each item comes
// in through the problem's own TMA map as the GEMM's 128 x 16 slabs, into a
// ring of ENC_STAGES slabs with bounded waits, so the loads of later slabs
// overlap the sums of the current one.  Per group G:
//   gsum[G][k] = sum over the group's x of X(x, k)        (FP64)
//   absv[x]    = sum over k of |X(x, k)|                   (per x)
//   gmax[G]    = max over k of sum over the group's x of |X(x, k)|
// The checksum sums are FP64.  The absolute sums, which only bound the
// rounding in the detection thresholds, run on the FP32 pipe with upward
// rounding (each partial stays an upper bound of the FP64 sum); where FP32's
// range makes one overflow or leaves it tiny (below 2^-90, where terms under
// FP32's normal range were rounded up to its smallest numbers), the block
// takes its absolute sums again in FP64 from global memory.  The host orders
// the items by their k extent, longest first, so the long blocks start in
// the first wave.
constexpr int ENC_STAGES = 3;
constexpr int ENC_SLAB = BM * BK * 8;  // one 128 x 16 slab, 16 KiB
constexpr int ENC_SMEM_BYTES = ENC_STAGES * ENC_SLAB + 1024;

struct EncItem {
  const CUtensorMap *map;  // the operand's TMA map (128 x 16 boxes), in global memory
  const double *X;         // the operand, column-major (for the FP64 absolute sums)
  long long ld;
  long long W, L;          // extents of x and k
  double *gsum;            // gsum[G * gstride + k], k < 16 * ceil(L / 16)
  long long gstride;
  double *absv;            // absv[x]
  double *gmax;            // gmax[G]
  int *err;                // the problem's report flag (a wait that timed out)
  int first_block;         // prefix sum of the items' group counts
  int kfirst;              // 1: X(x, k) = X[k + x ld], slab [128 x][16 k] 128-byte swizzled
                           // 0: X(x, k) = X[x + k ld], slab [16 k][128 x]
};

// 256 threads: thread t takes x = t mod 128 and the 8 k's 8h..8h+7 of every
// slab (h = t / 128).  A warp's 32 x's reduce each k by the transposing
// butterfly; the 4 warps of a half add their parts through shared memory in
// a fixed order.  A warp whose x's all lie past the group's last valid x
// skips its loads and sums.
// block_item[b]: the item of block b (a host-built map: one load instead of a
// search at the start of every block).
__global__ void __launch_bounds__(256) enc_batched_kernel(const EncItem *__restrict__ items,
                                                         const int *__restrict__ block_item, int *gerr,
                                                         unsigned long long limit_ns) {
  extern __shared__ unsigned char enc_smem_raw[];
  unsigned char *ring =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(enc_smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ double s_part[2][2][4][8];  // [slab parity][half][warp of the half][k]
  __shared__ float s_apart[2][2][4][8];
  __shared__ float s_xabs[128];
  __shared__ double s_md[8];
  __shared__ __align__(8) uint64_t s_full[ENC_STAGES];
  __shared__ int s_stop;
  const EncItem E = items[block_item[blockIdx.x]];
  const int G = blockIdx.x - E.first_block;
  const long long x0 = (long long)G * 128;
  const int xv = (int)min(128LL, E.W - x0);
  const int nsl = (int)((E.L + BK - 1) / BK);
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31, x = tid & 127, h = tid >> 7;
  const bool wact = 32 * (w & 3) < xv;
  const uint32_t full0 = smem_u32(s_full);
  if (tid == 0) {
    s_stop = *reinterpret_cast<volatile int *>(gerr) != 0;
    for (int s = 0; s < ENC_STAGES; ++s) mbar_init(full0 + 8 * s, 1);
    fence_mbar_init();
    prefetch_tmap(E.map);
  }
  __syncthreads();
  if (s_stop) return;
  auto issue = [&](int s) {
    const int st = s % ENC_STAGES;
    const uint32_t fb = full0 + 8 * st, sb = smem_u32(ring + st * ENC_SLAB);
    mbar_arrive_expect_tx(fb, ENC_SLAB);
    if (E.kfirst) tma_load_2d(sb, E.map, fb, BK * s, (int)x0);
    else tma_load_2d(sb, E.map, fb, (int)x0, BK * s);
  };
  int issued = 0;
  if (tid == 0)
    for (; issued < ENC_STAGES && issued < nsl; ++issued) issue(issued);
  float xa = 0.0f;    // this thread's x: |X(x, k)| over its k's, rounded upward
  float kmax = 0.0f;  // threads < 16: the largest group absolute sum of the k's they finished
  bool ok = true;
  int s = 0;
  for (; s < nsl; ++s) {
    const int st = s % ENC_STAGES;
    if (!mbar_wait_bounded(full0 + 8 * st, (s / ENC_STAGES) & 1, limit_ns, E.err)) ok = false;
    double ps[8];
    float pa[8];
    if (ok && wact) {
      const unsigned char *sl = ring + st * ENC_SLAB;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = 8 * h + c;
        const double v = E.kfirst ? *reinterpret_cast<const double *>(sl + swz_off(x, k))
                                  : reinterpret_cast<const double *>(sl)[k * BM + x];
        ps[c] = v;
        pa[c] = f32_ru_abs(v);
        xa = __fadd_ru(xa, pa[c]);
      }
      const double cs = colsum8<double, false>(ps, lane);
      const float ca = colsum8<float, true>(pa, lane);
      if (lane < 8) {
        s_part[s & 1][h][w & 3][lane] = cs;
        s_apart[s & 1][h][w & 3][lane] = ca;
      }
    } else if (lane < 8) {
      s_part[s & 1][h][w & 3][lane] = 0.0;
      s_apart[s & 1][h][w & 3][lane] = 0.0f;
    }
    // one barrier per slab: stage st is read and the partials are in; the
    // partials alternate between two buffers, so the next slab's cannot
    // overwrite these before they are read (a thread writes slab s + 2's
    // only after passing slab s + 1's barrier, which the readers of slab s
    // reach after reading)
    if (__syncthreads_or(!ok)) break;
    if (tid == 0 && issued < nsl) issue(issued++);
    if (tid < 16) {
      const int hh = tid >> 3, c = tid & 7;
      const double(*pp)[8] = s_part[s & 1][hh];
      const float(*pa2)[8] = s_apart[s & 1][hh];
      const double g = ((pp[0][c] + pp[1][c]) + pp[2][c]) + pp[3][c];
      const float ga = __fadd_ru(__fadd_ru(pa2[0][c], pa2[1][c]), __fadd_ru(pa2[2][c], pa2[3][c]));
      E.gsum[(long long)G * E.gstride + BK * s + tid] = g;
      kmax = fmaxf(kmax, ga);
    }
  }
  if (s < nsl) {  // a wait timed out: stop the batch; the copies in flight get a bounded chance to land
    if (tid == 0) {
      atomicExch(gerr, ERR_TIMEOUT);
      for (int q = s; q < issued; ++q)
        mbar_wait_bounded(full0 + 8 * (q % ENC_STAGES), (q / ENC_STAGES) & 1, limit_ns, E.err);
    }
    return;
  }
  if (h) s_xabs[x] = xa;
  __syncthreads();
  float xs = 0.0f, gm = 0.0f;
  bool loose = false;
  if (!h) {
    xs = __fadd_ru(xa, s_xabs[x]);
    loose = x < xv && abs32_loose(xs);
  }
  if (w == 0) {
    gm = warp_max(kmax);
    loose = loose || (lane == 0 && abs32_loose(gm));
  }
  if (!__syncthreads_or(loose)) {
    if (!h && x < xv) E.absv[x0 + x] = (double)xs;
    if (tid == 0) E.gmax[G] = (double)gm;
    return;
  }
  enc_abs64_group(E.X, E.ld, E.kfirst != 0, x0, xv, E.L, E.absv, E.gmax + G, s_md);
}

// One pass over C that takes, per 128x128 tile, the column sums over the
// tile's rows and the row sums over its columns (and the absolute sums, FP32
// with upward rounding), with the fused epilogue's thread mapping and order,
// so the sums have the epilogue's bits.  The unfused ablation also keeps a
// copy of C_in in Cc (needed to recompute an element after the GEMM overwrote
// C); the split-K reduction of small grids takes the sums alone (Cc null).
// grid = tiles, 256 threads, 128 KiB dynamic shared memory.
__global__ void __launch_bounds__(256) enc_c_kernel(const double *__restrict__ C, long long ldc,
                                                    double *__restrict__ Cc, long long ldcc, long long M,
                                                    long long N, int nI, double *__restrict__ ccs,
                                                    double *__restrict__ ccsa, double *__restrict__ crs,
                                                    double *__restrict__ crsa) {
  extern __shared__ double tbuf[];  // [128 columns][128 rows]
  __shared__ double part[4][128];
  const int tile = blockIdx.x, I = tile % nI, J = tile / nI;
  const long long i0 = (long long)I * 128, j0 = (long long)J * 128;
  const int mI = (int)min(128LL, M - i0), nJt = (int)min(128LL, N - j0);
  for (int e = threadIdx.x; e < 128 * 128; e += 256) {
    const int il = e & 127, jl = e >> 7;
    double v = 0.0;
    if (il < mI && jl < nJt) {
      v = C[(i0 + il) + (j0 + jl) * ldc];
      if (Cc) Cc[(i0 + il) + (j0 + jl) * ldcc] = v;
    }
    tbuf[jl * 128 + il] = v;
  }
  __syncthreads();
  const int r = threadIdx.x & 127, h = threadIdx.x >> 7;
  double rs = 0.0, cs = 0.0;
  float ra = 0.0f, ca = 0.0f;
  for (int q = 0; q < 64; ++q) {
    const double vr = tbuf[(64 * h + q) * 128 + r];
    const double vc = tbuf[r * 128 + 64 * h + ((q + r) & 63)];
    rs += vr;
    cs += vc;
    ra = __fadd_ru(ra, f32_ru_abs(vr));
    ca = __fadd_ru(ca, f32_ru_abs(vc));
  }
  if (h) { part[0][r] = rs; part[1][r] = cs; part[2][r] = (double)ra; part[3][r] = (double)ca; }
  __syncthreads();
  if (!h) {
    if (r < mI) {
      crs[(long long)J * M + i0 + r] = rs + part[0][r];
      crsa[(long long)J * M + i0 + r] = (double)__fadd_ru(ra, (float)part[2][r]);
    }
    if (r < nJt) {
      ccs[(long long)I * N + j0 + r] = cs + part[1][r];
      ccsa[(long long)I * N + j0 + r] = (double)__fadd_ru(ca, (float)part[3][r]);
    }
  }
}

// Split-K partial tiles (nsplit x ntile slots of BM x BN doubles, slot
// split * ntile + tile) summed into slot 0 of each tile in ascending split
// order, as the reduction kernel adds them (0 + W0 + W1 + ...: the same bits),
// spread over the whole GPU instead of one CTA per tile.
__global__ void splitk_sum_kernel(double *__restrict__ W, long long ntile, int nsplit) {
  const long long total = ntile * BM * BN;  // doubles per split; even
  for (long long e = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); e < total;
       e += 2LL * gridDim.x * blockDim.x) {
    double x = 0.0, y = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) {
      const double2 v = *reinterpret_cast<const double2 *>(W + (long long)sp * total + e);
      x += v.x;
      y += v.y;
    }
    *reinterpret_cast<double2 *>(W + e) = make_double2(x, y);
  }
}

// C <- beta*C (beta == 0 writes zeros without reading C)
__global__ void scale_kernel(double *C, long long M, long long N, long long ldc, double beta) {
  const long long total = M * N;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e % M, j = e / M;
    double *c = C + i + j * ldc;
    *c = (beta == 0.0) ? 0.0 : beta * *c;
  }
}

// dst[r + c*ldd] = src[r + c*lds] for r < rows, c < cols
__global__ void copy2d_kernel(const double *__restrict__ src, long long lds, double *__restrict__ dst, long long ldd,
                              long long rows, long long cols) {
  const long long total = rows * cols;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e % rows, c = e / rows;
    dst[r + c * ldd] = src[r + c * lds];
  }
}

// One block waits on an mbarrier that nothing completes (test of the bounded wait).
__global__ void wait_timeout_kernel(DevReport *rep, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait_bounded(smem_u32(&bar), 0, limit_ns, &rep->err);
}

}  // namespace ftg
