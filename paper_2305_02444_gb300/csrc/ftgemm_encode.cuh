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

// The finish of a group of the pass, run by the block that completes the
// group last (the others' partials are visible: each block fences its
// partials before counting itself done): abs_out[x] = sum over the chunks c
// of part_abs[c * L + x] for the group's 128 entries x0 .. (ascending c: a
// fixed order), gmax[G] = max over c of part_max[c * nG + G].  The counter
// goes back to zero for the next pass.
__device__ __forceinline__ void enc_group_finish(unsigned int *cnt, int G, int nG, int nch, long long x0,
                                                 long long L, const double *part_abs, const double *part_max,
                                                 double *abs_out, double *gmax) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&cnt[G], 1u) == (unsigned)(nch - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x < 128 && x0 + threadIdx.x < L) {
    const long long x = x0 + threadIdx.x;
    double t = 0.0;
    for (int c = 0; c < nch; ++c) t += __ldcg(part_abs + (long long)c * L + x);
    abs_out[x] = t;
  }
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int c = 0; c < nch; ++c) m = fmax(m, __ldcg(part_max + (long long)c * nG + G));
    gmax[G] = m;
    cnt[G] = 0u;
  }
}

// grid (nG, ceil(S / cw)), 256 threads; block (G, c) covers columns c*cw ..
// c*cw + cw - 1 of the 128-row group G.  Warp w takes batches of 16 columns
// (16w, 16w + 128, ...), lane l the rows l + 32q (q < 4) of each column; a
// column's sum and absolute sum are the lanes' 4-row partials reduced by the
// transposing butterfly (16 shuffled adds per 16 columns, not 5 per column:
// this pass runs on the FP64 pipe, GB300's scarcest unit).
__global__ void __launch_bounds__(256) enc_seg_kernel(const double *__restrict__ X, long long R, long long S,
                                                      long long ld, double *__restrict__ gsum, long long gstride,
                                                      double *__restrict__ part_rabs, double *__restrict__ part_max,
                                                      int cw, unsigned int *__restrict__ cnt,
                                                      double *__restrict__ rabs_out, double *__restrict__ gmax) {
  __shared__ double sh[8][128];
  __shared__ double smx[8];
  const int G = blockIdx.x, c = blockIdx.y, nG = gridDim.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)G * 128;
  double rabs[4] = {0.0, 0.0, 0.0, 0.0};
  double mx = 0.0;
  const long long c0 = (long long)c * cw, s1 = min(S, c0 + cw);
  for (long long sb = c0 + 16 * w; sb < s1; sb += 128) {
    double ps[16], pa[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long s = sb + j;
      double v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long r = r0 + lane + 32 * q;
        v[q] = (s < s1 && r < R) ? X[r + s * ld] : 0.0;
        rabs[q] += fabs(v[q]);
      }
      ps[j] = (v[0] + v[1]) + (v[2] + v[3]);
      pa[j] = (fabs(v[0]) + fabs(v[1])) + (fabs(v[2]) + fabs(v[3]));
    }
    const double sum = colsum16(ps, lane), ab = colsum16(pa, lane);
    const long long s = sb + (lane & 15);
    if (lane < 16 && s < s1) {
      gsum[(long long)G * gstride + s] = sum;
      mx = fmax(mx, ab);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[w][lane + 32 * q] = rabs[q];
  mx = warp_max(mx);
  if (lane == 0) smx[w] = mx;
  __syncthreads();
  if (threadIdx.x < 128) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += sh[q][threadIdx.x];
    const long long r = r0 + threadIdx.x;
    if (r < R) part_rabs[(long long)c * R + r] = t;
  }
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < 8; ++q) m = fmax(m, smx[q]);
    part_max[(long long)c * nG + G] = m;
  }
  enc_group_finish(cnt, G, nG, (int)gridDim.y, r0, R, part_rabs, part_max, rabs_out, gmax);
}

// grid (nG, ceil(R / (64 nsub))), 256 threads: a block covers nsub chunks of
// 64 rows of one 128-column group; warp w takes the group's columns
// 16w..16w+15, lane l the rows l and l + 32 of a chunk.  A column's absolute
// sum is kept per lane over the block's rows and reduced once at the end (the
// transposing butterfly over the warp's 16 columns).
__global__ void __launch_bounds__(256) enc_str_kernel(const double *__restrict__ X, long long R, long long S,
                                                      long long ld, double *__restrict__ gsum, long long gstride,
                                                      double *__restrict__ part_cabs, double *__restrict__ part_max,
                                                      int nsub, unsigned int *__restrict__ cnt,
                                                      double *__restrict__ cabs_out, double *__restrict__ gmax) {
  static_assert(ENC_CHUNK == 64, "two rows per lane");
  __shared__ double srs[8][64], sra[8][64];
  __shared__ double smx[2];
  const int G = blockIdx.x, c = blockIdx.y, nG = gridDim.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = (long long)G * 128;
  const int ns = (int)min(128LL, S - s0);
  double cab[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) cab[q] = 0.0;
  double mloc = 0.0;  // largest row absolute sum seen by this thread (threads < 64)
  for (int sub = 0; sub < nsub; ++sub) {
    const long long r0 = ((long long)c * nsub + sub) * 64, ra = r0 + lane, rb = ra + 32;
    if (r0 >= R) break;
    double rs_a = 0.0, rs_b = 0.0, ab_a = 0.0, ab_b = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int sl = w * 16 + q;
      double va = 0.0, vb = 0.0;
      if (sl < ns) {
        const double *col = X + (s0 + sl) * ld;
        if (ra < R) va = col[ra];
        if (rb < R) vb = col[rb];
      }
      rs_a += va;
      rs_b += vb;
      ab_a += fabs(va);
      ab_b += fabs(vb);
      cab[q] += fabs(va) + fabs(vb);
    }
    srs[w][lane] = rs_a;
    srs[w][lane + 32] = rs_b;
    sra[w][lane] = ab_a;
    sra[w][lane + 32] = ab_b;
    __syncthreads();
    if (threadIdx.x < 64) {
      const long long r = r0 + threadIdx.x;
      double t = 0.0, ta = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        t += srs[q][threadIdx.x];
        ta += sra[q][threadIdx.x];
      }
      if (r < R) {
        gsum[(long long)G * gstride + r] = t;
        mloc = fmax(mloc, ta);
      }
    }
    __syncthreads();
  }
  const double cs = colsum16(cab, lane);
  if (lane < 16 && w * 16 + lane < ns) part_cabs[(long long)c * S + s0 + w * 16 + lane] = cs;
  if (threadIdx.x < 64) {
    const double m = warp_max(mloc);
    if (lane == 0) smx[w] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) part_max[(long long)c * nG + G] = fmax(smx[0], smx[1]);
  enc_group_finish(cnt, G, nG, (int)gridDim.y, s0, S, part_cabs, part_max, cabs_out, gmax);
}

// Batched checksum pass: one item per operand of each problem of a batch, of
// the SEG or the STR shape; every block covers one 128-wide group of one item
// over the item's whole other dimension, so each result is written once (no
// partials).  The host orders the items by the length of their blocks,
// longest first, so that the long blocks start in the first wave.
//
// The checksum sums are FP64.  The absolute sums, which only bound the
// rounding in the detection thresholds, run on the FP32 pipe with upward
// rounding (each partial stays an upper bound of the FP64 sum), which leaves
// about one FP64 add per operand element.  Where the range makes an FP32
// absolute sum overflow or leaves it tiny (below 2^-90, where terms under
// FP32's normal range were rounded up to its smallest numbers), the block
// takes its absolute sums again in FP64.
struct EncItem {
  const double *X;       // column-major R x S
  long long R, S, ld;
  double *gsum;          // group sums, gsum[G * gstride + (s or r)]
  long long gstride;
  double *absv;          // SEG: row abs sums (R); STR: column abs sums (S)
  double *gmax;          // per group: max of the group's abs sums
  int first_block;       // prefix sum of the items' group counts
  int seg;               // 1: SEG, 0: STR
};

__device__ __forceinline__ int find_item(const EncItem *items, int nitems, int b) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].first_block <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// colsum16 on the FP32 pipe, every addition rounded upward.
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

// An FP32 absolute sum that does not stand for the FP64 one (see above).  A
// NaN (from a NaN operand) stands: the FP64 sum is NaN as well.
__device__ __forceinline__ bool abs32_loose(float s) { return isinf(s) || (s > 0.0f && s < 0x1p-90f); }

// Elements r and r + 1 (r even) of a column as one 16-byte load (the batched
// operands are 16-byte aligned with even leading dimensions); an element past
// the last row reads as zero.
__device__ __forceinline__ double2 load_pair(const double *col, long long r, long long R) {
  double2 v = make_double2(0.0, 0.0);
  if (r < R) {
    v = __ldg(reinterpret_cast<const double2 *>(col + r));
    if (r + 1 >= R) v.y = 0.0;
  }
  return v;
}

// SEG over the 128-row group G, all columns of the item: warp w takes batches
// of 8 columns (8w, 8w + 64, ...), lane l the rows 2l, 2l + 1, 2l + 64 and
// 2l + 65 of each column (two 16-byte loads; a batch's 16 loads are issued
// before any is used); a column's sum is the lanes' 4-row partials reduced by
// the transposing butterfly.
__device__ __forceinline__ void enc_seg_group(const EncItem &E, int G, float (*s_abs)[128], float *s_mx,
                                              double *s_md) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)G * 128;
  float rabs[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // rows 2l, 2l + 1, 2l + 64, 2l + 65
  float mx = 0.0f;
  for (long long sb = 8 * w; sb < E.S; sb += 64) {
    double2 v[8][2];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long s = sb + j;
      const double *col = E.X + min(s, E.S - 1) * E.ld;
#pragma unroll
      for (int h = 0; h < 2; ++h) v[j][h] = load_pair(col, r0 + 64 * h + 2 * lane, s < E.S ? E.R : 0);
    }
    double ps[8];
    float pa[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float a0 = f32_ru_abs(v[j][0].x), a1 = f32_ru_abs(v[j][0].y);
      const float a2 = f32_ru_abs(v[j][1].x), a3 = f32_ru_abs(v[j][1].y);
      rabs[0] = __fadd_ru(rabs[0], a0);
      rabs[1] = __fadd_ru(rabs[1], a1);
      rabs[2] = __fadd_ru(rabs[2], a2);
      rabs[3] = __fadd_ru(rabs[3], a3);
      ps[j] = (v[j][0].x + v[j][0].y) + (v[j][1].x + v[j][1].y);
      pa[j] = __fadd_ru(__fadd_ru(a0, a1), __fadd_ru(a2, a3));
    }
    const double sum = colsum8<double, false>(ps, lane);
    const float ab = colsum8<float, true>(pa, lane);
    const long long s = sb + (lane & 7);
    if (lane < 8 && s < E.S) {
      E.gsum[(long long)G * E.gstride + s] = sum;
      mx = fmaxf(mx, ab);
    }
  }
  s_abs[w][2 * lane] = rabs[0];
  s_abs[w][2 * lane + 1] = rabs[1];
  s_abs[w][2 * lane + 64] = rabs[2];
  s_abs[w][2 * lane + 65] = rabs[3];
  mx = warp_max(mx);
  if (lane == 0) s_mx[w] = mx;
  __syncthreads();
  float t = 0.0f, m = 0.0f;
  bool loose = false;
  const long long r = r0 + threadIdx.x;
  if (threadIdx.x < 128) {
#pragma unroll
    for (int q = 0; q < 8; ++q) t = __fadd_ru(t, s_abs[q][threadIdx.x]);
    loose = r < E.R && abs32_loose(t);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 8; ++q) m = fmaxf(m, s_mx[q]);
    loose = loose || abs32_loose(m);
  }
  if (!__syncthreads_or(loose)) {
    if (threadIdx.x < 128 && r < E.R) E.absv[r] = (double)t;
    if (threadIdx.x == 0) E.gmax[G] = (double)m;
    return;
  }
  // FP64 absolute sums: thread t the row r0 + t; warp w the columns w, w + 8, ...
  if (threadIdx.x < 128 && r < E.R) {
    double a = 0.0;
    for (long long s = 0; s < E.S; ++s) a += fabs(E.X[r + s * E.ld]);
    E.absv[r] = a;
  }
  double md = 0.0;
  for (long long s = w; s < E.S; s += 8) {
    double a = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long rr = r0 + lane + 32 * q;
      if (rr < E.R) a += fabs(E.X[rr + s * E.ld]);
    }
    md = fmax(md, warp_sum(a));
  }
  if (lane == 0) s_md[w] = md;
  __syncthreads();
  if (threadIdx.x == 0) {
    double g = 0.0;
    for (int q = 0; q < 8; ++q) g = fmax(g, s_md[q]);
    E.gmax[G] = g;
  }
}

// STR over the 128-column group G, all rows of the item: warp w takes the
// 64-row chunks w, w + 8, ..., lane l the rows 2l and 2l + 1 of a chunk over
// all of the group's columns (one 16-byte load per column; 16 columns' loads
// are issued before any is used), so a row's sum over the group stays in one
// lane (columns in ascending order).  The columns' absolute sums over the
// chunk are reduced across the warp by the transposing butterfly and kept per
// lane; the warps' parts are added once at the end.
__device__ __forceinline__ void enc_str_group(const EncItem &E, int G, float (*s_cab)[128], float *s_mx,
                                              double *s_md) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = (long long)G * 128;
  const int ns = (int)min(128LL, E.S - s0);
  // s_cab[w][c]: column c's absolute sum over warp w's chunks (the warp's own row)
  if (lane < 16) {
#pragma unroll
    for (int b = 0; b < 8; ++b) s_cab[w][16 * b + lane] = 0.0f;
  }
  __syncwarp();
  float mloc = 0.0f;
  for (long long r0 = 64LL * w; r0 < E.R; r0 += 512) {
    const long long r = r0 + 2 * lane;
    double rs0 = 0.0, rs1 = 0.0;
    float ra0 = 0.0f, ra1 = 0.0f;
#pragma unroll 1
    for (int b = 0; 16 * b < ns; ++b) {
      double2 v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int sl = 16 * b + q;
        v[q] = load_pair(E.X + (s0 + min(sl, ns - 1)) * E.ld, r, sl < ns ? E.R : 0);
      }
      float pc[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        rs0 += v[q].x;
        rs1 += v[q].y;
        const float fa = f32_ru_abs(v[q].x), fb = f32_ru_abs(v[q].y);
        ra0 = __fadd_ru(ra0, fa);
        ra1 = __fadd_ru(ra1, fb);
        pc[q] = __fadd_ru(fa, fb);
      }
      const float cs = colsum16_ru(pc, lane);
      if (lane < 16) s_cab[w][16 * b + lane] = __fadd_ru(s_cab[w][16 * b + lane], cs);
    }
    if (r < E.R) {
      E.gsum[(long long)G * E.gstride + r] = rs0;
      mloc = fmaxf(mloc, ra0);
    }
    if (r + 1 < E.R) {
      E.gsum[(long long)G * E.gstride + r + 1] = rs1;
      mloc = fmaxf(mloc, ra1);
    }
  }
  mloc = warp_max(mloc);
  if (lane == 0) s_mx[w] = mloc;
  __syncthreads();
  float cs = 0.0f, gm = 0.0f;
  bool loose = false;
  if (threadIdx.x < ns) {
#pragma unroll
    for (int q = 0; q < 8; ++q) cs = __fadd_ru(cs, s_cab[q][threadIdx.x]);
    loose = abs32_loose(cs);
  }
  if (threadIdx.x == 0) {
    for (int q = 0; q < 8; ++q) gm = fmaxf(gm, s_mx[q]);
    loose = loose || abs32_loose(gm);
  }
  if (!__syncthreads_or(loose)) {
    if (threadIdx.x < ns) E.absv[s0 + threadIdx.x] = (double)cs;
    if (threadIdx.x == 0) E.gmax[G] = (double)gm;
    return;
  }
  // FP64 absolute sums: thread t the column s0 + t; rows strided over the block
  if ((int)threadIdx.x < ns) {
    const double *col = E.X + (s0 + threadIdx.x) * E.ld;
    double a = 0.0;
    for (long long rr = 0; rr < E.R; ++rr) a += fabs(col[rr]);
    E.absv[s0 + threadIdx.x] = a;
  }
  double md = 0.0;
  for (long long rr = threadIdx.x; rr < E.R; rr += 256) {
    double a = 0.0;
    for (int sl = 0; sl < ns; ++sl) a += fabs(E.X[rr + (s0 + sl) * E.ld]);
    md = fmax(md, a);
  }
  md = warp_max(md);
  if (lane == 0) s_md[w] = md;
  __syncthreads();
  if (threadIdx.x == 0) {
    double g = 0.0;
    for (int q = 0; q < 8; ++q) g = fmax(g, s_md[q]);
    E.gmax[G] = g;
  }
}

__global__ void __launch_bounds__(256, 2) enc_batched_kernel(const EncItem *__restrict__ items, int nitems) {
  __shared__ float s_abs[8][128];
  __shared__ float s_mx[8];
  __shared__ double s_md[8];
  const int it = find_item(items, nitems, blockIdx.x);
  const EncItem &E = items[it];
  const int G = blockIdx.x - E.first_block;
  if (E.seg) enc_seg_group(E, G, s_abs, s_mx, s_md);
  else enc_str_group(E, G, s_abs, s_mx, s_md);
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
