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

// Batched checksum pass: one item per operand of each problem of a batch;
// every block covers one 128-wide group of one item over the item's whole
// other dimension, so each result is written once (no partials).
struct EncItem {
  const double *X;       // column-major R x S
  long long R, S, ld;
  double *gsum;          // group sums, gsum[G * gstride + (s or r)]
  long long gstride;
  double *absv;          // SEG: row abs sums (R); STR: column abs sums (S)
  double *gmax;          // per group: max of the group's abs sums
  int first_block;       // prefix sum of the items' group counts
  int pad;
};

__device__ __forceinline__ int find_item(const EncItem *items, int nitems, int b) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].first_block <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// SEG over groups of 128 rows, all columns of the item in one block; warp w
// takes batches of 16 columns (16w, 16w + 128, ...), reduced by the
// transposing butterfly as in enc_seg_kernel.
__global__ void __launch_bounds__(256) enc_seg_batched_kernel(const EncItem *__restrict__ items, int nitems) {
  __shared__ double sh[8][128];
  __shared__ double smx[8];
  const int it = find_item(items, nitems, blockIdx.x);
  const EncItem &E = items[it];
  const int G = blockIdx.x - E.first_block;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long r0 = (long long)G * 128;
  double rabs[4] = {0.0, 0.0, 0.0, 0.0};
  double mx = 0.0;
  for (long long sb = 16 * w; sb < E.S; sb += 128) {
    double ps[16], pa[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const long long s = sb + j;
      double v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long r = r0 + lane + 32 * q;
        v[q] = (r < E.R && s < E.S) ? E.X[r + s * E.ld] : 0.0;
        rabs[q] += fabs(v[q]);
      }
      ps[j] = (v[0] + v[1]) + (v[2] + v[3]);
      pa[j] = (fabs(v[0]) + fabs(v[1])) + (fabs(v[2]) + fabs(v[3]));
    }
    const double sum = colsum16(ps, lane), ab = colsum16(pa, lane);
    const long long s = sb + (lane & 15);
    if (lane < 16 && s < E.S) {
      E.gsum[(long long)G * E.gstride + s] = sum;
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
    if (r < E.R) E.absv[r] = t;
  }
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < 8; ++q) m = fmax(m, smx[q]);
    E.gmax[G] = m;
  }
}

// STR over groups of 128 columns, all rows of the item in one block, in
// chunks of 64 rows: warp w takes the group's columns 16w..16w+15, lane l the
// rows l and l + 32 of a chunk; the columns' absolute sums stay per lane in
// registers and are reduced once at the end (transposing butterfly), the
// rows' sums go through shared memory once per chunk.
__global__ void __launch_bounds__(256) enc_str_batched_kernel(const EncItem *__restrict__ items, int nitems) {
  __shared__ double srs[8][64], sra[8][64];
  __shared__ double smx[2];
  const int it = find_item(items, nitems, blockIdx.x);
  const EncItem &E = items[it];
  const int G = blockIdx.x - E.first_block;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = (long long)G * 128;
  const int ns = (int)min(128LL, E.S - s0);
  double cab[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) cab[q] = 0.0;
  double mloc = 0.0;
  for (long long r0 = 0; r0 < E.R; r0 += 64) {
    const long long ra = r0 + lane, rb = ra + 32;
    double rs_a = 0.0, rs_b = 0.0, ab_a = 0.0, ab_b = 0.0;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int sl = w * 16 + q;
      double va = 0.0, vb = 0.0;
      if (sl < ns) {
        const double *col = E.X + (s0 + sl) * E.ld;
        if (ra < E.R) va = col[ra];
        if (rb < E.R) vb = col[rb];
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
      if (r < E.R) {
        E.gsum[(long long)G * E.gstride + r] = t;
        mloc = fmax(mloc, ta);
      }
    }
    __syncthreads();
  }
  const double cs = colsum16(cab, lane);
  if (lane < 16 && w * 16 + lane < ns) E.absv[s0 + w * 16 + lane] = cs;
  if (threadIdx.x < 64) {
    const double m = warp_max(mloc);
    if (lane == 0) smx[w] = m;
  }
  __syncthreads();
  if (threadIdx.x == 0) E.gmax[G] = fmax(smx[0], smx[1]);
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
