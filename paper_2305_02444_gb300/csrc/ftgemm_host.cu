// Host side of libftgemm: the C ABI declared in include/ftgemm.h, argument
// checks, workspace, TMA descriptors, the operand checksum pass, the fault
// injection table and the report.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "ftgemm.h"
#include "ftgemm_common.cuh"
#include "ftgemm_encode.cuh"

namespace ftg {
// FP64 kernel launchers, one translation unit per operand layout
// (ftgemm_launch.cuh): any mode (0 whole tiles, 1 split-K partials, 2 split-K
// reduction, 3 verify-only pass), modes 0 and 1 optionally with the
// per-k-panel checks; and the persistent batched kernel
#define FTG_DECLARE_LAYOUT(XX)                                                                                     \
  cudaError_t launch_gemm_##XX(bool ft, bool inj, int mode, bool panel, const CUtensorMap &, const CUtensorMap &,  \
                               const CUtensorMap &, const CUtensorMap &, const Params &, cudaStream_t);            \
  cudaError_t launch_batched_##XX(bool, bool, const BatchProblem *, const int *, const int *, const int *, int,    \
                                  int, int *, int *, int, cudaStream_t);
FTG_DECLARE_LAYOUT(nn)
FTG_DECLARE_LAYOUT(nt)
FTG_DECLARE_LAYOUT(tn)
FTG_DECLARE_LAYOUT(tt)
#undef FTG_DECLARE_LAYOUT
cudaError_t launch_split(bool ta, bool tb, int ck, bool i8, const CUtensorMap &a, const CUtensorMap &b,
                         const SplitParams &p, cudaStream_t s);
cudaError_t launch_split_tc(bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &b,
                            const SplitParams &p, cudaStream_t s);
cudaError_t launch_split_tcp(bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &b,
                             const SplitParams &p, int nctas, cudaStream_t s);
cudaError_t launch_slicing(const double *X, long long ld, int trans, long long R, long long K, long long Kp, int *e,
                           int S, int w, int plain, int i8, void *out, unsigned long long *mb, int nsm,
                           cudaStream_t s);
long long bf16_checksum_scratch(long long R, long long Kp);
cudaError_t launch_bf16_checksums(const void *X, long long R, long long Kp, void *pieces, double *rowabs,
                                  double *gmax, float *part, cudaStream_t s);
}  // namespace ftg

using namespace ftg;

namespace {

constexpr long long LOC_CAP_DEV = 65536;
constexpr int MAX_DEV = 64;

std::atomic<long long> g_launches{0};
std::mutex g_mu;

struct Buf {
  void *p = nullptr;
  size_t cap = 0;
};

struct Workspace {
  bool init = false;
  Buf acs, bcs, arowabs, aabsmax, bcolabs, babsmax, part_abs, part_max;
  Buf part_abs2, part_max2, enc_cnt;  // op(B)'s partials, group counters of the checksum pass
  Buf rep, loc, flips;              // flips: the injection table, then its per-tile offsets
  Buf stA, stB, stC;        // aligned copies of unaligned operands
  Buf hA, hB, hC;           // device copies for ftgemm_d_host
  Buf W, wpc, wpr;          // split-K partial tiles and predicted-checksum partials
  Buf uC, uccs, uccsa, ucrs, ucrsa, uP1, uP2;  // unfused ablation: copy of C, C sums, skinny GEMMs
  Buf spA, spB, spEA, spEB;  // split precision: bf16 slices and row/column exponents
  Buf spPA, spPB, spEPA, spEPB;  // slices / exponents of the checksum operands (tcgen05 engine, ft = 2)
  Buf tscr;                      // persistent split kernel: one FP64 tile per CTA for flagged tiles
  Buf spMB;                      // row maxima of the slicing passes
  cudaStream_t side = nullptr;   // second stream for independent work inside one call (fork / join)
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int nsm = 0;              // SM count
  Buf pin;                  // pinned host staging of the report and location copies
  Buf ipin[2];              // pinned staging of the injection upload, used in turn
  cudaEvent_t ipin_ev[2] = {nullptr, nullptr};  // recorded after each staging buffer's copies
  int ipin_next = 0;
  bool encc_attr = false;   // enc_c_kernel's shared-memory attribute set on this device
  // ftgemm_d_host with column panels: copy streams, events, the panels'
  // report regions and fault tables
  cudaStream_t up = nullptr, down = nullptr;
  std::vector<cudaEvent_t> pev;
  Buf prep, ploc, pfl;
  Buf ppin;  // pinned staging of the panels' fault tables, one region per panel
  // the last injected call, for ftgemm_injection_log: one segment per fault
  // table (a call of panels has one per panel)
  struct LogSeg {
    const DevFlip *dev;
    std::vector<long long> orig;  // sorted position in the table -> index of the fault in the call
    long long col_off;            // added to the table's columns (the panel's first column)
  };
  long long last_nflips = 0;
  std::vector<LogSeg> last_log;
};
Workspace g_ws[MAX_DEV];

// Optional CUDA-event timing of the library's own kernels (ftgemm_timing).
struct TimingState {
  bool on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> main_ev, aux_ev;
} g_tim;

void timing_record(std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &v, cudaEvent_t *a, cudaEvent_t *b) {
  cudaEventCreate(a);
  cudaEventCreate(b);
  v.emplace_back(*a, *b);
}

struct InjState {
  int mode = 0;
  unsigned long long seed = 0;
  long long count = 0;
  std::vector<ftgemm_flip> list;
} g_inj;

bool is_n(char t) { return t == 'N' || t == 'n'; }
bool is_t(char t) { return t == 'T' || t == 't' || t == 'C' || t == 'c'; }

int check_args(char ta, char tb, long long M, long long N, long long K, long long lda, long long ldb,
               long long ldc) {
  if (!is_n(ta) && !is_t(ta)) return -1;
  if (!is_n(tb) && !is_t(tb)) return -2;
  if (M < 0) return -3;
  if (N < 0) return -4;
  if (K < 0) return -5;
  const long long arows = is_n(ta) ? M : K, brows = is_n(tb) ? K : N;
  if (lda < std::max(1LL, arows)) return -8;
  if (ldb < std::max(1LL, brows)) return -10;
  if (ldc < std::max(1LL, M)) return -13;
  return 0;
}

int ensure(Buf &b, size_t bytes) {
  if (b.cap >= bytes && b.p) return 0;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t n = std::max<size_t>(bytes, 256);
  if (cudaMalloc(&b.p, n) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_NOMEM;
  }
  b.cap = n;
  return 0;
}

int ensure_pinned(Buf &b, size_t bytes) {
  if (b.cap >= bytes && b.p) return 0;
  if (b.p) cudaFreeHost(b.p);
  b.p = nullptr;
  b.cap = 0;
  size_t n = std::max<size_t>(bytes, 4096);
  if (cudaMallocHost(&b.p, n) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_NOMEM;
  }
  b.cap = n;
  return 0;
}

Workspace *workspace(int *dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) {
    cudaGetLastError();
    return nullptr;
  }
  *dev_out = dev;
  Workspace &w = g_ws[dev];
  if (!w.init) {
    if (ensure(w.rep, sizeof(DevReport)) || ensure(w.loc, sizeof(DevLoc) * LOC_CAP_DEV)) return nullptr;
    w.init = true;
  }
  return &w;
}

unsigned long long wait_limit_ns() {
  static unsigned long long v = [] {
    const char *e = getenv("FTGEMM_WAIT_LIMIT_NS");
    unsigned long long x = e ? strtoull(e, nullptr, 10) : 0;
    return x ? x : 2000000000ull;  // 2 s: a slab normally lands within microseconds
  }();
  return v;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// 2-D fp64 tensor map of a column-major matrix with `rows` x `cols` and leading dimension ld.
int make_map(CUtensorMap *m, const double *ptr, long long rows, long long cols, long long ld, int box0, int box1,
             bool swizzle128) {
  auto fn = encode_fn();
  if (!fn) return FTGEMM_ERR_TENSORMAP;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {(cuuint32_t)box0, (cuuint32_t)box1};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : FTGEMM_ERR_TENSORMAP;
}

bool tma_ok(const void *p, long long ld) {
  return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && (ld % 2 == 0) && (ld * 8 < (1LL << 40));
}

int grid_for(long long n) { return (int)std::min<long long>(std::max<long long>((n + 255) / 256, 1), 152 * 16); }

// split precision: 0 default (persistent tcgen05), 1 mma.sync, 2 tcgen05 with one CTA per tile,
// 5 persistent tcgen05, 7 mma.sync with INT8 slices
int g_split_engine = 0;
int g_correct = 0;  // correction rule of the FP64 kernels (ftgemm_set_correction)
int g_splitk = 0;  // 0 automatic, 1 never split, n >= 2 force n splits (ftgemm_set_splitk)
int g_panel = 0;   // verify the accumulators every g_panel k-slabs (0: only at the end of the tile)

// Number of k-splits for a grid of `ntiles` tiles and `nks` k-slabs on `nsm`
// SMs.  One CTA per SM: a grid of few tiles leaves SMs idle (64 tiles of a
// 1024^3 problem on 152 SMs), so the k loop is split and the partial tiles
// summed in a reduction kernel.  Cost model in units of one k-slab of one
// tile: waves x (slabs per split + per-CTA overhead) + reduction.
int choose_splits(long long ntiles, long long nks, int nsm) {
  if (g_splitk == 1) return 1;
  if (g_splitk >= 2) {
    const long long ks = (nks + g_splitk - 1) / g_splitk;
    return (int)((nks + ks - 1) / ks);
  }
  if (ntiles >= 4LL * nsm || nks < 8) return 1;
  double best = 1e300;
  int bestS = 1;
  for (int S = 1; S <= 32 && S <= nks; ++S) {
    const long long ks = (nks + S - 1) / S, Se = (nks + ks - 1) / ks;
    if (Se != S) continue;
    const long long waves = (ntiles * Se + nsm - 1) / nsm;
    double T = waves * (ks + 0.07);
    if (Se > 1) T += (double)((ntiles + nsm - 1) / nsm) * (0.03 * Se + 0.3);
    if (T < best - 1e-9) { best = T; bestS = (int)Se; }
  }
  return bestS;
}

// K-splits for the tail of a large grid (ntiles >= 4 x nsm, which
// choose_splits never splits): when the last wave holds rem = ntiles mod nsm
// tiles, splitting K of those tiles over S x rem CTAs costs ceil(S rem / nsm)
// waves of 1/S of a tile instead of one whole wave.  Returns the best S
// (1: leave the tail whole) when it saves at least 0.15 of a tile's time.
int choose_tail_splits(long long ntiles, long long nks, int nsm) {
  if (g_splitk != 0 || ntiles < 4LL * nsm) return 1;
  const long long rem = ntiles % nsm;
  if (rem == 0) return 1;
  double best = 1.0;
  int bestS = 1;
  for (int S = 2; S <= 16 && S <= nks / 8; ++S) {
    const long long ks = (nks + S - 1) / S;
    if ((nks + ks - 1) / ks != S) continue;
    const double waves = (double)((rem * S + nsm - 1) / nsm);
    const double T = waves * ((double)ks + 0.07) / (double)nks + (0.03 * S + 0.3) / (double)nks;
    if (T < best - 1e-9) { best = T; bestS = S; }
  }
  return best <= 0.85 ? bestS : 1;
}

// The k-split plan of one FP64 call: S splits (1: none) of the tiles
// [tail_base, ntiles), the tiles before tail_base whole.  (With per-k-panel
// verification each k-split checks its own panels.)
struct KSplit {
  int S;
  long long tail_base;
};
KSplit plan_ksplit(long long ntiles, long long nks, int nsm) {
  KSplit k{choose_splits(ntiles, nks, nsm), 0};
  // Large grids whose last wave is partly empty: the full waves take whole
  // tiles, the tail tiles split K over the idle SMs (then a verifying reduction).
  if (k.S <= 1) {
    const int St = choose_tail_splits(ntiles, nks, nsm);
    if (St > 1) {
      k.S = St;
      k.tail_base = ntiles - ntiles % nsm;
    }
  }
  return k;
}

// 3-D fp64 tensor map over nz column-major matrices of rows x cols (ld), stacked.
int make_map3(CUtensorMap *m, const double *ptr, long long rows, long long cols, long long nz, long long ld) {
  auto fn = encode_fn();
  if (!fn) return FTGEMM_ERR_TENSORMAP;
  cuuint64_t dims[3] = {(cuuint64_t)rows, (cuuint64_t)cols, (cuuint64_t)nz};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 8, (cuuint64_t)ld * cols * 8};
  cuuint32_t box[3] = {(cuuint32_t)BM, (cuuint32_t)BN, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : FTGEMM_ERR_TENSORMAP;
}

cudaError_t launch_copy(const double *src, long long lds, double *dst, long long ldd, long long rows,
                        long long cols, cudaStream_t s) {
  copy2d_kernel<<<grid_for(rows * cols), 256, 0, s>>>(src, lds, dst, ldd, rows, cols);
  g_launches++;
  return cudaGetLastError();
}

uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Encode the operand checksum vectors (see ftgemm_encode.cuh).  Writes
// acs (nI x Kp), aabsmax, arowabs, bcs (nJ x Kp), babsmax, bcolabs.
// Chunking of the operand checksum pass for one operand: a SEG pass (column
// sums of 128-row groups, over stored R x S with the S columns chunked) or a
// STR pass (row sums of 128-column groups, rows chunked).  A block takes
// `sub` chunks of ENC_CHUNK: the largest of 4, 2, 1 that still gives two
// blocks per SM, so that small operands spread over the SMs and large ones
// keep the partial buffers small.
struct EncOp {
  bool seg;
  long long R, S, nG, nch;
  int sub;
  long long part_len() const { return nch * (seg ? R : S); }
  long long max_len() const { return nch * nG; }
};

EncOp enc_op(bool seg, long long R, long long S, int nsm) {
  EncOp o;
  o.seg = seg;
  o.R = R;
  o.S = S;
  o.nG = seg ? (R + 127) / 128 : (S + 127) / 128;
  const long long L = seg ? S : R;
  o.sub = 1;
  for (int sub : {4, 2})
    if (o.nG * ((L + ENC_CHUNK * sub - 1) / (ENC_CHUNK * sub)) >= 2LL * nsm) {
      o.sub = sub;
      break;
    }
  o.nch = (L + ENC_CHUNK * o.sub - 1) / (ENC_CHUNK * o.sub);
  return o;
}

// The passes of op(A) and op(B): op(A) is SEG over stored A (M x K) for 'N',
// STR over stored A (K x M) for 'T'; op(B) is STR over stored B (K x N) for
// 'N', SEG over stored B (N x K) for 'T'.
void enc_ops(bool ta_t, bool tb_t, long long M, long long N, long long K, int nsm, EncOp &oa, EncOp &ob) {
  oa = ta_t ? enc_op(false, K, M, nsm) : enc_op(true, M, K, nsm);
  ob = tb_t ? enc_op(true, N, K, nsm) : enc_op(false, K, N, nsm);
}

// One operand's pass: gsum = group sums (stride gstride), absv = row (SEG) /
// column (STR) absolute sums, gmax = per group maximum; part_abs / part_max
// hold the chunks' partials, cnt (o.nG counters, zero between passes) counts
// each group's finished chunks.  abs32: the absolute sums as FP32 upper
// bounds (the thresholds' use), else exact FP64 sums.
void launch_enc(const EncOp &o, const double *X, long long ld, double *gsum, long long gstride, double *part_abs,
                double *part_max, unsigned int *cnt, double *absv, double *gmax, cudaStream_t s, bool abs32 = false) {
  const dim3 grid((unsigned)o.nG, (unsigned)o.nch);
  const int cw = ENC_CHUNK * o.sub;
  if (o.seg && abs32)
    enc_seg_kernel<true><<<grid, 256, 0, s>>>(X, o.R, o.S, ld, gsum, gstride, part_abs, part_max, cw, cnt, absv, gmax);
  else if (o.seg)
    enc_seg_kernel<false><<<grid, 256, 0, s>>>(X, o.R, o.S, ld, gsum, gstride, part_abs, part_max, cw, cnt, absv, gmax);
  else if (abs32)
    enc_str_kernel<true><<<grid, 256, 0, s>>>(X, o.R, o.S, ld, gsum, gstride, part_abs, part_max, o.sub, cnt, absv,
                                              gmax);
  else
    enc_str_kernel<false><<<grid, 256, 0, s>>>(X, o.R, o.S, ld, gsum, gstride, part_abs, part_max, o.sub, cnt, absv,
                                               gmax);
}

// The second stream of a call (independent work inside one call runs on it
// between a fork and a join event).
int ensure_side(Workspace &w) {
  if (w.side) return 0;
  if (cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&w.fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&w.join_ev, cudaEventDisableTiming) != cudaSuccess)
    return FTGEMM_ERR_CUDA;
  return 0;
}

int device_sms(int dev) {
  static int cached[MAX_DEV] = {0};
  if (dev < 0 || dev >= MAX_DEV) return 152;
  if (!cached[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

// Encode the operand checksum vectors (see ftgemm_encode.cuh).  Writes
// acs (nI x Kp), aabsmax, arowabs, bcs (nJ x Kp), babsmax, bcolabs; the
// absolute sums as FP32 upper bounds (abs32: what the thresholds need) or as
// exact FP64 sums (ftgemm_encode_operands).
int run_encode(bool ta_t, bool tb_t, long long M, long long N, long long K, const double *A, long long lda,
               const double *B, long long ldb, long long Kp, double *acs, double *aabsmax, double *arowabs,
               double *bcs, double *babsmax, double *bcolabs, Workspace &w, cudaStream_t s,
               bool concurrent = true, bool abs32 = true) {
  const long long nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN;
  int dev = 0;
  cudaGetDevice(&dev);
  EncOp oa, ob;
  enc_ops(ta_t, tb_t, M, N, K, device_sms(dev), oa, ob);
  // op(A)'s pass on s and op(B)'s on the second stream (concurrent), or both
  // on s, each with its own partials and group counters (zeroed when
  // allocated, reset by each pass)
  const size_t ncnt = (size_t)(oa.nG + ob.nG);
  if (ensure(w.part_abs, sizeof(double) * oa.part_len()) || ensure(w.part_max, sizeof(double) * oa.max_len()) ||
      ensure(w.part_abs2, sizeof(double) * ob.part_len()) || ensure(w.part_max2, sizeof(double) * ob.max_len()))
    return FTGEMM_ERR_NOMEM;
  if (w.enc_cnt.cap < sizeof(unsigned int) * ncnt) {
    if (ensure(w.enc_cnt, sizeof(unsigned int) * ncnt)) return FTGEMM_ERR_NOMEM;
    if (cudaMemset(w.enc_cnt.p, 0, w.enc_cnt.cap) != cudaSuccess) return FTGEMM_ERR_CUDA;
  }
  if (concurrent)
    if (int rc = ensure_side(w)) return rc;
  unsigned int *cnt = (unsigned int *)w.enc_cnt.p;
  if (Kp != K) {
    cudaMemsetAsync(acs, 0, sizeof(double) * nI * Kp, s);
    cudaMemsetAsync(bcs, 0, sizeof(double) * nJ * Kp, s);
  }
  const cudaStream_t sb = concurrent ? w.side : s;
  if (concurrent) {
    cudaEventRecord(w.fork_ev, s);
    cudaStreamWaitEvent(w.side, w.fork_ev, 0);
  }
  launch_enc(oa, A, lda, acs, Kp, (double *)w.part_abs.p, (double *)w.part_max.p, cnt, arowabs, aabsmax, s,
             abs32);
  launch_enc(ob, B, ldb, bcs, Kp, (double *)w.part_abs2.p, (double *)w.part_max2.p, cnt + oa.nG, bcolabs, babsmax,
             sb, abs32);
  if (concurrent) {
    cudaEventRecord(w.join_ev, w.side);
    cudaStreamWaitEvent(s, w.join_ev, 0);
  }
  g_launches += 2;
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}

void zero_report(ftgemm_report *rep) {
  if (!rep) return;
  rep->detected = rep->corrected = rep->checksum_only = rep->unverifiable = 0;
  rep->flagged_rows = rep->flagged_cols = rep->recomputed = rep->n_loc = 0;
  rep->panel_detected = 0;
}

// The faults of one M x N call under the injection setting: drawn (mode 1)
// or listed (mode 2); FTGEMM_ERR_INJECT when one lies outside the problem.
int injection_list(long long M, long long N, long long nks, std::vector<ftgemm_flip> &L) {
  L.clear();
  if (g_inj.mode == 1) {
    L.resize((size_t)std::max(0LL, g_inj.count));
    for (long long f = 0; f < (long long)L.size(); ++f) {
      L[f].row = (long long)(splitmix64(g_inj.seed, 4 * (uint64_t)f + 0) % (uint64_t)M);
      L[f].col = (long long)(splitmix64(g_inj.seed, 4 * (uint64_t)f + 1) % (uint64_t)N);
      L[f].kstep = (long long)(splitmix64(g_inj.seed, 4 * (uint64_t)f + 2) % (uint64_t)nks);
      L[f].bit = (int)(splitmix64(g_inj.seed, 4 * (uint64_t)f + 3) % 63u);
      L[f].problem = 0;
    }
  } else if (g_inj.mode == 2) {
    L = g_inj.list;
  }
  for (const auto &f : L)
    if (f.row < 0 || f.row >= M || f.col < 0 || f.col >= N || f.kstep < 0 || f.kstep >= nks || f.bit < 0 ||
        f.bit > 62)
      return FTGEMM_ERR_INJECT;
  return 0;
}

// Where one call's fault table comes from and goes (ftgemm_d_host's panels):
// an explicit list in the call's own coordinates, the device memory that
// holds the table (and stays there for the log), the original index of each
// listed fault and the column offset the log adds back.
struct InjPanel {
  const std::vector<ftgemm_flip> *list;
  const std::vector<long long> *orig;
  void *table;
  long long col_off;
  const std::vector<long long> *perm;  // set: the table is on the device already, in this order
};

// The fault table of list L for a grid of ntiles tiles (nI tile rows), in
// host memory at `stage`: the faults sorted by tile, then k-step, then the
// per-tile offsets at a 256-byte aligned position (one copy moves both).
// perm[q] is the list position of table entry q.  Returns the table's bytes
// before the offsets.
size_t stage_injection_table(const std::vector<ftgemm_flip> &L, long long nI, long long ntiles, void *stage,
                             std::vector<long long> &perm) {
  const long long nf = (long long)L.size();
  perm.resize((size_t)nf);
  for (long long q = 0; q < nf; ++q) perm[q] = q;
  auto tile_of = [&](const ftgemm_flip &f) { return (f.row / BM) + (f.col / BN) * nI; };
  std::stable_sort(perm.begin(), perm.end(), [&](long long a, long long b) {
    const long long ta = tile_of(L[a]), tb = tile_of(L[b]);
    return ta != tb ? ta < tb : L[a].kstep < L[b].kstep;
  });
  const size_t fbytes = (sizeof(DevFlip) * (size_t)std::max(1LL, nf) + 255) & ~(size_t)255;
  DevFlip *hf = (DevFlip *)stage;
  int *ho = (int *)((char *)stage + fbytes);
  std::fill(ho, ho + ntiles + 1, 0);
  for (long long q = 0; q < nf; ++q) {
    const ftgemm_flip &f = L[perm[q]];
    hf[q].row = f.row; hf[q].col = f.col; hf[q].kstep = f.kstep; hf[q].bit = f.bit;
    hf[q].applied = 0; hf[q].before = 0.0; hf[q].after = 0.0; hf[q].kfirst = 0;
    ho[tile_of(f) + 1]++;
  }
  for (long long t = 0; t < ntiles; ++t) ho[t + 1] += ho[t];
  return fbytes;
}

// Build and upload the injection table for this call (FT path only); with
// `pan`, the panel's table, appended to the call's log (already on the
// device when pan->perm is set).
int upload_injection(long long M, long long N, long long nks, long long nI, long long ntiles, Workspace &w,
                     cudaStream_t s, Params &p, bool *inj, const InjPanel *pan = nullptr) {
  *inj = false;
  if (g_inj.mode == 0) return 0;
  std::vector<ftgemm_flip> L;
  if (pan) {
    L = *pan->list;
  } else if (int rc = injection_list(M, N, nks, L)) {
    return rc;
  }
  const long long nf = (long long)L.size();
  const size_t fbytes = (sizeof(DevFlip) * (size_t)std::max(1LL, nf) + 255) & ~(size_t)255;
  const size_t obytes = sizeof(int) * (size_t)(ntiles + 1);
  void *table = pan ? pan->table : w.flips.p;
  std::vector<long long> perm;
  if (pan && pan->perm) {
    perm = *pan->perm;
  } else {
    // two pinned staging buffers in turn: the one taken now may still be read
    // by the copies of the call before the previous one, so wait for its event
    // (recorded after those copies; long complete when calls follow each other)
    const int k = w.ipin_next;
    w.ipin_next ^= 1;
    if (!w.ipin_ev[k] && cudaEventCreateWithFlags(&w.ipin_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return FTGEMM_ERR_CUDA;
    if (cudaEventSynchronize(w.ipin_ev[k]) != cudaSuccess) return FTGEMM_ERR_CUDA;
    if ((!pan && ensure(w.flips, fbytes + obytes)) || ensure_pinned(w.ipin[k], fbytes + obytes + 4096))
      return FTGEMM_ERR_NOMEM;
    table = pan ? pan->table : w.flips.p;
    stage_injection_table(L, nI, ntiles, w.ipin[k].p, perm);
    cudaMemcpyAsync(table, w.ipin[k].p, fbytes + obytes, cudaMemcpyHostToDevice, s);
    cudaEventRecord(w.ipin_ev[k], s);
  }
  Workspace::LogSeg seg;
  seg.dev = (const DevFlip *)table;
  seg.orig.resize((size_t)nf);
  for (long long q = 0; q < nf; ++q) seg.orig[q] = pan ? (*pan->orig)[perm[q]] : perm[q];
  seg.col_off = pan ? pan->col_off : 0;
  if (!pan) {
    w.last_log.clear();
    w.last_nflips = 0;
  }
  w.last_log.push_back(std::move(seg));
  w.last_nflips += nf;
  p.flips = (DevFlip *)table;
  p.tile_off = (const int *)((const char *)table + fbytes);
  *inj = true;
  return 0;
}

// Bytes of one fault table (upload_injection's layout) of nf faults over
// ntiles tiles.
size_t injection_table_bytes(long long nf, long long ntiles) {
  return ((sizeof(DevFlip) * (size_t)std::max(1LL, nf) + 255) & ~(size_t)255) +
         ((sizeof(int) * (size_t)(ntiles + 1) + 255) & ~(size_t)255);
}

// Copy the device report (and up to rep->cap location records) into rep,
// waiting for the stream.
int copy_report(Workspace &w, ftgemm_report *rep, cudaStream_t s) {
  const long long ncopy = std::min<long long>(std::max<long long>(rep->cap, 0), LOC_CAP_DEV);
  const size_t need = sizeof(DevReport) + sizeof(DevLoc) * (size_t)ncopy;
  if (ensure_pinned(w.pin, need + 4096)) return FTGEMM_ERR_NOMEM;
  DevReport *hr = (DevReport *)w.pin.p;
  DevLoc *hl = (DevLoc *)((char *)w.pin.p + sizeof(DevReport));
  cudaMemcpyAsync(hr, w.rep.p, sizeof(DevReport), cudaMemcpyDeviceToHost, s);
  if (ncopy > 0 && rep->loc) cudaMemcpyAsync(hl, w.loc.p, sizeof(DevLoc) * ncopy, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return FTGEMM_ERR_CUDA;
  rep->detected = (long long)hr->detected;
  rep->corrected = (long long)hr->corrected;
  rep->checksum_only = (long long)hr->checksum_only;
  rep->unverifiable = (long long)hr->unverifiable;
  rep->flagged_rows = (long long)hr->flagged_rows;
  rep->flagged_cols = (long long)hr->flagged_cols;
  rep->recomputed = (long long)hr->recomputed;
  rep->panel_detected = (long long)hr->panel_detected;
  rep->n_loc = (long long)hr->n_loc;
  if (rep->loc)
    for (long long q = 0; q < std::min<long long>(ncopy, rep->n_loc); ++q) {
      rep->loc[q].row = hl[q].row;
      rep->loc[q].col = hl[q].col;
      rep->loc[q].tile = hl[q].tile;
      rep->loc[q].kind = hl[q].kind;
      rep->loc[q].delta = hl[q].delta;
    }
  if (hr->err) return FTGEMM_ERR_TIMEOUT;
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}

// One column panel of ftgemm_d_host: its own device report and location
// records, and its faults (none: no injection in this panel).
struct GemmPanel {
  DevReport *rep;
  DevLoc *loc;
  long long loc_cap;
  const InjPanel *inj;
};

int gemm_impl(char transA, char transB, long long M, long long N, long long K, double alpha, const double *A,
              long long lda, const double *B, long long ldb, double beta, double *C, long long ldc,
              ftgemm_report *rep, cudaStream_t s, bool ft, const GemmPanel *gp = nullptr) {
  int rc = check_args(transA, transB, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  zero_report(rep);
  if (M == 0 || N == 0) return 0;
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return FTGEMM_ERR_NODEVICE;
  Workspace &w = *wp;
  if (K == 0 || alpha == 0.0) {
    if (beta != 1.0) {
      scale_kernel<<<grid_for(M * N), 256, 0, s>>>(C, M, N, ldc, beta);
      g_launches++;
    }
    if (rep && cudaStreamSynchronize(s) != cudaSuccess) return FTGEMM_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
  }
  const bool ta_t = is_t(transA), tb_t = is_t(transB);
  const long long arows = ta_t ? K : M, acols = ta_t ? M : K;
  const long long brows = tb_t ? N : K, bcols = tb_t ? K : N;

  // operands the TMA cannot address directly are copied to aligned workspace
  const double *Ause = A, *Buse = B;
  double *Cuse = C;
  long long ldaU = lda, ldbU = ldb, ldcU = ldc;
  bool c_staged = false;
  if (!tma_ok(A, lda)) {
    ldaU = (arows + 1) & ~1LL;
    if (ensure(w.stA, sizeof(double) * ldaU * acols)) return FTGEMM_ERR_NOMEM;
    launch_copy(A, lda, (double *)w.stA.p, ldaU, arows, acols, s);
    Ause = (const double *)w.stA.p;
  }
  if (!tma_ok(B, ldb)) {
    ldbU = (brows + 1) & ~1LL;
    if (ensure(w.stB, sizeof(double) * ldbU * bcols)) return FTGEMM_ERR_NOMEM;
    launch_copy(B, ldb, (double *)w.stB.p, ldbU, brows, bcols, s);
    Buse = (const double *)w.stB.p;
  }
  if (!tma_ok(C, ldc)) {
    ldcU = (M + 1) & ~1LL;
    if (ensure(w.stC, sizeof(double) * ldcU * N)) return FTGEMM_ERR_NOMEM;
    if (beta != 0.0) launch_copy(C, ldc, (double *)w.stC.p, ldcU, M, N, s);
    Cuse = (double *)w.stC.p;
    c_staged = true;
  }

  CUtensorMap mA, mB, mC;
  if (ta_t) rc = make_map(&mA, Ause, K, M, ldaU, BK, BM, true);
  else rc = make_map(&mA, Ause, M, K, ldaU, BM, BK, false);
  if (!rc) {
    if (tb_t) rc = make_map(&mB, Buse, N, K, ldbU, BN, BK, false);
    else rc = make_map(&mB, Buse, K, N, ldbU, BK, BN, true);
  }
  if (!rc) rc = make_map(&mC, Cuse, M, N, ldcU, BM, BN, false);
  if (rc) return rc;

  const long long nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN, ntiles = nI * nJ;
  const long long nks = (K + BK - 1) / BK, Kp = nks * BK;
  Params p;
  memset(&p, 0, sizeof(p));
  p.M = M; p.N = N; p.K = K; p.alpha = alpha; p.beta = beta;
  p.A = Ause; p.B = Buse; p.C = Cuse; p.lda = ldaU; p.ldb = ldbU; p.ldc = ldcU;
  p.nI = (int)nI; p.nJ = (int)nJ; p.nks = (int)nks; p.Kp = Kp;
  p.rep = gp ? gp->rep : (DevReport *)w.rep.p;
  p.loc = gp ? gp->loc : (DevLoc *)w.loc.p;
  p.loc_cap = gp ? gp->loc_cap : LOC_CAP_DEV;
  p.wait_limit_ns = wait_limit_ns();
  p.correct_mode = g_correct;
  cudaMemsetAsync(p.rep, 0, sizeof(DevReport), s);

  cudaEvent_t ea0 = nullptr, ea1 = nullptr, em0 = nullptr, em1 = nullptr;
  if (g_tim.on) {
    timing_record(g_tim.aux_ev, &ea0, &ea1);
    timing_record(g_tim.main_ev, &em0, &em1);
    cudaEventRecord(ea0, s);
  }
  bool inj = false;
  if (ft) {
    if (ensure(w.acs, sizeof(double) * nI * Kp) || ensure(w.bcs, sizeof(double) * nJ * Kp) ||
        ensure(w.arowabs, sizeof(double) * M) || ensure(w.aabsmax, sizeof(double) * nI) ||
        ensure(w.bcolabs, sizeof(double) * N) || ensure(w.babsmax, sizeof(double) * nJ))
      return FTGEMM_ERR_NOMEM;
    rc = run_encode(ta_t, tb_t, M, N, K, Ause, ldaU, Buse, ldbU, Kp, (double *)w.acs.p, (double *)w.aabsmax.p,
                    (double *)w.arowabs.p, (double *)w.bcs.p, (double *)w.babsmax.p, (double *)w.bcolabs.p, w, s);
    if (rc) return rc;
    p.acs = (const double *)w.acs.p; p.bcs = (const double *)w.bcs.p;
    p.arowabs = (const double *)w.arowabs.p; p.aabsmax = (const double *)w.aabsmax.p;
    p.bcolabs = (const double *)w.bcolabs.p; p.babsmax = (const double *)w.babsmax.p;
    if (!gp) rc = upload_injection(M, N, nks, nI, ntiles, w, s, p, &inj);
    else if (gp->inj) rc = upload_injection(M, N, nks, nI, ntiles, w, s, p, &inj, gp->inj);
    if (rc) return rc;
  }

  if (g_tim.on) {
    cudaEventRecord(ea1, s);
    cudaEventRecord(em0, s);
  }
  if (!w.nsm) {
    if (cudaDeviceGetAttribute(&w.nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || w.nsm <= 0) {
      cudaGetLastError();
      w.nsm = 152;
    }
  }
  const bool panel = ft && g_panel > 0 && nks > g_panel;
  const KSplit ksp = plan_ksplit(ntiles, nks, w.nsm);
  int S = ksp.S;
  const long long tail_base = ksp.tail_base, tail_count = ntiles - ksp.tail_base;
  p.panel_slabs = panel ? g_panel : 0;
  cudaError_t e;
  auto launch = [&](int mode, const CUtensorMap &mW) {
    const bool pk = panel && mode < 2;  // the panel checks run in the kernels with a k-loop
    if (!ta_t && !tb_t) return launch_gemm_nn(ft, inj, mode, pk, mA, mB, mC, mW, p, s);
    if (!ta_t && tb_t) return launch_gemm_nt(ft, inj, mode, pk, mA, mB, mC, mW, p, s);
    if (ta_t && !tb_t) return launch_gemm_tn(ft, inj, mode, pk, mA, mB, mC, mW, p, s);
    return launch_gemm_tt(ft, inj, mode, pk, mA, mB, mC, mW, p, s);
  };
  if (S <= 1) {
    e = launch(0, mC);
    g_launches++;
  } else {
    e = cudaSuccess;
    if (tail_base > 0) {  // whole tiles first
      p.tile_base = 0;
      p.tile_count = (int)tail_base;
      e = launch(0, mC);
      g_launches++;
    }
    // split-K over tiles [tail_base, tail_base + tail_count): partial tiles
    // (128 x 128 slots) into workspace, then the verifying reduction
    if (ensure(w.W, sizeof(double) * BM * BN * S * tail_count) || ensure(w.wpc, sizeof(double) * S * nI * N) ||
        ensure(w.wpr, sizeof(double) * S * nJ * M))
      return FTGEMM_ERR_NOMEM;
    CUtensorMap mW;
    if ((rc = make_map3(&mW, (const double *)w.W.p, BM, BN, S * tail_count, BM))) return rc;
    p.tile_base = (int)tail_base;
    p.tile_count = (int)tail_count;
    p.nsplit = S;
    p.ks_slabs = (int)((nks + S - 1) / S);
    p.W = (double *)w.W.p;
    p.wpc = (double *)w.wpc.p;
    p.wpr = (double *)w.wpr.p;
    // a small split grid (all tiles split, fewer than the SMs): the
    // reduction's C-side checksum sums come from a pass over C on the second
    // stream while the partial kernel runs (C is not written before the
    // reduction), instead of from the reduction's few CTAs
    const bool csums = ft && beta != 0.0 && tail_base == 0 && tail_count < w.nsm;
    if (csums) {
      if (ensure(w.uccs, sizeof(double) * nI * N) || ensure(w.uccsa, sizeof(double) * nI * N) ||
          ensure(w.ucrs, sizeof(double) * nJ * M) || ensure(w.ucrsa, sizeof(double) * nJ * M))
        return FTGEMM_ERR_NOMEM;
      if ((rc = ensure_side(w))) return rc;
      cudaEventRecord(w.fork_ev, s);
    }
    if (e == cudaSuccess) e = launch(1, mW);
    if (csums && e == cudaSuccess) {
      if (!w.encc_attr) {
        cudaFuncSetAttribute(enc_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 8);
        w.encc_attr = true;
      }
      cudaStreamWaitEvent(w.side, w.fork_ev, 0);
      enc_c_kernel<<<(unsigned)ntiles, 256, 128 * 128 * 8, w.side>>>(Cuse, ldcU, nullptr, 0, M, N, (int)nI,
                                                                      (double *)w.uccs.p, (double *)w.uccsa.p,
                                                                      (double *)w.ucrs.p, (double *)w.ucrsa.p);
      e = cudaGetLastError();
      cudaEventRecord(w.join_ev, w.side);
      cudaStreamWaitEvent(s, w.join_ev, 0);
      p.csums = 1;
      p.ccs = (const double *)w.uccs.p; p.ccsa = (const double *)w.uccsa.p;
      p.crs = (const double *)w.ucrs.p; p.crsa = (const double *)w.ucrsa.p;
      g_launches++;
    }
    // fewer tiles than SMs: sum the partial tiles over the whole GPU first
    // (the reduction has one CTA per tile and is FP64-add bound)
    p.presummed = tail_count < w.nsm ? 1 : 0;
    if (e == cudaSuccess && p.presummed) {
      const long long pairs = BM * BN * tail_count / 2;
      splitk_sum_kernel<<<(unsigned)std::min<long long>((pairs + 255) / 256, 8LL * w.nsm), 256, 0, s>>>(
          (double *)w.W.p, tail_count, S);
      e = cudaGetLastError();
      g_launches++;
    }
    if (e == cudaSuccess) e = launch(2, mW);
    g_launches += 2;
  }
  if (g_tim.on) cudaEventRecord(em1, s);
  if (e != cudaSuccess) return FTGEMM_ERR_CUDA;
  if (c_staged) launch_copy(Cuse, ldcU, C, ldc, M, N, s);

  if (rep) return copy_report(w, rep, s);
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}

// ftgemm_d_host's column panels: 0 automatic, n >= 1 that many panels (at
// most one per tile column) -- ftgemm_set_host_panels.
int g_host_panels = 0;

// Columns per panel of an M x N host-buffer call (N: one panel, no
// pipeline).  Automatic: up to 8 panels, each at least four waves of tiles,
// so that the panels keep the whole-launch efficiency of the grid.
long long host_panel_cols(long long M, long long N, int nsm) {
  const long long nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN;
  const long long P = g_host_panels > 0 ? std::min<long long>(g_host_panels, nJ)
                                        : std::min<long long>({8LL, nJ, (nI * nJ) / (4LL * nsm)});
  if (P <= 1) return N;
  return (nJ + P - 1) / P * BN;
}

int ensure_copy_streams(Workspace &w, size_t nev) {
  if (!w.up && cudaStreamCreateWithFlags(&w.up, cudaStreamNonBlocking) != cudaSuccess) return FTGEMM_ERR_CUDA;
  if (!w.down && cudaStreamCreateWithFlags(&w.down, cudaStreamNonBlocking) != cudaSuccess) return FTGEMM_ERR_CUDA;
  while (w.pev.size() < nev) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return FTGEMM_ERR_CUDA;
    w.pev.push_back(e);
  }
  return 0;
}

// ftgemm_d_host in column panels of NB columns of op(B) and C: op(A) goes up
// first, then each panel's op(B) and C columns, on a copy stream; a panel's
// FT-DGEMM runs on the caller's stream as soon as its columns have landed
// and its result goes down on a second copy stream while the next panel
// computes.  Output tiles are independent, so the results equal those of one
// call.  The faults of the call are drawn (or listed) over the whole M x N
// problem and each runs in the panel that holds its column; every panel
// reports into its own device region, merged (columns and tile numbers
// shifted back) after the last panel.
int host_panels(char transA, char transB, long long M, long long N, long long K, double alpha, const double *A,
                long long lda, const double *B, long long ldb, double beta, double *C, long long ldc,
                ftgemm_report *r, cudaStream_t s, Workspace &w, long long NB) {
  const long long P = (N + NB - 1) / NB;
  const bool tb_n = is_n(transB);
  const long long acols = is_n(transA) ? K : M, bcols = tb_n ? N : K;
  const size_t abytes = sizeof(double) * (size_t)(lda * acols), bbytes = sizeof(double) * (size_t)(ldb * bcols);
  const size_t cbytes = sizeof(double) * (size_t)(ldc * N);
  if (ensure(w.hA, abytes) || ensure(w.hB, bbytes) || ensure(w.hC, cbytes)) return FTGEMM_ERR_NOMEM;
  const long long nks = (K + BK - 1) / BK, nI = (M + BM - 1) / BM;
  std::vector<ftgemm_flip> all;
  if (int rc = injection_list(M, N, nks, all)) return rc;
  std::vector<std::vector<ftgemm_flip>> pl((size_t)P);
  std::vector<std::vector<long long>> po((size_t)P);
  for (long long q = 0; q < (long long)all.size(); ++q) {
    ftgemm_flip f = all[q];
    const long long pp = f.col / NB;
    f.col -= pp * NB;
    pl[pp].push_back(f);
    po[pp].push_back(q);
  }
  const long long capp = LOC_CAP_DEV / P;
  std::vector<size_t> toff((size_t)P + 1, 0);
  for (long long pp = 0; pp < P; ++pp) {
    const long long nc = std::min(N, (pp + 1) * NB) - pp * NB;
    toff[pp + 1] = toff[pp] + injection_table_bytes((long long)pl[pp].size(), nI * ((nc + BN - 1) / BN));
  }
  if (ensure(w.prep, sizeof(DevReport) * (size_t)P) || ensure(w.ploc, sizeof(DevLoc) * (size_t)(capp * P)) ||
      ensure(w.pfl, toff[P]) || (!all.empty() && ensure_pinned(w.ppin, toff[P])))
    return FTGEMM_ERR_NOMEM;
  if (int rc = ensure_side(w)) return rc;
  if (int rc = ensure_copy_streams(w, (size_t)(2 * P + 2))) return rc;
  // ev[0] fork (later: the upload stream's join), ev[1 + p] panel p landed, ev[1 + P + p] panel p
  // computed, ev[2 P + 1] the download stream's join
  cudaEvent_t *ev = w.pev.data();
  cudaEventRecord(ev[0], s);
  cudaStreamWaitEvent(w.up, ev[0], 0);
  cudaStreamWaitEvent(w.down, ev[0], 0);
  double *hA = (double *)w.hA.p, *hB = (double *)w.hB.p, *hC = (double *)w.hC.p;
  // the panels' fault tables travel first, in one copy on the upload stream:
  // a small copy queued on the compute stream would wait in the copy engine
  // behind the panels' uploads, and the first panel with it
  std::vector<std::vector<long long>> perms((size_t)P);
  if (!all.empty()) {
    for (long long pp = 0; pp < P; ++pp) {
      const long long nc = std::min(N, (pp + 1) * NB) - pp * NB;
      if (!pl[pp].empty())
        stage_injection_table(pl[pp], nI, nI * ((nc + BN - 1) / BN), (char *)w.ppin.p + toff[pp], perms[pp]);
    }
    cudaMemcpyAsync(w.pfl.p, w.ppin.p, toff[P], cudaMemcpyHostToDevice, w.up);
  }
  cudaMemcpyAsync(hA, A, abytes, cudaMemcpyHostToDevice, w.up);
  for (long long pp = 0; pp < P; ++pp) {
    const long long j0 = pp * NB, nc = std::min(N, j0 + NB) - j0;
    if (tb_n)
      cudaMemcpyAsync(hB + j0 * ldb, B + j0 * ldb, sizeof(double) * (size_t)(ldb * nc), cudaMemcpyHostToDevice,
                      w.up);
    else
      cudaMemcpy2DAsync(hB + j0, sizeof(double) * (size_t)ldb, B + j0, sizeof(double) * (size_t)ldb,
                        sizeof(double) * (size_t)nc, (size_t)K, cudaMemcpyHostToDevice, w.up);
    if (beta != 0.0)
      cudaMemcpyAsync(hC + j0 * ldc, C + j0 * ldc, sizeof(double) * (size_t)(ldc * nc), cudaMemcpyHostToDevice,
                      w.up);
    cudaEventRecord(ev[1 + pp], w.up);
  }
  if (g_inj.mode) {  // this call's log is built panel by panel
    w.last_log.clear();
    w.last_nflips = 0;
  }
  int rc = 0;
  for (long long pp = 0; pp < P && !rc; ++pp) {
    const long long j0 = pp * NB, nc = std::min(N, j0 + NB) - j0;
    cudaStreamWaitEvent(s, ev[1 + pp], 0);
    InjPanel ip{&pl[pp], &po[pp], (char *)w.pfl.p + toff[pp], j0, &perms[pp]};
    GemmPanel gp{(DevReport *)w.prep.p + pp, (DevLoc *)w.ploc.p + pp * capp, capp,
                 (g_inj.mode && !pl[pp].empty()) ? &ip : nullptr};
    rc = gemm_impl(transA, transB, M, nc, K, alpha, hA, lda, hB + (tb_n ? j0 * ldb : j0), ldb, beta, hC + j0 * ldc,
                   ldc, nullptr, s, true, &gp);
    if (rc) break;
    cudaEventRecord(ev[1 + P + pp], s);
    cudaStreamWaitEvent(w.down, ev[1 + P + pp], 0);
    // only the M x nc block goes back: rows M..ldc-1 of the caller's C are
    // not the call's to write
    if (ldc == M)
      cudaMemcpyAsync(C + j0 * ldc, hC + j0 * ldc, sizeof(double) * (size_t)(ldc * nc), cudaMemcpyDeviceToHost,
                      w.down);
    else
      cudaMemcpy2DAsync(C + j0 * ldc, sizeof(double) * (size_t)ldc, hC + j0 * ldc, sizeof(double) * (size_t)ldc,
                        sizeof(double) * (size_t)M, (size_t)nc, cudaMemcpyDeviceToHost, w.down);
  }
  // join both copy streams back into the caller's stream
  cudaEventRecord(ev[2 * P + 1], w.down);
  cudaStreamWaitEvent(s, ev[2 * P + 1], 0);
  cudaEventRecord(ev[0], w.up);
  cudaStreamWaitEvent(s, ev[0], 0);
  if (rc) {
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return rc;
  }
  // the panels' reports and location records, in one copy after the last panel
  const long long cap = std::max<long long>(r->loc ? r->cap : 0, 0), per = std::min(capp, cap);
  const size_t need = sizeof(DevReport) * (size_t)P + sizeof(DevLoc) * (size_t)(per * P);
  if (ensure_pinned(w.pin, need + 4096)) return FTGEMM_ERR_NOMEM;
  DevReport *hr = (DevReport *)w.pin.p;
  DevLoc *hl = (DevLoc *)(hr + P);
  cudaMemcpyAsync(hr, w.prep.p, sizeof(DevReport) * (size_t)P, cudaMemcpyDeviceToHost, s);
  for (long long pp = 0; pp < P && per > 0; ++pp)
    cudaMemcpyAsync(hl + pp * per, (DevLoc *)w.ploc.p + pp * capp, sizeof(DevLoc) * (size_t)per,
                    cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_CUDA;
  }
  long long nout = 0;
  bool timeout = false;
  for (long long pp = 0; pp < P; ++pp) {
    const DevReport &d = hr[pp];
    r->detected += (long long)d.detected;
    r->corrected += (long long)d.corrected;
    r->checksum_only += (long long)d.checksum_only;
    r->unverifiable += (long long)d.unverifiable;
    r->flagged_rows += (long long)d.flagged_rows;
    r->flagged_cols += (long long)d.flagged_cols;
    r->recomputed += (long long)d.recomputed;
    r->panel_detected += (long long)d.panel_detected;
    r->n_loc += (long long)d.n_loc;
    timeout = timeout || d.err;
    const long long j0 = pp * NB;
    for (long long q = 0; q < std::min<long long>(per, (long long)d.n_loc) && nout < cap; ++q, ++nout) {
      const DevLoc &l = hl[pp * per + q];
      r->loc[nout].row = l.row;
      r->loc[nout].col = l.col + j0;
      r->loc[nout].tile = (int)(l.tile + (j0 / BN) * nI);
      r->loc[nout].kind = l.kind;
      r->loc[nout].delta = l.delta;
    }
  }
  if (timeout) return FTGEMM_ERR_TIMEOUT;
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}

}  // namespace

extern "C" {

int ftgemm_d(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
             int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, ftgemm_report *rep,
             void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  return gemm_impl(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rep, (cudaStream_t)stream, true);
}

int ftgemm_d_noft(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                  int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  return gemm_impl(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, (cudaStream_t)stream,
                   false);
}

int ftgemm_d_host(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                  int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc, ftgemm_report *rep,
                  void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = check_args(transA, transB, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  zero_report(rep);
  if (M == 0 || N == 0) return 0;
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return FTGEMM_ERR_NODEVICE;
  Workspace &w = *wp;
  cudaStream_t s = (cudaStream_t)stream;
  if (K > 0 && alpha != 0.0) {
    const long long NB = host_panel_cols(M, N, device_sms(dev));
    if (NB < N) {
      ftgemm_report local;
      memset(&local, 0, sizeof(local));
      return host_panels(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rep ? rep : &local, s, w,
                         NB);
    }
  }
  const long long acols = is_n(transA) ? K : M, bcols = is_n(transB) ? N : K;
  const size_t abytes = sizeof(double) * (size_t)(lda * acols), bbytes = sizeof(double) * (size_t)(ldb * bcols);
  const size_t cbytes = sizeof(double) * (size_t)(ldc * N);
  if (ensure(w.hA, abytes) || ensure(w.hB, bbytes) || ensure(w.hC, cbytes)) return FTGEMM_ERR_NOMEM;
  if ((rc = ensure_side(w))) return rc;
  // op(B) goes up on the second stream, beside op(A) and C (two copy engines)
  cudaEventRecord(w.fork_ev, s);
  cudaStreamWaitEvent(w.side, w.fork_ev, 0);
  if (K > 0 && alpha != 0.0) {
    if (abytes) cudaMemcpyAsync(w.hA.p, A, abytes, cudaMemcpyHostToDevice, s);
    if (bbytes) cudaMemcpyAsync(w.hB.p, B, bbytes, cudaMemcpyHostToDevice, w.side);
  }
  if (beta != 0.0) cudaMemcpyAsync(w.hC.p, C, cbytes, cudaMemcpyHostToDevice, s);
  cudaEventRecord(w.join_ev, w.side);
  cudaStreamWaitEvent(s, w.join_ev, 0);
  ftgemm_report local;
  memset(&local, 0, sizeof(local));
  ftgemm_report *r = rep ? rep : &local;
  rc = gemm_impl(transA, transB, M, N, K, alpha, (const double *)w.hA.p, lda, (const double *)w.hB.p, ldb, beta,
                 (double *)w.hC.p, ldc, r, s, true);
  if (rc && rc != FTGEMM_ERR_TIMEOUT) return rc;
  // only the M x N block goes back: rows M..ldc-1 of the caller's C are not
  // the call's to write (with beta == 0 the workspace never held them)
  const cudaError_t ce =
      ldc == M ? cudaMemcpyAsync(C, w.hC.p, cbytes, cudaMemcpyDeviceToHost, s)
               : cudaMemcpy2DAsync(C, sizeof(double) * (size_t)ldc, w.hC.p, sizeof(double) * (size_t)ldc,
                                   sizeof(double) * (size_t)M, (size_t)N, cudaMemcpyDeviceToHost, s);
  if (ce != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_CUDA;
  }
  return rc;
}

int ftgemm_d_unfused(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha, const double *A,
                     int64_t lda, const double *B, int64_t ldb, double beta, double *C, int64_t ldc,
                     ftgemm_report *rep, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = check_args(transA, transB, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  zero_report(rep);
  if (M == 0 || N == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0 || alpha == 0.0)  // BLAS quick return: same path as ftgemm_d
    return gemm_impl(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rep, s, true);
  if (!tma_ok(A, lda) || !tma_ok(B, ldb) || !tma_ok(C, ldc)) return FTGEMM_ERR_UNALIGNED;
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return FTGEMM_ERR_NODEVICE;
  Workspace &w = *wp;
  const bool ta_t = is_t(transA), tb_t = is_t(transB);
  const long long nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN, ntiles = nI * nJ;
  const long long nks = (K + BK - 1) / BK, Kp = nks * BK;
  const long long ldcc = (M + 1) & ~1LL, ldp1 = (nI + 1) & ~1LL, ldp2 = (M + 1) & ~1LL;
  // pass 1: operand checksum vectors (as in ftgemm_d)
  if (ensure(w.acs, sizeof(double) * nI * Kp) || ensure(w.bcs, sizeof(double) * nJ * Kp) ||
      ensure(w.arowabs, sizeof(double) * M) || ensure(w.aabsmax, sizeof(double) * nI) ||
      ensure(w.bcolabs, sizeof(double) * N) || ensure(w.babsmax, sizeof(double) * nJ) ||
      ensure(w.uC, sizeof(double) * ldcc * N) || ensure(w.uccs, sizeof(double) * nI * N) ||
      ensure(w.uccsa, sizeof(double) * nI * N) || ensure(w.ucrs, sizeof(double) * nJ * M) ||
      ensure(w.ucrsa, sizeof(double) * nJ * M) || ensure(w.uP1, sizeof(double) * ldp1 * N) ||
      ensure(w.uP2, sizeof(double) * ldp2 * nJ))
    return FTGEMM_ERR_NOMEM;
  if ((rc = run_encode(ta_t, tb_t, M, N, K, A, lda, B, ldb, Kp, (double *)w.acs.p, (double *)w.aabsmax.p,
                       (double *)w.arowabs.p, (double *)w.bcs.p, (double *)w.babsmax.p, (double *)w.bcolabs.p,
                       w, s)))
    return rc;
  // pass 2: copy of C_in and its per-tile row/column sums
  if (beta != 0.0) {
    if (!w.encc_attr) {
      cudaFuncSetAttribute(enc_c_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 8);
      w.encc_attr = true;
    }
    enc_c_kernel<<<(unsigned)ntiles, 256, 128 * 128 * 8, s>>>(C, ldc, (double *)w.uC.p, ldcc, M, N, (int)nI,
                                                               (double *)w.uccs.p, (double *)w.uccsa.p,
                                                               (double *)w.ucrs.p, (double *)w.ucrsa.p);
    g_launches++;
  }
  // passes 3-4: predicted checksums as separate GEMMs on the unprotected kernel:
  // P1 = acs^T-view x op(B) (nI x N), P2 = op(A) x bcs-view (M x nJ)
  if ((rc = gemm_impl('T', transB, nI, N, K, 1.0, (const double *)w.acs.p, Kp, B, ldb, 0.0, (double *)w.uP1.p,
                      ldp1, nullptr, s, false)))
    return rc;
  if ((rc = gemm_impl(transA, 'N', M, nJ, K, 1.0, A, lda, (const double *)w.bcs.p, Kp, 0.0, (double *)w.uP2.p,
                      ldp2, nullptr, s, false)))
    return rc;
  // pass 5: the GEMM itself, unprotected
  if ((rc = gemm_impl(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nullptr, s, false))) return rc;
  // pass 6: verify / locate / correct on the finished C (MODE 3)
  CUtensorMap mC;
  if ((rc = make_map(&mC, C, M, N, ldc, BM, BN, false))) return rc;
  Params p;
  memset(&p, 0, sizeof(p));
  p.M = M; p.N = N; p.K = K; p.alpha = alpha; p.beta = beta;
  p.A = A; p.B = B; p.lda = lda; p.ldb = ldb;
  p.C = (double *)w.uC.p; p.ldc = ldcc;          // copy of C_in for recomputation
  p.Cout = C; p.ldcout = ldc;
  p.nI = (int)nI; p.nJ = (int)nJ; p.nks = (int)nks; p.Kp = Kp;
  p.arowabs = (const double *)w.arowabs.p; p.aabsmax = (const double *)w.aabsmax.p;
  p.bcolabs = (const double *)w.bcolabs.p; p.babsmax = (const double *)w.babsmax.p;
  p.P1 = (const double *)w.uP1.p; p.ldp1 = ldp1; p.P2 = (const double *)w.uP2.p; p.ldp2 = ldp2;
  p.ccs = (const double *)w.uccs.p; p.ccsa = (const double *)w.uccsa.p;
  p.crs = (const double *)w.ucrs.p; p.crsa = (const double *)w.ucrsa.p;
  p.rep = (DevReport *)w.rep.p;
  p.loc = (DevLoc *)w.loc.p;
  p.loc_cap = LOC_CAP_DEV;
  p.wait_limit_ns = wait_limit_ns();
  p.correct_mode = g_correct;
  p.nsplit = 1;
  cudaMemsetAsync(w.rep.p, 0, sizeof(DevReport), s);
  cudaError_t e;
  if (!ta_t && !tb_t) e = launch_gemm_nn(true, false, 3, false, mC, mC, mC, mC, p, s);
  else if (!ta_t && tb_t) e = launch_gemm_nt(true, false, 3, false, mC, mC, mC, mC, p, s);
  else if (ta_t && !tb_t) e = launch_gemm_tn(true, false, 3, false, mC, mC, mC, mC, p, s);
  else e = launch_gemm_tt(true, false, 3, false, mC, mC, mC, mC, p, s);
  g_launches++;
  if (e != cudaSuccess) return FTGEMM_ERR_CUDA;
  if (rep) return copy_report(w, rep, s);
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}

int ftgemm_encode_operands(char transA, char transB, int64_t M, int64_t N, int64_t K, const double *A, int64_t lda,
                           const double *B, int64_t ldb, double *acs, double *aabsmax, double *arowabs, double *bcs,
                           double *babsmax, double *bcolabs, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = check_args(transA, transB, M, N, K, lda, ldb, std::max<int64_t>(1, M));
  if (rc) return rc == -8 ? -7 : rc == -10 ? -9 : rc;  // lda, ldb are arguments 7 and 9 here
  if (M == 0 || N == 0 || K == 0) return 0;
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return FTGEMM_ERR_NODEVICE;
  return run_encode(is_t(transA), is_t(transB), M, N, K, A, lda, B, ldb, K, acs, aabsmax, arowabs, bcs, babsmax,
                    bcolabs, *wp, (cudaStream_t)stream, true, false);
}

int ftgemm_set_injection(const ftgemm_inject *cfg) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!cfg || cfg->mode == 0) {
    g_inj.mode = 0;
    g_inj.list.clear();
    return 0;
  }
  if (cfg->mode == 1) {
    if (cfg->count < 0) return -1;
    g_inj.mode = 1;
    g_inj.seed = cfg->seed;
    g_inj.count = cfg->count;
    g_inj.list.clear();
    return 0;
  }
  if (cfg->mode == 2) {
    if (cfg->n_list < 0 || (cfg->n_list > 0 && !cfg->list)) return -1;
    g_inj.mode = 2;
    g_inj.list.assign(cfg->list, cfg->list + cfg->n_list);
    return 0;
  }
  return -1;
}

int64_t ftgemm_injection_log(ftgemm_flip_log *out, int64_t cap) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap > 0 && !out) return -1;
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return -FTGEMM_ERR_NODEVICE;
  Workspace &w = *wp;
  const long long nf = w.last_nflips;
  if (nf == 0 || cap <= 0) return nf;
  if (cudaDeviceSynchronize() != cudaSuccess) return -FTGEMM_ERR_CUDA;
  for (const auto &seg : w.last_log) {
    const long long n = (long long)seg.orig.size();
    if (n == 0) continue;
    std::vector<DevFlip> h((size_t)n);
    if (cudaMemcpy(h.data(), seg.dev, sizeof(DevFlip) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
      return -FTGEMM_ERR_CUDA;
    for (long long q = 0; q < n; ++q) {
      const long long o = seg.orig[q];
      if (o >= cap) continue;
      out[o].row = h[q].row;
      out[o].col = h[q].col + seg.col_off;
      out[o].kstep = h[q].kstep;
      out[o].bit = h[q].bit;
      out[o].applied = h[q].applied;
      out[o].before = h[q].before;
      out[o].after = h[q].after;
      out[o].kfirst = h[q].kfirst;
    }
  }
  return nf;
}

int ftgemm_selftest_wait_timeout(int64_t limit_ns, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return FTGEMM_ERR_NODEVICE;
  cudaStream_t s = (cudaStream_t)stream;
  DevReport *r = (DevReport *)wp->rep.p;
  cudaMemsetAsync(r, 0, sizeof(DevReport), s);
  wait_timeout_kernel<<<1, 32, 0, s>>>(r, (unsigned long long)std::max<int64_t>(limit_ns, 1));
  g_launches++;
  int err = 0;
  if (cudaMemcpyAsync(&err, &r->err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return FTGEMM_ERR_CUDA;
  return err == ERR_TIMEOUT ? FTGEMM_ERR_TIMEOUT : (err ? err : 0);
}

int64_t ftgemm_launch_count(void) { return g_launches.load(); }

int ftgemm_set_panel_check(int kslabs) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (kslabs < 0) return -1;
  g_panel = kslabs;
  return 0;
}

int ftgemm_set_split_engine(int engine) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (engine != 0 && engine != 1 && engine != 2 && engine != 5 && engine != 7) return -1;
  g_split_engine = engine;
  return 0;
}

int ftgemm_set_correction(int mode) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (mode < 0 || mode > 1) return -1;
  g_correct = mode;
  return 0;
}

int ftgemm_query_ksplit(int64_t M, int64_t N, int64_t K, int nsm, int *splits, int64_t *first_split_tile) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (M < 0) return -1;
  if (N < 0) return -2;
  if (K < 0) return -3;
  if (nsm <= 0) return -4;
  if (!splits) return -5;
  if (!first_split_tile) return -6;
  const long long ntiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN), nks = (K + BK - 1) / BK;
  if (ntiles == 0 || nks == 0) {  // quick returns: no GEMM kernel
    *splits = 1;
    *first_split_tile = ntiles;
    return 0;
  }
  const KSplit k = plan_ksplit(ntiles, nks, nsm);
  *splits = k.S;
  *first_split_tile = k.S > 1 ? k.tail_base : ntiles;
  return 0;
}

int ftgemm_set_host_panels(int panels) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (panels < 0) return -1;
  g_host_panels = panels;
  return 0;
}

int ftgemm_set_splitk(int nsplit) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (nsplit < 0 || nsplit > 64) return -1;
  g_splitk = nsplit;
  return 0;
}

int ftgemm_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto *v : {&g_tim.main_ev, &g_tim.aux_ev}) {
    for (auto &pr : *v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    v->clear();
  }
  g_tim.on = enable != 0;
  return 0;
}

int ftgemm_timing_read(double *main_ms, int64_t *main_launches, double *aux_ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  double tm = 0.0, ta = 0.0;
  for (auto &pr : g_tim.main_ev) {
    float ms = 0.0f;
    if (cudaEventSynchronize(pr.second) != cudaSuccess || cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess)
      return FTGEMM_ERR_CUDA;
    tm += ms;
  }
  for (auto &pr : g_tim.aux_ev) {
    float ms = 0.0f;
    if (cudaEventSynchronize(pr.second) != cudaSuccess || cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess)
      return FTGEMM_ERR_CUDA;
    ta += ms;
  }
  if (main_ms) *main_ms = tm;
  if (aux_ms) *aux_ms = ta;
  if (main_launches) *main_launches = (int64_t)g_tim.main_ev.size();
  return 0;
}

const char *ftgemm_strerror(int code) {
  if (code == 0) return "success";
  if (code < 0) return "invalid argument (see the BLAS argument number)";
  switch (code) {
    case FTGEMM_ERR_CUDA: return "CUDA runtime call or kernel launch failed";
    case FTGEMM_ERR_TIMEOUT: return "bounded device pipeline wait expired";
    case FTGEMM_ERR_NODEVICE: return "no usable CUDA device";
    case FTGEMM_ERR_NOMEM: return "workspace allocation failed";
    case FTGEMM_ERR_INJECT: return "injected fault outside the problem";
    case FTGEMM_ERR_TENSORMAP: return "TMA descriptor encoding failed";
    case FTGEMM_ERR_SCRATCH: return "problem needs more scratch than ftgemm_d_noalloc holds";
    case FTGEMM_ERR_UNALIGNED: return "operand not 16-byte aligned or leading dimension odd";
    case FTGEMM_ERR_BATCH: return "invalid batch: count < 0, or a NULL plan pointer or per-problem array";
    case FTGEMM_ERR_TOO_LARGE: return "ftgemm_d_split: M or N above FTGEMM_SPLIT_MAX_ROWS";
    case FTGEMM_ERR_CAPTURE: return "ftgemm_d_noalloc: a report cannot be read back inside a stream capture";
    default: return "unknown error";
  }
}

int ftgemm_finalize(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) return FTGEMM_ERR_NODEVICE;
  Workspace &w = g_ws[dev];
  cudaDeviceSynchronize();
  Buf *dbufs[] = {&w.prep, &w.ploc, &w.pfl,
                  &w.acs, &w.bcs, &w.arowabs, &w.aabsmax, &w.bcolabs, &w.babsmax, &w.part_abs, &w.part_max,
                  &w.rep, &w.loc, &w.flips, &w.stA, &w.stB, &w.stC, &w.hA, &w.hB, &w.hC,
                  &w.W, &w.wpc, &w.wpr, &w.uC, &w.uccs, &w.uccsa, &w.ucrs, &w.ucrsa, &w.uP1, &w.uP2,
                  &w.spA, &w.spB, &w.spEA, &w.spEB, &w.spPA, &w.spPB, &w.spEPA, &w.spEPB, &w.tscr, &w.spMB,
                  &w.part_abs2, &w.part_max2, &w.enc_cnt};
  for (Buf *b : dbufs) {
    if (b->p) cudaFree(b->p);
    b->p = nullptr;
    b->cap = 0;
  }
  if (w.pin.p) cudaFreeHost(w.pin.p);
  w.pin.p = nullptr;
  if (w.ppin.p) cudaFreeHost(w.ppin.p);
  w.ppin.p = nullptr;
  w.ppin.cap = 0;
  for (int k = 0; k < 2; ++k) {
    if (w.ipin[k].p) cudaFreeHost(w.ipin[k].p);
    w.ipin[k].p = nullptr;
    w.ipin[k].cap = 0;
    if (w.ipin_ev[k]) cudaEventDestroy(w.ipin_ev[k]);
    w.ipin_ev[k] = nullptr;
  }
  w.ipin_next = 0;
  if (w.side) cudaStreamDestroy(w.side);
  if (w.up) cudaStreamDestroy(w.up);
  if (w.down) cudaStreamDestroy(w.down);
  for (cudaEvent_t e : w.pev) cudaEventDestroy(e);
  w.pev.clear();
  w.up = w.down = nullptr;
  if (w.fork_ev) cudaEventDestroy(w.fork_ev);
  if (w.join_ev) cudaEventDestroy(w.join_ev);
  w.side = nullptr;
  w.fork_ev = w.join_ev = nullptr;
  w.pin.cap = 0;
  w.init = false;
  w.last_nflips = 0;
  w.last_log.clear();
  return 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ftgemm_d_noalloc: the fault-tolerant DGEMM for callers that cannot allocate
// device memory.  All of its scratch (operand checksum vectors, the partial
// sums of the checksum pass, the device report and location records) lives in
// the file-scope array below, which every GPU that loads this library holds
// until the process exits.  No cudaMalloc, cudaFree or allocating library
// routine is called on this path.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FTGEMM_NOALLOC_SCRATCH_BYTES];

constexpr long long NOALLOC_LOC_CAP = 1024;

// Device address of g_noalloc_scratch per device, looked up on the first call
// made with that device current (host code may not use the symbol itself).
unsigned char *g_noalloc_ptr[MAX_DEV] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Scratch layout for one call; returns the bytes needed.
struct NoallocLayout {
  size_t rep, loc, acs, bcs, arowabs, aabsmax, bcolabs, babsmax, part_abs, part_max, enc_cnt, total;
};

NoallocLayout noalloc_layout(bool ta_t, bool tb_t, long long M, long long N, long long K, int nsm) {
  const long long nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN, Kp = (K + BK - 1) / BK * BK;
  // partial buffers of the checksum pass: worst case over the two operands
  EncOp oa, ob;
  enc_ops(ta_t, tb_t, M, N, K, nsm, oa, ob);
  const long long pa = std::max(oa.part_len(), ob.part_len()), pm = std::max(oa.max_len(), ob.max_len());
  NoallocLayout L;
  size_t o = 0;
  L.rep = o; o = align256(o + sizeof(DevReport));
  L.loc = o; o = align256(o + sizeof(DevLoc) * NOALLOC_LOC_CAP);
  L.acs = o; o = align256(o + sizeof(double) * nI * Kp);
  L.bcs = o; o = align256(o + sizeof(double) * nJ * Kp);
  L.arowabs = o; o = align256(o + sizeof(double) * M);
  L.aabsmax = o; o = align256(o + sizeof(double) * nI);
  L.bcolabs = o; o = align256(o + sizeof(double) * N);
  L.babsmax = o; o = align256(o + sizeof(double) * nJ);
  L.part_abs = o; o = align256(o + sizeof(double) * pa);
  L.part_max = o; o = align256(o + sizeof(double) * pm);
  L.enc_cnt = o; o = align256(o + sizeof(unsigned int) * std::max(oa.nG, ob.nG));
  L.total = o;
  return L;
}

}  // namespace

extern "C" int ftgemm_d_noalloc(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                                const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                                int64_t ldc, ftgemm_report *rep, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = check_args(transA, transB, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  zero_report(rep);
  if (M == 0 || N == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0 || alpha == 0.0) {
    if (beta != 1.0) {
      scale_kernel<<<grid_for(M * N), 256, 0, s>>>(C, M, N, ldc, beta);
      g_launches++;
    }
    if (rep && cudaStreamSynchronize(s) != cudaSuccess) return FTGEMM_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
  }
  const bool ta_t = is_t(transA), tb_t = is_t(transB);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV) {
    cudaGetLastError();
    return FTGEMM_ERR_NODEVICE;
  }
  const int nsm = device_sms(dev);
  const NoallocLayout L = noalloc_layout(ta_t, tb_t, M, N, K, nsm);
  if (L.total > (size_t)FTGEMM_NOALLOC_SCRATCH_BYTES) return FTGEMM_ERR_SCRATCH;
  if (!tma_ok(A, lda) || !tma_ok(B, ldb) || !tma_ok(C, ldc)) return FTGEMM_ERR_UNALIGNED;
  if (rep) {
    // reading the report back waits for the stream, which a stream capture
    // does not allow: refuse before anything is enqueued
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      return FTGEMM_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return FTGEMM_ERR_CAPTURE;
  }

  if (!g_noalloc_ptr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return FTGEMM_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<unsigned char *>(ptr);
  }
  unsigned char *base = g_noalloc_ptr[dev];

  const long long nI = (M + BM - 1) / BM, nJ = (N + BN - 1) / BN;
  const long long nks = (K + BK - 1) / BK, Kp = nks * BK;
  double *acs = (double *)(base + L.acs), *bcs = (double *)(base + L.bcs);
  double *arowabs = (double *)(base + L.arowabs), *aabsmax = (double *)(base + L.aabsmax);
  double *bcolabs = (double *)(base + L.bcolabs), *babsmax = (double *)(base + L.babsmax);
  double *part_abs = (double *)(base + L.part_abs), *part_max = (double *)(base + L.part_max);
  DevReport *drep = (DevReport *)(base + L.rep);
  DevLoc *dloc = (DevLoc *)(base + L.loc);

  // the array keeps the previous call's contents: clear what must start at zero
  cudaMemsetAsync(drep, 0, sizeof(DevReport), s);
  if (Kp != K) {
    cudaMemsetAsync(acs, 0, sizeof(double) * nI * Kp, s);
    cudaMemsetAsync(bcs, 0, sizeof(double) * nJ * Kp, s);
  }
  // operand checksum pass (same kernels as ftgemm_d), partials and group
  // counters in the array, both operands on the caller's stream
  {
    EncOp oa, ob;
    enc_ops(ta_t, tb_t, M, N, K, nsm, oa, ob);
    unsigned int *cnt = (unsigned int *)(base + L.enc_cnt);
    cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * std::max(oa.nG, ob.nG), s);
    launch_enc(oa, A, lda, acs, Kp, part_abs, part_max, cnt, arowabs, aabsmax, s);
    launch_enc(ob, B, ldb, bcs, Kp, part_abs, part_max, cnt, bcolabs, babsmax, s);
  }
  g_launches += 2;

  CUtensorMap mA, mB, mC;
  if (ta_t) rc = make_map(&mA, A, K, M, lda, BK, BM, true);
  else rc = make_map(&mA, A, M, K, lda, BM, BK, false);
  if (!rc) {
    if (tb_t) rc = make_map(&mB, B, N, K, ldb, BN, BK, false);
    else rc = make_map(&mB, B, K, N, ldb, BK, BN, true);
  }
  if (!rc) rc = make_map(&mC, C, M, N, ldc, BM, BN, false);
  if (rc) return rc;

  Params p;
  memset(&p, 0, sizeof(p));
  p.M = M; p.N = N; p.K = K; p.alpha = alpha; p.beta = beta;
  p.A = A; p.B = B; p.C = C; p.lda = lda; p.ldb = ldb; p.ldc = ldc;
  p.nI = (int)nI; p.nJ = (int)nJ; p.nks = (int)nks; p.Kp = Kp;
  p.acs = acs; p.bcs = bcs; p.arowabs = arowabs; p.aabsmax = aabsmax; p.bcolabs = bcolabs; p.babsmax = babsmax;
  p.rep = drep;
  p.loc = dloc;
  p.loc_cap = NOALLOC_LOC_CAP;
  p.wait_limit_ns = wait_limit_ns();
  p.correct_mode = g_correct;
  cudaError_t e;
  if (!ta_t && !tb_t) e = launch_gemm_nn(true, false, 0, false, mA, mB, mC, mC, p, s);
  else if (!ta_t && tb_t) e = launch_gemm_nt(true, false, 0, false, mA, mB, mC, mC, p, s);
  else if (ta_t && !tb_t) e = launch_gemm_tn(true, false, 0, false, mA, mB, mC, mC, p, s);
  else e = launch_gemm_tt(true, false, 0, false, mA, mB, mC, mC, p, s);
  g_launches++;
  if (e != cudaSuccess) return FTGEMM_ERR_CUDA;

  if (rep) {
    // copy the report into host variables of this call (no pinned staging)
    DevReport hr;
    DevLoc hl[64];
    const long long ncopy = std::min<long long>(std::max<long long>(rep->cap, 0), NOALLOC_LOC_CAP);
    if (cudaMemcpyAsync(&hr, drep, sizeof(DevReport), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return FTGEMM_ERR_CUDA;
    rep->detected = (long long)hr.detected;
    rep->corrected = (long long)hr.corrected;
    rep->checksum_only = (long long)hr.checksum_only;
    rep->unverifiable = (long long)hr.unverifiable;
    rep->flagged_rows = (long long)hr.flagged_rows;
    rep->flagged_cols = (long long)hr.flagged_cols;
    rep->recomputed = (long long)hr.recomputed;
    rep->panel_detected = (long long)hr.panel_detected;
    rep->n_loc = (long long)hr.n_loc;
    const long long nrec = std::min<long long>(ncopy, rep->n_loc);
    for (long long q0 = 0; rep->loc && q0 < nrec; q0 += 64) {
      const long long nq = std::min<long long>(64, nrec - q0);
      if (cudaMemcpy(hl, dloc + q0, sizeof(DevLoc) * nq, cudaMemcpyDeviceToHost) != cudaSuccess)
        return FTGEMM_ERR_CUDA;
      for (long long q = 0; q < nq; ++q) {
        rep->loc[q0 + q].row = hl[q].row;
        rep->loc[q0 + q].col = hl[q].col;
        rep->loc[q0 + q].tile = hl[q].tile;
        rep->loc[q0 + q].kind = hl[q].kind;
        rep->loc[q0 + q].delta = hl[q].delta;
      }
    }
    if (hr.err) return FTGEMM_ERR_TIMEOUT;
  }
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Batched FT-DGEMM: many independent problems in one persistent launch per
// operand layout, captured once into a CUDA graph.
namespace {

constexpr int PLAN_LOC_CAP = 64;  // location records kept per problem

}  // namespace

struct ftgemm_batched_plan_s {
  int dev = 0;
  long long count = 0;
  bool ft = true, inj = false;
  int kernels = 0;                       // kernels per graph launch
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void *> bufs;              // device allocations owned by the plan
  DevReport *reps = nullptr;
  DevLoc *locs = nullptr;
  DevFlip *flips = nullptr;
  long long nflips = 0;
  std::vector<long long> flip_perm;      // sorted position -> original index
  std::vector<int> flip_problem;         // original index -> problem
};

namespace {

void plan_free(ftgemm_batched_plan_s *P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  for (void *b : P->bufs) cudaFree(b);
  delete P;
}

template <typename T>
int plan_alloc(ftgemm_batched_plan_s *P, T **out, size_t n) {
  void *q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(n * sizeof(T), 256)) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_NOMEM;
  }
  P->bufs.push_back(q);
  *out = (T *)q;
  return 0;
}

long long round32(long long n) { return (n + 31) / 32 * 32; }

}  // namespace

extern "C" {

int ftgemm_batched_plan_create(ftgemm_batched_plan *plan_out, int64_t count, const char *transA,
                               const char *transB, const int64_t *M, const int64_t *N, const int64_t *K,
                               const double *alpha, const double *const *A, const int64_t *lda,
                               const double *const *B, const int64_t *ldb, const double *beta, double *const *C,
                               const int64_t *ldc, int ft, int schedule, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!plan_out) return FTGEMM_ERR_BATCH;
  *plan_out = nullptr;
  if (count < 0) return FTGEMM_ERR_BATCH;
  if (count > 0 && (!transA || !transB || !M || !N || !K || !alpha || !A || !lda || !B || !ldb || !beta || !C ||
                    !ldc))
    return FTGEMM_ERR_BATCH;
  for (long long q = 0; q < count; ++q) {
    const int rc = check_args(transA[q], transB[q], M[q], N[q], K[q], lda[q], ldb[q], ldc[q]);
    if (rc) return (int)(rc - 100 * q);  // -(100*problem + argument)
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_NODEVICE;
  }
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 152;
  const int order_kind = schedule < 0 ? 1 : (schedule & 15);
  const int chunk = schedule < 0 ? 1 : (1 << ((schedule >> 4) & 3));
  auto *P = new ftgemm_batched_plan_s();
  P->dev = dev;
  P->count = count;
  P->ft = ft != 0;
  int rc = 0;
#define PLAN_TRY(x)        \
  do {                     \
    if ((rc = (x))) {      \
      plan_free(P);        \
      return rc;           \
    }                      \
  } while (0)

  // problems with work, their tiles and checksum-vector offsets
  std::vector<char> work(count, 0);
  std::vector<long long> nI(count), nJ(count), nks(count), Kp(count), tiles(count);
  std::vector<long long> off_acs(count), off_bcs(count), off_ar(count), off_am(count), off_bc(count), off_bm(count);
  long long enc_total = 0;
  for (long long q = 0; q < count; ++q) {
    work[q] = M[q] > 0 && N[q] > 0 && K[q] > 0 && alpha[q] != 0.0;
    nI[q] = (M[q] + BM - 1) / BM; nJ[q] = (N[q] + BN - 1) / BN;
    nks[q] = (K[q] + BK - 1) / BK; Kp[q] = nks[q] * BK;
    tiles[q] = work[q] ? nI[q] * nJ[q] : 0;
    if (work[q] && (!tma_ok(A[q], lda[q]) || !tma_ok(B[q], ldb[q]) || !tma_ok(C[q], ldc[q]))) {
      plan_free(P);
      return FTGEMM_ERR_UNALIGNED;
    }
    if (!work[q] || !P->ft) continue;
    off_acs[q] = enc_total; enc_total += round32(nI[q] * Kp[q]);
    off_bcs[q] = enc_total; enc_total += round32(nJ[q] * Kp[q]);
    off_ar[q] = enc_total; enc_total += round32(M[q]);
    off_am[q] = enc_total; enc_total += round32(nI[q]);
    off_bc[q] = enc_total; enc_total += round32(N[q]);
    off_bm[q] = enc_total; enc_total += round32(nJ[q]);
  }
  double *enc = nullptr;
  PLAN_TRY(plan_alloc(P, &enc, (size_t)std::max<long long>(1, enc_total)));
  PLAN_TRY(plan_alloc(P, &P->reps, (size_t)std::max<long long>(1, count)));
  PLAN_TRY(plan_alloc(P, &P->locs, (size_t)std::max<long long>(1, count) * PLAN_LOC_CAP));
  int *gerr = nullptr;
  PLAN_TRY(plan_alloc(P, &gerr, 1));

  // injection table: sorted by (problem, tile, k-step); per-problem tile offsets
  std::vector<long long> tile_base(count + 1, 0);
  for (long long q = 0; q < count; ++q) tile_base[q + 1] = tile_base[q] + tiles[q] + 1;
  std::vector<ftgemm_flip> L;
  std::vector<int> Lp;
  if (P->ft && g_inj.mode == 1 && count > 0) {
    for (long long f = 0; f < g_inj.count; ++f) {
      const long long q = (long long)(splitmix64(g_inj.seed, 5 * (uint64_t)f) % (uint64_t)count);
      if (!work[q]) continue;
      ftgemm_flip x;
      x.row = (long long)(splitmix64(g_inj.seed, 5 * (uint64_t)f + 1) % (uint64_t)M[q]);
      x.col = (long long)(splitmix64(g_inj.seed, 5 * (uint64_t)f + 2) % (uint64_t)N[q]);
      x.kstep = (long long)(splitmix64(g_inj.seed, 5 * (uint64_t)f + 3) % (uint64_t)nks[q]);
      x.bit = (int)(splitmix64(g_inj.seed, 5 * (uint64_t)f + 4) % 63u);
      x.problem = (int)q;
      L.push_back(x);
      Lp.push_back((int)q);
    }
  } else if (P->ft && g_inj.mode == 2) {
    for (const auto &x : g_inj.list) {
      const long long q = x.problem;
      if (q < 0 || q >= count || !work[q] || x.row < 0 || x.row >= M[q] || x.col < 0 || x.col >= N[q] ||
          x.kstep < 0 || x.kstep >= nks[q] || x.bit < 0 || x.bit > 62) {
        plan_free(P);
        return FTGEMM_ERR_INJECT;
      }
      L.push_back(x);
      Lp.push_back((int)q);
    }
  }
  P->nflips = (long long)L.size();
  P->inj = P->nflips > 0;
  P->flip_problem = Lp;
  P->flip_perm.resize(P->nflips);
  for (long long q = 0; q < P->nflips; ++q) P->flip_perm[q] = q;
  auto ltile = [&](const ftgemm_flip &f) { return (f.row / BM) + (f.col / BN) * nI[f.problem]; };
  std::stable_sort(P->flip_perm.begin(), P->flip_perm.end(), [&](long long a, long long b) {
    if (L[a].problem != L[b].problem) return L[a].problem < L[b].problem;
    const long long ta = ltile(L[a]), tb = ltile(L[b]);
    return ta != tb ? ta < tb : L[a].kstep < L[b].kstep;
  });
  std::vector<DevFlip> hf(std::max<long long>(1, P->nflips));
  std::vector<int> hoff(tile_base[count] + 1, 0);
  for (long long q = 0; q < P->nflips; ++q) {
    const ftgemm_flip &f = L[P->flip_perm[q]];
    hf[q].row = f.row; hf[q].col = f.col; hf[q].kstep = f.kstep; hf[q].bit = f.bit;
    hf[q].applied = 0; hf[q].before = 0.0; hf[q].after = 0.0; hf[q].kfirst = 0;
    hoff[tile_base[f.problem] + ltile(f) + 1]++;
  }
  // offsets are global flip indices; each problem's segment starts where the previous ended
  {
    long long run = 0;
    for (long long q = 0; q < count; ++q) {
      hoff[tile_base[q]] = (int)run;
      for (long long t = 0; t < tiles[q]; ++t) {
        run += hoff[tile_base[q] + t + 1];
        hoff[tile_base[q] + t + 1] = (int)run;
      }
    }
  }
  int *doff = nullptr;
  PLAN_TRY(plan_alloc(P, &P->flips, hf.size()));
  PLAN_TRY(plan_alloc(P, &doff, hoff.size()));
  cudaMemcpy(P->flips, hf.data(), sizeof(DevFlip) * hf.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(doff, hoff.data(), sizeof(int) * hoff.size(), cudaMemcpyHostToDevice);

  // problem descriptors (TMA maps + parameters)
  std::vector<BatchProblem> hp(std::max<long long>(1, count));
  for (long long q = 0; q < count; ++q) {
    memset(&hp[q], 0, sizeof(BatchProblem));
    if (!work[q]) continue;
    const bool ta_t = is_t(transA[q]), tb_t = is_t(transB[q]);
    if (ta_t) rc = make_map(&hp[q].tmA, A[q], K[q], M[q], lda[q], BK, BM, true);
    else rc = make_map(&hp[q].tmA, A[q], M[q], K[q], lda[q], BM, BK, false);
    if (!rc) rc = tb_t ? make_map(&hp[q].tmB, B[q], N[q], K[q], ldb[q], BN, BK, false)
                       : make_map(&hp[q].tmB, B[q], K[q], N[q], ldb[q], BK, BN, true);
    if (!rc) rc = make_map(&hp[q].tmC, C[q], M[q], N[q], ldc[q], BM, BN, false);
    if (rc) {
      plan_free(P);
      return rc;
    }
    Params &pp = hp[q].p;
    pp.M = M[q]; pp.N = N[q]; pp.K = K[q]; pp.alpha = alpha[q]; pp.beta = beta[q];
    pp.A = A[q]; pp.B = B[q]; pp.C = C[q]; pp.lda = lda[q]; pp.ldb = ldb[q]; pp.ldc = ldc[q];
    pp.nI = (int)nI[q]; pp.nJ = (int)nJ[q]; pp.nks = (int)nks[q]; pp.Kp = Kp[q];
    if (P->ft) {
      pp.acs = enc + off_acs[q]; pp.bcs = enc + off_bcs[q];
      pp.arowabs = enc + off_ar[q]; pp.aabsmax = enc + off_am[q];
      pp.bcolabs = enc + off_bc[q]; pp.babsmax = enc + off_bm[q];
    }
    pp.rep = P->reps + q;
    pp.loc = P->locs + q * PLAN_LOC_CAP;
    pp.loc_cap = PLAN_LOC_CAP;
    pp.flips = P->flips;
    pp.tile_off = doff + tile_base[q];
    pp.wait_limit_ns = wait_limit_ns();
    pp.correct_mode = g_correct;
    pp.nsplit = 1;
  }
  BatchProblem *dprobs = nullptr;
  PLAN_TRY(plan_alloc(P, &dprobs, hp.size()));
  cudaMemcpy(dprobs, hp.data(), sizeof(BatchProblem) * hp.size(), cudaMemcpyHostToDevice);

  // checksum-pass items, one per operand, read through the problem's own TMA
  // maps (in dprobs); one block per 128-wide group, the items ordered by their
  // k extent, longest first
  std::vector<EncItem> items;
  int enc_blocks = 0;
  for (long long q = 0; q < count && P->ft; ++q) {
    if (!work[q]) continue;
    EncItem a{}, b{};
    a.map = &dprobs[q].tmA; a.X = A[q]; a.ld = lda[q]; a.W = M[q]; a.L = K[q]; a.kfirst = is_t(transA[q]) ? 1 : 0;
    a.gsum = enc + off_acs[q]; a.gstride = Kp[q]; a.absv = enc + off_ar[q]; a.gmax = enc + off_am[q];
    b.map = &dprobs[q].tmB; b.X = B[q]; b.ld = ldb[q]; b.W = N[q]; b.L = K[q]; b.kfirst = is_t(transB[q]) ? 0 : 1;
    b.gsum = enc + off_bcs[q]; b.gstride = Kp[q]; b.absv = enc + off_bc[q]; b.gmax = enc + off_bm[q];
    a.err = b.err = &P->reps[q].err;
    a.first_block = (int)nI[q];   // group counts until the prefix sums below
    b.first_block = (int)nJ[q];
    items.push_back(a);
    items.push_back(b);
  }
  std::stable_sort(items.begin(), items.end(), [](const EncItem &x, const EncItem &y) { return x.L > y.L; });
  std::vector<int> block_item;
  for (size_t q = 0; q < items.size(); ++q) {
    EncItem &e = items[q];
    const int groups = e.first_block;
    e.first_block = enc_blocks;
    enc_blocks += groups;
    block_item.insert(block_item.end(), (size_t)groups, (int)q);
  }
  EncItem *ditems = nullptr;
  int *dblock_item = nullptr;
  PLAN_TRY(plan_alloc(P, &ditems, std::max<size_t>(1, items.size())));
  PLAN_TRY(plan_alloc(P, &dblock_item, std::max<size_t>(1, block_item.size())));
  if (!items.empty()) cudaMemcpy(ditems, items.data(), sizeof(EncItem) * items.size(), cudaMemcpyHostToDevice);
  if (!block_item.empty())
    cudaMemcpy(dblock_item, block_item.data(), sizeof(int) * block_item.size(), cudaMemcpyHostToDevice);
  if (enc_blocks && cudaFuncSetAttribute(enc_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         ENC_SMEM_BYTES) != cudaSuccess) {
    cudaGetLastError();
    plan_free(P);
    return FTGEMM_ERR_CUDA;
  }

  // work lists per operand layout, in the scheduled order
  struct Group { std::vector<int> prob, local, order; };
  Group grp[4];
  for (long long q = 0; q < count; ++q) {
    if (!work[q]) continue;
    Group &g = grp[(is_t(transA[q]) ? 2 : 0) + (is_t(transB[q]) ? 1 : 0)];
    for (long long t = 0; t < tiles[q]; ++t) { g.prob.push_back((int)q); g.local.push_back((int)t); }
  }
  int *counters = nullptr;
  PLAN_TRY(plan_alloc(P, &counters, 4));
  int *dgrp[4][3] = {};
  for (int gi = 0; gi < 4; ++gi) {
    Group &g = grp[gi];
    const int total = (int)g.prob.size();
    g.order.resize(total);
    for (int i = 0; i < total; ++i) g.order[i] = i;
    if (order_kind == 1) {  // longest first: k-slabs of the tile, largest first
      std::stable_sort(g.order.begin(), g.order.end(), [&](int a, int b) { return nks[g.prob[a]] > nks[g.prob[b]]; });
    } else if (order_kind == 2) {  // round robin over problems
      std::stable_sort(g.order.begin(), g.order.end(), [&](int a, int b) { return g.local[a] < g.local[b]; });
    }
    if (!total) continue;
    PLAN_TRY(plan_alloc(P, &dgrp[gi][0], total));
    PLAN_TRY(plan_alloc(P, &dgrp[gi][1], total));
    PLAN_TRY(plan_alloc(P, &dgrp[gi][2], total));
    cudaMemcpy(dgrp[gi][0], g.order.data(), sizeof(int) * total, cudaMemcpyHostToDevice);
    cudaMemcpy(dgrp[gi][1], g.prob.data(), sizeof(int) * total, cudaMemcpyHostToDevice);
    cudaMemcpy(dgrp[gi][2], g.local.data(), sizeof(int) * total, cudaMemcpyHostToDevice);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    plan_free(P);
    return FTGEMM_ERR_CUDA;
  }

  // capture: reset, checksum pass, quick returns, one persistent kernel per layout
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    plan_free(P);
    return FTGEMM_ERR_CUDA;
  }
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    cudaMemsetAsync(counters, 0, 4 * sizeof(int), cs);
    cudaMemsetAsync(gerr, 0, sizeof(int), cs);
    cudaMemsetAsync(P->reps, 0, sizeof(DevReport) * std::max<long long>(1, count), cs);
    if (P->ft && enc_total) {
      cudaMemsetAsync(enc, 0, sizeof(double) * enc_total, cs);
      if (enc_blocks) {
        enc_batched_kernel<<<enc_blocks, 256, ENC_SMEM_BYTES, cs>>>(ditems, dblock_item, gerr, wait_limit_ns());
        P->kernels++;
      }
    }
    for (long long q = 0; q < count; ++q)
      if (!work[q] && M[q] > 0 && N[q] > 0 && beta[q] != 1.0) {
        scale_kernel<<<grid_for(M[q] * N[q]), 256, 0, cs>>>(C[q], M[q], N[q], ldc[q], beta[q]);
        P->kernels++;
      }
    for (int gi = 0; gi < 4; ++gi) {
      const int total = (int)grp[gi].prob.size();
      if (!total) continue;
      const int grid = std::min(nsm, (total + chunk - 1) / chunk);
      auto launch = gi == 0 ? launch_batched_nn : gi == 1 ? launch_batched_nt : gi == 2 ? launch_batched_tn
                                                                                    : launch_batched_tt;
      const cudaError_t e = launch(P->ft, P->inj, dprobs, dgrp[gi][0], dgrp[gi][1], dgrp[gi][2], total, chunk,
                                   counters + gi, gerr, grid, cs);
      ok = ok && e == cudaSuccess;
      P->kernels++;
    }
    ok = (cudaStreamEndCapture(cs, &P->graph) == cudaSuccess) && ok;
  }
  if (ok) ok = cudaGraphInstantiate(&P->exec, P->graph, 0) == cudaSuccess;
  cudaStreamDestroy(cs);
  if (!ok) {
    cudaGetLastError();
    plan_free(P);
    return FTGEMM_ERR_CUDA;
  }
  (void)stream;
#undef PLAN_TRY
  *plan_out = P;
  return 0;
}

int ftgemm_batched_plan_launch(ftgemm_batched_plan plan, void *stream) {
  if (!plan || !plan->exec) return -1;
  if (cudaGraphLaunch(plan->exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_CUDA;
  }
  g_launches += plan->kernels;
  return 0;
}

int ftgemm_batched_plan_report(ftgemm_batched_plan plan, ftgemm_report *reps, void *stream) {
  if (!plan) return -1;
  cudaStream_t s = (cudaStream_t)stream;
  const long long n = plan->count;
  std::vector<DevReport> hr(std::max<long long>(1, n));
  std::vector<DevLoc> hl(std::max<long long>(1, n) * PLAN_LOC_CAP);
  if (cudaMemcpyAsync(hr.data(), plan->reps, sizeof(DevReport) * hr.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(hl.data(), plan->locs, sizeof(DevLoc) * hl.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return FTGEMM_ERR_CUDA;
  }
  int err = 0;
  for (long long q = 0; q < n; ++q) {
    if (hr[q].err) err = FTGEMM_ERR_TIMEOUT;
    if (!reps) continue;
    ftgemm_report &r = reps[q];
    r.detected = (long long)hr[q].detected;
    r.corrected = (long long)hr[q].corrected;
    r.checksum_only = (long long)hr[q].checksum_only;
    r.unverifiable = (long long)hr[q].unverifiable;
    r.flagged_rows = (long long)hr[q].flagged_rows;
    r.flagged_cols = (long long)hr[q].flagged_cols;
    r.recomputed = (long long)hr[q].recomputed;
    r.panel_detected = (long long)hr[q].panel_detected;
    r.n_loc = (long long)hr[q].n_loc;
    if (r.loc)
      for (long long k = 0; k < std::min<long long>({r.cap, (long long)PLAN_LOC_CAP, r.n_loc}); ++k) {
        const DevLoc &d = hl[q * PLAN_LOC_CAP + k];
        r.loc[k].row = d.row; r.loc[k].col = d.col; r.loc[k].tile = d.tile; r.loc[k].kind = d.kind;
        r.loc[k].delta = d.delta;
      }
  }
  return err;
}

int64_t ftgemm_batched_plan_injection_log(ftgemm_batched_plan plan, ftgemm_flip_log *out, int64_t cap) {
  if (!plan) return -1;
  const long long nf = plan->nflips;
  if (nf == 0 || cap <= 0 || !out) return nf;
  std::vector<DevFlip> h((size_t)nf);
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(h.data(), plan->flips, sizeof(DevFlip) * nf, cudaMemcpyDeviceToHost) != cudaSuccess)
    return -FTGEMM_ERR_CUDA;
  for (long long q = 0; q < nf; ++q) {
    const long long o = plan->flip_perm[q];
    if (o >= cap) continue;
    out[o].row = h[q].row; out[o].col = h[q].col; out[o].kstep = h[q].kstep; out[o].bit = h[q].bit;
    out[o].applied = h[q].applied; out[o].before = h[q].before; out[o].after = h[q].after;
    out[o].kfirst = h[q].kfirst;
    out[o].problem = plan->flip_problem[o];
  }
  return nf;
}

int ftgemm_batched_plan_destroy(ftgemm_batched_plan plan) {
  if (!plan) return -1;
  cudaDeviceSynchronize();
  plan_free(plan);
  return 0;
}

int ftgemm_batched(int64_t count, const char *transA, const char *transB, const int64_t *M, const int64_t *N,
                   const int64_t *K, const double *alpha, const double *const *A, const int64_t *lda,
                   const double *const *B, const int64_t *ldb, const double *beta, double *const *C,
                   const int64_t *ldc, ftgemm_report *reps, void *stream) {
  ftgemm_batched_plan plan = nullptr;
  int rc = ftgemm_batched_plan_create(&plan, count, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                      1, -1, stream);
  if (rc) return rc;
  rc = ftgemm_batched_plan_launch(plan, stream);
  if (!rc) rc = ftgemm_batched_plan_report(plan, reps, stream);
  ftgemm_batched_plan_destroy(plan);
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Split-precision FT-GEMM (BF16 tensor cores; see ftgemm_split.cuh).
namespace {

// 3-D map {Kp, R, S} of slices: bf16, or bytes (INT8 slices, i8); the box is
// one 128-byte row of k by box_rows rows, with the 128-byte swizzle.
int make_map_slices(CUtensorMap *m, const void *ptr, long long Kp, long long R, long long S, int box_rows,
                    bool i8 = false) {
  auto fn = encode_fn();
  if (!fn) return FTGEMM_ERR_TENSORMAP;
  const long long esz = i8 ? 1 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)R, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)(Kp * esz), (cuuint64_t)(R * Kp * esz)};
  cuuint32_t box[3] = {(cuuint32_t)(i8 ? SP_BK_I8 : SP_BK), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, i8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void *>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : FTGEMM_ERR_TENSORMAP;
}

}  // namespace

extern "C" int ftgemm_d_split(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                              const double *A, int64_t lda, const double *B, int64_t ldb, double beta, double *C,
                              int64_t ldc, int nslices, int ft, ftgemm_report *rep, void *stream) {
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = check_args(transA, transB, M, N, K, lda, ldb, ldc);
  if (rc) return rc;
  if (nslices < 0 || nslices > 15) return -14;
  if (ft < 0 || ft > 2 || (ft == 2 && nslices == 0)) return -15;
  zero_report(rep);
  if (M == 0 || N == 0) return 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (K == 0 || alpha == 0.0)
    return gemm_impl(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, rep, s, true);
  // the slicing passes give each 8 rows of an operand one block along grid y
  static_assert(FTGEMM_SPLIT_MAX_ROWS == 8LL * 65535, "largest row count of the slicing grids");
  if (M > FTGEMM_SPLIT_MAX_ROWS || N > FTGEMM_SPLIT_MAX_ROWS) return FTGEMM_ERR_TOO_LARGE;
  int dev = 0;
  Workspace *wp = workspace(&dev);
  if (!wp) return FTGEMM_ERR_NODEVICE;
  Workspace &w = *wp;
  const bool ta_t = is_t(transA), tb_t = is_t(transB);
  const bool plain = nslices == 0;
  const int S = plain ? 1 : nslices;
  // INT8 slices (engine 7, emulated forms): 7 bits each, exact INT32 sums
  const bool i8 = g_split_engine == 7 && !plain;
  if (i8 && ft == 1) return -15;
  const long long sbk = i8 ? SP_BK_I8 : SP_BK, esz = i8 ? 1 : 2;
  const long long Kp = (K + sbk - 1) / sbk * sbk;
  // bits per slice: the FP32 (INT32) accumulation of a pair stays exact over
  // kchunk products
  int wbits = 0;
  long long kchunk = Kp;
  if (i8) {
    wbits = 7;
    kchunk = std::min<long long>(Kp, ((1LL << 31) - 1) / (127 * 127) / SP_BK_I8 * SP_BK_I8);
  } else if (!plain) {
    wbits = K <= 256 ? 8 : K <= 1024 ? 7 : K <= 4096 ? 6 : 5;
    const long long lim = (1LL << 24) / (((1LL << wbits) - 1) * ((1LL << wbits) - 1));
    kchunk = std::max<long long>(SP_BK, lim / SP_BK * SP_BK);
  }
  const long long nI = (M + SP_BM - 1) / SP_BM, nJ = (N + SP_BN - 1) / SP_BN;
  if (ensure(w.spA, (size_t)(S * M * Kp * esz)) || ensure(w.spB, (size_t)(S * N * Kp * esz)) ||
      ensure(w.spEA, sizeof(int) * M) || ensure(w.spEB, sizeof(int) * N))
    return FTGEMM_ERR_NOMEM;
  if (plain) {
    cudaMemsetAsync(w.spEA.p, 0, sizeof(int) * M, s);
    cudaMemsetAsync(w.spEB.p, 0, sizeof(int) * N, s);
  }
  // ft 2: the operand checksum pass (FP64 adds) runs on the second stream
  // while the slicing passes (integer and memory work) run on s
  // tcgen05 kernels (ft 0 / 2, and the plain form with ft 1) or the mma.sync
  // kernel; ck: the kernels' check mode (2: verification against the
  // checksum products P1 / P2 computed before the product)
  const bool tc = !i8 && g_split_engine != 1 && g_split_engine != 7 && (ft != 1 || plain);
  const int ck = tc ? (ft ? 2 : 0) : ft;
  // the plain form on tcgen05 with checks: P1 / P2 are plain BF16 products of
  // the two bf16 pieces of the checksum vectors (P1 with 2 nI rows, P2 with
  // 2 nJ columns), computed from the bf16 operands
  const bool plain_ck = plain && ft == 1 && tc;
  const long long Kq = (K + BK - 1) / BK * BK, ldp1 = ((plain_ck ? 2 * nI : nI) + 1) & ~1LL,
                  ldp2 = (M + 1) & ~1LL;
  if (ft == 2) {
    if (ensure(w.acs, sizeof(double) * nI * Kq) || ensure(w.bcs, sizeof(double) * nJ * Kq) ||
        ensure(w.arowabs, sizeof(double) * M) || ensure(w.aabsmax, sizeof(double) * nI) ||
        ensure(w.bcolabs, sizeof(double) * N) || ensure(w.babsmax, sizeof(double) * nJ) ||
        ensure(w.uP1, sizeof(double) * ldp1 * N) || ensure(w.uP2, sizeof(double) * ldp2 * nJ))
      return FTGEMM_ERR_NOMEM;
    if (!tma_ok(A, lda) || !tma_ok(B, ldb)) return FTGEMM_ERR_UNALIGNED;
    if ((rc = ensure_side(w))) return rc;
    cudaEventRecord(w.fork_ev, s);
    cudaStreamWaitEvent(w.side, w.fork_ev, 0);
    if ((rc = run_encode(ta_t, tb_t, M, N, K, A, lda, B, ldb, Kq, (double *)w.acs.p, (double *)w.aabsmax.p,
                         (double *)w.arowabs.p, (double *)w.bcs.p, (double *)w.babsmax.p, (double *)w.bcolabs.p,
                         w, w.side, false)))
      return rc;
  }
  // op(A)(i, k): 'T' has k contiguous; op(B)(k, j) seen as row j: 'N' has k contiguous
  const int nsm = device_sms(dev);
  if (ensure(w.spMB, (sizeof(unsigned long long) + sizeof(unsigned int)) * (size_t)std::max(M, N)))
    return FTGEMM_ERR_NOMEM;
  unsigned long long *mb = (unsigned long long *)w.spMB.p;
  if (launch_slicing(A, lda, ta_t ? 1 : 0, M, K, Kp, (int *)w.spEA.p, S, wbits, plain, i8, w.spA.p, mb, nsm, s) !=
          cudaSuccess ||
      launch_slicing(B, ldb, tb_t ? 0 : 1, N, K, Kp, (int *)w.spEB.p, S, wbits, plain, i8, w.spB.p, mb, nsm, s) !=
          cudaSuccess)
    return FTGEMM_ERR_CUDA;
  g_launches += plain ? 2 : 4;
  // tcgen05 kernel (ft 0 / 2): persistent (at most one CTA per SM, the
  // default) or one CTA per tile
  const bool persist = tc && g_split_engine != 2;
  auto run_tc = [&](bool ta, bool tb, int ck, const CUtensorMap &a, const CUtensorMap &b, const SplitParams &q,
                    cudaStream_t st) {
    if (persist)
      return launch_split_tcp(ta, tb, ck, a, b, q, (int)std::min<long long>((long long)q.nI * q.nJ, nsm), st);
    return launch_split_tc(ta, tb, ck, a, b, q, st);
  };
  CUtensorMap mA, mB;
  if ((rc = make_map_slices(&mA, w.spA.p, Kp, M, S, SP_BM, i8)) ||
      (rc = make_map_slices(&mB, w.spB.p, Kp, N, S, SP_BN, i8)))
    return rc;

  SplitParams p;
  memset(&p, 0, sizeof(p));
  p.M = M; p.N = N; p.K = K; p.Kp = Kp; p.alpha = alpha; p.beta = beta;
  p.S = plain ? 0 : S; p.w = wbits; p.kchunk = (int)kchunk;
  // kept pairs s + t < S, smallest weights (largest s + t) first
  int np = 0;
  for (int d = S - 1; d >= 0; --d)
    for (int a = 0; a <= d; ++a) { p.pair_s[np] = a; p.pair_t[np] = d - a; ++np; }
  p.npairs = np;
  p.eA = (const int *)w.spEA.p; p.eB = (const int *)w.spEB.p;
  p.A = A; p.B = B; p.lda = lda; p.ldb = ldb; p.ta = ta_t; p.tb = tb_t;
  p.C = C; p.ldc = ldc; p.nI = (int)nI; p.nJ = (int)nJ;
  p.i8 = i8 ? 1 : 0;
  p.rep = (DevReport *)w.rep.p; p.loc = (DevLoc *)w.loc.p; p.loc_cap = LOC_CAP_DEV;
  p.wait_limit_ns = wait_limit_ns();
  p.verify = ft;
  if (plain && ft) {  // flagged elements are recomputed from the bf16 operands
    p.Ab = (const uint16_t *)w.spA.p;
    p.Bb = (const uint16_t *)w.spB.p;
    p.ldk = Kp;
  }
  if (plain_ck) {
    // the checksum vectors of the bf16 operands (op(A)'s on s, op(B)'s on the
    // second stream), then P1 = pieces(acs) op(B) on s and P2 = op(A)
    // pieces(bcs) on the second stream, as plain products
    const long long sa = bf16_checksum_scratch(M, Kp), sb = bf16_checksum_scratch(N, Kp);
    if (ensure(w.spPA, (size_t)2 * nI * Kp * 2) || ensure(w.spPB, (size_t)2 * nJ * Kp * 2) ||
        ensure(w.spEPA, sizeof(int) * 2 * nI) || ensure(w.spEPB, sizeof(int) * 2 * nJ) ||
        ensure(w.arowabs, sizeof(double) * M) || ensure(w.aabsmax, sizeof(double) * nI) ||
        ensure(w.bcolabs, sizeof(double) * N) || ensure(w.babsmax, sizeof(double) * nJ) ||
        ensure(w.uP1, sizeof(double) * ldp1 * N) || ensure(w.uP2, sizeof(double) * ldp2 * 2 * nJ) ||
        ensure(w.part_abs, sizeof(float) * sa) || ensure(w.part_abs2, sizeof(float) * sb))
      return FTGEMM_ERR_NOMEM;
    if ((rc = ensure_side(w))) return rc;
    cudaMemsetAsync(w.spEPA.p, 0, sizeof(int) * 2 * nI, s);
    cudaMemsetAsync(w.spEPB.p, 0, sizeof(int) * 2 * nJ, s);
    cudaEventRecord(w.fork_ev, s);
    cudaStreamWaitEvent(w.side, w.fork_ev, 0);
    if (launch_bf16_checksums(w.spA.p, M, Kp, w.spPA.p, (double *)w.arowabs.p, (double *)w.aabsmax.p,
                              (float *)w.part_abs.p, s) != cudaSuccess ||
        launch_bf16_checksums(w.spB.p, N, Kp, w.spPB.p, (double *)w.bcolabs.p, (double *)w.babsmax.p,
                              (float *)w.part_abs2.p, w.side) != cudaSuccess)
      return FTGEMM_ERR_CUDA;
    g_launches += 4;
    CUtensorMap mPA, mPB;
    if ((rc = make_map_slices(&mPA, w.spPA.p, Kp, 2 * nI, 1, SP_BM)) ||
        (rc = make_map_slices(&mPB, w.spPB.p, Kp, 2 * nJ, 1, SP_BN)))
      return rc;
    SplitParams q1 = p, q2 = p;
    q1.M = 2 * nI; q1.nI = (int)((2 * nI + SP_BM - 1) / SP_BM);
    q1.eA = (const int *)w.spEPA.p; q1.C = (double *)w.uP1.p; q1.ldc = ldp1;
    q2.N = 2 * nJ; q2.nJ = (int)((2 * nJ + SP_BN - 1) / SP_BN);
    q2.eB = (const int *)w.spEPB.p; q2.C = (double *)w.uP2.p; q2.ldc = ldp2;
    for (SplitParams *q : {&q1, &q2}) { q->alpha = 1.0; q->beta = 0.0; q->verify = 0; q->inj = 0; }
    if (run_tc(false, false, 0, mPA, mB, q1, s) != cudaSuccess ||
        run_tc(false, false, 0, mA, mPB, q2, w.side) != cudaSuccess)
      return FTGEMM_ERR_CUDA;
    cudaEventRecord(w.join_ev, w.side);
    cudaStreamWaitEvent(s, w.join_ev, 0);
    g_launches += 2;
    p.P1 = (const double *)w.uP1.p; p.ldp1 = ldp1; p.p1_lo = nI;
    p.P2 = (const double *)w.uP2.p; p.ldp2 = ldp2; p.p2_lo = nJ * ldp2;
    p.arowabs = (const double *)w.arowabs.p; p.aabsmax = (const double *)w.aabsmax.p;
    p.bcolabs = (const double *)w.bcolabs.p; p.babsmax = (const double *)w.babsmax.p;
  }
  cudaMemsetAsync(w.rep.p, 0, sizeof(DevReport), s);
  if (ft == 2) {
    // FP64 predicted checksums of the 128 x 128 tiles from the original
    // operands: the checksum pass (side stream) joins here
    cudaEventRecord(w.join_ev, w.side);
    cudaStreamWaitEvent(s, w.join_ev, 0);
    p.P1 = (const double *)w.uP1.p; p.ldp1 = ldp1; p.P2 = (const double *)w.uP2.p; p.ldp2 = ldp2;
    if (tc) {
      // P1 = acs^T op(B) and P2 = op(A) bcs by the same emulated product on the
      // tensor cores: slice the checksum operands (rows I of acs^T, columns J
      // of bcs), reuse op(B)'s and op(A)'s slices
      if (ensure(w.spPA, (size_t)S * nI * Kp * 2) || ensure(w.spPB, (size_t)S * nJ * Kp * 2) ||
          ensure(w.spEPA, sizeof(int) * nI) || ensure(w.spEPB, sizeof(int) * nJ))
        return FTGEMM_ERR_NOMEM;
      if (launch_slicing((const double *)w.acs.p, Kq, 1, nI, K, Kp, (int *)w.spEPA.p, S, wbits, 0, 0, w.spPA.p, mb,
                         nsm, s) != cudaSuccess ||
          launch_slicing((const double *)w.bcs.p, Kq, 1, nJ, K, Kp, (int *)w.spEPB.p, S, wbits, 0, 0, w.spPB.p, mb,
                         nsm, s) != cudaSuccess)
        return FTGEMM_ERR_CUDA;
      g_launches += 4;
      CUtensorMap mPA, mPB;
      if ((rc = make_map_slices(&mPA, w.spPA.p, Kp, nI, S, SP_BM)) ||
          (rc = make_map_slices(&mPB, w.spPB.p, Kp, nJ, S, SP_BN)))
        return rc;
      SplitParams q1 = p, q2 = p;
      q1.M = nI; q1.nI = (int)((nI + SP_BM - 1) / SP_BM);
      q1.eA = (const int *)w.spEPA.p; q1.C = (double *)w.uP1.p; q1.ldc = ldp1;
      q2.N = nJ; q2.nJ = (int)((nJ + SP_BN - 1) / SP_BN);
      q2.eB = (const int *)w.spEPB.p; q2.C = (double *)w.uP2.p; q2.ldc = ldp2;
      for (SplitParams *q : {&q1, &q2}) { q->alpha = 1.0; q->beta = 0.0; q->verify = 0; q->inj = 0; }
      // P1 and P2 are independent one-wave grids: P2 runs on a second stream
      if ((rc = ensure_side(w))) return rc;
      cudaEventRecord(w.fork_ev, s);
      cudaStreamWaitEvent(w.side, w.fork_ev, 0);
      if (run_tc(false, false, 0, mPA, mB, q1, s) != cudaSuccess ||
          run_tc(false, false, 0, mA, mPB, q2, w.side) != cudaSuccess)
        return FTGEMM_ERR_CUDA;
      cudaEventRecord(w.join_ev, w.side);
      cudaStreamWaitEvent(s, w.join_ev, 0);
      g_launches += 2;
      p.ePA = (const int *)w.spEPA.p; p.ePB = (const int *)w.spEPB.p;
    } else {
      if ((rc = gemm_impl('T', transB, nI, N, K, 1.0, (const double *)w.acs.p, Kq, B, ldb, 0.0, (double *)w.uP1.p,
                          ldp1, nullptr, s, false)))
        return rc;
      if ((rc = gemm_impl(transA, 'N', M, nJ, K, 1.0, A, lda, (const double *)w.bcs.p, Kq, 0.0,
                          (double *)w.uP2.p, ldp2, nullptr, s, false)))
        return rc;
    }
    p.arowabs = (const double *)w.arowabs.p; p.aabsmax = (const double *)w.aabsmax.p;
    p.bcolabs = (const double *)w.bcolabs.p; p.babsmax = (const double *)w.babsmax.p;
  }
  bool inj = false;
  if (ft) {
    Params tmp;
    memset(&tmp, 0, sizeof(tmp));
    if ((rc = upload_injection(M, N, np, nI, nI * nJ, w, s, tmp, &inj))) return rc;
    p.flips = tmp.flips; p.tile_off = tmp.tile_off; p.inj = inj ? 1 : 0;
  }
  if (persist && ck == 2) {
    // one tile per CTA of the grid
    const long long ctas = std::min<long long>(nI * nJ, nsm);
    if (ensure(w.tscr, sizeof(double) * SP_BM * SP_BN * (size_t)ctas))
      return FTGEMM_ERR_NOMEM;
    p.tscratch = (double *)w.tscr.p;
  }
  cudaEvent_t em0 = nullptr, em1 = nullptr;
  if (g_tim.on) {
    timing_record(g_tim.main_ev, &em0, &em1);
    cudaEventRecord(em0, s);
  }
  if ((tc ? run_tc(ta_t, tb_t, ck, mA, mB, p, s) : launch_split(ta_t, tb_t, ft, i8, mA, mB, p, s)) !=
      cudaSuccess)
    return FTGEMM_ERR_CUDA;
  if (g_tim.on) cudaEventRecord(em1, s);
  g_launches++;
  if (rep) return copy_report(w, rep, s);
  return cudaGetLastError() == cudaSuccess ? 0 : FTGEMM_ERR_CUDA;
}
