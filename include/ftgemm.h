/*
 * ftgemm.h -- C ABI of libftgemm, a fault-tolerant FP64 GEMM for one NVIDIA
 * GB300 (sm_103a).
 *
 * The operation is the BLAS DGEMM of FT-GEMM (Wu et al., HPDC'23, abstract
 * and §2.1):
 *
 *     C <- alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T,
 *
 * protected by algorithm-based fault tolerance (§2.2, after Huang and Abraham
 * 1984): for every BM x BN output tile the library predicts the column and
 * row checksums of the result from checksums of the operands and of beta*C,
 * sums the reference checksums from the computed tile before it leaves the
 * chip, and on a mismatch locates the wrong elements and rewrites them with a
 * recomputed value.  Faults are injected at source level (§3.2) by flipping
 * seeded bits of accumulator values.
 *
 * Conventions (all entry points):
 *  - Column-major storage.  trans is 'N'/'n' (op(X) = X) or 'T'/'t'/'C'/'c'
 *    (op(X) = X^T; real data, so 'C' equals 'T').  op(A) is M x K, op(B) is
 *    K x N, C is M x N.
 *  - Matrix pointers of ftgemm_d* are DEVICE pointers owned by the caller;
 *    they must stay valid until the stream reaches the end of the call.
 *    ftgemm_d_host takes HOST pointers instead.  Report and injection structs
 *    are HOST memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is stream-ordered.  A call with rep == NULL returns after
 *    enqueueing (no host synchronisation); a call with rep != NULL waits for
 *    its own stream so that the report is complete on return.
 *  - Return value: 0 on success; -i when argument i is invalid (BLAS xerbla
 *    numbering: 1 transA, 2 transB, 3 M, 4 N, 5 K, 8 lda, 10 ldb, 13 ldc);
 *    a positive FTGEMM_ERR_* code otherwise.  A detected and corrected fault
 *    is not an error: the call returns 0 and the report counts it.
 *  - BLAS quick returns: M == 0 or N == 0 does nothing; K == 0 or alpha == 0
 *    gives C = beta*C; beta == 0 never reads C (NaN in C does not propagate).
 *  - The library owns a lazily grown per-device workspace (operand checksum
 *    vectors, the device report, the injection table, staging for unaligned
 *    operands and for ftgemm_d_host) and a second stream on which a call runs
 *    independent parts of its work (forked from and joined back into the
 *    caller's stream by events, so the call stays stream-ordered), released
 *    by ftgemm_finalize().  Calls share them, so calls must not run
 *    concurrently on different streams or host threads.
 *  - Operands whose base address is not 16-byte aligned or whose leading
 *    dimension is odd are first copied into aligned workspace (the tensor
 *    memory accelerator needs 16-byte aligned rows); results are the same.
 */
#ifndef FTGEMM_H
#define FTGEMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Output tile of the checksum scheme, and the k-step (products accumulated
 * between two points where a fault may be injected). */
#define FTGEMM_BM 128
#define FTGEMM_BN 128
#define FTGEMM_KSTEP 16

/* Positive error codes. */
#define FTGEMM_ERR_CUDA 1       /* a CUDA runtime call or kernel launch failed */
#define FTGEMM_ERR_TIMEOUT 2    /* a bounded pipeline wait expired on the device */
#define FTGEMM_ERR_NODEVICE 4   /* no usable CUDA device */
#define FTGEMM_ERR_NOMEM 5      /* workspace allocation failed */
#define FTGEMM_ERR_INJECT 6     /* an explicit fault lies outside the problem */
#define FTGEMM_ERR_TENSORMAP 7  /* a TMA descriptor could not be encoded */
#define FTGEMM_ERR_SCRATCH 8    /* ftgemm_d_noalloc: the problem needs more scratch than it holds */
#define FTGEMM_ERR_UNALIGNED 9  /* ftgemm_d_noalloc, ftgemm_d_unfused, the batched calls and
                                   ftgemm_d_split with ft = 2: an operand is not 16-byte
                                   aligned or its leading dimension is odd */
#define FTGEMM_ERR_BATCH 10     /* batched calls: count < 0, or a NULL plan pointer or
                                   per-problem array (count > 0) */
#define FTGEMM_ERR_TOO_LARGE 11 /* ftgemm_d_split: M or N above FTGEMM_SPLIT_MAX_ROWS */
#define FTGEMM_ERR_CAPTURE 12   /* ftgemm_d_noalloc: a report was requested (rep != NULL) on a
                                   stream that is being captured; nothing was enqueued */

/* Largest M and N of ftgemm_d_split (the slicing passes run one block per 8
 * operand rows along the 65535-block y dimension of their grids). */
#define FTGEMM_SPLIT_MAX_ROWS 524280

/* Size of the device array that ftgemm_d_noalloc uses as scratch. */
#define FTGEMM_NOALLOC_SCRATCH_BYTES (32u << 20)

/* One located fault: element (row, col) of C, 0-based. */
typedef struct {
  int64_t row, col;
  int32_t tile;  /* tile id: I + J * ceil(M / FTGEMM_BM) */
  int32_t kind;  /* 0: found at a flagged row x flagged column intersection;
                    1: found by the fallback that recomputes whole row/column
                       segments of a tile;
                    2: found by a per-k-panel check (accumulator corrected
                       before the end of K);
                    3: corrected by subtracting the column checksum residual
                       (ftgemm_set_correction(1)) */
  double delta;  /* stored value minus recomputed value (may be Inf/NaN); for
                    kind 3 the subtracted residual */
} ftgemm_loc;

/* Fault report of one call.  The caller sets cap and loc (loc may be NULL
 * with cap 0); the library fills the rest.  Every count is exact even when
 * n_loc > cap (then only the first cap records, in no particular order, are
 * written). */
typedef struct {
  int64_t detected;      /* elements whose recomputed value differed from the
                            computed one by more than the element bound */
  int64_t corrected;     /* of those, rewritten with the recomputed value */
  int64_t checksum_only; /* rows + columns whose mismatch survived every
                            recomputation: a fault in a checksum, data intact */
  int64_t unverifiable;  /* rows + columns (per tile) whose predicted checksum
                            was not finite because the inputs are not */
  int64_t flagged_rows;  /* row mismatches raised by the first verification */
  int64_t flagged_cols;  /* column mismatches raised by the first verification */
  int64_t recomputed;    /* elements recomputed, wrong or not */
  int64_t panel_detected; /* of `detected`, found by a per-k-panel check
                            (ftgemm_set_panel_check) before the end of K */
  int64_t n_loc;         /* location records produced */
  int64_t cap;           /* capacity of loc (input) */
  ftgemm_loc *loc;       /* caller-owned host array of cap records (input) */
} ftgemm_report;

/* One fault to inject: flip bit `bit` (0..62; the sign bit is excluded) of
 * the accumulator of C(row, col) right after its k-step `kstep`, i.e. after
 * its first min(K, FTGEMM_KSTEP * (kstep + 1)) products (source-level
 * injection, §3.2). */
typedef struct {
  int64_t row, col, kstep;
  int32_t bit;
  int32_t problem;  /* batched calls: index of the problem; otherwise ignored */
} ftgemm_flip;

/* Injection setting, process-global, applied to every later call that checks
 * its result: ftgemm_d, ftgemm_d_host, ftgemm_d_split with ft != 0, and the
 * batched calls (a plan takes the setting when it is created); not to
 * ftgemm_d_noft, ftgemm_d_noalloc or ftgemm_d_unfused.  mode 0: off.  mode 1: `count` faults per call at
 * positions drawn from splitmix64(seed): fault f takes outputs 4f..4f+3 of the
 * generator, n-th output = mix(seed + (n+1) * 0x9E3779B97F4A7C15), as
 * (row mod M, col mod N, kstep mod ceil(K/16), bit mod 63).  mode 2: the
 * explicit `list` of n_list faults (copied at the call). */
typedef struct {
  int32_t mode, pad;
  uint64_t seed;
  int64_t count;
  const ftgemm_flip *list;
  int64_t n_list;
} ftgemm_inject;

/* What happened to one injected fault of the last injected call. */
typedef struct {
  int64_t row, col, kstep;
  int32_t bit;
  int32_t applied;  /* 1 when the flip was made */
  double before;    /* accumulator value before the flip */
  double after;     /* accumulator value after the flip */
  int64_t kfirst;   /* first product the flipped accumulator holds: 0, or the
                       start of its k-split when the call split K */
  int64_t problem;  /* batched calls: the problem the fault was injected in */
} ftgemm_flip_log;

/* Fault-tolerant DGEMM (abstract; §2.2).  Encodes, verifies, locates and
 * corrects per FTGEMM_BM x FTGEMM_BN tile; rep may be NULL. */
int ftgemm_d(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
             const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
             double *C, int64_t ldc, ftgemm_report *rep, void *stream);

/* The same DGEMM with the fault tolerance compiled out: the same tiles,
 * pipeline and epilogue without checksums, verification or injection (the
 * baseline the ABFT overhead is measured against, §3.1 "FT-GEMM: Ori"). */
int ftgemm_d_noft(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                  const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                  double *C, int64_t ldc, void *stream);

/* ftgemm_d for callers that cannot allocate device memory.  (The paper has no
 * counterpart: it is an interface for this library's users.)
 *
 * Who needs it: callers whose device memory is owned and budgeted by their own
 * pool allocator (a framework's caching allocator, an inference server with a
 * fixed memory plan), which must not see a foreign cudaMalloc; callers that
 * cannot afford the device-wide synchronisation that cudaMalloc/cudaFree
 * imply in a latency-critical loop; and callers recovering from an
 * out-of-memory error, where any new allocation may fail.  ftgemm_d grows a
 * workspace with cudaMalloc on first use and when a problem is larger.
 *
 * This entry point calls no cudaMalloc, cudaFree or other allocating routine.
 * Its scratch is one static device array of FTGEMM_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that every GPU which loads the library holds until the process
 * exits.  The caller still owns A, B and C (device pointers) and the report.
 *  - Limit: the scratch needed is about 8 * (ceil(M/128) + ceil(N/128)) *
 *    ceil(K/16)*16 bytes of checksum vectors plus 8 * ceil(K/256) *
 *    max(M, N) bytes of partial sums plus small terms; a problem that needs
 *    more returns FTGEMM_ERR_SCRATCH and touches nothing (M = N = K = 8192
 *    needs about 10.5 MiB; 16384^3 does not fit).
 *  - A, B and C must be 16-byte aligned with even leading dimensions (no
 *    aligned copies can be made without memory): FTGEMM_ERR_UNALIGNED
 *    otherwise.
 *  - No fault injection (the injection table needs allocated memory); at
 *    most 1024 location records per call.
 *  - The first call on each device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *    The address is kept for the life of the process: a cudaDeviceReset
 *    between calls is not supported (the kept address would be stale).
 *  - With rep != NULL the call waits for its stream to read the report back;
 *    on a stream that is being captured it returns FTGEMM_ERR_CAPTURE before
 *    enqueueing anything.  With rep == NULL it does not wait, so it cannot
 *    return FTGEMM_ERR_TIMEOUT either: a pipeline wait that expired on the
 *    device shows only in a report.
 *  - Every call shares the one array and it keeps the last call's contents;
 *    the call clears what must start at zero.  Calls that overlap on the GPU
 *    (different streams, threads or processes' graphs) race on it.
 * Same kernels as ftgemm_d, always on whole tiles: where ftgemm_d splits K
 * (grids of few tiles) the two sum in different orders and agree within the
 * parity bound; elsewhere their results are equal.  Returns as ftgemm_d does. */
int ftgemm_d_noalloc(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                     const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                     double *C, int64_t ldc, ftgemm_report *rep, void *stream);

/* The unfused ablation: the same ABFT scheme and result as ftgemm_d, but
 * computed in separate passes, as FT-GEMM's unfused baseline (§2.2: fusing
 * the memory-bound checksum work into the GEMM took the ABFT overhead from
 * about 15% to 2.94% on Cascade Lake): the operand checksum pass; one pass
 * over C that copies it and takes its tile row/column sums; two skinny GEMMs
 * for the predicted checksums; the unprotected GEMM; a verify / locate /
 * correct pass over the finished C.  For measuring what fusion saves on
 * GB300.  Operands must be 16-byte aligned with even leading dimensions
 * (FTGEMM_ERR_UNALIGNED otherwise); fault injection does not apply. */
int ftgemm_d_unfused(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                     const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                     double *C, int64_t ldc, ftgemm_report *rep, void *stream);

/* Batched FT-DGEMM: `count` independent problems (arrays of per-problem
 * arguments on the host; matrix pointers are device pointers) computed by one
 * persistent kernel per operand layout present (one for an all-'N' batch):
 * one CTA per SM takes (problem, tile) work items from a global counter, in
 * an order fixed by the schedule.  Each problem gets its own report
 * (reps[p], cap/loc set by the caller; up to 64 locations per problem).
 * Argument errors return -(100*p + i) for argument i of problem p, numbered
 * as in ftgemm_d (so -(100*p + 8) is a bad lda); count < 0 or a NULL array
 * (count > 0) returns FTGEMM_ERR_BATCH; all of these are found before any
 * device work.  Operands must be 16-byte aligned with even leading
 * dimensions (FTGEMM_ERR_UNALIGNED).
 * Injection (the process-global setting): mode 1 draws `count` faults over
 * the batch, fault f taking splitmix64 outputs 5f..5f+4 as (problem mod count,
 * row, col, kstep, bit) of that problem; mode 2 uses ftgemm_flip.problem.
 * ftgemm_batched = plan create + launch + report + destroy. */
int ftgemm_batched(int64_t count, const char *transA, const char *transB, const int64_t *M,
                   const int64_t *N, const int64_t *K, const double *alpha,
                   const double *const *A, const int64_t *lda, const double *const *B,
                   const int64_t *ldb, const double *beta, double *const *C, const int64_t *ldc,
                   ftgemm_report *reps, void *stream);

/* A batch prepared once and launched many times: plan_create validates the
 * problems, builds their TMA descriptors, checksum-pass work lists, work
 * order and injection table in device memory owned by the plan, and captures
 * one CUDA graph (counter reset, batched checksum pass, persistent kernels).
 * ft = 0 builds the same batch without fault tolerance (overhead baseline).
 * schedule: -1 default; otherwise (order) | (log2(chunk) << 4) with order
 * 0 = problem order, 1 = tiles with the longest K first, 2 = round robin
 * over problems, and chunk = work items taken per counter access (1, 2, 4,
 * 8) -- the knob the autotuner searches.  plan_launch enqueues the graph on a
 * stream; plan_report waits for that stream and fills reps (may be NULL);
 * the matrices must stay valid while the plan lives. */
typedef struct ftgemm_batched_plan_s *ftgemm_batched_plan;
int ftgemm_batched_plan_create(ftgemm_batched_plan *plan, int64_t count, const char *transA,
                               const char *transB, const int64_t *M, const int64_t *N,
                               const int64_t *K, const double *alpha, const double *const *A,
                               const int64_t *lda, const double *const *B, const int64_t *ldb,
                               const double *beta, double *const *C, const int64_t *ldc, int ft,
                               int schedule, void *stream);
int ftgemm_batched_plan_launch(ftgemm_batched_plan plan, void *stream);
int ftgemm_batched_plan_report(ftgemm_batched_plan plan, ftgemm_report *reps, void *stream);
int64_t ftgemm_batched_plan_injection_log(ftgemm_batched_plan plan, ftgemm_flip_log *out, int64_t cap);
int ftgemm_batched_plan_destroy(ftgemm_batched_plan plan);

/* Split-precision FT-GEMM on the BF16 tensor cores (FP32 accumulation):
 *  - nslices = 0: the plain BF16 form: op(A) and op(B) rounded to bf16, FP32
 *    accumulation over K, out = alpha * acc + beta * C in FP64;
 *  - nslices = S in 1..15: FP64 emulated by error-free splitting (Ozaki,
 *    Ogita, Oishi, Rump 2012): every row of op(A) and column of op(B) is
 *    scaled by a power of two and split into S integer slices of w bits
 *    (w = 8, 7, 6, 5 for K <= 256, 1024, 4096, larger: the FP32 accumulation
 *    of a slice pair stays exact over the chunk of K it covers); the
 *    S(S+1)/2 slice pairs with s + t < S are bf16 tensor-core products folded
 *    into FP64 with their power-of-two weights.  S = 11 (w = 5) keeps about
 *    55 bits of every row's largest element; entries far smaller than their
 *    row's (column's) largest keep fewer bits.
 * ft = 1: checksums carried in FP32, reference sums, verification and
 * correction in FP64.  Emulated forms (mma.sync kernel): predicted checksums
 * summed in FP32 from the staged slices, flagged elements recomputed from the
 * original FP64 operands.  Plain form: on the tcgen05 engines the predicted
 * checksums are tensor-core products of the FP32 checksum vectors of the bf16
 * operands (each split into two bf16 pieces), on the mma.sync engine they are
 * summed from the staged slices; flagged elements are recomputed in FP64
 * from the same bf16 operands (the form's own value without its FP32
 * accumulation error), and an element counts as detected when it differs from
 * that by more than the FP32 accumulation bound (K + 16) 2^-22 sum_k |a~||b~|.
 * ft = 2 (emulated forms only): FP64 predicted checksums from the original
 * operands (operand checksum pass + two skinny products before the kernel),
 * verified against the scaled result with the FP64 threshold plus the
 * splitting bound -- far more sensitive than FP32 checksums; ft = 0 compiles
 * the checks out (overhead baseline).  Injection
 * (ftgemm_set_injection) flips bits of the FP64 accumulator after the slice
 * pair numbered `kstep` has been folded in (kstep < number of pairs; the
 * plain form has one pair, and the flip applies to the FP64 value of its FP32
 * accumulator).
 * Returns -14 for an invalid nslices, -15 for an invalid ft (0, 1 or 2;
 * ft = 2 needs nslices >= 1), FTGEMM_ERR_TOO_LARGE when M or N exceeds
 * FTGEMM_SPLIT_MAX_ROWS (before any device work), FTGEMM_ERR_UNALIGNED when
 * ft = 2 and an operand is not 16-byte aligned or has an odd leading
 * dimension. */
int ftgemm_d_split(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                   const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                   double *C, int64_t ldc, int nslices, int ft, ftgemm_report *rep, void *stream);

/* ftgemm_d on HOST matrices: copies A, B (and C unless beta == 0) to device
 * workspace, runs ftgemm_d, copies the M x N result back (rows M..ldc-1 of C
 * are left as they were), and waits for the stream.  Pinned host memory
 * makes the copies fastest; pageable memory also works.
 * Large problems run in column panels so that the copies overlap the
 * compute: op(A) goes up first, then each panel's columns of op(B) and C on
 * a copy stream; each panel's FT-DGEMM starts as soon as its columns have
 * landed, and its result goes back on a second copy stream while the next
 * panel computes.  The results equal those of ftgemm_d (output tiles are
 * independent); injected faults are drawn or listed over the whole M x N
 * problem as for ftgemm_d and the report and injection log cover the whole
 * call.  ftgemm_set_host_panels chooses the number of panels. */
int ftgemm_d_host(char transA, char transB, int64_t M, int64_t N, int64_t K, double alpha,
                  const double *A, int64_t lda, const double *B, int64_t ldb, double beta,
                  double *C, int64_t ldc, ftgemm_report *rep, void *stream);

/* The operand checksum pass on its own (the A and B checksum vectors of
 * §2.2/§2.3 per FTGEMM_BM-row / FTGEMM_BN-column tile, and the absolute sums
 * the detection threshold uses).  All outputs are device arrays owned by the
 * caller: acs (ceil(M/BM) x K, row stride K), aabsmax (ceil(M/BM)), arowabs
 * (M), bcs (ceil(N/BN) x K, row stride K), babsmax (ceil(N/BN)), bcolabs (N):
 *   acs[I*K+k] = sum_{i in I} op(A)(i,k),   aabsmax[I] = max_k sum_{i in I} |op(A)(i,k)|,
 *   arowabs[i] = sum_k |op(A)(i,k)|,        and symmetrically for op(B).
 * Returns 0, -i for a bad argument i (this function's numbering: lda is 7,
 * ldb is 9), or a positive FTGEMM_ERR_* code; M, N or K = 0 does nothing. */
int ftgemm_encode_operands(char transA, char transB, int64_t M, int64_t N, int64_t K,
                           const double *A, int64_t lda, const double *B, int64_t ldb,
                           double *acs, double *aabsmax, double *arowabs, double *bcs,
                           double *babsmax, double *bcolabs, void *stream);

/* Set (cfg != NULL) or clear (cfg == NULL or mode 0) fault injection. */
int ftgemm_set_injection(const ftgemm_inject *cfg);

/* Copy up to cap records of the last injected call's faults, in the order
 * they were drawn or listed, into out; returns the number of faults of that
 * call (or a negative value if out is NULL while cap > 0).  Waits for the
 * device. */
int64_t ftgemm_injection_log(ftgemm_flip_log *out, int64_t cap);

/* Test hook for the bounded waits: launches one block that waits on an
 * mbarrier nothing ever completes, with a limit of limit_ns nanoseconds.
 * Returns FTGEMM_ERR_TIMEOUT when the wait gave up and the context is still
 * usable (the expected result), another code otherwise. */
int ftgemm_selftest_wait_timeout(int64_t limit_ns, void *stream);

/* K splitting (a tuning knob; results stay within the same bound): 0 picks
 * the number of k-splits automatically (the default: grids with fewer than
 * 4 tiles per SM split K so that every SM gets work; larger grids whose last
 * wave is partly empty run their full waves whole and split K of the tail
 * tiles over the idle SMs; a reduction kernel sums the partial tiles and runs
 * the verification on the whole tile), 1 never splits, n >= 2 forces n
 * splits of every tile (fewer when K is short).  ftgemm_d_noalloc never
 * splits; with per-k-panel verification (ftgemm_set_panel_check) each k-split
 * checks the panels of its own k-range. */
int ftgemm_set_splitk(int nsplit);

/* Column panels of ftgemm_d_host: 0 (default) picks them automatically (up to
 * 8, each at least four waves of 128 x 128 tiles on the GPU; one panel, i.e.
 * no overlap, for smaller problems), n >= 1 uses n panels (at most one per
 * 128 columns).  Process-global; returns -1 for a negative value. */
int ftgemm_set_host_panels(int panels);

/* The K split that ftgemm_d (and ftgemm_d_host) would use for an M x N x K
 * problem on a GPU with nsm SMs under the current settings (host only, no
 * device work): *splits k-ranges (1: none) for the tiles from
 * *first_split_tile on, in the kernels' tile order; the tiles before it run
 * whole (*first_split_tile = 0: every tile split; = the tile count: none).
 * ftgemm_d_noft plans the same way.  Returns 0, or -i for a bad argument i
 * (M, N, K < 0, nsm <= 0, NULL outputs). */
int ftgemm_query_ksplit(int64_t M, int64_t N, int64_t K, int nsm, int *splits,
                        int64_t *first_split_tile);

/* Engine of ftgemm_d_split (results: the same bits for the emulated forms
 * on every engine, and for the plain BF16 form on the tcgen05 engines).
 * The tcgen05 engines run the slice products on the 5th-generation tensor
 * cores with the FP32 accumulators and the FP64 fold in tensor memory, when
 * ft is 0 or 2:
 *   2: one CTA per 128 x 128 tile;
 *   5: persistent, one CTA per SM walking its tiles, each tile finished
 *      from tensor memory while the next one's loads and MMAs run;
 *   0 (default): engine 5.
 * 1: every call on the mma.sync kernel.  The emulated forms with ft = 1 (FP32
 * checksums summed from the staged slices on the CUDA cores) always run on
 * the mma.sync kernel; the plain form with ft = 1 runs on the engine chosen.
 * 7: the emulated forms with INT8 slices on the mma.sync kernel (m16n8k32 s8
 *    MMAs; 7 bits per slice, exact INT32 sums over up to 133 120 products;
 *    ft 0 or 2, ft = 1 returns -15); a row of op(A) or column of op(B) that
 *    holds Inf or NaN is multiplied in FP64 instead (INT8 cannot carry it);
 *    the plain form runs as on engine 1.
 * Every CTA loads its own operand tiles (no thread-block clusters, no TMA
 * multicast).  Process-global; returns -1 for another value. */
int ftgemm_set_split_engine(int engine);

/* Per-k-panel verification (FT-BLAS style; FT-GEMM blocks K by K_C, §2.1):
 * kslabs > 0 makes later ftgemm_d calls also verify every tile's
 * accumulators after every kslabs k-slabs (kslabs * 16 products) against the
 * predicted checksums of the products done so far, correcting a located
 * accumulator in place, so that faults arriving at different times stay
 * separable and are caught before they spread through the remaining sum.
 * The end-of-tile verification still runs.  0 (default) turns it off.  In a
 * call that splits K (grids of few tiles, ftgemm_set_splitk) each k-split
 * checks every kslabs k-slabs of its own k-range. */
int ftgemm_set_panel_check(int kslabs);

/* Correction rule of the FP64 FT-GEMM kernels (ftgemm_d and the calls built
 * on the same kernels): 0 (default) recomputes every located element from
 * the original operands (exact to the element's rounding bound, robust to
 * Inf / NaN faults); 1 is FT-BLAS's rule, kept for comparison: when exactly
 * one row and one column of a tile are flagged, their intersection is
 * corrected by subtracting the column's checksum residual (reference minus
 * predicted column sum), which costs no recomputation but carries the
 * rounding of the 128-term sums and cancels badly for huge faults; a
 * non-finite residual, several faults in a tile, or a corrected row / column
 * that still fails its check fall back to recomputation.  Returns -1 for
 * another value.  The split-precision path always recomputes. */
int ftgemm_set_correction(int mode);

/* Number of kernels this library has launched in this process. */
int64_t ftgemm_launch_count(void);

/* Event timing of the library's own kernels, for benchmarks: enable != 0
 * starts recording CUDA events on the launching stream around every later
 * main GEMM kernel and around the work before it (operand checksum pass,
 * report reset, injection upload); any call clears what was recorded. */
int ftgemm_timing(int enable);

/* Wait for the recorded events and return the summed main-kernel time, the
 * number of main-kernel launches timed, and the summed time of the work
 * before each launch (milliseconds; any pointer may be NULL). */
int ftgemm_timing_read(double *main_ms, int64_t *main_launches, double *aux_ms);

/* Static description of an error code. */
const char *ftgemm_strerror(int code);

/* Release the workspace of the current device. */
int ftgemm_finalize(void);

#ifdef __cplusplus
}
#endif

#endif /* FTGEMM_H */
