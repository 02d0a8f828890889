"""Python binding of libftgemm (argument marshalling only).

Every function calls the C entry point of the same name declared in
include/ftgemm.h; all arithmetic runs in the CUDA kernels of the library.
Matrix arguments are device pointers given as torch CUDA tensors (their
data_ptr) or plain integers; the `_host` variant takes CPU tensors or numpy
arrays.  Streams are torch.cuda.Stream objects, raw cudaStream_t integers, or
None for torch's current stream.  There is no fallback: a missing library
raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libftgemm.so")

BM = BN = 128
KSTEP = 16
ERR_CUDA, ERR_TIMEOUT, ERR_NODEVICE, ERR_NOMEM, ERR_INJECT, ERR_TENSORMAP = 1, 2, 4, 5, 6, 7
ERR_SCRATCH, ERR_UNALIGNED, ERR_BATCH, ERR_TOO_LARGE, ERR_CAPTURE = 8, 9, 10, 11, 12
SPLIT_MAX_ROWS = 524280

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_vp = ctypes.c_void_p


class Loc(ctypes.Structure):
    _fields_ = [("row", _i64), ("col", _i64), ("tile", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("delta", _dbl)]


class Report(ctypes.Structure):
    _fields_ = [("detected", _i64), ("corrected", _i64), ("checksum_only", _i64),
                ("unverifiable", _i64), ("flagged_rows", _i64), ("flagged_cols", _i64),
                ("recomputed", _i64), ("panel_detected", _i64), ("n_loc", _i64), ("cap", _i64),
                ("loc", ctypes.POINTER(Loc))]


class Flip(ctypes.Structure):
    _fields_ = [("row", _i64), ("col", _i64), ("kstep", _i64), ("bit", ctypes.c_int32),
                ("problem", ctypes.c_int32)]


class Inject(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("pad", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("count", _i64), ("list", ctypes.POINTER(Flip)), ("n_list", _i64)]


class FlipLog(ctypes.Structure):
    _fields_ = [("row", _i64), ("col", _i64), ("kstep", _i64), ("bit", ctypes.c_int32),
                ("applied", ctypes.c_int32), ("before", _dbl), ("after", _dbl), ("kfirst", _i64),
                ("problem", _i64)]


_lib = None

_GEMM_ARGS = [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _dbl, _vp, _i64, _vp, _i64, _dbl, _vp, _i64]


def lib():
    """Load libftgemm.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first")
        L = ctypes.CDLL(LIB_PATH)
        L.ftgemm_d.argtypes = _GEMM_ARGS + [ctypes.POINTER(Report), _vp]
        L.ftgemm_d_noft.argtypes = _GEMM_ARGS + [_vp]
        L.ftgemm_d_host.argtypes = _GEMM_ARGS + [ctypes.POINTER(Report), _vp]
        L.ftgemm_d_noalloc.argtypes = _GEMM_ARGS + [ctypes.POINTER(Report), _vp]
        L.ftgemm_d_unfused.argtypes = _GEMM_ARGS + [ctypes.POINTER(Report), _vp]
        L.ftgemm_d_split.argtypes = _GEMM_ARGS + [ctypes.c_int, ctypes.c_int, ctypes.POINTER(Report), _vp]
        L.ftgemm_d_split.restype = ctypes.c_int
        L.ftgemm_encode_operands.argtypes = [ctypes.c_char, ctypes.c_char, _i64, _i64, _i64, _vp, _i64,
                                             _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.ftgemm_set_injection.argtypes = [ctypes.POINTER(Inject)]
        L.ftgemm_injection_log.argtypes = [ctypes.POINTER(FlipLog), _i64]
        L.ftgemm_injection_log.restype = _i64
        L.ftgemm_selftest_wait_timeout.argtypes = [_i64, _vp]
        L.ftgemm_launch_count.restype = _i64
        L.ftgemm_set_host_panels.argtypes = [ctypes.c_int]
        L.ftgemm_set_host_panels.restype = ctypes.c_int
        L.ftgemm_set_panel_check.argtypes = [ctypes.c_int]
        L.ftgemm_set_panel_check.restype = ctypes.c_int
        L.ftgemm_query_ksplit.argtypes = [_i64, _i64, _i64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(_i64)]
        L.ftgemm_query_ksplit.restype = ctypes.c_int
        L.ftgemm_set_splitk.argtypes = [ctypes.c_int]
        L.ftgemm_set_splitk.restype = ctypes.c_int
        L.ftgemm_set_correction.argtypes = [ctypes.c_int]
        L.ftgemm_set_correction.restype = ctypes.c_int
        L.ftgemm_set_split_engine.argtypes = [ctypes.c_int]
        L.ftgemm_set_split_engine.restype = ctypes.c_int
        L.ftgemm_timing.argtypes = [ctypes.c_int]
        L.ftgemm_timing.restype = ctypes.c_int
        L.ftgemm_timing_read.argtypes = [ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_dbl)]
        L.ftgemm_timing_read.restype = ctypes.c_int
        _pp = ctypes.POINTER(ctypes.c_void_p)
        _pc = ctypes.c_char_p
        _pi = ctypes.POINTER(_i64)
        _pd = ctypes.POINTER(_dbl)
        L.ftgemm_batched.argtypes = [_i64, _pc, _pc, _pi, _pi, _pi, _pd, _pp, _pi, _pp, _pi, _pd, _pp, _pi,
                                     ctypes.POINTER(Report), _vp]
        L.ftgemm_batched.restype = ctypes.c_int
        L.ftgemm_batched_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), _i64, _pc, _pc, _pi, _pi, _pi,
                                                 _pd, _pp, _pi, _pp, _pi, _pd, _pp, _pi, ctypes.c_int,
                                                 ctypes.c_int, _vp]
        L.ftgemm_batched_plan_create.restype = ctypes.c_int
        L.ftgemm_batched_plan_launch.argtypes = [ctypes.c_void_p, _vp]
        L.ftgemm_batched_plan_launch.restype = ctypes.c_int
        L.ftgemm_batched_plan_report.argtypes = [ctypes.c_void_p, ctypes.POINTER(Report), _vp]
        L.ftgemm_batched_plan_report.restype = ctypes.c_int
        L.ftgemm_batched_plan_injection_log.argtypes = [ctypes.c_void_p, ctypes.POINTER(FlipLog), _i64]
        L.ftgemm_batched_plan_injection_log.restype = _i64
        L.ftgemm_batched_plan_destroy.argtypes = [ctypes.c_void_p]
        L.ftgemm_batched_plan_destroy.restype = ctypes.c_int
        L.ftgemm_strerror.argtypes = [ctypes.c_int]
        L.ftgemm_strerror.restype = ctypes.c_char_p
        for f in ("ftgemm_d", "ftgemm_d_noft", "ftgemm_d_host", "ftgemm_d_noalloc", "ftgemm_d_unfused", "ftgemm_encode_operands",
                  "ftgemm_set_injection", "ftgemm_selftest_wait_timeout", "ftgemm_finalize"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(x, device: bool = True) -> int | None:
    """Address of a matrix argument: None, a raw pointer (int), a float64 torch
    tensor on the GPU (device arguments) or on the CPU (host arguments), or a
    float64 numpy array (host arguments).  A tensor on the wrong side or of
    another dtype raises instead of giving a kernel an address it cannot use."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if bool(x.is_cuda) != device:
            raise ValueError(f"expected a {'CUDA' if device else 'CPU'} tensor, got one on {x.device}")
        if str(x.dtype) != "torch.float64":
            raise ValueError(f"expected a float64 tensor, got {x.dtype}")
        return x.data_ptr()
    if hasattr(x, "ctypes") and hasattr(x, "dtype"):
        if device:
            raise ValueError("a numpy array is host memory; this argument is a device pointer")
        if str(x.dtype) != "float64":
            raise ValueError(f"expected a float64 array, got {x.dtype}")
        return x.ctypes.data
    raise TypeError(type(x))


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _report(cap: int):
    locs = (Loc * max(1, cap))()
    r = Report()
    r.cap = cap
    r.loc = ctypes.cast(locs, ctypes.POINTER(Loc))
    return r, locs


def _report_dict(r: Report, locs, cap: int) -> dict:
    d = {f: getattr(r, f) for f, _ in Report._fields_ if f not in ("cap", "loc")}
    d["locs"] = [(locs[q].row, locs[q].col, locs[q].tile, locs[q].kind, locs[q].delta)
                 for q in range(min(cap, r.n_loc))]
    return d


def _c(t: str) -> bytes:
    return t.encode() if isinstance(t, str) else t


def ftgemm_d(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, report=True,
             loc_cap=4096, stream=None):
    """Fault-tolerant DGEMM on device buffers; returns (rc, report dict or None)."""
    if report:
        r, locs = _report(loc_cap)
        rc = lib().ftgemm_d(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                            _ptr(C), ldc, ctypes.byref(r), _stream(stream))
        return rc, _report_dict(r, locs, loc_cap)
    rc = lib().ftgemm_d(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                        _ptr(C), ldc, None, _stream(stream))
    return rc, None


def ftgemm_d_noft(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """The same DGEMM without fault tolerance (overhead baseline); returns rc."""
    return lib().ftgemm_d_noft(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb,
                               beta, _ptr(C), ldc, _stream(stream))


def ftgemm_d_host(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, loc_cap=4096,
                  stream=None):
    """ftgemm_d on host buffers (copies in and out); returns (rc, report dict)."""
    r, locs = _report(loc_cap)
    rc = lib().ftgemm_d_host(_c(transA), _c(transB), M, N, K, alpha, _ptr(A, False), lda, _ptr(B, False), ldb,
                             beta, _ptr(C, False), ldc, ctypes.byref(r), _stream(stream))
    return rc, _report_dict(r, locs, loc_cap)


def ftgemm_d_unfused(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, report=True,
                     loc_cap=4096, stream=None):
    """The unfused ablation (separate checksum, GEMM and verify passes);
    returns (rc, report dict or None)."""
    if report:
        r, locs = _report(loc_cap)
        rc = lib().ftgemm_d_unfused(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb,
                                    beta, _ptr(C), ldc, ctypes.byref(r), _stream(stream))
        return rc, _report_dict(r, locs, loc_cap)
    rc = lib().ftgemm_d_unfused(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                                _ptr(C), ldc, None, _stream(stream))
    return rc, None


def ftgemm_d_split(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, nslices=11, ft=True,
                   report=True, loc_cap=4096, stream=None):
    """Split-precision FT-GEMM on the BF16 tensor cores (nslices 0: plain BF16;
    S >= 1: FP64 emulated with S slices; ft 0 none, 1/True FP32 checksums,
    2 FP64 checksums); returns (rc, report dict or None)."""
    if report:
        r, locs = _report(loc_cap)
        rc = lib().ftgemm_d_split(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                                  _ptr(C), ldc, nslices, int(ft), ctypes.byref(r), _stream(stream))
        return rc, _report_dict(r, locs, loc_cap)
    rc = lib().ftgemm_d_split(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                              _ptr(C), ldc, nslices, int(ft), None, _stream(stream))
    return rc, None


def ftgemm_d_noalloc(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, report=True,
                     loc_cap=1024, stream=None):
    """ftgemm_d without any device allocation (scratch in a static device
    array, see include/ftgemm.h); returns (rc, report dict or None)."""
    if report:
        r, locs = _report(loc_cap)
        rc = lib().ftgemm_d_noalloc(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb,
                                    beta, _ptr(C), ldc, ctypes.byref(r), _stream(stream))
        return rc, _report_dict(r, locs, loc_cap)
    rc = lib().ftgemm_d_noalloc(_c(transA), _c(transB), M, N, K, alpha, _ptr(A), lda, _ptr(B), ldb, beta,
                                _ptr(C), ldc, None, _stream(stream))
    return rc, None


def ftgemm_encode_operands(transA, transB, M, N, K, A, lda, B, ldb, acs, aabsmax, arowabs, bcs,
                           babsmax, bcolabs, stream=None):
    return lib().ftgemm_encode_operands(_c(transA), _c(transB), M, N, K, _ptr(A), lda, _ptr(B), ldb,
                                        _ptr(acs), _ptr(aabsmax), _ptr(arowabs), _ptr(bcs),
                                        _ptr(babsmax), _ptr(bcolabs), _stream(stream))


def ftgemm_set_injection(mode=0, seed=0, count=0, flips=None):
    """mode 0 off, 1 seeded random (count per call), 2 explicit list of
    (row, col, kstep, bit) or, for batched calls, (row, col, kstep, bit, problem)."""
    cfg = Inject()
    cfg.mode = mode
    cfg.seed = seed & (2 ** 64 - 1)
    cfg.count = count
    keep = None
    if mode == 2:
        fl = list(flips or [])
        keep = (Flip * max(1, len(fl)))()
        for q, f in enumerate(fl):
            keep[q].row, keep[q].col, keep[q].kstep, keep[q].bit = (int(x) for x in f[:4])
            keep[q].problem = int(f[4]) if len(f) > 4 else 0
        cfg.list = ctypes.cast(keep, ctypes.POINTER(Flip))
        cfg.n_list = len(fl)
    return lib().ftgemm_set_injection(ctypes.byref(cfg))


def ftgemm_injection_log():
    """Faults of the last injected call, in list/draw order, as dicts."""
    n = lib().ftgemm_injection_log(None, 0)
    if n <= 0:
        return []
    buf = (FlipLog * n)()
    lib().ftgemm_injection_log(buf, n)
    return [{f: getattr(buf[q], f) for f, _ in FlipLog._fields_} for q in range(n)]


def ftgemm_selftest_wait_timeout(limit_ns: int, stream=None) -> int:
    return lib().ftgemm_selftest_wait_timeout(limit_ns, _stream(stream))


def ftgemm_set_panel_check(kslabs: int) -> int:
    """Verify accumulators every kslabs k-slabs (0: only at the end of K)."""
    return lib().ftgemm_set_panel_check(kslabs)


def ftgemm_set_host_panels(panels: int) -> int:
    """ftgemm_d_host's column panels: 0 automatic, n >= 1 that many."""
    return lib().ftgemm_set_host_panels(panels)


def ftgemm_set_splitk(nsplit: int) -> int:
    """0 automatic k-splitting, 1 never, n >= 2 force n splits."""
    return lib().ftgemm_set_splitk(nsplit)


def ftgemm_set_correction(mode: int) -> int:
    """0 recompute located elements (default), 1 subtract the checksum residual."""
    return lib().ftgemm_set_correction(mode)


def ftgemm_set_split_engine(engine: int) -> int:
    """Split precision: 0 default (= 5), 1 mma.sync, 2 tcgen05 one CTA per tile, 5 persistent
    tcgen05, 7 mma.sync with INT8 slices (emulated forms; ft 0 or 2); other values return -1."""
    return lib().ftgemm_set_split_engine(engine)


def ftgemm_query_ksplit(M, N, K, nsm=152):
    """(rc, splits, first_split_tile): the K split ftgemm_d would use (host only)."""
    sp = ctypes.c_int(0)
    first = _i64(0)
    rc = lib().ftgemm_query_ksplit(M, N, K, nsm, ctypes.byref(sp), ctypes.byref(first))
    return rc, sp.value, first.value


def ftgemm_launch_count() -> int:
    return lib().ftgemm_launch_count()


def ftgemm_timing(enable: bool) -> int:
    return lib().ftgemm_timing(1 if enable else 0)


def ftgemm_timing_read():
    """(main-kernel ms summed, main launches, pre-launch work ms summed)."""
    m, a, n = _dbl(), _dbl(), _i64()
    rc = lib().ftgemm_timing_read(ctypes.byref(m), ctypes.byref(n), ctypes.byref(a))
    if rc:
        raise RuntimeError(ftgemm_strerror(rc))
    return m.value, n.value, a.value


def ftgemm_strerror(code: int) -> str:
    return lib().ftgemm_strerror(code).decode()


def ftgemm_finalize() -> int:
    return lib().ftgemm_finalize()


class _BatchArgs:
    """ctypes arrays for a list of problems (ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc)."""

    def __init__(self, problems):
        n = len(problems)
        self.n = n
        self.ta = ctypes.create_string_buffer(bytes("".join(p[0] for p in problems), "ascii"), max(1, n))
        self.tb = ctypes.create_string_buffer(bytes("".join(p[1] for p in problems), "ascii"), max(1, n))
        I64 = _i64 * max(1, n)
        D = _dbl * max(1, n)
        P = ctypes.c_void_p * max(1, n)
        self.M = I64(*[p[2] for p in problems]); self.N = I64(*[p[3] for p in problems])
        self.K = I64(*[p[4] for p in problems]); self.alpha = D(*[p[5] for p in problems])
        self.A = P(*[_ptr(p[6]) for p in problems]); self.lda = I64(*[p[7] for p in problems])
        self.B = P(*[_ptr(p[8]) for p in problems]); self.ldb = I64(*[p[9] for p in problems])
        self.beta = D(*[p[10] for p in problems])
        self.C = P(*[_ptr(p[11]) for p in problems]); self.ldc = I64(*[p[12] for p in problems])

    def args(self):
        c = ctypes.cast
        pp = ctypes.POINTER(ctypes.c_void_p)
        return (self.n, self.ta, self.tb, self.M, self.N, self.K, self.alpha, c(self.A, pp), self.lda,
                c(self.B, pp), self.ldb, self.beta, c(self.C, pp), self.ldc)


def _reports(n, cap):
    reps = (Report * max(1, n))()
    keep = []
    for q in range(n):
        locs = (Loc * max(1, cap))()
        keep.append(locs)
        reps[q].cap = cap
        reps[q].loc = ctypes.cast(locs, ctypes.POINTER(Loc))
    return reps, keep


def ftgemm_batched(problems, loc_cap=16, stream=None):
    """Batched FT-DGEMM; returns (rc, list of per-problem report dicts)."""
    a = _BatchArgs(problems)
    reps, keep = _reports(a.n, loc_cap)
    rc = lib().ftgemm_batched(*a.args(), reps, _stream(stream))
    return rc, [_report_dict(reps[q], keep[q], loc_cap) for q in range(a.n)]


class BatchedPlan:
    """A batch captured once into a CUDA graph (see ftgemm_batched_plan_create)."""

    def __init__(self, problems, ft=True, schedule=-1, stream=None):
        self._args = _BatchArgs(problems)
        self.n = self._args.n
        self.h = ctypes.c_void_p()
        rc = lib().ftgemm_batched_plan_create(ctypes.byref(self.h), *self._args.args(), 1 if ft else 0,
                                              schedule, _stream(stream))
        if rc:
            raise RuntimeError(f"ftgemm_batched_plan_create: {rc} {ftgemm_strerror(rc)}")

    def launch(self, stream=None):
        rc = lib().ftgemm_batched_plan_launch(self.h, _stream(stream))
        if rc:
            raise RuntimeError(f"ftgemm_batched_plan_launch: {ftgemm_strerror(rc)}")

    def report(self, loc_cap=16, stream=None):
        reps, keep = _reports(self.n, loc_cap)
        rc = lib().ftgemm_batched_plan_report(self.h, reps, _stream(stream))
        return rc, [_report_dict(reps[q], keep[q], loc_cap) for q in range(self.n)]

    def injection_log(self):
        n = lib().ftgemm_batched_plan_injection_log(self.h, None, 0)
        if n <= 0:
            return []
        buf = (FlipLog * n)()
        lib().ftgemm_batched_plan_injection_log(self.h, buf, n)
        return [{f: getattr(buf[q], f) for f, _ in FlipLog._fields_} for q in range(n)]

    def destroy(self):
        if self.h:
            lib().ftgemm_batched_plan_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
