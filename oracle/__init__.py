"""FT-DGEMM oracle: plain CPU statement of FT-GEMM's fault-tolerant DGEMM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs (the ``cpu_baseline`` sample, the reference arm, and
the sampled-row accuracy checks of its optional ``--split`` / ``--config5``
reports, outside any timed region) may import this package.  The GPU library
(``paper_2305_02444_gb300``) shares no code with it and never imports it.

The arithmetic lives in ``ftgemm_oracle.c`` (compiled with contraction off so
every operation rounds once); this module only marshals numpy arrays.  Each
function cites the passage it follows:

* ``gemm``             -- C = alpha*op(A)*op(B) + beta*C  (abstract, §2.1), plus
                          the bound matrix E = |alpha||A||B| + |beta||C|.
* ``pred_checksums``   -- Huang-Abraham column/row checksum invariants (§2.2).
* ``encode_operands``  -- per-tile A and B checksum vectors (§2.2, §2.3).
* ``ft_gemm``          -- the whole encode / verify / locate / correct scheme
                          with source-level fault injection (§2.2, §3.2).
* ``partial``          -- the accumulator value after the first kend products.
* ``random_flips``     -- the seeded fault list (splitmix64, counter based).
* ``split``            -- the split-precision form (module ``split.py``,
                          numpy and Python integers): the BF16-slice
                          emulation of the product evaluated exactly
                          (``split_gemm``) and the plain BF16 form
                          (``bf16_round``, ``bf16_gemm``).

The paper prints no worked example and no numeric output to compare with,
so every function is pinned by what the mathematics fixes: closed forms,
exact rational arithmetic, integer-exact cases, the checksum invariants and
brute force on tiny inputs (``tests/test_oracle.py``,
``tests/test_oracle_split.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ftgemm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)
_pi64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-shared",
           "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Counts(ctypes.Structure):
    _fields_ = [("detected", _i64), ("corrected", _i64), ("checksum_only", _i64),
                ("unverifiable", _i64), ("flagged_rows", _i64), ("flagged_cols", _i64),
                ("recomputed", _i64)]


class Loc(ctypes.Structure):
    _fields_ = [("row", _i64), ("col", _i64), ("tile", ctypes.c_int32),
                ("kind", ctypes.c_int32), ("delta", _dbl)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        c = ctypes.c_char
        _lib.orc_gemm.argtypes = [c, c, _i64, _i64, _i64, _dbl, _pd, _i64, _pd, _i64, _dbl,
                                  _pd, _i64, _pd, _i64, ctypes.c_int]
        _lib.orc_gemm.restype = ctypes.c_int
        _lib.orc_partial.argtypes = [c, c, _i64, _i64, _i64, _pd, _i64, _pd, _i64]
        _lib.orc_partial.restype = _dbl
        _lib.orc_pred_checksums.argtypes = [c, c, _i64, _i64, _i64, _dbl, _pd, _i64, _pd, _i64,
                                            _dbl, _pd, _i64, _pd, _pd]
        _lib.orc_pred_checksums.restype = ctypes.c_int
        _lib.orc_encode_operands.argtypes = [c, c, _i64, _i64, _i64, _pd, _i64, _pd, _i64,
                                             _i64, _i64, _pd, _pd, _pd, _pd, _pd, _pd]
        _lib.orc_encode_operands.restype = ctypes.c_int
        _lib.orc_tau.argtypes = [_i64, _i64, _dbl, _dbl, _dbl, _dbl, _dbl]
        _lib.orc_tau.restype = _dbl
        _lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib.orc_splitmix64.restype = ctypes.c_uint64
        _lib.orc_random_flips.argtypes = [ctypes.c_uint64, _i64, _i64, _i64, _i64, _pi64]
        _lib.orc_random_flips.restype = None
        _lib.orc_ft_gemm.argtypes = [c, c, _i64, _i64, _i64, _dbl, _pd, _i64, _pd, _i64, _dbl,
                                     _pd, _i64, _i64, _i64, _i64, _pi64, _i64, _pd, _pd,
                                     ctypes.POINTER(Counts), ctypes.POINTER(Loc), _i64, _pi64,
                                     ctypes.c_int]
        _lib.orc_ft_gemm.restype = ctypes.c_int
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_pd)


def _colmajor(x: np.ndarray) -> np.ndarray:
    """A float64 Fortran-ordered copy (column-major storage, ld = rows)."""
    return np.asfortranarray(np.asarray(x, dtype=np.float64))


def _ld(x: np.ndarray) -> int:
    """Leading dimension of a Fortran-ordered 2-D float64 array."""
    assert x.flags.f_contiguous or x.ndim == 2
    return max(1, x.shape[0]) if x.flags.f_contiguous else x.strides[1] // 8


def _t(c: str) -> bytes:
    return c.encode()


def gemm(ta: str, tb: str, alpha: float, A: np.ndarray, B: np.ndarray, beta: float,
         C: np.ndarray, want_E: bool = False, nthreads: int = 0, k: int | None = None):
    """Return (C_out, E or None): C_out = alpha*op(A)*op(B) + beta*C (§2.1).

    A, B, C are 2-D arrays holding the stored (not transposed) matrices; they
    are copied to column-major.  E(i,j) = |alpha| sum_k |op(A)_ik||op(B)_kj|
    + |beta||C_ij|, the componentwise bound the parity rule scales.
    """
    A = _colmajor(A); B = _colmajor(B); C = _colmajor(C).copy(order="F")
    M, N = C.shape
    K = (A.shape[1] if ta.upper() == "N" else A.shape[0]) if k is None else k
    E = np.zeros((M, N), dtype=np.float64, order="F") if want_E else None
    rc = lib().orc_gemm(_t(ta), _t(tb), M, N, K, alpha, _p(A), _ld(A), _p(B), _ld(B), beta,
                        _p(C), _ld(C), _p(E), max(1, M), nthreads)
    if rc != 0:
        raise ValueError(f"orc_gemm argument {-rc} invalid")
    return C, E


def gemm_raw(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, E=None, lde=1, nthreads=0):
    """orc_gemm on raw Fortran buffers (1-D float64 arrays); returns the BLAS info code."""
    return lib().orc_gemm(_t(ta), _t(tb), M, N, K, alpha, _p(A), lda, _p(B), ldb, beta, _p(C),
                          ldc, _p(E), lde, nthreads)


def partial(ta: str, tb: str, i: int, j: int, kend: int, A: np.ndarray, B: np.ndarray) -> float:
    """Accumulator after its first kend products, ascending k."""
    A = _colmajor(A); B = _colmajor(B)
    return lib().orc_partial(_t(ta), _t(tb), i, j, kend, _p(A), _ld(A), _p(B), _ld(B))


def pred_checksums(ta, tb, alpha, A, B, beta, C, k=None):
    """(colpred, rowpred) = (alpha (e^T opA) opB + beta e^T C, alpha opA (opB e) + beta C e)."""
    A = _colmajor(A); B = _colmajor(B); C = _colmajor(C)
    M, N = C.shape
    K = (A.shape[1] if ta.upper() == "N" else A.shape[0]) if k is None else k
    col = np.zeros(N); row = np.zeros(M)
    rc = lib().orc_pred_checksums(_t(ta), _t(tb), M, N, K, alpha, _p(A), _ld(A), _p(B), _ld(B),
                                  beta, _p(C), _ld(C), _p(col), _p(row))
    if rc != 0:
        raise ValueError(f"orc_pred_checksums argument {-rc} invalid")
    return col, row


@dataclass
class Encoded:
    acs: np.ndarray       # (nI, K)  sum over tile rows of op(A)
    aabsmax: np.ndarray   # (nI,)    max_k sum over tile rows of |op(A)|
    arowabs: np.ndarray   # (M,)     sum_k |op(A)_ik|
    bcs: np.ndarray       # (nJ, K)  sum over tile columns of op(B)
    babsmax: np.ndarray   # (nJ,)
    bcolabs: np.ndarray   # (N,)


def encode_operands(ta, tb, M, N, K, A, B, BM, BN) -> Encoded:
    A = _colmajor(A); B = _colmajor(B)
    nI = -(-M // BM); nJ = -(-N // BN)
    e = Encoded(np.zeros((nI, K)), np.zeros(nI), np.zeros(M), np.zeros((nJ, K)), np.zeros(nJ),
                np.zeros(N))
    rc = lib().orc_encode_operands(_t(ta), _t(tb), M, N, K, _p(A), _ld(A), _p(B), _ld(B), BM, BN,
                                   _p(e.acs), _p(e.aabsmax), _p(e.arowabs), _p(e.bcs),
                                   _p(e.babsmax), _p(e.bcolabs))
    if rc != 0:
        raise ValueError(f"orc_encode_operands argument {-rc} invalid")
    return e


def tau(K, L, alpha, absrow, absmax, beta, abscsum) -> float:
    return lib().orc_tau(K, L, alpha, absrow, absmax, beta, abscsum)


def splitmix64(seed: int, n: int) -> int:
    return lib().orc_splitmix64(seed & (2**64 - 1), n)


def random_flips(seed: int, count: int, M: int, N: int, nksteps: int) -> np.ndarray:
    out = np.zeros((count, 4), dtype=np.int64)
    lib().orc_random_flips(seed & (2**64 - 1), count, M, N, nksteps,
                           out.ctypes.data_as(_pi64))
    return out


@dataclass
class FTResult:
    C: np.ndarray
    counts: dict
    locs: list
    n_loc: int
    before: np.ndarray
    after: np.ndarray


def ft_gemm(ta, tb, alpha, A, B, beta, C, BM=128, BN=128, BK=16, flips=None, cap=4096,
            nthreads=0, k=None) -> FTResult:
    """Fault-tolerant DGEMM on the CPU (§2.2) with source-level injection (§3.2)."""
    A = _colmajor(A); B = _colmajor(B); C = _colmajor(C).copy(order="F")
    M, N = C.shape
    K = (A.shape[1] if ta.upper() == "N" else A.shape[0]) if k is None else k
    fl = np.zeros((0, 4), dtype=np.int64) if flips is None else np.ascontiguousarray(flips, dtype=np.int64).reshape(-1, 4)
    nf = fl.shape[0]
    before = np.full(nf, np.nan); after = np.full(nf, np.nan)
    cnt = Counts()
    locs = (Loc * max(1, cap))()
    nloc = ctypes.c_int64(0)
    rc = lib().orc_ft_gemm(_t(ta), _t(tb), M, N, K, alpha, _p(A), _ld(A), _p(B), _ld(B), beta,
                           _p(C), _ld(C), BM, BN, BK, fl.ctypes.data_as(_pi64), nf, _p(before),
                           _p(after), ctypes.byref(cnt), locs, cap, ctypes.byref(nloc), nthreads)
    if rc != 0:
        raise ValueError(f"orc_ft_gemm argument {-rc} invalid")
    counts = {f: getattr(cnt, f) for f, _ in Counts._fields_}
    ll = [(locs[q].row, locs[q].col, locs[q].tile, locs[q].kind, locs[q].delta)
          for q in range(min(nloc.value, cap))]
    return FTResult(C, counts, sorted(ll), nloc.value, before, after)


U = 2.0 ** -53


def parity_tol(K: int, E: np.ndarray) -> np.ndarray:
    """Componentwise parity bound max(4K, 2K+6) * u * E (4Ku as the target
    states; for K < 3 the rigorous two-sided bound (2K+5)u is larger)."""
    return max(4 * K, 2 * K + 6) * U * E


from .split import bf16_gemm, bf16_round, row_exponents, slices, split_gemm, split_width  # noqa: E402
