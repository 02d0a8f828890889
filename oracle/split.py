"""Split-precision oracle: what the BF16-slice form of the DGEMM computes.

TEST INFRASTRUCTURE ONLY, under the same rule as the rest of ``oracle``: only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it.

The protected DGEMM (§2.1, §2.2) can run its products on the BF16 tensor
cores by emulating FP64 with the error-free splitting of Ozaki, Ogita, Oishi
and Rump (2012), in a fixed-point form.  This module states that form plainly
and evaluates it exactly, so a kernel can be compared with it element by
element (their difference is only the kernel's own FP64 roundings) instead of
with the FP64 product under the splitting bound:

* row exponent: e_r is the smallest integer with |x| < 2^e_r for every entry
  x of row r (0 for a row of zeros); rows of op(A), columns of op(B);
* slice width: w = 8, 7, 6, 5 bits for K <= 256, 1024, 4096 and above (the
  sum of a k-chunk's products of two w-bit integers is an exact FP32
  integer);
* slice s (0 <= s < S) of an entry x of row r:
      n_s(x) = sign(x) (floor(|x| 2^(w(s+1) - e_r)) mod 2^w),
  an integer with |n_s| < 2^w, so that
      x = 2^e_r (sum_s n_s 2^-w(s+1) + rest),   |rest| < 2^-wS;
* product: the slice pairs whose weight 2^-w(s+t+2) is at least 2^-w(S+1),
  i.e. s + t < S, the rest dropped:
      V_ij = 2^(e_i + f_j) sum_{s+t<S} 2^-w(s+t+2) sum_k n_s(a_ik) n_t(b_kj);
* result: alpha V + beta C, rounded once to FP64.

The plain BF16 form rounds every operand entry to bf16 (``bf16_round``:
8 significant bits, FP32's exponent range, nearest with ties to even) and
multiplies; ``bf16_gemm`` is the FP64 oracle on the rounded operands.

Every step before the final rounding is exact: slices come from power-of-two
scalings, floors and fmods of FP64 values; the pair sums are FP64 matrix
products of integers whose every partial sum stays below 2^53; the weighted
sum over pairs and the epilogue use Python integers.  Pinned in
``tests/test_oracle.py`` by closed forms (digit patterns of 1 - 2^-wS,
products of powers of two where the rule s + t < S decides each term), the
reconstruction of x from its slices within 2^(e-wS), the splitting error
bound against the FP64 oracle, and torch's float32 -> bfloat16 conversion.
"""
from __future__ import annotations

import numpy as np


def split_width(K: int) -> int:
    """Bits per slice for a contraction of length K."""
    return 8 if K <= 256 else 7 if K <= 1024 else 6 if K <= 4096 else 5


def row_exponents(X: np.ndarray) -> np.ndarray:
    """e_r for every row of X: the smallest integer with max_k |X_rk| < 2^e_r
    (0 for a row of zeros).  Operands must be finite."""
    X = np.asarray(X, dtype=np.float64)
    if not np.all(np.isfinite(X)):
        raise ValueError("the split oracle takes finite operands")
    m = np.abs(X).max(axis=1) if X.shape[1] else np.zeros(X.shape[0])
    return np.frexp(m)[1].astype(np.int64)        # m = f 2^e with 1/2 <= f < 1


def slices(X: np.ndarray, S: int, w: int, e: np.ndarray | None = None) -> np.ndarray:
    """(S, rows, cols) array of the slices n_s of every entry of X (integers
    held in FP64), with the row exponents e (computed when not given)."""
    X = np.asarray(X, dtype=np.float64)
    e = row_exponents(X) if e is None else np.asarray(e, dtype=np.int64)
    ax = np.abs(X)
    out = np.empty((S,) + X.shape)
    for s in range(S):
        # |x| 2^(w(s+1) - e_r) is exact (a power-of-two scaling below 2^w(s+1);
        # a result below the normal range is below 1 and floors to 0 anyway)
        y = np.floor(np.ldexp(ax, (w * (s + 1) - e)[:, None]))
        out[s] = np.copysign(np.fmod(y, 2.0 ** w), X)
    return out


def _op(X: np.ndarray, t: str) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    return X if t.upper() == "N" else X.T


def _dyadic(x: float) -> tuple[int, int]:
    """(m, p) with x = m 2^p exactly."""
    n, d = float(x).as_integer_ratio()
    return n, -(d.bit_length() - 1)


def _to_float(m: int, p: int) -> float:
    """m 2^p rounded once to FP64 (Python's int -> float conversion and int
    true division round to nearest, ties to even)."""
    return float(m << p) if p >= 0 else m / (1 << -p)


def split_product(opA: np.ndarray, opB: np.ndarray, S: int, w: int | None = None):
    """The emulated product as exact integers: (Nmat, P) with
    V_ij = Nmat[i, j] 2^P[i, j] (Nmat an object array of Python ints)."""
    opA = np.asarray(opA, dtype=np.float64)
    opB = np.asarray(opB, dtype=np.float64)
    M, K = opA.shape
    N = opB.shape[1]
    w = split_width(K) if w is None else w
    if K * S * (2 ** w - 1) ** 2 >= 2 ** 53:
        raise ValueError("pair sums would leave the exact FP64 integers")
    eA = row_exponents(opA)
    eB = row_exponents(opB.T)
    a = slices(opA, S, w, eA)                      # (S, M, K)
    b = slices(opB.T, S, w, eB)                    # (S, N, K)
    # Q_d = sum_{s+t=d} sum_k n_s(a_ik) n_t(b_kj): integers of magnitude below
    # K S 2^2w < 2^53, so every partial sum is exact in any order
    Nmat = np.zeros((M, N), dtype=object)
    for d in range(S):
        q = np.zeros((M, N))
        for s in range(d + 1):
            q += a[s] @ b[d - s].T
        # sum_d Q_d 2^-w(d+2) = (sum_d Q_d 2^w(S-1-d)) 2^-w(S+1)
        Nmat = Nmat + q.astype(np.int64).astype(object) * (1 << (w * (S - 1 - d)))
    P = eA[:, None] + eB[None, :] - w * (S + 1)
    return Nmat, P


def split_gemm(ta: str, tb: str, alpha: float, A: np.ndarray, B: np.ndarray, beta: float,
               C: np.ndarray, S: int, w: int | None = None) -> np.ndarray:
    """alpha V + beta C rounded once to FP64, V the emulated product of
    op(A) op(B) from S slices of w bits.  A, B, C are the stored matrices
    (2-D arrays indexed [row, col]); C is not read when beta == 0."""
    opA, opB = _op(A, ta), _op(B, tb)
    Nmat, P = split_product(opA, opB, S, w)
    M, N = Nmat.shape
    ma, pa = _dyadic(alpha)
    C = np.asarray(C, dtype=np.float64)
    out = np.empty((M, N))
    for i in range(M):
        for j in range(N):
            m1, p1 = ma * int(Nmat[i, j]), pa + int(P[i, j])
            if beta != 0.0:
                mb, pb = _dyadic(beta)
                mc, pc = _dyadic(C[i, j])
                m2, p2 = mb * mc, pb + pc
            else:
                m2, p2 = 0, p1
            p = min(p1, p2)
            out[i, j] = _to_float((m1 << (p1 - p)) + (m2 << (p2 - p)), p)
    return out


def bf16_round(X) -> np.ndarray:
    """Every entry rounded to bf16 (8 significant bits and FP32's exponent
    range: normal values from 2^-126, below it multiples of 2^-133), to
    nearest with ties to even; values that round to 2^128 or beyond become
    +-Inf; zeros, Inf and NaN stay."""
    X = np.asarray(X, dtype=np.float64)
    out = X.copy()
    sel = np.isfinite(X) & (X != 0)
    x = X[sel]
    e = np.frexp(x)[1]                              # x = f 2^e, 1/2 <= |f| < 1
    q = np.maximum(e - 8, -133)                     # the bf16 spacing at x
    v = np.ldexp(np.rint(np.ldexp(x, -q)), q)       # rint: nearest, ties to even
    out[sel] = np.where(np.abs(v) >= 2.0 ** 128, np.copysign(np.inf, x), v)
    return out


def bf16_gemm(ta: str, tb: str, alpha: float, A, B, beta: float, C, want_E: bool = False):
    """The plain BF16 form: the FP64 oracle on bf16-rounded operands,
    alpha bf16(op(A)) bf16(op(B)) + beta C, with its bound matrix E."""
    from . import gemm
    return gemm(ta, tb, alpha, bf16_round(A), bf16_round(B), beta, C, want_E=want_E)


# ---------------------------------------------------------------------------
# Fault tolerance of the plain BF16 form (checksums carried in FP32).
#
# The plain form sums exact products of bf16 values (8-bit significands, so
# every product is exact in FP32) in an FP32 accumulator.  How a tensor core
# adds within one instruction is not documented, so the bound below assumes
# only that the accumulation proceeds in blocks of n >= 2 inputs (the running
# sum and n - 1 or more products), each block aligned to its largest input
# with at least 24 bits kept, summed, and rounded or truncated once to FP32.
# One block then errs by at most (n + 2) 2^-23 times the sum of its inputs'
# magnitudes, and K products in blocks of n by at most
#     (K / n) (n + 2) 2^-23 sum_k |a_k b_k|  <=  2 K 2^-23 sum_k |a_k b_k|;
# plain recursive FP32 summation (n = 2, rounding to nearest) is within it.
# With 16 more products of slack for ragged blocks:
#     e32(K) = (K + 16) 2^-22.
#
# Checksums of one 128 x 128 tile (I, J), column j (rows symmetric):
#   reference  sum_{i in I} out_ij, out_ij = fl64(alpha v_ij + beta c_ij),
#              v_ij the FP32 accumulator;
#   predicted  alpha P1_Ij + beta cs_j, cs_j = fl32(sum_i fl32(c_ij)) (within
#              (L + 1) 2^-24 sum_i |c_ij|), P1_Ij = sum_k acs_I[k] b_kj with
#              acs_I[k] = fl32(sum_{i in I} a_ik) split into two bf16 pieces
#              (hi = bf16(acs), lo = bf16(acs - hi); |acs - hi - lo| <=
#              2^-16 |acs|), each piece's product accumulated in FP32 and
#              the two results added in FP64.
# With H >= sum_k sum_{i in I} |a_ik||b_kj| (the Hoelder bound
# max_k sum_{i in I} |a_ik| * sum_k |b_kj|) and L the rows of the tile:
#   |ref - alpha X| <= |alpha| e32 H                       (X the exact sums)
#   |P1 - X|        <= (1.02 e32 + 1.01 (L - 1) 2^-24 + 1.01 2^-16) H
# plus the FP64 roundings of the L-term sums and the epilogue, and an
# absolute term for FP32 results below the normal range.  A fault whose
# effect on the column sum exceeds tau_plain is seen by the check.
# ---------------------------------------------------------------------------

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def bf16_acc_bound(K: int) -> float:
    """e32(K): |fl32-accumulated sum of K exact products - exact sum| <=
    e32(K) * sum of the products' magnitudes, under the block model above."""
    return (K + 16) * 2.0 ** -22


def bf16_tau(K: int, L: int, alpha: float, gmax: float, vsum: float, beta: float, abscsum: float) -> float:
    """Detection threshold of one row or column checksum of a plain-BF16 tile.
    K: contraction length; L: the tile's rows (column check) or columns (row
    check); gmax: max_k of the tile group's absolute sums of the summed
    operand (max_k sum_{i in I} |a_ik| for a column check); vsum: the other
    operand's absolute sum along k for this column or row (sum_k |b_kj|), so
    that H = gmax * vsum bounds the absolute checksum; abscsum: sum of |C_in|
    over the same row/column segment.  The last terms cover FP32 results
    below the normal range: flushed products and checksum pieces that lose
    bits there (at most 2^-134 per piece entry, times |b_kj|)."""
    e32 = bf16_acc_bound(K)
    H = gmax * vsum
    fp32 = (abs(alpha) * H * (2.04 * e32 + 1.01 * (L + 1) * U32 + 1.01 * 2.0 ** -16)
            + abs(beta) * abscsum * 1.01 * (L + 1) * U32)
    fp64 = 2.01 * (L + 40) * U64 * (abs(alpha) * H * (1.0 + e32) + abs(beta) * abscsum)
    tiny = abs(alpha) * ((L + 2) * (K + 16) * 2.0 ** -124 + vsum * 2.0 ** -130) + (L + 40) * 2.0 ** -1021
    return fp32 + fp64 + tiny


def bf16_elem_tol(K: int, alpha: float, ab: float, beta: float, c: float) -> float:
    """Largest difference between the plain form's output element
    fl64(alpha v + beta c) and its FP64 recomputation from the bf16 operands
    fl64(alpha fl64(sum_k a_k b_k) + beta c), ab = sum_k |a_k b_k|."""
    e32 = bf16_acc_bound(K)
    return (abs(alpha) * ab * 1.01 * e32 + 2.01 * (K + 4) * U64 * (abs(alpha) * ab + abs(beta * c))
            + abs(alpha) * (K + 16) * 2.0 ** -124)


def bf16_pieces(x) -> tuple[np.ndarray, np.ndarray]:
    """The two bf16 pieces of FP32 values x: hi = bf16(x), lo = bf16(x - hi)
    (x - hi is exact in FP32)."""
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    hi = bf16_round(x)
    lo = bf16_round((x - hi).astype(np.float32).astype(np.float64))
    return hi, lo
