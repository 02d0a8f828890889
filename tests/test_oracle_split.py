"""Pins for the split-precision oracle (no GPU).

The splitting (Ozaki, Ogita, Oishi, Rump 2012, in fixed point) is pinned by
what the mathematics fixes, not by restating its formula:
  - closed forms: the base-2^w digits of 1 - 2^-53 and of powers of two, the
    all-(2^w - 1) digit pattern of 1 - 2^-wS whose product has a closed sum
    over the kept slice pairs, and products of powers of two where each term
    survives exactly when its two slice indices sum below S;
  - the digits reconstruct x truncated to wS bits below the row's exponent
    (a base-2^w expansion), so |x - sum| < 2^(e - wS);
  - the splitting error bound against the FP64 oracle, attained within a
    factor that a misplaced slice would break;
  - exact rational brute force on tiny inputs;
  - bf16 rounding against torch's float32 -> bfloat16 conversion (a library
    routine) and its halfway and overflow cases.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -53


def test_width_table(orc):
    """The width bands as stated (8, 7, 6, 5 bits up to K = 256, 1024, 4096,
    above), and for each the products of two w-bit integers over 64 k stay
    an exact FP32 integer sum (the k-slab a kernel accumulates at least)."""
    want = {1: 8, 256: 8, 257: 7, 1024: 7, 1025: 6, 4096: 6, 4097: 5, 10 ** 6: 5}
    for K, w in want.items():
        assert orc.split_width(K) == w
        assert 64 * (2 ** w - 1) ** 2 <= 2 ** 24


def test_row_exponents_closed_form(orc):
    X = np.array([[1.0, 0.5, -0.25],            # max exactly 2^0: e = 1 (|x| < 2^e strictly)
                  [1.0 - 2.0 ** -53, 0.0, 0.0],  # just below 1: e = 0
                  [0.0, 0.0, 0.0],               # zero row: e = 0
                  [3.0, -5.0, 7.9],              # max 7.9 < 8: e = 3
                  [-2.0 ** -1074, 0.0, 0.0],     # smallest subnormal: e = -1073
                  [2.0 ** 1023, 1.0, 0.0]])      # largest power of two: e = 1024
    np.testing.assert_array_equal(orc.row_exponents(X), [1, 0, 0, 3, -1073, 1024])
    with pytest.raises(ValueError):
        orc.row_exponents(np.array([[1.0, np.inf]]))


@pytest.mark.parametrize("w", [5, 6, 7, 8])
def test_digits_of_one_minus_ulp(orc, w):
    """1 - 2^-53 has 53 one bits below the point: slice s is all ones while
    w(s+1) <= 53, the slice that straddles bit 53 keeps its top bits, the rest
    are zero; the negated entry has the negated digits."""
    x = 1.0 - 2.0 ** -53
    S = 15
    d = orc.slices(np.array([[x, -x]]), S, w)
    for s in range(S):
        if w * (s + 1) <= 53:
            want = 2 ** w - 1
        elif w * s < 53:
            want = 2 ** w - 2 ** (w * (s + 1) - 53)
        else:
            want = 0
        assert d[s, 0, 0] == want and d[s, 0, 1] == -want, (w, s)


@pytest.mark.parametrize("w", [5, 8])
def test_digits_of_powers_of_two(orc, w):
    """2^p in a row whose largest entry is 2^q has its one bit at position
    b = q + 1 - p below the point of the scaled row: slice (b - 1) // w holds
    2^(w((b-1)//w + 1) - b), the others 0 (nothing when (b - 1) // w >= S)."""
    S = 4
    q = 3
    ps = list(range(q, q - w * S - 3, -1))
    row = np.array([[2.0 ** p for p in ps]])
    d = orc.slices(row, S, w)
    for c, p in enumerate(ps):
        b = q + 1 - p
        s0 = (b - 1) // w
        for s in range(S):
            want = 2 ** (w * (s + 1) - b) if s == s0 else 0
            assert d[s, 0, c] == want, (p, s)


@pytest.mark.parametrize("dist", ["uniform", "loguniform", "wide"])
@pytest.mark.parametrize("w,S", [(5, 3), (7, 2), (8, 7), (6, 11)])
def test_slices_reconstruct_truncation(orc, dist, w, S):
    """sum_s n_s 2^(e - w(s+1)) (exact, in fractions) is x truncated toward
    zero to a multiple of 2^(e - wS), every digit lies in (-2^w, 2^w) with
    the sign of x, and |x - sum| < 2^(e - wS)."""
    rng = np.random.default_rng(w * 100 + S)
    R, K = 4, 40
    if dist == "uniform":
        X = rng.uniform(-1, 1, (R, K))
    elif dist == "loguniform":
        X = rng.choice([-1.0, 1.0], (R, K)) * 10.0 ** rng.uniform(-3, 3, (R, K))
    else:
        X = rng.choice([-1.0, 1.0], (R, K)) * 2.0 ** rng.integers(-300, 300, (R, K)) * rng.uniform(1, 2, (R, K))
    X[1, 3] = 0.0
    e = orc.row_exponents(X)
    d = orc.slices(X, S, w)
    assert np.all(np.abs(d) < 2 ** w)
    assert np.all((d == 0) | (np.sign(d) == np.sign(X)[None]))
    for r in range(R):
        ulp = Fraction(2) ** (int(e[r]) - w * S)
        for k in range(K):
            x = Fraction(float(X[r, k]))
            tot = sum(Fraction(int(d[s, r, k])) * Fraction(2) ** (int(e[r]) - w * (s + 1)) for s in range(S))
            q = abs(x) / ulp
            trunc = (q.numerator // q.denominator) * ulp * (1 if x >= 0 else -1)
            assert tot == trunc
            assert abs(x - tot) < ulp


@pytest.mark.parametrize("K,S", [(3, 4), (256, 3), (300, 3), (1500, 2), (5000, 2)])
def test_all_max_digits_product_closed_form(orc, K, S):
    """Entries 1 - 2^-wS have every one of their S digits equal to 2^w - 1,
    so every pair sum is K (2^w - 1)^2 and the kept pairs s + t = d number
    d + 1: V = K (2^w - 1)^2 sum_{d<S} (d + 1) 2^-w(d+2), rounded once after
    alpha V + beta C."""
    w = orc.split_width(K)
    x = 1.0 - 2.0 ** (-w * S)
    M, N = 2, 3
    A = np.full((M, K), x)
    B = np.full((K, N), -x)
    C = np.full((M, N), 0.75)
    V = -K * (2 ** w - 1) ** 2 * sum(Fraction(d + 1, 2 ** (w * (d + 2))) for d in range(S))
    got = orc.split_gemm("N", "N", 1.5, A, B, 0.0, C, S)
    assert np.all(got == float(Fraction(3, 2) * V))
    got = orc.split_gemm("N", "N", 1.5, A, B, -0.25, C, S)
    assert np.all(got == float(Fraction(3, 2) * V - Fraction(3, 16)))
    # the dropped pairs (s + t >= S) are what separates V from the exact product
    exact = -K * Fraction(x) ** 2
    dropped = -K * (2 ** w - 1) ** 2 * sum(Fraction(1, 2 ** (w * (s + t + 2)))
                                           for s in range(S) for t in range(S) if s + t >= S)
    assert V == exact - dropped


@pytest.mark.parametrize("w,S", [(8, 3), (8, 1), (7, 2)])
def test_powers_of_two_product_pair_rule(orc, w, S):
    """With entries +-2^p every term a_ik b_kj is one digit product: it is kept
    exactly when the slice index of a_ik in its row plus that of b_kj in its
    column is below S, and then enters exactly.  Row (column) exponents
    follow from the largest power in the row (column)."""
    rng = np.random.default_rng(w + 10 * S)
    M, N, K = 5, 4, 24
    K = min(K, 256 if w == 8 else 1024)
    pa = rng.integers(-3 * w, 4, (M, K))
    pb = rng.integers(-3 * w, 4, (K, N))
    A = rng.choice([-1.0, 1.0], (M, K)) * np.ldexp(1.0, pa)
    B = rng.choice([-1.0, 1.0], (K, N)) * np.ldexp(1.0, pb)
    got = orc.split_gemm("N", "N", 1.0, A, B, 0.0, np.zeros((M, N)), S, w=w)
    kept_any = dropped_any = False
    for i in range(M):
        ea = int(pa[i].max()) + 1
        for j in range(N):
            eb = int(pb[:, j].max()) + 1
            tot = Fraction(0)
            for k in range(K):
                s = (ea - int(pa[i, k]) - 1) // w
                t = (eb - int(pb[k, j]) - 1) // w
                if s + t < S:
                    tot += Fraction(float(A[i, k])) * Fraction(float(B[k, j]))
                    kept_any = True
                else:
                    dropped_any = True
            assert got[i, j] == float(tot), (i, j)
    assert kept_any and dropped_any


def test_brute_force_tiny(orc):
    """Tiny random operands: the definition evaluated entry by entry in
    rational arithmetic (digits by integer floor division)."""
    rng = np.random.default_rng(5)
    for ta, tb, S in [("N", "N", 2), ("T", "N", 3), ("N", "T", 1), ("T", "T", 4)]:
        M, N, K = 3, 2, 5
        opA = rng.uniform(-4, 4, (M, K)) * 10.0 ** rng.integers(-2, 3, (M, K))
        opB = rng.uniform(-1, 1, (K, N))
        C = rng.uniform(-1, 1, (M, N))
        A = opA if ta == "N" else opA.T.copy()
        B = opB if tb == "N" else opB.T.copy()
        w = orc.split_width(K)

        def digits(x, e):
            a = abs(Fraction(float(x))) / Fraction(2) ** e
            sg = -1 if x < 0 else 1
            return [sg * ((a * 2 ** (w * (s + 1))).__floor__() % 2 ** w) for s in range(S)]

        def rexp(v):
            m = max(abs(float(t)) for t in v)
            e = 0
            if m == 0:
                return 0
            while Fraction(m) >= Fraction(2) ** e:
                e += 1
            while Fraction(m) < Fraction(2) ** (e - 1):
                e -= 1
            return e

        got = orc.split_gemm(ta, tb, -1.25, A, B, 0.5, C, S)
        for i in range(M):
            ei = rexp(opA[i])
            for j in range(N):
                fj = rexp(opB[:, j])
                V = Fraction(0)
                for k in range(K):
                    da, db = digits(opA[i, k], ei), digits(opB[k, j], fj)
                    for s in range(S):
                        for t in range(S - s):
                            V += Fraction(da[s] * db[t]) / Fraction(2) ** (w * (s + t + 2))
                V *= Fraction(2) ** (ei + fj)
                want = float(Fraction(-5, 4) * V + Fraction(1, 2) * Fraction(float(C[i, j])))
                assert got[i, j] == want


@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
def test_split_error_bound_against_fp64(orc, dist):
    """|split - FP64| stays within |alpha| 2^(e_i + f_j) K (S + 4) 2^-wS plus
    the FP64 parity bound, and reaches at least 1/(10 K) of the splitting
    part somewhere (a product kept one slice finer would sit 2^w lower)."""
    rng = np.random.default_rng(11)
    M, N, K = 12, 10, 50
    if dist == "uniform":
        opA = rng.uniform(-1, 1, (M, K)); opB = rng.uniform(-1, 1, (K, N))
    else:
        opA = rng.choice([-1.0, 1.0], (M, K)) * 10.0 ** rng.uniform(-3, 3, (M, K))
        opB = rng.choice([-1.0, 1.0], (K, N)) * 10.0 ** rng.uniform(-3, 3, (K, N))
    C = rng.uniform(-1, 1, (M, N))
    alpha, beta = 1.5, 0.5
    ref, E = orc.gemm("N", "N", alpha, opA, opB, beta, C, want_E=True)
    sa = np.ldexp(1.0, orc.row_exponents(opA))
    sb = np.ldexp(1.0, orc.row_exponents(opB.T))
    w = orc.split_width(K)
    for S in range(1, 8):
        got = orc.split_gemm("N", "N", alpha, opA, opB, beta, C, S)
        split = alpha * np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-w * S)
        err = np.abs(got - ref)
        assert np.all(err <= split + orc.parity_tol(K, E)), S
        if w * S <= 40:   # the splitting error well above FP64 rounding
            assert (err / split).max() > 1.0 / (10 * K), S


def test_bf16_round_matches_torch_float32_conversion(orc):
    """For FP32-exact inputs a single rounding to bf16 is what torch's
    float32 -> bfloat16 conversion does (nearest, ties to even): random FP32
    bit patterns over the whole range, subnormals and near-overflow values."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    bits[:1000] &= 0x807FFFFF                      # FP32 subnormals
    bits[1000:2000] = (bits[1000:2000] & 0x8000FFFF) | 0x7F7F0000   # near the largest bf16
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    want = torch.from_numpy(f.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = orc.bf16_round(f.astype(np.float64))
    np.testing.assert_array_equal(got, want)


def test_bf16_round_halfway_and_limits(orc):
    vals = [1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 255.5, 256.5, 2.0 ** -134,
            3 * 2.0 ** -134, (2 - 2.0 ** -8) * 2.0 ** 127, (2 - 2.0 ** -8 - 2.0 ** -40) * 2.0 ** 127,
            -1e300, 1e-300, 0.0, -0.0, math.inf, -math.inf]
    want = [1.0, 1 + 2.0 ** -6, -1.0, 256.0, 256.0, 0.0, 2.0 ** -132, math.inf,
            (2 - 2.0 ** -7) * 2.0 ** 127, -math.inf, 0.0, 0.0, -0.0, math.inf, -math.inf]
    got = orc.bf16_round(np.array(vals))
    np.testing.assert_array_equal(got, want)
    assert math.copysign(1.0, got[12]) == -1.0
    assert np.isnan(orc.bf16_round(np.array([math.nan])))[0]


def test_plain_form_is_exact_on_bf16_values(orc):
    """Operands already on the bf16 grid (8 significant bits) are not changed
    by the rounding: the plain form then equals the FP64 product."""
    rng = np.random.default_rng(21)
    A = rng.integers(-255, 256, (9, 13)) * 2.0 ** rng.integers(-20, 20, (9, 13))
    B = rng.integers(-255, 256, (13, 7)) * 2.0 ** rng.integers(-20, 20, (13, 7))
    C = rng.uniform(-1, 1, (9, 7))
    np.testing.assert_array_equal(orc.bf16_round(A), A)
    got, _ = orc.bf16_gemm("N", "N", 1.5, A, B, 0.5, C)
    ref, _ = orc.gemm("N", "N", 1.5, A, B, 0.5, C)
    np.testing.assert_array_equal(got, ref)


def test_split_beta_zero_never_reads_c(orc):
    rng = np.random.default_rng(22)
    A = rng.uniform(-1, 1, (4, 6)); B = rng.uniform(-1, 1, (6, 5))
    got = orc.split_gemm("N", "N", 1.0, A, B, 0.0, np.full((4, 5), np.nan), 3)
    assert np.all(np.isfinite(got))
    np.testing.assert_array_equal(got, orc.split_gemm("N", "N", 1.0, A, B, 0.0, np.zeros((4, 5)), 3))


@pytest.mark.parametrize("ta,tb", [("T", "N"), ("N", "T"), ("T", "T")])
def test_split_layouts_agree(orc, ta, tb):
    """op(X) = X^T for 'T': every layout gives the bits of the 'N','N'
    product of the transposed storage."""
    rng = np.random.default_rng(23)
    opA = rng.uniform(-1, 1, (7, 30)) * 10.0 ** rng.integers(-2, 3, (7, 30))
    opB = rng.uniform(-1, 1, (30, 5))
    C = rng.uniform(-1, 1, (7, 5))
    A = opA if ta == "N" else opA.T.copy()
    B = opB if tb == "N" else opB.T.copy()
    np.testing.assert_array_equal(orc.split_gemm(ta, tb, 1.25, A, B, -0.5, C, 4),
                                  orc.split_gemm("N", "N", 1.25, opA, opB, -0.5, C, 4))


# ---------------------------------------------------------------------------
# Fault tolerance of the plain BF16 form: the FP32 accumulation bound, the
# two-piece split of the checksum vectors and the detection threshold,
# pinned against models of an FP32 accumulator written here from their
# definitions (Python integers and fractions, or numpy float32 adds).

def _fp32_round_nearest(x: Fraction) -> Fraction:
    """x rounded to the nearest FP32 value (ties to even), normal range."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    q = Fraction(2) ** (e - 23)                   # the spacing of 24-bit significands at a
    n = a / q
    f = math.floor(n)
    r = n - f
    f = f + 1 if (r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1)) else f
    return s * f * q


def _exp_of(a: Fraction) -> int:
    e = math.floor(math.log2(a.numerator) - math.log2(a.denominator))
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    return e


def _trunc_block_sum(vals, n: int) -> Fraction:
    """A truncating fused accumulator: the running sum and the next n - 1
    products are aligned to the largest of them, each truncated toward zero
    to 24 bits below that largest exponent, summed exactly, and the block's
    result truncated toward zero to 24 significant bits."""
    acc = Fraction(0)
    vals = [Fraction(v) for v in vals]
    for b0 in range(0, len(vals), n - 1):
        block = [acc] + vals[b0:b0 + n - 1]
        m = max(abs(v) for v in block)
        if m == 0:
            continue
        q = Fraction(2) ** (_exp_of(m) - 23)
        s = sum((abs(v) // q) * q * (1 if v >= 0 else -1) for v in block)
        if s == 0:
            acc = Fraction(0)
            continue
        qs = Fraction(2) ** (_exp_of(abs(s)) - 23)
        acc = (abs(s) // qs) * qs * (1 if s >= 0 else -1)
    return acc


def _bf16_products(rng, K, kind):
    from oracle import split
    if kind == "positive":
        a, b = rng.random(K) + 0.5, rng.random(K) + 0.5
    elif kind == "loguniform":
        a = rng.choice([-1.0, 1.0], K) * 10.0 ** rng.uniform(-3, 3, K)
        b = rng.choice([-1.0, 1.0], K) * 10.0 ** rng.uniform(-3, 3, K)
    elif kind == "one_large":        # 1 first, then products just below one FP32 ulp of 1 (2^-23)
        a = np.full(K, 1.9921875); b = np.full(K, 2.0 ** -24)
        a[0], b[0] = 1.0, 1.0
    else:
        a, b = rng.uniform(-1, 1, K), rng.uniform(-1, 1, K)
    a, b = split.bf16_round(a), split.bf16_round(b)
    return a * b                                  # exact: two 8-bit significands


@pytest.mark.parametrize("kind", ["uniform", "positive", "loguniform", "one_large"])
@pytest.mark.parametrize("K", [16, 100, 1024])
def test_bf16_accumulation_bound_holds_for_fp32_accumulators(orc, kind, K):
    """e32(K) bounds the error of sequential round-to-nearest FP32 sums and
    of truncating fused blocks of 2, 4, 16 and 17 inputs; on the adversarial
    'one large product first' input the truncating accumulator reaches a
    fair share of the bound, so the bound is not loose by orders of
    magnitude."""
    from oracle import split
    rng = np.random.default_rng(K + len(kind))
    p = _bf16_products(rng, K, kind)
    exact = sum(Fraction(float(x)) for x in p)
    mag = float(np.abs(p).sum())
    e32 = split.bf16_acc_bound(K)
    seq = np.float32(0)
    for x in p.astype(np.float32):
        seq = np.float32(seq + x)
    worst = abs(float(Fraction(float(seq)) - exact)) / mag
    for n in (2, 4, 16, 17):
        worst = max(worst, abs(float(_trunc_block_sum(p, n) - exact)) / mag)
    assert worst <= e32, (worst, e32)
    if kind == "one_large" and K >= 100:
        assert worst >= 0.2 * e32, (worst, e32)


def test_bf16_pieces_remainder(orc):
    """FP32 = hi + lo + r with hi = bf16(x), lo = bf16(x - hi): |r| <= 2^-16
    |x| over random FP32 bit patterns of normal magnitude, with cases near
    the bound; hi + lo recovers every FP32 value with at most 16 significant
    bits exactly."""
    from oracle import split
    rng = np.random.default_rng(3)
    bits = rng.integers(0x0C000000, 0x72000000, 200000).astype(np.uint32)   # 2^-103 .. 2^101
    x = bits.view(np.float32).astype(np.float64) * rng.choice([-1.0, 1.0], 200000)
    hi, lo = split.bf16_pieces(x)
    r = np.abs(x - hi - lo)
    assert np.all(r <= 2.0 ** -16 * np.abs(x))
    assert r.max() / np.abs(x)[np.argmax(r / np.abs(x))] > 2.0 ** -18          # the bound is nearly reached
    short = (rng.integers(1 << 15, 1 << 16, 1000) * 2.0 ** rng.integers(-40, 40, 1000))
    hi, lo = split.bf16_pieces(short)
    np.testing.assert_array_equal(hi + lo, short)


def _simulate_plain_tile(rng, K, L, alpha, beta, kind, acc):
    """The plain form's column check of one L x L tile with the accumulator
    model `acc` (a function of a vector of exact products): returns the
    residuals |ref_j - pred_j| and the thresholds tau_j (bf16_tau)."""
    from oracle import split
    if kind == "loguniform":
        A = rng.choice([-1.0, 1.0], (L, K)) * 10.0 ** rng.uniform(-3, 3, (L, K))
        B = rng.choice([-1.0, 1.0], (K, L)) * 10.0 ** rng.uniform(-3, 3, (K, L))
    elif kind == "positive":
        A, B = rng.random((L, K)) + 0.5, rng.random((K, L)) + 0.5
    else:
        A, B = rng.uniform(-1, 1, (L, K)), rng.uniform(-1, 1, (K, L))
    C = rng.uniform(-1, 1, (L, L))
    a, b = split.bf16_round(A), split.bf16_round(B)
    V = np.array([[acc(a[i] * b[:, j]) for j in range(L)] for i in range(L)])   # FP32 accumulators
    out = alpha * V + beta * C                                                   # the epilogue, FP64
    ref = out.sum(axis=0)
    acs = np.zeros(K, dtype=np.float32)
    for i in range(L):                                                           # FP32 group sums
        acs = (acs + a[i].astype(np.float32)).astype(np.float32)
    hi, lo = split.bf16_pieces(acs)
    P1 = np.array([acc(hi * b[:, j]) + acc(lo * b[:, j]) for j in range(L)])
    cs = np.zeros(L, dtype=np.float32)
    for i in range(L):                                                           # FP32 sums of C
        cs = (cs + C[i].astype(np.float32)).astype(np.float32)
    pred = alpha * P1 + beta * cs.astype(np.float64)
    gmax = np.abs(a).sum(axis=0).max()
    tau = np.array([split.bf16_tau(K, L, alpha, gmax, np.abs(b[:, j]).sum(), beta, np.abs(C[:, j]).sum())
                    for j in range(L)])
    return np.abs(ref - pred), tau


def _acc_seq32(p):
    s = np.float32(0)
    for x in np.asarray(p, dtype=np.float32):
        s = np.float32(s + x)
    return float(s)


def _acc_trunc16(p):
    return float(_trunc_block_sum(p, 17))


@pytest.mark.parametrize("kind", ["uniform", "positive", "loguniform"])
@pytest.mark.parametrize("acc", [_acc_seq32, _acc_trunc16])
def test_bf16_tau_sound_under_fp32_accumulators(orc, kind, acc):
    """No fault-free column check of the simulated plain form exceeds its
    threshold, for round-to-nearest and truncating accumulators, uniform,
    all-positive and six-decade log-uniform operands; the residual uses a
    visible share of the threshold on all-positive data under truncation
    (where both sides' errors pile up) but stays below it."""
    rng = np.random.default_rng(11)
    K, L = (96, 12) if acc is _acc_trunc16 else (300, 16)
    res, tau = _simulate_plain_tile(rng, K, L, 1.5, -0.5, kind, acc)
    assert np.all(res <= tau), (res / tau).max()
    assert np.all(tau > 0)


def test_bf16_elem_tol_sound(orc):
    """The element bound covers the difference between the FP32-accumulated
    output and its FP64 recomputation from the bf16 operands, under both
    accumulator models, and a change of twice the bound exceeds it."""
    from oracle import split
    rng = np.random.default_rng(5)
    for kind in ("uniform", "positive", "loguniform", "one_large"):
        for K in (16, 200):
            p = _bf16_products(rng, K, kind)
            ab = float(np.abs(p).sum())
            c = float(rng.uniform(-1, 1))
            recomputed = math.fma(1.5, math.fsum(p), -0.5 * c) if hasattr(math, "fma") else 1.5 * math.fsum(p) - 0.5 * c
            tol = split.bf16_elem_tol(K, 1.5, ab, -0.5, c)
            for acc in (_acc_seq32, _acc_trunc16):
                out = 1.5 * acc(p) + -0.5 * c
                assert abs(out - recomputed) <= tol, (kind, K)
            assert tol < 2.0 ** -20 * 1.5 * ab * K + 1e-300 or kind == "loguniform"
