"""Split-precision FT-GEMM on the BF16 tensor cores against the FP64 oracle.

Tolerances (stated, not tuned):
  emulated FP64 with S slices of w bits: the parity bound of the FP64 path
  plus the splitting bound |alpha| sigma_i tau_j K (S + 4) 2^(-wS), where
  sigma_i, tau_j are the power-of-two row/column scales (every row of op(A)
  and column of op(B) keeps w*S bits relative to its largest element);
  plain BF16: |alpha| (2^-7 + 2.01 (K+2) 2^-24) sum_k |a_ik||b_kj| (bf16
  input rounding + FP32 accumulation) plus the FP64 parity bound.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_02444_gb300 import build
    build.build()
    from paper_2305_02444_gb300 import ftgemm
    ftgemm.lib()
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_split_engine(0)
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_split_engine(0)


def wbits(K):
    return 8 if K <= 256 else 7 if K <= 1024 else 6 if K <= 4096 else 5


def problem(ta, tb, M, N, K, seed, dist="uniform"):
    from paper_2305_02444_gb300 import inputs
    ar, ac = (M, K) if ta == "N" else (K, M)
    br, bc = (K, N) if tb == "N" else (N, K)
    A = inputs.matrix(ar, ac, seed, dist)
    B = inputs.matrix(br, bc, seed + 1, dist)
    C = inputs.matrix(M, N, seed + 2, dist)
    return A, B, C, ar, br


def run(ft, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, S, ftflag=True):
    dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
    rc, rep = ft.ftgemm_d_split(ta, tb, M, N, K, alpha, dA, ar, dB, br, beta, dC, M, nslices=S,
                                ft=ftflag)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    return dC.cpu().T.numpy(), rep


def scales(ta, tb, A, B, ar, br):
    opA = A[:, :ar].T.numpy(); opA = opA if ta == "N" else opA.T
    opB = B[:, :br].T.numpy(); opB = opB if tb == "N" else opB.T
    sa = np.array([2.0 ** math.frexp(float(np.abs(r).max()))[1] if np.abs(r).max() > 0 else 1.0 for r in opA])
    sb = np.array([2.0 ** math.frexp(float(np.abs(c).max()))[1] if np.abs(c).max() > 0 else 1.0 for c in opB.T])
    return opA, opB, sa, sb


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("M,N,K,S", [(300, 260, 200, 7), (130, 257, 1000, 8), (256, 128, 5000, 11)])
def test_emulated_fp64_parity(ft, orc, ta, tb, M, N, K, S):
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=M + K)
    alpha, beta = 1.5, 0.5
    got, rep = run(ft, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, S)
    ref, E = orc.gemm(ta, tb, alpha, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), beta, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales(ta, tb, A, B, ar, br)
    w = wbits(K)
    split = abs(alpha) * np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-w * S)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0 and rep["detected"] == 0


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_plain_bf16_form(ft, orc, ta, tb):
    M, N, K = 300, 200, 700
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=31)
    alpha, beta = 1.0, 1.0
    got, rep = run(ft, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, 0)
    ref, E = orc.gemm(ta, tb, alpha, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), beta, C.T.numpy(), want_E=True)
    opA, opB, _, _ = scales(ta, tb, A, B, ar, br)
    absab = np.abs(opA) @ np.abs(opB)
    tol = abs(alpha) * (2.0 ** -7 + 2.01 * (K + 2) * 2.0 ** -24) * absab + orc.parity_tol(K, E)
    assert np.all(np.abs(got - ref) <= tol)
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    assert 1e-6 < rel < 1e-2   # really BF16: far from FP64, well inside its own bound
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0


def test_ft_and_unprotected_give_the_same_bits(ft):
    A, B, C, ar, br = problem("N", "N", 200, 200, 300, seed=3)
    g1, _ = run(ft, "N", "N", 200, 200, 300, 1.25, -0.5, A, B, C, ar, br, 8, ftflag=True)
    g0, _ = run(ft, "N", "N", 200, 200, 300, 1.25, -0.5, A, B, C, ar, br, 8, ftflag=False)
    np.testing.assert_array_equal(g0, g1)


def test_split_injection_detected_and_corrected(ft, orc):
    """Flips of the top exponent bit of the FP64 accumulator after chosen slice
    pairs (the first, a middle and the last of the 36 pairs): each moves the
    value by at least 2 (or to a huge value / Inf / NaN), above the FP32
    checksums' threshold, so each is detected and corrected by the FP64
    recomputation.  (Flips far below that threshold, e.g. low exponent bits of
    a small partial sum, are not detectable with FP32 checksums: their band is
    stated with the design.)"""
    M, N, K, S = 256, 256, 512, 8
    A, B, C, ar, br = problem("N", "N", M, N, K, seed=17)
    flips = [(5, 6, 0, 62), (100, 200, 20, 62), (250, 3, 35, 62)]   # kstep = pair index (36 pairs)
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        got, rep = run(ft, "N", "N", M, N, K, 1.0, 1.0, A, B, C, ar, br, S)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert [L["applied"] for L in log] == [1, 1, 1]
    ref, E = orc.gemm("N", "N", 1.0, A.T.numpy(), B.T.numpy(), 1.0, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales("N", "N", A, B, ar, br)
    split = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
    assert rep["detected"] == 3
    assert sorted(l[:2] for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)


def test_loguniform_error_is_stated(ft, orc):
    """Six-decade log-uniform entries: the emulation keeps w*S bits relative to
    each row's (column's) largest entry; the error stays within the stated
    bound and is far below the plain BF16 form's."""
    M = N = 256
    K = 2048
    A, B, C, ar, br = problem("N", "N", M, N, K, seed=99, dist="loguniform")
    ref, E = orc.gemm("N", "N", 1.0, A.T.numpy(), B.T.numpy(), 0.0, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales("N", "N", A, B, ar, br)
    errs = {}
    for S in (0, 6, 9):
        got, rep = run(ft, "N", "N", M, N, K, 1.0, 0.0, A, B, C, ar, br, S)
        errs[S] = float(np.abs(got - ref).max() / np.abs(ref).max())
        if S:
            split = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
            assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
        assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0
    assert errs[9] < errs[6] < errs[0]


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T")])
def test_emulated_with_fp64_checksums(ft, orc, ta, tb):
    M, N, K, S = 300, 260, 1000, 8
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=77)
    got, rep = run(ft, ta, tb, M, N, K, 1.5, 0.5, A, B, C, ar, br, S, ftflag=2)
    ref, E = orc.gemm(ta, tb, 1.5, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), 0.5, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales(ta, tb, A, B, ar, br)
    split = 1.5 * np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0 and rep["detected"] == 0


def test_fp64_checksums_see_what_fp32_checksums_miss(ft, orc):
    """Mantissa flips (bits 40..50) of the full-magnitude accumulator after the
    last slice pair change an element by 2^-12..2^-2 of its value: the FP64
    checksums (ft=2) detect and correct every one; the FP32 checksums (ft=1)
    cannot see changes that small."""
    M, N, K, S = 256, 256, 512, 8
    npairs = S * (S + 1) // 2
    A, B, C, ar, br = problem("N", "N", M, N, K, seed=23)
    ref, E = orc.gemm("N", "N", 1.0, A.T.numpy(), B.T.numpy(), 0.0, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales("N", "N", A, B, ar, br)
    split = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    rng = np.random.default_rng(5)
    flips = [(int(rng.integers(M)), int(rng.integers(N)), npairs - 1, bit) for bit in range(40, 51)]
    detected = {}
    for mode in (1, 2):
        assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
        try:
            got, rep = run(ft, "N", "N", M, N, K, 1.0, 0.0, A, B, C, ar, br, S, ftflag=mode)
        finally:
            ft.ftgemm_set_injection(mode=0)
        detected[mode] = rep["detected"]
        if mode == 2:
            assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
            assert sorted(l[:2] for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)
    assert detected[2] == len(flips)
    assert detected[1] < len(flips) // 2


# default, mma.sync, tcgen05 with one CTA per tile, persistent tcgen05
ENGINES = (0, 1, 2, 5)


def run_engine(ft, engine, *a, **kw):
    assert ft.ftgemm_set_split_engine(engine) == 0
    try:
        return run(ft, *a, **kw)
    finally:
        ft.ftgemm_set_split_engine(0)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("M,N,K,S,ck", [(300, 260, 200, 7, 0), (130, 258, 1000, 8, 2), (256, 384, 640, 3, 2),
                                        (1, 129, 65, 4, 0), (2, 130, 5000, 11, 2)])
def test_tcgen05_and_mma_sync_give_the_same_bits(ft, orc, ta, tb, M, N, K, S, ck):
    """The emulated pair products are exact integers in FP32 on both engines and
    the FP64 fold has the same order and arithmetic: identical outputs.  (FP64
    checksums need even leading dimensions: those shapes are even.)"""
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=M + N + K)
    outs = {e: run_engine(ft, e, ta, tb, M, N, K, 1.5, 0.5, A, B, C, ar, br, S, ftflag=ck) for e in ENGINES}
    g_tc = outs[0][0]
    for e, (g, r) in outs.items():   # tcgen05 one CTA per tile / persistent, mma.sync
        np.testing.assert_array_equal(g, g_tc)
        assert r["flagged_rows"] == 0 and r["flagged_cols"] == 0
    ref, E = orc.gemm(ta, tb, 1.5, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), 0.5, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales(ta, tb, A, B, ar, br)
    split = 1.5 * np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    assert np.all(np.abs(g_tc - ref) <= orc.parity_tol(K, E) + split)


def test_tcgen05_several_k_chunks(ft, orc):
    """K = 18000 > 17408 products per exact FP32 chunk at w = 5: every pair is
    folded in two chunks, through both tensor-memory accumulators (a 2 x 2
    tile grid)."""
    M, N, K, S = 130, 140, 18000, 3
    A, B, C, ar, br = problem("N", "N", M, N, K, seed=5)
    outs = {e: run_engine(ft, e, "N", "N", M, N, K, 1.0, 1.0, A, B, C, ar, br, S, ftflag=2)[0] for e in ENGINES}
    g_tc = outs[0]
    for g in outs.values():
        np.testing.assert_array_equal(g, g_tc)
    ref, E = orc.gemm("N", "N", 1.0, A.T.numpy(), B.T.numpy(), 1.0, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales("N", "N", A, B, ar, br)
    split = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    assert np.all(np.abs(g_tc - ref) <= orc.parity_tol(K, E) + split)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
def test_tcgen05_plain_bf16(ft, orc, ta, tb):
    M, N, K = 300, 200, 700
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=41)
    got, rep = run_engine(ft, 0, ta, tb, M, N, K, 1.0, 1.0, A, B, C, ar, br, 0, ftflag=0)
    ref, E = orc.gemm(ta, tb, 1.0, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), 1.0, C.T.numpy(), want_E=True)
    opA, opB, _, _ = scales(ta, tb, A, B, ar, br)
    absab = np.abs(opA) @ np.abs(opB)
    tol = (2.0 ** -7 + 2.01 * (K + 2) * 2.0 ** -24) * absab + orc.parity_tol(K, E)
    assert np.all(np.abs(got - ref) <= tol)
    rel = np.abs(got - ref).max() / np.abs(ref).max()
    assert 1e-6 < rel < 1e-2


@pytest.mark.parametrize("engine", [2, 5])
def test_tcgen05_injection_log_and_correction(ft, orc, engine):
    """Flips of the tensor-memory FP64 accumulators after chosen slice pairs
    (first, middle, last of 36; one element in each lane quadrant): logged
    with the value they changed, detected by the FP64 checksums, located and
    corrected."""
    M, N, K, S = 256, 256, 512, 8
    A, B, C, ar, br = problem("N", "N", M, N, K, seed=19)
    flips = [(5, 6, 0, 62), (100, 200, 20, 62), (250, 3, 35, 62), (70, 129, 35, 52)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        got, rep = run_engine(ft, engine, "N", "N", M, N, K, 1.0, 1.0, A, B, C, ar, br, S, ftflag=2)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert [L["applied"] for L in log] == [1] * len(flips)
    for L, (i, j, q, bit) in zip(log, flips):
        assert (L["row"], L["col"], L["kstep"], L["bit"]) == (i, j, q, bit)
        before, after = np.float64(L["before"]), np.float64(L["after"])
        assert before.view(np.int64) ^ after.view(np.int64) == np.int64(1) << bit
    ref, E = orc.gemm("N", "N", 1.0, A.T.numpy(), B.T.numpy(), 1.0, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales("N", "N", A, B, ar, br)
    split = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
    assert rep["detected"] == len(flips)
    assert sorted(l[:2] for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)


@pytest.mark.parametrize("ck,S", [(0, 0), (0, 4), (2, 4)])
def test_persistent_many_tiles_per_cta(ft, orc, ck, S):
    """2560 x 2690: 420 tiles (ragged last tile column), so each CTA of the
    persistent grid (one per SM) finishes two or three tiles and the ring and
    accumulators pass between tiles.  Same bits as one CTA per tile, for the
    plain BF16 form (finished from the FP32 accumulator), the emulated form
    without checks and with FP64 checksums."""
    M, N, K = 2560, 2690, 192
    A, B, C, ar, br = problem("N", "T", M, N, K, seed=77)
    outs = {e: run_engine(ft, e, "N", "T", M, N, K, 1.5, -0.5, A, B, C, ar, br, S, ftflag=ck) for e in (2, 5)}
    np.testing.assert_array_equal(outs[5][0], outs[2][0])
    for g, r in outs.values():
        assert r["flagged_rows"] == 0 and r["flagged_cols"] == 0 and r["unverifiable"] == 0
    if S:
        ref, E = orc.gemm("N", "T", 1.5, A.T.numpy(), B[:, :br].T.numpy(), -0.5, C.T.numpy(), want_E=True)
        _, _, sa, sb = scales("N", "T", A, B, ar, br)
        split = 1.5 * np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
        assert np.all(np.abs(outs[5][0] - ref) <= orc.parity_tol(K, E) + split)


@pytest.mark.parametrize("engine", [5])
def test_persistent_flips_in_later_tiles(ft, orc, engine):
    """Flips in tiles that a persistent CTA reaches first, second and third
    (tile t goes to CTA t mod grid): each tile with a fault is recomputed in
    the CTA's scratch tile, the others are stored directly; all are located
    and corrected, and the report counts each once."""
    M, N, K, S = 2048, 2560, 256, 5
    A, B, C, ar, br = problem("N", "N", M, N, K, seed=91)
    # (row, col, pair, bit): tiles (0,0), (8,3) and (15,19) of the 16 x 20 grid, two faults in one tile
    flips = [(3, 4, 0, 62), (1030, 400, 7, 62), (1100, 450, 14, 61), (1990, 2500, 14, 62)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        got, rep = run_engine(ft, engine, "N", "N", M, N, K, 1.0, 1.0, A, B, C, ar, br, S, ftflag=2)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert [L["applied"] for L in log] == [1] * len(flips)
    ref, E = orc.gemm("N", "N", 1.0, A.T.numpy(), B.T.numpy(), 1.0, C.T.numpy(), want_E=True)
    _, _, sa, sb = scales("N", "N", A, B, ar, br)
    split = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-wbits(K) * S)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split)
    assert rep["detected"] == len(flips) and rep["corrected"] == len(flips)
    assert sorted(l[:2] for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)


def bf16_nearest_even(x: float) -> float:
    """x rounded to bf16 (8 significant bits, exponents of FP32), to nearest
    with ties to even, from the definition: Python's round() of an exactly
    scaled double is round-half-even."""
    if x == 0.0 or not math.isfinite(x):
        return x
    f, e = math.frexp(x)                  # x = f 2^e, 1/2 <= |f| < 1
    if e - 1 < -126:                      # below the normal range: multiples of 2^-133
        v = round(x * 2.0 ** 133) * 2.0 ** -133
    else:
        v = math.ldexp(round(math.ldexp(f, 8)), e - 8)
    return math.copysign(math.inf, x) if abs(v) >= 2.0 ** 128 else v


@pytest.mark.parametrize("side,trans", [("A", "N"), ("A", "T"), ("B", "N"), ("B", "T")])
def test_plain_bf16_rounding_is_nearest_even(ft, side, trans):
    """A rank-1 product with K = 1 and a unit other operand returns the bf16
    rounding of each entry (exact in FP32 and FP64 after it): halfway cases
    (ties to even, both parities, with carries into the exponent), values just
    off the halfway points, overflow to Inf, zeros and random magnitudes, in
    both layouts of both operands (the two slicing paths)."""
    rng = np.random.default_rng(7)
    q = rng.integers(0x0080, 0x7F7F, 600).astype(np.uint32) << 16          # normal bf16 values
    base = q.view(np.float32).astype(np.float64) * rng.choice([-1.0, 1.0], 600)
    ulp = np.array([math.ldexp(1.0, math.frexp(b)[1] - 8) for b in base])
    vals = np.concatenate([
        base + np.sign(base) * ulp / 2,                                      # exact ties
        base + np.sign(base) * ulp / 2 * (1 + 2.0 ** -40),                   # just above
        base + np.sign(base) * ulp / 2 * (1 - 2.0 ** -40),                   # just below
        rng.standard_normal(300) * 10.0 ** rng.integers(-30, 30, 300),
        [0.0, -0.0, 3.4e38, -3.39e38, 3.3961e38, 1.0, 255.5, 256.5, 1.9921875 + 2 ** -8, 1.99609375],
    ])
    n = len(vals)
    x = torch.tensor(vals, dtype=torch.float64)
    one = torch.ones(1, dtype=torch.float64)
    if side == "A":   # op(A) n x 1, op(B) = [1]
        M, N = n, 1
        A = x.reshape(1, n) if trans == "N" else x.reshape(n, 1)   # column-major (cols, ld) storage
        lda = n if trans == "N" else 1
        B, ldb, tb, ta = one.reshape(1, 1), 1, "N", trans
    else:             # op(A) = [1], op(B) 1 x n
        M, N = 1, n
        B = x.reshape(n, 1) if trans == "N" else x.reshape(1, n)
        ldb = 1 if trans == "N" else n
        A, lda, ta, tb = one.reshape(1, 1), 1, "N", trans
    dC = torch.zeros(N, M, dtype=torch.float64, device="cuda")
    rc, _ = ft.ftgemm_d_split(ta, tb, M, N, 1, 1.0, A.cuda(), lda, B.cuda(), ldb, 0.0, dC, M, nslices=0, ft=0)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    got = dC.cpu().numpy().reshape(-1)
    want = np.array([bf16_nearest_even(float(v)) for v in vals])
    np.testing.assert_array_equal(got, want)
