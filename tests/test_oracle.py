"""Pins for the CPU oracle (no GPU).

The paper prints no worked example, so the oracle is pinned by what the
mathematics fixes: exact rational arithmetic (fractions.Fraction) on tiny
cases, integer-exact and dyadic-exact closed forms (identity, all-ones,
rank-1), an exact integer matmul from numpy as an independent library step,
BLAS quick returns and argument codes, the Huang-Abraham checksum
invariants, and exhaustive single-fault recovery on tiny tiles.
"""
from __future__ import annotations

import itertools
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

U = 2.0 ** -53
TRANS = ["N", "T"]


def stored(opX: np.ndarray, t: str) -> np.ndarray:
    """Stored matrix whose op() is opX."""
    return np.asfortranarray(opX if t == "N" else opX.T)


def dyadic(rng, shape, bits=6, scale=3):
    """Random dyadic rationals m / 2^bits with |m| < 2^scale * 2^bits (exact in fp64)."""
    return rng.integers(-(2 ** (bits + scale)), 2 ** (bits + scale), size=shape).astype(np.float64) / 2 ** bits


# --------------------------------------------------------------------------- gemm closed forms

@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
def test_identity_operand_exact(orc, ta, tb):
    rng = np.random.default_rng(1)
    M, N = 7, 5
    opA = np.eye(M)
    opB = dyadic(rng, (M, N))
    C = dyadic(rng, (M, N))
    alpha, beta = 2.0, 0.5
    out, _ = orc.gemm(ta, tb, alpha, stored(opA, ta), stored(opB, tb), beta, C)
    # I*B is exact and alpha*B + beta*C is exact for these dyadic values
    np.testing.assert_array_equal(out, alpha * opB + beta * C)


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
def test_all_ones_closed_form(orc, ta, tb):
    M, N, K = 6, 9, 37
    c = 0.75
    out, E = orc.gemm(ta, tb, 1.5, stored(np.ones((M, K)), ta), stored(np.ones((K, N)), tb), -0.25,
                      np.full((M, N), c), want_E=True)
    assert np.all(out == 1.5 * K - 0.25 * c)
    assert np.all(E == 1.5 * K + 0.25 * c)


def test_rank1_powers_of_two_exact(orc):
    rng = np.random.default_rng(2)
    x = 2.0 ** rng.integers(-20, 20, size=(11, 1)) * rng.choice([-1, 1], size=(11, 1))
    y = 2.0 ** rng.integers(-20, 20, size=(1, 13)) * rng.choice([-1, 1], size=(1, 13))
    C = np.zeros((11, 13))
    out, _ = orc.gemm("N", "N", 0.5, x, y, 0.0, C)
    for i in range(11):
        for j in range(13):
            assert out[i, j] == 0.5 * x[i, 0] * y[0, j]


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (17, 3, 29), (33, 40, 7), (5, 64, 65)])
def test_small_integer_exact_vs_integer_matmul(orc, ta, tb, M, N, K):
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    opA = rng.integers(-8, 9, size=(M, K))
    opB = rng.integers(-8, 9, size=(K, N))
    C = rng.integers(-8, 9, size=(M, N))
    alpha, beta = 3, -2
    expect = alpha * (opA @ opB) + beta * C          # numpy int64 matmul: exact
    eabs = abs(alpha) * (np.abs(opA) @ np.abs(opB)) + abs(beta) * np.abs(C)
    out, E = orc.gemm(ta, tb, float(alpha), stored(opA.astype(float), ta),
                      stored(opB.astype(float), tb), float(beta), C.astype(float), want_E=True)
    np.testing.assert_array_equal(out, expect.astype(float))
    np.testing.assert_array_equal(E, eabs.astype(float))


def _exact(opA, opB, C, alpha, beta):
    M, K = opA.shape
    N = opB.shape[1]
    ex = np.empty((M, N), dtype=object)
    for i in range(M):
        for j in range(N):
            s = sum((Fraction(opA[i, k]) * Fraction(opB[k, j]) for k in range(K)), Fraction(0))
            ex[i, j] = Fraction(alpha) * s + (Fraction(beta) * Fraction(C[i, j]) if beta != 0 else 0)
    return ex


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (1.5, 0.5), (-0.3, 0.0), (0.7, -1.25)])
def test_brute_force_rational(orc, ta, tb, alpha, beta):
    rng = np.random.default_rng(7)
    for trial in range(4):
        M, N, K = rng.integers(1, 6, size=3)
        opA = rng.uniform(-1, 1, (M, K))
        opB = rng.uniform(-1, 1, (K, N))
        C = rng.uniform(-1, 1, (M, N))
        out, E = orc.gemm(ta, tb, alpha, stored(opA, ta), stored(opB, tb), beta, C, want_E=True)
        ex = _exact(opA, opB, C, alpha, beta)
        g = (K + 3) * U / (1 - (K + 3) * U)
        for i in range(M):
            for j in range(N):
                err = abs(Fraction(out[i, j]) - ex[i, j])
                assert err <= Fraction(g) * Fraction(E[i, j]) * Fraction(101, 100)


# --------------------------------------------------------------------------- BLAS contract

def test_quick_returns_and_beta_zero(orc):
    rng = np.random.default_rng(3)
    A = rng.uniform(-1, 1, (4, 0)); B = rng.uniform(-1, 1, (0, 3)); C = rng.uniform(-1, 1, (4, 3))
    out, _ = orc.gemm("N", "N", 2.0, A, B, 0.5, C)                # K = 0: beta*C
    np.testing.assert_array_equal(out, 0.5 * C)
    A = rng.uniform(-1, 1, (4, 5)); B = rng.uniform(-1, 1, (5, 3))
    out, _ = orc.gemm("N", "N", 0.0, A, B, -2.0, C)               # alpha = 0: beta*C
    np.testing.assert_array_equal(out, -2.0 * C)
    Cn = C.copy(); Cn[1, 1] = np.nan; Cn[2, 0] = np.inf
    out, E = orc.gemm("N", "N", 1.0, A, B, 0.0, Cn, want_E=True)  # beta = 0: C is not read
    assert np.all(np.isfinite(out)) and np.all(np.isfinite(E))
    out, _ = orc.gemm("N", "N", 0.0, A, B, 0.0, Cn)
    assert np.all(out == 0.0)
    # M = 0 / N = 0: nothing touched (no crash on empty)
    out, _ = orc.gemm("N", "N", 1.0, np.zeros((0, 5)), B, 1.0, np.zeros((0, 3)))
    assert out.shape == (0, 3)


def test_argument_codes(orc):
    A = np.zeros(64); B = np.zeros(64); C = np.zeros(64)
    g = orc.gemm_raw
    assert g("X", "N", 2, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == -1
    assert g("N", "Q", 2, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == -2
    assert g("N", "N", -1, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == -3
    assert g("N", "N", 2, -1, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == -4
    assert g("N", "N", 2, 2, -1, 1.0, A, 2, B, 2, 0.0, C, 2) == -5
    assert g("N", "N", 3, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 3) == -8
    assert g("T", "N", 2, 2, 3, 1.0, A, 2, B, 3, 0.0, C, 2) == -8
    assert g("N", "N", 2, 2, 3, 1.0, A, 2, B, 2, 0.0, C, 2) == -10
    assert g("N", "T", 2, 3, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == -10
    assert g("N", "N", 3, 2, 2, 1.0, A, 3, B, 2, 0.0, C, 2) == -13
    assert g("n", "t", 2, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == 0
    assert g("C", "c", 2, 2, 2, 1.0, A, 2, B, 2, 0.0, C, 2) == 0


def test_leading_dimension_padding(orc):
    rng = np.random.default_rng(4)
    M, N, K = 5, 4, 6
    lda, ldb, ldc = 9, 8, 7
    opA = rng.integers(-5, 6, (M, K)).astype(float); opB = rng.integers(-5, 6, (K, N)).astype(float)
    C0 = rng.integers(-5, 6, (M, N)).astype(float)
    Abuf = np.full(lda * K, 1e300); Bbuf = np.full(ldb * N, 1e300); Cbuf = np.full(ldc * N, 7.0)
    for k in range(K):
        Abuf[k * lda:k * lda + M] = opA[:, k]
    for j in range(N):
        Bbuf[j * ldb:j * ldb + K] = opB[:, j]
        Cbuf[j * ldc:j * ldc + M] = C0[:, j]
    assert orc.gemm_raw("N", "N", M, N, K, 2.0, Abuf, lda, Bbuf, ldb, 1.0, Cbuf, ldc) == 0
    out = np.stack([Cbuf[j * ldc:j * ldc + M] for j in range(N)], axis=1)
    np.testing.assert_array_equal(out, 2 * opA @ opB + C0)
    for j in range(N):                                   # padding rows untouched
        assert np.all(Cbuf[j * ldc + M:(j + 1) * ldc] == 7.0)


def test_partial_is_accumulator(orc):
    rng = np.random.default_rng(5)
    A = rng.uniform(-1, 1, (6, 40)); B = rng.uniform(-1, 1, (40, 3))
    out, _ = orc.gemm("N", "N", 1.0, A, B, 0.0, np.zeros((6, 3)))
    for i in range(6):
        for j in range(3):
            assert orc.partial("N", "N", i, j, 40, A, B) == out[i, j]
            assert orc.partial("N", "N", i, j, 0, A, B) == 0.0
    ex = sum(Fraction(A[2, k]) * Fraction(B[k, 1]) for k in range(17))
    assert abs(Fraction(orc.partial("N", "N", 2, 1, 17, A, B)) - ex) <= Fraction(17 * U) * sum(
        Fraction(abs(A[2, k] * B[k, 1])) for k in range(17)) * 2


# --------------------------------------------------------------------------- checksum invariants

@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
def test_pred_checksums_exact_integers(orc, ta, tb):
    rng = np.random.default_rng(6)
    M, N, K = 13, 11, 9
    opA = rng.integers(-7, 8, (M, K)); opB = rng.integers(-7, 8, (K, N)); C = rng.integers(-7, 8, (M, N))
    col, row = orc.pred_checksums(ta, tb, 2.0, stored(opA.astype(float), ta), stored(opB.astype(float), tb),
                                  -3.0, C.astype(float))
    np.testing.assert_array_equal(col, (2 * (np.ones(M) @ opA) @ opB - 3 * C.sum(0)).astype(float))
    np.testing.assert_array_equal(row, (2 * opA @ (opB @ np.ones(N)) - 3 * C.sum(1)).astype(float))
    col0, row0 = orc.pred_checksums(ta, tb, 2.0, stored(opA.astype(float), ta), stored(opB.astype(float), tb),
                                    0.0, np.full((M, N), np.nan))
    assert np.all(np.isfinite(col0)) and np.all(np.isfinite(row0))


def test_invariants_hold_on_output(orc):
    rng = np.random.default_rng(8)
    M, N, K = 40, 30, 500
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    out, E = orc.gemm("N", "N", 1.5, A, B, 0.5, C, want_E=True)
    col, row = orc.pred_checksums("N", "N", 1.5, A, B, 0.5, C)
    # e^T C_out = alpha (e^T A) B + beta e^T C within the two-sided rounding bound
    assert np.all(np.abs(out.sum(0) - col) <= 2 * (K + M + 3) * U * E.sum(0) * 1.01)
    assert np.all(np.abs(out.sum(1) - row) <= 2 * (K + N + 3) * U * E.sum(1) * 1.01)


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
def test_encode_operands_definition(orc, ta, tb):
    rng = np.random.default_rng(9)
    M, N, K, BM, BN = 21, 19, 7, 8, 6
    opA = rng.integers(-9, 10, (M, K)).astype(float); opB = rng.integers(-9, 10, (K, N)).astype(float)
    e = orc.encode_operands(ta, tb, M, N, K, stored(opA, ta), stored(opB, tb), BM, BN)
    for I in range(-(-M // BM)):
        blk = opA[I * BM:(I + 1) * BM]
        np.testing.assert_array_equal(e.acs[I], blk.sum(0))
        assert e.aabsmax[I] == np.abs(blk).sum(0).max()
    for J in range(-(-N // BN)):
        blk = opB[:, J * BN:(J + 1) * BN]
        np.testing.assert_array_equal(e.bcs[J], blk.sum(1))
        assert e.babsmax[J] == np.abs(blk).sum(1).max()
    np.testing.assert_array_equal(e.arowabs, np.abs(opA).sum(1))
    np.testing.assert_array_equal(e.bcolabs, np.abs(opB).sum(0))


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
def test_encode_vectors_predict_tile_checksums(orc, ta, tb):
    """Huang-Abraham invariant of the per-tile scheme (§2.2): a_I^T op(B)
    is the column checksum e^T (op(A) op(B))_IJ of every tile, op(A) b_J its
    row checksum; exact on integers, so a vector summed over the wrong rows,
    the wrong axis or a shifted tile boundary fails."""
    rng = np.random.default_rng(10)
    M, N, K, BM, BN = 23, 17, 11, 8, 5
    opA = rng.integers(-9, 10, (M, K)).astype(float); opB = rng.integers(-9, 10, (K, N)).astype(float)
    e = orc.encode_operands(ta, tb, M, N, K, stored(opA, ta), stored(opB, tb), BM, BN)
    P = opA.astype(np.int64) @ opB.astype(np.int64)
    for I in range(-(-M // BM)):
        rows = slice(I * BM, min(M, (I + 1) * BM))
        for J in range(-(-N // BN)):
            cols = slice(J * BN, min(N, (J + 1) * BN))
            np.testing.assert_array_equal(e.acs[I] @ opB[:, cols], P[rows, cols].sum(0))
            np.testing.assert_array_equal(opA[rows] @ e.bcs[J], P[rows, cols].sum(1))


# --------------------------------------------------------------------------- seeded fault list

def test_splitmix64_golden(orc):
    here = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    rows = [l.split() for l in open(here) if l.strip() and not l.startswith("#")]
    for seed, n, hx in rows:
        assert orc.splitmix64(int(seed), int(n)) == int(hx, 16)


def _golden_splitmix64():
    here = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    rows = [l.split() for l in open(here) if l.strip() and not l.startswith("#")]
    return {(int(seed), int(n)): int(hx, 16) for seed, n, hx in rows}


def test_random_flips_field_mapping_from_golden_outputs(orc):
    """Fault f takes generator outputs 4f, 4f+1, 4f+2, 4f+3 as (row mod M,
    col mod N, k-step mod nks, bit mod 63): checked against the published
    outputs themselves (not the oracle's generator), for fault 0 of two
    seeds and the row of fault 1 (output 4) -- a mistake in the stride, the
    field order or a modulus fails here."""
    g = _golden_splitmix64()
    for seed in (0, 1234567):
        M, N, nks = 1000003, 999983, 517       # primes: no modulus hides another
        f = orc.random_flips(seed, 2, M, N, nks)
        assert tuple(f[0]) == (g[(seed, 0)] % M, g[(seed, 1)] % N, g[(seed, 2)] % nks, g[(seed, 3)] % 63)
        assert f[1][0] == g[(seed, 4)] % M


def test_random_flips_ranges_and_determinism(orc):
    f1 = orc.random_flips(1234, 500, 100, 37, 9)
    f2 = orc.random_flips(1234, 500, 100, 37, 9)
    np.testing.assert_array_equal(f1, f2)
    assert f1[:, 0].min() >= 0 and f1[:, 0].max() < 100
    assert f1[:, 1].max() < 37 and f1[:, 2].max() < 9 and f1[:, 3].max() <= 62
    assert len(set(f1[:, 3].tolist())) > 50          # the bits spread over [0, 62]
    assert not np.array_equal(f1, orc.random_flips(1235, 500, 100, 37, 9))


# --------------------------------------------------------------------------- the FT scheme

def _ft_vs_plain(orc, ta, tb, M, N, K, alpha, beta, BM, BN, BK, seed, dist="uniform"):
    rng = np.random.default_rng(seed)
    if dist == "uniform":
        opA = rng.uniform(-1, 1, (M, K)); opB = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    elif dist == "normal":
        opA = rng.normal(size=(M, K)); opB = rng.normal(size=(K, N)); C = rng.normal(size=(M, N))
    else:  # sign-random, log-uniform magnitudes over six decades
        def lu(shape):
            return rng.choice([-1, 1], size=shape) * 10 ** rng.uniform(-3, 3, shape)
        opA = lu((M, K)); opB = lu((K, N)); C = lu((M, N))
    A, B = stored(opA, ta), stored(opB, tb)
    plain, _ = orc.gemm(ta, tb, alpha, A, B, beta, C)
    r = orc.ft_gemm(ta, tb, alpha, A, B, beta, C, BM=BM, BN=BN, BK=BK)
    return A, B, C, plain, r


@pytest.mark.parametrize("ta,tb", list(itertools.product(TRANS, TRANS)))
@pytest.mark.parametrize("dist", ["uniform", "normal", "loguniform"])
def test_ft_fault_free_equals_plain_and_no_false_positive(orc, ta, tb, dist):
    for seed in range(3):
        _, _, _, plain, r = _ft_vs_plain(orc, ta, tb, 37, 29, 300, 1.5, 0.5, 16, 8, 16, seed, dist)
        np.testing.assert_array_equal(r.C, plain)
        assert r.counts["flagged_rows"] == 0 and r.counts["flagged_cols"] == 0
        assert r.counts["detected"] == 0 and r.counts["unverifiable"] == 0


def test_ft_no_false_positive_long_k(orc):
    for seed in range(2):
        _, _, _, plain, r = _ft_vs_plain(orc, "N", "N", 24, 24, 4096, 1.0, 1.0, 8, 8, 16, seed, "normal")
        np.testing.assert_array_equal(r.C, plain)
        assert r.counts["flagged_rows"] == 0 and r.counts["flagged_cols"] == 0


def _tile_taus(orc, ta, tb, alpha, beta, A, B, C, K, BM, BN, i, j):
    """tau_row(i) and tau_col(j) of the tile holding (i,j), from the definitions."""
    M, N = C.shape
    opA = A if ta == "N" else A.T
    opB = B if tb == "N" else B.T
    I, J = i // BM, j // BN
    rows = slice(I * BM, min(M, (I + 1) * BM)); cols = slice(J * BN, min(N, (J + 1) * BN))
    mI = rows.stop - rows.start; nJ = cols.stop - cols.start
    tr = orc.tau(K, nJ, alpha, np.abs(opA[i]).sum(), np.abs(opB[:, cols]).sum(1).max(), beta,
                 np.abs(C[i, cols]).sum())
    tc = orc.tau(K, mI, alpha, np.abs(opB[:, j]).sum(), np.abs(opA[rows]).sum(0).max(), beta,
                 np.abs(C[rows, j]).sum())
    return tr, tc


@pytest.mark.parametrize("ta,tb,alpha,beta", [("N", "N", 1.0, 1.0), ("T", "N", 1.5, 0.5),
                                              ("N", "T", -0.75, 0.0), ("T", "T", 2.0, -1.0)])
def test_every_single_flip_on_tiny_tiles(orc, ta, tb, alpha, beta):
    """All positions x k-steps x bits 0..62 of a 4x4x4 problem with 2x2 tiles
    and k-steps of 2: every flip whose effect clears both thresholds with
    margin is detected, located at its (i,j) and corrected to the fault-free
    bits; every flip far below both thresholds leaves the tile unflagged."""
    rng = np.random.default_rng(11)
    M = N = K = 4
    BM = BN = BK = 2
    opA = rng.uniform(-1, 1, (M, K)); opB = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    A, B = stored(opA, ta), stored(opB, tb)
    plain, E = orc.gemm(ta, tb, alpha, A, B, beta, C, want_E=True)
    n_big = n_small = 0
    for i, j, s, bit in itertools.product(range(M), range(N), range(K // BK), range(63)):
        r = orc.ft_gemm(ta, tb, alpha, A, B, beta, C, BM=BM, BN=BN, BK=BK,
                        flips=np.array([[i, j, s, bit]]))
        before, after = r.before[0], r.after[0]
        assert before == orc.partial(ta, tb, i, j, (s + 1) * BK, A, B)
        assert struct.unpack("<Q", struct.pack("<d", before))[0] ^ struct.unpack(
            "<Q", struct.pack("<d", after))[0] == 1 << bit
        with np.errstate(invalid="ignore", over="ignore"):   # flips to Inf / NaN are part of the sweep
            d = after - before
            eff = abs(alpha * d) if math.isfinite(d) else math.inf
        tr, tc = _tile_taus(orc, ta, tb, alpha, beta, A, B, C, K, BM, BN, i, j)
        if eff > 4 * max(tr, tc) + 1e-300:
            n_big += 1
            assert r.counts["detected"] == 1, (i, j, s, bit, r.counts)
            assert r.counts["corrected"] == 1
            assert r.locs[0][:2] == (i, j) and r.locs[0][3] == 0
            np.testing.assert_array_equal(r.C, plain)
        elif eff < 0.25 * min(tr, tc):
            n_small += 1
            assert r.counts["flagged_rows"] == 0 and r.counts["flagged_cols"] == 0
            assert r.counts["detected"] == 0
            tol = orc.parity_tol(K, E) + 2 * eff
            assert np.all(np.abs(r.C - plain) <= tol)
        else:   # inside the threshold band: any outcome must leave a sane result
            bad = np.abs(r.C - plain) > orc.parity_tol(K, E) + 2 * eff
            assert not np.any(bad)
    assert n_big > 1000 and n_small > 100


def test_nonfinite_and_huge_flips_recovered(orc):
    rng = np.random.default_rng(12)
    M = N = 16; K = 64
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    plain, _ = orc.gemm("N", "N", 1.0, A, B, 1.0, C)
    seen = set()
    for (i, j, s) in [(0, 0, 0), (5, 9, 2), (15, 15, 3), (7, 3, 1)]:
        for bit in (52, 57, 60, 61, 62):
            r = orc.ft_gemm("N", "N", 1.0, A, B, 1.0, C, BM=8, BN=8, BK=16,
                            flips=np.array([[i, j, s, bit]]))
            a = r.after[0]
            seen.add("nan" if math.isnan(a) else "inf" if math.isinf(a) else
                     "huge" if abs(a) > 1e100 else "tiny" if abs(a) < 1e-100 else "other")
            np.testing.assert_array_equal(r.C, plain)
            assert r.counts["detected"] == 1 and r.locs[0][:2] == (i, j)
    assert {"huge", "tiny"} <= seen


def test_multiple_flips_one_tile(orc):
    rng = np.random.default_rng(13)
    M = N = 32; K = 48
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    plain, _ = orc.gemm("N", "N", 1.5, A, B, 0.5, C)
    # two faults in distinct rows and columns: 4 intersections, 2 wrong
    fl = np.array([[1, 2, 0, 55], [5, 6, 1, 58]])
    r = orc.ft_gemm("N", "N", 1.5, A, B, 0.5, C, BM=16, BN=16, BK=16, flips=fl)
    np.testing.assert_array_equal(r.C, plain)
    assert r.counts["detected"] == 2 and r.counts["recomputed"] == 4
    assert [l[:2] for l in r.locs] == [(1, 2), (5, 6)]
    # same row, two columns
    fl = np.array([[3, 2, 0, 59], [3, 9, 2, 59]])
    r = orc.ft_gemm("N", "N", 1.5, A, B, 0.5, C, BM=16, BN=16, BK=16, flips=fl)
    np.testing.assert_array_equal(r.C, plain)
    assert r.counts["detected"] == 2
    # 9 x 9 flagged rows/columns exceed the 64-intersection cap: segment fallback
    fl = np.array([[q, q, 1, 60] for q in range(9)])
    r = orc.ft_gemm("N", "N", 1.5, A, B, 0.5, C, BM=16, BN=16, BK=16, flips=fl)
    np.testing.assert_array_equal(r.C, plain)
    assert r.counts["detected"] == 9 and all(l[3] == 1 for l in r.locs)
    # faults in two different tiles are handled independently
    fl = np.array([[1, 1, 0, 61], [20, 30, 2, 61]])
    r = orc.ft_gemm("N", "N", 1.5, A, B, 0.5, C, BM=16, BN=16, BK=16, flips=fl)
    np.testing.assert_array_equal(r.C, plain)
    assert r.counts["detected"] == 2 and len({l[2] for l in r.locs}) == 2


def test_row_only_flag_uses_segment_fallback(orc):
    """A fault whose size lies between a small row threshold and a large column
    threshold flags only its row; the segment fallback still repairs it."""
    rng = np.random.default_rng(14)
    M = N = 8; K = 32
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    A[3] *= 1e-6            # row 3: tiny values -> tiny row threshold
    B[:, 5] *= 1e6          # column 5: huge values -> huge column threshold
    plain, _ = orc.gemm("N", "N", 1.0, A, B, 0.0, C)
    hits = 0
    for bit in range(63):
        r = orc.ft_gemm("N", "N", 1.0, A, B, 0.0, C, BM=8, BN=8, BK=8, flips=np.array([[3, 5, 1, bit]]))
        if r.counts["flagged_rows"] == 1 and r.counts["flagged_cols"] == 0:
            hits += 1
            np.testing.assert_array_equal(r.C, plain)
            assert r.counts["detected"] == 1 and r.locs[0][:2] == (3, 5) and r.locs[0][3] == 1
            assert r.counts["checksum_only"] == 0
    assert hits >= 3


def test_nonfinite_inputs_unverifiable(orc):
    rng = np.random.default_rng(15)
    M = N = 8; K = 16
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    A[2, 3] = np.inf
    plain, _ = orc.gemm("N", "N", 1.0, A, B, 1.0, C)
    r = orc.ft_gemm("N", "N", 1.0, A, B, 1.0, C, BM=4, BN=4, BK=8)
    np.testing.assert_array_equal(np.isnan(r.C), np.isnan(plain))
    fin = np.isfinite(plain)
    np.testing.assert_array_equal(r.C[fin], plain[fin])
    assert r.counts["unverifiable"] > 0 and r.counts["detected"] == 0


def test_ragged_tiles_and_quick_returns(orc):
    for (M, N, K) in [(37, 23, 19), (1, 50, 3), (50, 1, 40), (17, 17, 1)]:
        for ta, tb in itertools.product(TRANS, TRANS):
            _, _, _, plain, r = _ft_vs_plain(orc, ta, tb, M, N, K, 1.5, 0.5, 16, 8, 16, M + N + K)
            np.testing.assert_array_equal(r.C, plain)
            assert r.counts["flagged_rows"] == 0 and r.counts["flagged_cols"] == 0
    C = np.ones((3, 4))
    r = orc.ft_gemm("N", "N", 1.0, np.zeros((3, 0)), np.zeros((0, 4)), 0.5, C)
    np.testing.assert_array_equal(r.C, 0.5 * C)


def test_threshold_is_tight(orc):
    """The miss band is bounded independently of orc_tau: every flip whose
    effect exceeds 10 * n * u * S (n = K + L + 3, S the Hoelder bound of the
    checksum's terms, computed here with numpy) must be detected, so a
    threshold looser than about 5x the two-sided rounding bound fails."""
    rng = np.random.default_rng(16)
    M = N = 8; K = 64; BM = BN = 8; BK = 16
    A = rng.uniform(-1, 1, (M, K)); B = rng.uniform(-1, 1, (K, N)); C = rng.uniform(-1, 1, (M, N))
    alpha, beta = 1.25, 0.5
    n = K + BN + 3
    checked = 0
    for (i, j, s) in [(0, 0, 0), (3, 5, 1), (7, 2, 3), (4, 4, 2)]:
        Srow = abs(alpha) * np.abs(A[i]).sum() * np.abs(B).sum(1).max() + abs(beta) * np.abs(C[i]).sum()
        Scol = abs(alpha) * np.abs(B[:, j]).sum() * np.abs(A).sum(0).max() + abs(beta) * np.abs(C[:, j]).sum()
        lim = 10 * n * U * max(Srow, Scol)
        for bit in range(20, 52):
            r = orc.ft_gemm("N", "N", alpha, A, B, beta, C, BM=BM, BN=BN, BK=BK,
                            flips=np.array([[i, j, s, bit]]))
            if abs(alpha * (r.after[0] - r.before[0])) > lim:
                checked += 1
                assert r.counts["detected"] == 1, (i, j, s, bit)
    assert checked > 40
