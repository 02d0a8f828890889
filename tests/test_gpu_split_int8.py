"""Emulated FP64 from INT8 slices (split engine 7: mma.sync m16n8k32 s8,
exact INT32 pair sums) through the C ABI.

The splitting is the oracle's fixed-point form (oracle.split_gemm) with
w = 7 bits per slice: every slice is an integer of magnitude below 128 (an
INT8), every pair's INT32 sum over the k-chunk is exact, and each enters
one FP64 sum with its power-of-two weight (one addition per slice pair and
k-chunk, n = S(S+1)/2 ceil(K / 133120) in all).

Tolerances (stated, not tuned):
  against the exact evaluation of the splitting: 1.02 (n + 4) u E_ij,
  E = |alpha||A||B| + |beta||C| (the kernel's FP64 roundings);
  against the FP64 oracle: the FP64 parity bound plus the splitting bound
  |alpha| sigma_i tau_j K (S + 4) 2^(-7S), sigma_i / tau_j the power-of-two
  scales of the rows of op(A) / columns of op(B).
"""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
W = 7


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_02444_gb300 import build
    build.build()
    from paper_2305_02444_gb300 import ftgemm
    ftgemm.lib()
    ftgemm.ftgemm_set_injection(mode=0)
    assert ftgemm.ftgemm_set_split_engine(7) == 0
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_split_engine(0)


def _problem(ta, tb, M, N, K, seed, dist="uniform"):
    from paper_2305_02444_gb300 import inputs
    ar, ac = (M, K) if ta == "N" else (K, M)
    br, bc = (K, N) if tb == "N" else (N, K)
    return (inputs.matrix(ar, ac, seed, dist), inputs.matrix(br, bc, seed + 1, dist),
            inputs.matrix(M, N, seed + 2, dist), ar, br)


def _run(ft, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, S, ftflag):
    dC = C.cuda()
    rc, rep = ft.ftgemm_d_split(ta, tb, M, N, K, alpha, A.cuda(), ar, B.cuda(), br, beta, dC, M, nslices=S,
                                ft=ftflag, loc_cap=4096)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    return dC.cpu().T.numpy(), rep


def _ops(ta, tb, A, B, ar, br):
    opA = A[:, :ar].T.numpy(); opB = B[:, :br].T.numpy()
    return (opA if ta == "N" else opA.T), (opB if tb == "N" else opB.T)


def _scales(opA, opB):
    sa = np.array([2.0 ** math.frexp(float(np.abs(r).max()))[1] if np.abs(r).max() > 0 else 1.0 for r in opA])
    sb = np.array([2.0 ** math.frexp(float(np.abs(c).max()))[1] if np.abs(c).max() > 0 else 1.0 for c in opB.T])
    return sa, sb


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("M,N,K,S,dist,ftflag", [(300, 260, 200, 3, "uniform", 0), (130, 258, 1000, 5, "normal", 2),
                                                (256, 128, 640, 8, "loguniform", 2), (1, 129, 65, 2, "uniform", 0),
                                                (200, 200, 3000, 4, "loguniform", 0)])
def test_int8_equals_exact_emulation(ft, orc, ta, tb, M, N, K, S, dist, ftflag):
    """Every layout, ragged tiles, K not a multiple of the 128-entry slab,
    uniform, normal and six-decade log-uniform entries, without and with the
    FP64 checksums: within the kernel's own FP64 rounding bound of the
    oracle's exact evaluation of the same splitting, where the FP64 product
    lies far outside that bound (so the comparison checks the emulation)."""
    from oracle import split
    A, B, C, ar, br = _problem(ta, tb, M, N, K, seed=M + N + K + S, dist=dist)
    alpha, beta = 1.5, -0.5
    got, rep = _run(ft, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, S, ftflag)
    opA, opB = _ops(ta, tb, A, B, ar, br)
    exact = split.split_gemm("N", "N", alpha, opA, opB, beta, C.T.numpy(), S, w=W)
    _, E = orc.gemm("N", "N", alpha, opA, opB, beta, C.T.numpy(), want_E=True)
    n = S * (S + 1) // 2
    assert np.all(np.abs(got - exact) <= 1.02 * (n + 4) * U * E)
    ref = orc.gemm("N", "N", alpha, opA, opB, beta, C.T.numpy())[0]
    sa, sb = _scales(opA, opB)
    split_bound = abs(alpha) * np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-W * S)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + split_bound)
    if S <= 4:   # few slices: the FP64 product is far from the emulation, which the first check tells apart
        assert np.abs(ref - exact).max() > 100 * (1.02 * (n + 4) * U * E).max()
    for k in ("flagged_rows", "flagged_cols", "detected", "unverifiable"):
        assert rep[k] == 0, (k, rep)


def test_int8_fp64_checksums_detect_and_correct(ft, orc):
    """Flips of the top exponent bits of the FP64 accumulator after the first
    and the last of the 21 slice pairs, in three tiles (the last a ragged
    corner): each moves its element by at least its own magnitude, far
    above the FP64 checksums' threshold (a flip after a middle pair can
    change only the small-weight partial sum, which may lie below it), and
    each is detected, located and corrected."""
    M, N, K, S = 300, 260, 700, 6
    A, B, C, ar, br = _problem("N", "N", M, N, K, seed=9)
    flips = [(5, 6, 0, 62), (200, 100, 20, 62), (299, 259, 20, 61)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        got, rep = _run(ft, "N", "N", M, N, K, 1.0, 1.0, A, B, C, ar, br, S, 2)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert [L["applied"] for L in log] == [1, 1, 1]
    assert rep["detected"] == 3 and rep["corrected"] == 3
    assert sorted(l[:2] for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)
    opA, opB = _ops("N", "N", A, B, ar, br)
    ref, E = orc.gemm("N", "N", 1.0, opA, opB, 1.0, C.T.numpy(), want_E=True)
    sa, sb = _scales(opA, opB)
    assert np.all(np.abs(got - ref) <= orc.parity_tol(K, E) + np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-W * S))


def test_int8_nonfinite_rows_are_multiplied_in_fp64(ft, orc):
    """Inf in a row of op(A) and NaN in a column of op(B): INT8 slices cannot
    carry them, so those rows and columns come from an FP64 product with the
    FP64 oracle's Inf / NaN pattern; every other element keeps the emulated
    value (within its bound of the exact splitting of the finite data)."""
    M, N, K, S = 256, 200, 300, 5
    A, B, C, ar, br = _problem("N", "N", M, N, K, seed=13)
    A[7, 40] = float("inf")        # op(A)(40, 7)
    B[150, 3] = float("nan")       # op(B)(3, 150)
    got, rep = _run(ft, "N", "N", M, N, K, 1.0, 0.5, A, B, C, ar, br, S, 0)
    opA, opB = _ops("N", "N", A, B, ar, br)
    ref, E = orc.gemm("N", "N", 1.0, opA, opB, 0.5, C.T.numpy(), want_E=True)
    bad = np.zeros((M, N), bool); bad[40, :] = True; bad[:, 150] = True
    np.testing.assert_array_equal(np.isnan(got[bad]), np.isnan(ref[bad]))
    np.testing.assert_array_equal(np.isinf(got[bad]), np.isinf(ref[bad]))
    fin = bad & np.isfinite(ref)
    assert np.all(np.abs(got[fin] - ref[fin]) <= orc.parity_tol(K, E)[fin])
    assert np.isfinite(got[~bad]).all()
    sa, sb = _scales(np.nan_to_num(opA, posinf=0), np.nan_to_num(opB))
    split_bound = np.outer(sa, sb) * K * (S + 4) * 2.0 ** (-W * S)
    assert np.all((np.abs(got - ref) <= orc.parity_tol(K, E) + split_bound)[~bad])


def test_int8_engine_argument_rules(ft):
    """FP32 checksums (ft = 1) are not offered with INT8 slices; the plain
    BF16 form runs on the mma.sync kernel as on engine 1."""
    A, B, C, ar, br = _problem("N", "N", 64, 64, 64, seed=3)
    dC = C.cuda()
    rc, _ = ft.ftgemm_d_split("N", "N", 64, 64, 64, 1.0, A.cuda(), 64, B.cuda(), 64, 0.0, dC, 64, nslices=4, ft=1,
                              report=False)
    assert rc == -15
    rc, _ = ft.ftgemm_d_split("N", "N", 64, 64, 64, 1.0, A.cuda(), 64, B.cuda(), 64, 0.0, dC, 64, nslices=0, ft=1)
    assert rc == 0
