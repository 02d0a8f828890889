"""Split-precision kernels against the exact evaluation of the same method.

The oracle's split form (the fixed-point splitting of Ozaki, Ogita, Oishi,
Rump 2012: S slices of w bits per entry, the slice pairs with s + t < S)
gives alpha V + beta C rounded once; the kernels differ from it only by
their own FP64 roundings, far below the splitting error that separates both
from the FP64 product at small S.

Tolerances (stated, not tuned):
  emulated: every pair sum over a k-chunk is an exact FP32 integer and
  enters one FP64 sum with its power-of-two weight, at most one addition per
  slice pair and 64-wide k-slab, n = S(S+1)/2 ceil(K/64) in all; the terms'
  magnitudes add up to at most sum_k |a_ik||b_kj| (the digits of an entry
  have its sign), so with the epilogue's two roundings and the oracle's one
      |got - ref| <= 1.02 (n + 4) u E_ij,  E = |alpha||A||B| + |beta||C|;
  plain BF16: the products of bf16 entries are exact, their FP32 sum over K
  is within 2.01 (K + 2) 2^-24 sum_k |bf16(a)||bf16(b)|, plus the FP64
  parity bound of the reference and the epilogue.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U = 2.0 ** -53


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


def problem(ta, tb, M, N, K, seed, dist):
    from paper_2305_02444_gb300 import inputs
    ar, ac = (M, K) if ta == "N" else (K, M)
    br, bc = (K, N) if tb == "N" else (N, K)
    A = inputs.matrix(ar, ac, seed, dist)
    B = inputs.matrix(br, bc, seed + 1, dist)
    C = inputs.matrix(M, N, seed + 2, dist)
    return A, B, C, ar, br


def run(ft, engine, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, S, ftflag):
    ft.ftgemm_set_split_engine(engine)
    try:
        dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
        rc, rep = ft.ftgemm_d_split(ta, tb, M, N, K, alpha, dA, ar, dB, br, beta, dC, M, nslices=S,
                                    ft=ftflag)
        torch.cuda.synchronize()
    finally:
        ft.ftgemm_set_split_engine(0)
    assert rc == 0, ft.ftgemm_strerror(rc)
    return dC.cpu().T.numpy(), rep


def stored(A, rows):
    return A[:, :rows].T.numpy()


def emulated_tol(K, S, E):
    n = S * (S + 1) // 2 * (-(-K // 64))
    return 1.02 * (n + 4) * U * E


# (M, N, K, S, distribution, ft): every shape even (FP64 checksums want even
# leading dimensions), ragged against the 128 x 128 tiles and 64-wide k-slabs;
# w = 7, 7, 8, 5 for these K
CASES = [(200, 136, 300, 1, "uniform", 0), (200, 136, 300, 3, "loguniform", 2),
         (130, 258, 1000, 4, "normal", 2), (256, 130, 200, 5, "loguniform", 2),
         (66, 140, 5000, 2, "uniform", 0)]


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("M,N,K,S,dist,ftflag", CASES)
def test_emulated_equals_exact_emulation(ft, orc, ta, tb, M, N, K, S, dist, ftflag):
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=M + 3 * K + S, dist=dist)
    alpha, beta = 1.5, -0.5
    got, rep = run(ft, 0, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, S, ftflag)
    sA, sB, sC = stored(A, ar), stored(B, br), C.T.numpy()
    ref = orc.split_gemm(ta, tb, alpha, sA, sB, beta, sC, S)
    fp64, E = orc.gemm(ta, tb, alpha, sA, sB, beta, sC, want_E=True)
    tol = emulated_tol(K, S, E)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (err / tol).max()
    # the comparison discriminates: the FP64 product itself (what a kernel
    # keeping one slice more, or none dropped, would approach) lies far outside
    assert (np.abs(fp64 - ref) / tol).max() > 100
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0 and rep["detected"] == 0


@pytest.mark.parametrize("engine,ta,tb,M,N,K,S,dist,ftflag", [
    (1, "N", "N", 256, 130, 200, 7, "uniform", 1),      # mma.sync with FP32 checksums
    (1, "T", "N", 200, 136, 300, 3, "loguniform", 2),   # mma.sync, FP64 checksums
    (6, "N", "T", 256, 258, 300, 3, "loguniform", 2),   # tcgen05 on CTA pairs
    (2, "T", "T", 130, 258, 1000, 4, "normal", 0),      # tcgen05, one CTA per tile
])
def test_other_engines_equal_exact_emulation(ft, orc, engine, ta, tb, M, N, K, S, dist, ftflag):
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=7 * M + K, dist=dist)
    got, rep = run(ft, engine, ta, tb, M, N, K, 1.0, 1.0, A, B, C, ar, br, S, ftflag)
    sA, sB, sC = stored(A, ar), stored(B, br), C.T.numpy()
    ref = orc.split_gemm(ta, tb, 1.0, sA, sB, 1.0, sC, S)
    _, E = orc.gemm(ta, tb, 1.0, sA, sB, 1.0, sC, want_E=True)
    err = np.abs(got - ref)
    tol = emulated_tol(K, S, E)
    assert np.all(err <= tol), (err / tol).max()
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0 and rep["detected"] == 0


@pytest.mark.parametrize("ta,tb,dist", [("N", "N", "uniform"), ("T", "T", "loguniform"),
                                         ("N", "T", "normal")])
def test_plain_bf16_equals_rounded_operand_product(ft, orc, ta, tb, dist):
    """K = 200 (four k-slabs, the last ragged): short enough that the FP32
    accumulation bound stays well below the effect of rounding the inputs."""
    M, N, K = 300, 200, 200
    A, B, C, ar, br = problem(ta, tb, M, N, K, seed=53, dist=dist)
    alpha, beta = 1.25, 0.5
    got, rep = run(ft, 0, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, 0, 0)
    sA, sB, sC = stored(A, ar), stored(B, br), C.T.numpy()
    ref, E = orc.bf16_gemm(ta, tb, alpha, sA, sB, beta, sC, want_E=True)
    hA, hB = orc.bf16_round(sA), orc.bf16_round(sB)
    opA = hA if ta == "N" else hA.T
    opB = hB if tb == "N" else hB.T
    absab = np.abs(opA) @ np.abs(opB)
    tol = abs(alpha) * 2.01 * (K + 2) * 2.0 ** -24 * absab + orc.parity_tol(K, E)
    err = np.abs(got - ref)
    assert np.all(err <= tol), (err / tol).max()
    # and the unrounded FP64 product lies outside (the inputs really are bf16)
    fp64, _ = orc.gemm(ta, tb, alpha, sA, sB, beta, sC)
    assert (np.abs(fp64 - ref) / tol).max() > 10
