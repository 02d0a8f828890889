"""The two correction rules of the FP64 FT-GEMM kernels against the oracle.

- rule 0 (default): every located element is recomputed from the original
  operands, so the output meets the element-wise parity bound;
- rule 1 (FT-BLAS's, ftgemm_set_correction(1)): with one flagged row and one
  flagged column in a tile, the intersection is corrected by subtracting the
  column's checksum residual.  Its error is that of the checksum sums: the
  test allows the column's detection threshold (the oracle's tau for that
  column) on top of the parity bound.  Huge or non-finite faults end up
  recomputed (agreement test, non-finite residual, re-verification).
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BM = BN = 128


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_02444_gb300 import build
    build.build()
    from paper_2305_02444_gb300 import ftgemm
    ftgemm.lib()
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_correction(0)
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_correction(0)


def problem(M, N, K, seed):
    from paper_2305_02444_gb300 import inputs
    return inputs.matrix(M, K, seed), inputs.matrix(K, N, seed + 1), inputs.matrix(M, N, seed + 2)


def run(ft, rule, A, B, C, M, N, K, alpha, beta, flips):
    dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
    assert ft.ftgemm_set_correction(rule) == 0
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        rc, rep = ft.ftgemm_d("N", "N", M, N, K, alpha, dA, M, dB, K, beta, dC, M, loc_cap=256)
    finally:
        ft.ftgemm_set_injection(mode=0)
        ft.ftgemm_set_correction(0)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    return dC.cpu().T.numpy(), rep


def column_tau(orc, A, B, C, K, alpha, beta, i, j):
    a, b, c = A.T.numpy(), B.T.numpy(), C.T.numpy()
    M, N = a.shape[0], b.shape[1]
    enc = orc.encode_operands("N", "N", M, N, K, a, b, BM, BN)
    I = i // BM
    rows = slice(I * BM, min(M, (I + 1) * BM))
    return orc.tau(K, rows.stop - rows.start, alpha, enc.bcolabs[j], enc.aabsmax[I], beta,
                   np.abs(c[rows, j]).sum())


def test_subtraction_rule_on_moderate_faults(ft, orc):
    """Exponent bits 52-54 of an accumulator (its value times 2^+-1 .. 2^+-4),
    one fault in each of four tiles: rule 1 corrects each by subtraction
    (location kind 3) within the column threshold; rule 0 recomputes them
    (kind 0) to the element bound."""
    M = N = 256
    K = 512
    alpha, beta = 1.5, 0.5
    A, B, C = problem(M, N, K, seed=71)
    flips = [(10, 20, 31, 52), (200, 30, 5, 53), (40, 150, 20, 54), (130, 140, 10, 52)]
    ref, E = orc.gemm("N", "N", alpha, A.T.numpy(), B.T.numpy(), beta, C.T.numpy(), want_E=True)
    tol = orc.parity_tol(K, E)

    out0, rep0 = run(ft, 0, A, B, C, M, N, K, alpha, beta, flips)
    assert rep0["detected"] == 4 and rep0["corrected"] == 4
    assert sorted(l[:2] for l in rep0["locs"]) == sorted((i, j) for i, j, _, _ in flips)
    assert {l[3] for l in rep0["locs"]} == {0}
    assert np.all(np.abs(out0 - ref) <= tol)

    out1, rep1 = run(ft, 1, A, B, C, M, N, K, alpha, beta, flips)
    assert rep1["detected"] == 4 and rep1["corrected"] == 4 and rep1["recomputed"] == 0
    assert sorted(l[:2] for l in rep1["locs"]) == sorted((i, j) for i, j, _, _ in flips)
    assert {l[3] for l in rep1["locs"]} == {3}
    loose = tol.copy()
    for i, j, _, _ in flips:
        loose[i, j] += column_tau(orc, A, B, C, K, alpha, beta, i, j)
    assert np.all(np.abs(out1 - ref) <= loose)
    # elsewhere both rules leave the same bits
    mask = np.ones_like(out0, dtype=bool)
    for i, j, _, _ in flips:
        mask[i, j] = False
    np.testing.assert_array_equal(out0[mask], out1[mask])


def test_subtraction_rule_falls_back_for_huge_faults(ft, orc):
    """The top exponent bit (bit 62) makes an accumulator huge, Inf or NaN:
    the subtraction cannot restore it (non-finite residual, or the element's
    true value is lost to absorption), so rule 1 ends with every faulty
    element recomputed and the output within the element bound."""
    M = N = 256
    K = 512
    alpha, beta = 1.0, 1.0
    A, B, C = problem(M, N, K, seed=73)
    flips = [(3, 4, 7, 62), (150, 60, 15, 62), (70, 200, 28, 62)]
    ref, E = orc.gemm("N", "N", alpha, A.T.numpy(), B.T.numpy(), beta, C.T.numpy(), want_E=True)
    out1, rep1 = run(ft, 1, A, B, C, M, N, K, alpha, beta, flips)
    assert np.all(np.abs(out1 - ref) <= orc.parity_tol(K, E))
    located = {l[:2] for l in rep1["locs"]}
    assert {(i, j) for i, j, _, _ in flips} <= located
    assert rep1["detected"] >= 3 and rep1["recomputed"] >= 3
