"""Parity at full size, in the launch configuration bench.py times.

M = N = K = 8192, alpha = 1.5, beta = 0.5, U[-1,1], NN, one seeded flip per 64
tiles (64 per call).  The oracle cannot run the whole product in a test, so
it checks what it can compute one by one and what holds at any size:
  - sampled full rows and full columns of C against the oracle's DGEMM;
  - every injected element against the oracle's value for that element;
  - the Huang-Abraham invariants e^T C = alpha (e^T A) B + beta e^T C_in and
    C e = alpha A (B e) + beta C_in e over the whole matrix, within the
    two-sided rounding bound (plus the effect of below-threshold flips);
  - the report: every flip clearly above the oracle's threshold is detected,
    located and corrected; none clearly below is counted.
Also: the rank-k update 8192^2 x 256 (sampled + invariants) and 2048^3 in full.
"""
from __future__ import annotations

import math
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
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
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)


def _flip(x, bit):
    u = struct.unpack("<Q", struct.pack("<d", x))[0] ^ (1 << bit)
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def _run(ft, M, N, K, alpha, beta, seed, nflips):
    from paper_2305_02444_gb300 import inputs
    A = inputs.matrix(M, K, seed)
    B = inputs.matrix(K, N, seed + 1)
    C = inputs.matrix(M, N, seed + 2)
    dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
    if nflips:
        assert ft.ftgemm_set_injection(mode=1, seed=seed, count=nflips) == 0
    try:
        rc, rep = ft.ftgemm_d("N", "N", M, N, K, alpha, dA, M, dB, K, beta, dC, M, loc_cap=65536)
        log = ft.ftgemm_injection_log() if nflips else []
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert rc == 0, ft.ftgemm_strerror(rc)
    out = dC.cpu().T.numpy()
    return A.T.numpy(), B.T.numpy(), C.T.numpy(), out, rep, log


def _check_full_size(ft, orc, M, N, K, alpha, beta, seed, nflips, nsample=6):
    A, B, Cin, out, rep, log = _run(ft, M, N, K, alpha, beta, seed, nflips)
    rng = np.random.default_rng(seed)
    flips = orc.random_flips(seed, nflips, M, N, -(-K // 16)) if nflips else np.zeros((0, 4), np.int64)
    got_pos = np.array([[L["row"], L["col"], L["kstep"], L["bit"]] for L in log]).reshape(-1, 4)
    np.testing.assert_array_equal(got_pos, flips)

    # oracle view of each flip: its effect and the thresholds of its row/column
    enc = orc.encode_operands("N", "N", M, N, K, A, B, BM, BN)
    extra = {}
    n_above = n_not_below = 0
    above = set()
    for (i, j, s, bit) in flips.tolist():
        kend = min(K, 16 * (s + 1))
        kf = [L for L in log if (L["row"], L["col"], L["kstep"], L["bit"]) == (i, j, s, bit)][0]["kfirst"]
        part = orc.partial("N", "N", i, j, kend, A, B) if kf == 0 else float(np.dot(A[i, kf:kend], B[kf:kend, j]))
        d = _flip(part, bit) - part
        eff = abs(alpha * d) if math.isfinite(d) else math.inf
        I, J = i // BM, j // BN
        cols = slice(J * BN, min(N, (J + 1) * BN)); rows = slice(I * BM, min(M, (I + 1) * BM))
        tr = orc.tau(K, cols.stop - cols.start, alpha, enc.arowabs[i], enc.babsmax[J], beta,
                     np.abs(Cin[i, cols]).sum())
        tc = orc.tau(K, rows.stop - rows.start, alpha, enc.bcolabs[j], enc.aabsmax[I], beta,
                     np.abs(Cin[rows, j]).sum())
        if eff > 4 * max(tr, tc):
            n_above += 1
            above.add((i, j))
        if not eff < 0.25 * min(tr, tc):
            n_not_below += 1
        if (i, j) not in above:
            extra[(i, j)] = extra.get((i, j), 0.0) + 2 * eff
    assert n_above <= rep["detected"] <= n_not_below, (n_above, rep["detected"], n_not_below)
    assert rep["corrected"] == rep["detected"] and rep["checksum_only"] == 0
    located = {(l[0], l[1]) for l in rep["locs"]}
    assert above <= located

    def row_ref(i):
        r, E = orc.gemm("N", "N", alpha, A[i:i + 1], B, beta, Cin[i:i + 1], want_E=True)
        return r[0], E[0]

    # every injected element
    for (i, j, s, bit) in flips.tolist():
        a = A[i:i + 1]; b = B[:, j:j + 1]
        r, E = orc.gemm("N", "N", alpha, a, b, beta, Cin[i:i + 1, j:j + 1], want_E=True)
        tol = orc.parity_tol(K, E)[0, 0] + extra.get((i, j), 0.0)
        assert abs(out[i, j] - r[0, 0]) <= tol, (i, j, bit, out[i, j], r[0, 0], tol)
    # sampled full rows and columns
    for i in rng.choice(M, nsample, replace=False):
        r, E = row_ref(i)
        tol = orc.parity_tol(K, E)
        for (fi, fj), e in extra.items():
            if fi == i:
                tol[fj] += e
        assert np.all(np.abs(out[i] - r) <= tol), i
    for j in rng.choice(N, nsample, replace=False):
        r, E = orc.gemm("N", "N", alpha, A, B[:, j:j + 1], beta, Cin[:, j:j + 1], want_E=True)
        tol = orc.parity_tol(K, E[:, 0])
        for (fi, fj), e in extra.items():
            if fj == j:
                tol[fi] += e
        assert np.all(np.abs(out[:, j] - r[:, 0]) <= tol), j
    # whole-matrix invariants
    col, row = orc.pred_checksums("N", "N", alpha, A, B, beta, Cin)
    colE, rowE = orc.pred_checksums("N", "N", abs(alpha), np.abs(A), np.abs(B), abs(beta), np.abs(Cin))
    ecol = np.zeros(N); erow = np.zeros(M)
    for (fi, fj), e in extra.items():
        ecol[fj] += e; erow[fi] += e
    assert np.all(np.abs(out.sum(0) - col) <= 2.02 * (K + M + 3) * U * colE + ecol)
    assert np.all(np.abs(out.sum(1) - row) <= 2.02 * (K + N + 3) * U * rowE + erow)
    return rep


def test_bench_configuration_8192(ft, orc):
    rep = _check_full_size(ft, orc, 8192, 8192, 8192, 1.5, 0.5, seed=20230614, nflips=64)
    assert rep["detected"] >= 20


def test_rank_k_update_8192x8192x256(ft, orc):
    _check_full_size(ft, orc, 8192, 8192, 256, 1.5, 0.5, seed=7, nflips=64)


@pytest.mark.parametrize("n", [1024, 2048])
def test_full_oracle_small_squares(ft, orc, n):
    """The two sweep sizes with fewer tiles than 4 per SM (automatic k-split
    with the verifying reduction), against the whole oracle product."""
    A, B, Cin, out, rep, _ = _run(ft, n, n, n, 1.5, 0.5, seed=11, nflips=0)
    ref, E = orc.gemm("N", "N", 1.5, A, B, 0.5, Cin, want_E=True)
    assert np.all(np.abs(out - ref) <= orc.parity_tol(n, E))
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0


def test_wave_tail_split_with_flips(ft, orc):
    """3200^2 x 256: 625 tiles = 4 waves of 152 + 17, so the 17 tail tiles
    (I = 8..24 of tile column 24) split K in two and go through the verifying
    reduction while the others run whole.  Exponent-bit flips in a whole tile
    and in both k-halves of tail tiles are detected, located and corrected;
    the whole product matches the oracle."""
    from paper_2305_02444_gb300 import inputs
    M = N = 3200
    K = 256
    A = inputs.matrix(M, K, 31)
    B = inputs.matrix(K, N, 32)
    C = inputs.matrix(M, N, 33)
    dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
    flips = [(5, 7, 3, 62), (10 * BM + 5, 24 * BN + 3, 2, 62), (20 * BM + 9, 24 * BN + 28, 12, 62)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        rc, rep = ft.ftgemm_d("N", "N", M, N, K, 1.5, dA, M, dB, K, 0.5, dC, M, loc_cap=64)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert rc == 0, ft.ftgemm_strerror(rc)
    assert [L["applied"] for L in log] == [1, 1, 1]
    # tail tiles accumulate each half of K in its own CTA: the flip lands in
    # the half that holds its k-step
    assert [L["kfirst"] for L in log] == [0, 0, 128]
    assert rep["detected"] == 3 and rep["corrected"] == 3 and rep["checksum_only"] == 0
    assert sorted((l[0], l[1]) for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)
    out = dC.cpu().T.numpy()
    ref, E = orc.gemm("N", "N", 1.5, A.T.numpy(), B.T.numpy(), 0.5, C.T.numpy(), want_E=True)
    assert np.all(np.abs(out - ref) <= orc.parity_tol(K, E))
