"""The plain BF16 form with fault tolerance (ftgemm_d_split, nslices = 0,
ft = 1) against the oracle, through the C ABI.

The form: op(A) and op(B) rounded to bf16, products accumulated in FP32 on
the tensor cores, out = alpha acc + beta C in FP64.  Its checksums are
carried in FP32 and verified in FP64; a flagged element is recomputed in
FP64 from the same bf16 operands (the form's own value, without its FP32
accumulation error).  On the tcgen05 engines the predicted checksums are
tensor-core products of the checksum vectors' two bf16 pieces; on the
mma.sync engine they are summed from the staged slices on the CUDA cores.

Tolerances (stated, from the oracle):
  parity with oracle.bf16_gemm (the FP64 product of the rounded operands):
  1.01 |alpha| e32(K) |A~||B~| + the FP64 parity bound, e32 the FP32
  accumulation bound oracle.split.bf16_acc_bound;
  detection: oracle.split.bf16_tau per row and column, with a guard band of
  8x on each side (the mma.sync engine's own threshold lies inside it).
"""
from __future__ import annotations

import struct

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
    ftgemm.ftgemm_set_split_engine(0)
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_split_engine(0)


def _problem(ta, tb, M, N, K, seed, dist="uniform"):
    from paper_2305_02444_gb300 import inputs
    ar, ac = (M, K) if ta == "N" else (K, M)
    br, bc = (K, N) if tb == "N" else (N, K)
    A = inputs.matrix(ar, ac, seed, dist)
    B = inputs.matrix(br, bc, seed + 1, dist)
    C = inputs.matrix(M, N, seed + 2, dist)
    return A, B, C, ar, br


def _ops(ta, tb, A, B, ar, br):
    opA = A[:, :ar].T.numpy()
    opB = B[:, :br].T.numpy()
    return (opA if ta == "N" else opA.T), (opB if tb == "N" else opB.T)


def _run(ft, engine, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br, ftflag=1, loc_cap=4096):
    assert ft.ftgemm_set_split_engine(engine) == 0
    try:
        dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
        rc, rep = ft.ftgemm_d_split(ta, tb, M, N, K, alpha, dA, ar, dB, br, beta, dC, M, nslices=0, ft=ftflag,
                                    loc_cap=loc_cap)
        torch.cuda.synchronize()
    finally:
        ft.ftgemm_set_split_engine(0)
    assert rc == 0, ft.ftgemm_strerror(rc)
    return dC.cpu().T.numpy(), rep


def _tol(orc, K, alpha, opA, opB, E):
    from oracle import split
    absab = np.abs(split.bf16_round(opA)) @ np.abs(split.bf16_round(opB))
    return 1.01 * abs(alpha) * split.bf16_acc_bound(K) * absab + orc.parity_tol(K, E)


ENGINES = (0, 2, 1)   # persistent tcgen05 (default), tcgen05 one CTA per tile, mma.sync


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("M,N,K,alpha,beta", [(300, 260, 1000, 1.5, 0.5), (130, 385, 64, -0.75, 0.0),
                                              (256, 128, 5000, 1.0, 1.0)])
def test_plain_ft_parity_no_false_positives(ft, orc, engine, ta, tb, M, N, K, alpha, beta):
    """Ragged tiles, a single k-slab, long K and beta = 0: within the FP32
    accumulation bound of the exact product of the rounded operands, and no
    check raised."""
    A, B, C, ar, br = _problem(ta, tb, M, N, K, seed=M + N + K)
    if beta == 0.0:
        C = torch.full_like(C, float("nan"))          # beta == 0 never reads C
    got, rep = _run(ft, engine, ta, tb, M, N, K, alpha, beta, A, B, C, ar, br)
    opA, opB = _ops(ta, tb, A, B, ar, br)
    ref, E = orc.bf16_gemm("N", "N", alpha, opA, opB, beta, np.nan_to_num(C.T.numpy()), want_E=True)
    assert np.all(np.abs(got - ref) <= _tol(orc, K, alpha, opA, opB, E))
    for k in ("flagged_rows", "flagged_cols", "detected", "unverifiable", "checksum_only"):
        assert rep[k] == 0, (k, rep)


def test_plain_ft_tcgen05_engines_give_the_same_bits(ft, orc):
    """The two tcgen05 engines run the same MMAs in the same order, so their
    FP32 accumulators and outputs are equal bit for bit, with checks or
    without; the checked form writes the same values as the unchecked one."""
    M, N, K = 384, 300, 777
    A, B, C, ar, br = _problem("N", "T", M, N, K, seed=5)
    outs = {(e, f): _run(ft, e, "N", "T", M, N, K, 1.25, -0.5, A, B, C, ar, br, ftflag=f)[0]
            for e in (0, 2) for f in (0, 1)}
    base = outs[(0, 1)]
    for g in outs.values():
        np.testing.assert_array_equal(g, base)


def _flip(x, bit):
    u = struct.unpack("<Q", struct.pack("<d", x))[0] ^ (1 << bit)
    return struct.unpack("<d", struct.pack("<Q", u))[0]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("dist", ["uniform", "loguniform"])
def test_plain_ft_injection_classified_by_the_oracle(ft, orc, engine, dist):
    """Seeded flips of the FP64 value of the FP32 accumulator (every bit
    range, many tiles): each is classified by the oracle's own accumulator
    value (the exact product of the rounded operands) against bf16_tau of its
    row and column; every flip clearly above is detected, located and
    corrected to the oracle's value within the element bound, none clearly
    below is counted, and detected = above + the band flips found.  The log
    records the value each flip changed, within the FP32 accumulation bound
    of the oracle's."""
    from oracle import split
    M, N, K = 512, 384, 1000
    alpha, beta = 1.5, 0.5
    A, B, C, ar, br = _problem("N", "N", M, N, K, seed=41, dist=dist)
    nflips = 120
    assert ft.ftgemm_set_injection(mode=1, seed=2024 + engine, count=nflips) == 0
    try:
        got, rep = _run(ft, engine, "N", "N", M, N, K, alpha, beta, A, B, C, ar, br)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert len(log) == nflips and all(L["applied"] == 1 for L in log)
    opA, opB = _ops("N", "N", A, B, ar, br)
    a, b = split.bf16_round(opA), split.bf16_round(opB)
    Cin = C.T.numpy()
    V = orc.gemm("N", "N", 1.0, a, b, 0.0, np.zeros((M, N)))[0]       # the oracle's accumulator values
    ref, E = orc.bf16_gemm("N", "N", alpha, opA, opB, beta, Cin, want_E=True)
    tol = _tol(orc, K, alpha, opA, opB, E)
    enc = orc.encode_operands("N", "N", M, N, K, a, b, BM, BN)
    absab = np.abs(a) @ np.abs(b)
    e32 = split.bf16_acc_bound(K)
    above, band, below = set(), set(), set()
    extra = {}
    for L in log:
        i, j, bit = L["row"], L["col"], L["bit"]
        assert L["kstep"] == 0 and L["kfirst"] == 0
        assert abs(L["before"] - V[i, j]) <= 1.01 * e32 * absab[i, j] + 1e-300
        assert _flip(L["before"], bit) == L["after"] or np.isnan(L["after"])
        d = _flip(float(V[i, j]), bit) - float(V[i, j])
        eff = abs(alpha * d) if np.isfinite(d) else np.inf
        I, J = i // BM, j // BN
        cols = slice(J * BN, min(N, (J + 1) * BN)); rows = slice(I * BM, min(M, (I + 1) * BM))
        tr = split.bf16_tau(K, cols.stop - cols.start, alpha, enc.babsmax[J], enc.arowabs[i], beta,
                            float(np.abs(Cin[i, cols]).sum()))
        tc = split.bf16_tau(K, rows.stop - rows.start, alpha, enc.aabsmax[I], enc.bcolabs[j], beta,
                            float(np.abs(Cin[rows, j]).sum()))
        if eff > 8 * max(tr, tc):
            above.add((i, j))
        elif eff < min(tr, tc) / 8:
            below.add((i, j))
            extra[(i, j)] = extra.get((i, j), 0.0) + eff
        else:
            band.add((i, j))
            extra[(i, j)] = extra.get((i, j), 0.0) + eff
    assert len(above) >= 5 and len(below) >= 5, (len(above), len(band), len(below))
    located = {(l[0], l[1]) for l in rep["locs"]}
    assert above <= located
    assert not (below - above - band) & located
    assert rep["detected"] == len(located) == len(above) + len(band & located)
    assert rep["corrected"] == rep["detected"] and rep["checksum_only"] == 0
    for (i, j) in above:
        assert abs(got[i, j] - ref[i, j]) <= tol[i, j], (i, j, got[i, j], ref[i, j])
    for (i, j), e in extra.items():
        if (i, j) not in above:
            assert abs(got[i, j] - ref[i, j]) <= tol[i, j] + 2 * e
    mask = np.ones((M, N), bool)
    for (i, j) in above | band | below:
        mask[i, j] = False
    assert np.all(np.abs(got - ref)[mask] <= tol[mask])


def test_plain_ft_nonfinite_inputs_are_unverifiable(ft, orc):
    """An Inf in op(A) makes its tile row's checksums non-finite: those rows
    and columns are counted unverifiable, nothing is flagged or rewritten,
    and the rest of C is the plain product."""
    M, N, K = 256, 256, 300
    A, B, C, ar, br = _problem("N", "N", M, N, K, seed=8)
    A[3, 10] = float("inf")             # op(A)(10, 3): row 10 of tile row 0
    got, rep = _run(ft, 0, "N", "N", M, N, K, 1.0, 1.0, A, B, C, ar, br)
    assert rep["unverifiable"] > 0 and rep["detected"] == 0
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0
    opA, opB = _ops("N", "N", A, B, ar, br)
    ref, E = orc.bf16_gemm("N", "N", 1.0, opA, opB, 1.0, C.T.numpy(), want_E=True)
    fin = np.isfinite(ref)
    assert np.all(np.abs(got - ref)[fin] <= _tol(orc, K, 1.0, opA, opB, E)[fin])
