"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: |C_gpu - C_oracle| <= max(4K, 2K+6) * 2^-53 * E elementwise, with
E = |alpha||op(A)||op(B)| + |beta||C| (the componentwise bound of the target;
for K < 3 the two-sided rounding bound (2K+5)u exceeds 4Ku).  Fault reports
are compared with the oracle's scheme; flips are classified by the oracle's
own accumulator values.
"""
from __future__ import annotations

import itertools
import math
import struct

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BM = BN = 128
KSTEP = 16


@pytest.fixture(scope="module")
def ft():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_02444_gb300 import build
    build.build()
    from paper_2305_02444_gb300 import ftgemm
    ftgemm.lib()
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_splitk(0)
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_splitk(0)


class splitk:
    """Force a k-split setting for a block (0 auto, 1 off, n splits)."""
    def __init__(self, ft, n):
        self.ft, self.n = ft, n

    def __enter__(self):
        assert self.ft.ftgemm_set_splitk(self.n) == 0

    def __exit__(self, *a):
        self.ft.ftgemm_set_splitk(0)


def stored_dims(t, rows_op, cols_op):
    return (rows_op, cols_op) if t == "N" else (cols_op, rows_op)


def make_problem(ta, tb, M, N, K, seed, dist="uniform", pad=(0, 0, 0), c_nan=False):
    from paper_2305_02444_gb300 import inputs
    ar, ac = stored_dims(ta, M, K)
    br, bc = stored_dims(tb, K, N)
    lda, ldb, ldc = max(1, ar) + pad[0], max(1, br) + pad[1], max(1, M) + pad[2]
    A = inputs.matrix(ar, ac, seed, dist, lda)
    B = inputs.matrix(br, bc, seed + 1, dist, ldb)
    C = inputs.matrix(M, N, seed + 2, dist, ldc)
    if c_nan and M > 0 and N > 0:
        C[0, 0] = float("nan")
        C[N - 1, M - 1] = float("inf")
    return dict(ta=ta, tb=tb, M=M, N=N, K=K, A=A, B=B, C=C, lda=lda, ldb=ldb, ldc=ldc, ar=ar, br=br)


def np_logical(st, rows):
    return st[:, :rows].T.numpy()


def run_gpu(ft, P, alpha, beta, noft=False, offset=False, report=True):
    dev = "cuda"
    def up(st):
        if not offset:
            return st.to(dev), 0
        flat = torch.empty(st.numel() + 1, dtype=torch.float64, device=dev)
        flat[1:] = st.reshape(-1).to(dev)
        return flat, 8
    A, oa = up(P["A"]); B, ob = up(P["B"]); C, oc = up(P["C"])
    args = (P["ta"], P["tb"], P["M"], P["N"], P["K"], alpha, A.data_ptr() + oa, P["lda"],
            B.data_ptr() + ob, P["ldb"], beta, C.data_ptr() + oc, P["ldc"])
    if noft:
        rc, rep = ft.ftgemm_d_noft(*args), None
    else:
        rc, rep = ft.ftgemm_d(*args, report=report)
    torch.cuda.synchronize()
    out = C.cpu()
    if offset:
        out = out[1:].reshape(P["C"].shape)
    return rc, rep, out


def oracle_ref(orc, P, alpha, beta):
    ref, E = orc.gemm(P["ta"], P["tb"], alpha, np_logical(P["A"], P["ar"]), np_logical(P["B"], P["br"]),
                      beta, np_logical(P["C"], P["M"]), want_E=True, k=P["K"])
    return ref, E


def assert_parity(orc, P, out, ref, E, extra=None):
    got = np_logical(out, P["M"])
    tol = orc.parity_tol(P["K"], E)
    if extra is not None:
        tol = tol + extra
    both_nan = np.isnan(got) & np.isnan(ref)
    same_inf = np.isinf(got) & np.isinf(ref) & (np.sign(got) == np.sign(ref))
    with np.errstate(invalid="ignore"):   # Inf - Inf where both sides agree on the infinity
        ok = both_nan | same_inf | (np.abs(got - ref) <= tol)
    if not ok.all():
        i, j = np.argwhere(~ok)[0]
        raise AssertionError(f"mismatch at ({i},{j}): gpu {got[i, j]!r} oracle {ref[i, j]!r} tol {tol[i, j]!r}"
                             f" ({(~ok).sum()} bad)")
    # padding rows of C (ldc > M) untouched
    if P["ldc"] > P["M"]:
        pad_in = P["C"][:, P["M"]:]
        pad_out = out[:, P["M"]:]
        assert torch.equal(torch.isnan(pad_in), torch.isnan(pad_out))


CASES = [
    # (M, N, K): several tiles with ragged tails, partial k-steps, degenerate shapes
    (300, 260, 200), (128, 128, 16), (129, 257, 33), (256, 256, 256), (1, 1, 1), (1, 300, 7),
    (300, 1, 50), (17, 19, 1000), (384, 130, 3),
]


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("M,N,K", CASES)
def test_parity_ft_all_layouts(ft, orc, ta, tb, M, N, K):
    P = make_problem(ta, tb, M, N, K, seed=M * 7 + N * 3 + K)
    ref, E = oracle_ref(orc, P, 1.5, 0.5)
    rc, rep, out = run_gpu(ft, P, 1.5, 0.5)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)
    assert rep["detected"] == 0 and rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0
    assert rep["unverifiable"] == 0


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
def test_parity_noft(ft, orc, ta, tb):
    P = make_problem(ta, tb, 300, 260, 200, seed=99)
    ref, E = oracle_ref(orc, P, -0.75, 2.0)
    rc, _, out = run_gpu(ft, P, -0.75, 2.0, noft=True)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)


@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (1.5, 0.5), (-0.75, 0.0), (2.0, -1.0), (0.0, 0.5),
                                        (0.0, 0.0), (1.0, 0.0)])
def test_alpha_beta_and_nan_in_c(ft, orc, alpha, beta):
    P = make_problem("N", "N", 200, 150, 70, seed=5, c_nan=True)
    ref, E = oracle_ref(orc, P, alpha, beta)
    rc, rep, out = run_gpu(ft, P, alpha, beta)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)
    if beta == 0.0:
        assert np.isfinite(np_logical(out, 200)).all()   # C is not read when beta == 0


@pytest.mark.parametrize("dist", ["normal", "loguniform"])
def test_parity_distributions(ft, orc, dist):
    P = make_problem("T", "N", 257, 131, 500, seed=21, dist=dist)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    rc, rep, out = run_gpu(ft, P, 1.0, 1.0)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0


def test_quick_returns(ft, orc):
    for (M, N, K) in [(0, 5, 5), (5, 0, 5), (5, 5, 0)]:
        P = make_problem("N", "N", M, N, K, seed=3)
        ref, E = oracle_ref(orc, P, 1.5, 0.5)
        rc, rep, out = run_gpu(ft, P, 1.5, 0.5)
        assert rc == 0
        if M and N:
            assert_parity(orc, P, out, ref, E)


@pytest.mark.parametrize("pad,offset", [((1, 0, 0), False), ((0, 3, 1), False), ((2, 2, 2), True), ((0, 0, 0), True)])
def test_unaligned_operands(ft, orc, pad, offset):
    """Odd leading dimensions and 8-byte-offset base pointers (TMA needs
    16-byte rows: the library copies such operands to aligned workspace)."""
    for ta, tb in [("N", "N"), ("T", "T")]:
        P = make_problem(ta, tb, 131, 77, 45, seed=11, pad=pad)
        ref, E = oracle_ref(orc, P, 1.25, -0.5)
        rc, rep, out = run_gpu(ft, P, 1.25, -0.5, offset=offset)
        assert rc == 0
        assert_parity(orc, P, out, ref, E)
        rc, _, out = run_gpu(ft, P, 1.25, -0.5, offset=offset, noft=True)
        assert rc == 0
        assert_parity(orc, P, out, ref, E)


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("M,N,K", [(300, 200, 77), (2085, 1103, 3001)])
def test_encode_operands_vs_oracle(ft, orc, ta, tb, M, N, K):
    """The operand checksum pass against the oracle's, both operand layouts.
    The larger shape splits each 128-wide group into several chunks, so the
    group's finish (the last block to complete sums the chunks' partials)
    runs over many partials; the ragged sizes leave partial groups."""
    P = make_problem(ta, tb, M, N, K, seed=8)
    nI, nJ = -(-M // BM), -(-N // BN)
    d = dict(acs=(nI, K), aabsmax=(nI,), arowabs=(M,), bcs=(nJ, K), babsmax=(nJ,), bcolabs=(N,))
    outs = {k: torch.zeros(v, dtype=torch.float64, device="cuda") for k, v in d.items()}
    A, B = P["A"].cuda(), P["B"].cuda()
    rc = ft.ftgemm_encode_operands(ta, tb, M, N, K, A, P["lda"], B, P["ldb"], outs["acs"], outs["aabsmax"],
                                   outs["arowabs"], outs["bcs"], outs["babsmax"], outs["bcolabs"])
    torch.cuda.synchronize()
    assert rc == 0
    e = orc.encode_operands(ta, tb, M, N, K, np_logical(P["A"], P["ar"]), np_logical(P["B"], P["br"]), BM, BN)
    u = 2.0 ** -53
    opA = np_logical(P["A"], P["ar"]); opA = opA if ta == "N" else opA.T
    opB = np_logical(P["B"], P["br"]); opB = opB if tb == "N" else opB.T
    for I in range(nI):
        bound = 2 * 130 * u * np.abs(opA[I * BM:(I + 1) * BM]).sum(0)
        assert np.all(np.abs(outs["acs"][I].cpu().numpy() - e.acs[I]) <= bound)
    for J in range(nJ):
        bound = 2 * 130 * u * np.abs(opB[:, J * BN:(J + 1) * BN]).sum(1)
        assert np.all(np.abs(outs["bcs"][J].cpu().numpy() - e.bcs[J]) <= bound)
    rel = 2 * (K + 130) * u
    for k in ("aabsmax", "arowabs", "babsmax", "bcolabs"):
        np.testing.assert_allclose(outs[k].cpu().numpy(), getattr(e, k), rtol=rel, atol=0)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "T")])
@pytest.mark.parametrize("sa,sb", [(2.0 ** 140, 2.0 ** -140), (2.0 ** -400, 2.0 ** -400)])
def test_thresholds_at_the_edges_of_the_fp32_range(ft, orc, ta, tb, sa, sb):
    """The checksum pass of a call keeps the thresholds' absolute sums as FP32
    upper bounds and takes a group's again in FP64 where FP32's range would
    overflow them (operands near 2^140) or leave them loose (every |x| near
    2^-400, products near 2^-800).  With beta = 0 (C's own absolute sums are
    the epilogue's) the call stays verifiable, raises no check without
    faults, and detects, locates and corrects an exponent flip; K = 700 gives
    every group several chunks, both layouts both shapes of the pass."""
    P = make_problem(ta, tb, 300, 260, 700, seed=31)
    P["A"].mul_(sa)
    P["B"].mul_(sb)
    ref, E = oracle_ref(orc, P, 1.0, 0.0)
    with splitk(ft, 1):
        rc, rep, out = run_gpu(ft, P, 1.0, 0.0)
    assert rc == 0
    assert rep["unverifiable"] == 0 and rep["detected"] == 0 and rep["flagged_rows"] == 0, rep
    assert_parity(orc, P, out, ref, E)
    rc, rep, out, log = run_injected(ft, P, 1.0, 0.0, [(100, 50, 3, 61)])
    assert rc == 0 and log[0]["applied"] == 1
    assert rep["unverifiable"] == 0 and rep["detected"] == 1 and rep["corrected"] == 1, rep
    assert tuple(rep["locs"][0][:2]) == (100, 50)
    assert_parity(orc, P, out, ref, E)


# ------------------------------------------------------------------------------ injection

def flip_value(x: float, bit: int) -> float:
    u = struct.unpack("<Q", struct.pack("<d", x))[0] ^ (1 << bit)
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def run_injected(ft, P, alpha, beta, flips, nsplit=1):
    """Injected call; nsplit=1 keeps whole-K accumulators, as in the oracle's scheme."""
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        with splitk(ft, nsplit):
            rc, rep, out = run_gpu(ft, P, alpha, beta)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    return rc, rep, out, log


def tile_taus(orc, P, alpha, beta, i, j):
    """Oracle thresholds of row i / column j in their tile."""
    M, N, K = P["M"], P["N"], P["K"]
    opA = np_logical(P["A"], P["ar"]); opA = opA if P["ta"] == "N" else opA.T
    opB = np_logical(P["B"], P["br"]); opB = opB if P["tb"] == "N" else opB.T
    C = np_logical(P["C"], M)
    I, J = i // BM, j // BN
    rows = slice(I * BM, min(M, (I + 1) * BM)); cols = slice(J * BN, min(N, (J + 1) * BN))
    mI, nJ = rows.stop - rows.start, cols.stop - cols.start
    cterm = (lambda v: np.abs(v).sum()) if beta != 0 else (lambda v: 0.0)
    tr = orc.tau(K, nJ, alpha, np.abs(opA[i]).sum(), np.abs(opB[:, cols]).sum(1).max(), beta, cterm(C[i, cols]))
    tc = orc.tau(K, mI, alpha, np.abs(opB[:, j]).sum(), np.abs(opA[rows]).sum(0).max(), beta, cterm(C[rows, j]))
    return tr, tc


def check_log_against_oracle(orc, P, flips, log):
    assert len(log) == len(flips)
    opA = np_logical(P["A"], P["ar"]); opB = np_logical(P["B"], P["br"])
    for (i, j, s, bit), L in zip(flips, log):
        assert (L["row"], L["col"], L["kstep"], L["bit"]) == (i, j, s, bit)
        assert L["applied"] == 1
        assert struct.unpack("<Q", struct.pack("<d", L["before"]))[0] ^ \
            struct.unpack("<Q", struct.pack("<d", L["after"]))[0] == 1 << bit
        kend = min(P["K"], KSTEP * (s + 1))
        kf = L["kfirst"]
        assert 0 <= kf < kend and kf % KSTEP == 0
        a_row = (opA if P["ta"] == "N" else opA.T)[i, kf:kend]
        b_col = (opB if P["tb"] == "N" else opB.T)[kf:kend, j]
        if kf == 0:
            part = orc.partial(P["ta"], P["tb"], i, j, kend, opA, opB)
        else:   # the accumulator of a k-split holds products kf .. kend-1
            part = float(np.dot(a_row, b_col))
        bound = 2 * (kend - kf + 1) * 2.0 ** -53 * np.abs(a_row * b_col).sum()
        assert abs(L["before"] - part) <= bound


def test_single_flip_config1(ft, orc):
    """M=N=K=256, U[-1,1], alpha=beta=1: one seeded high-bit flip is detected,
    located and corrected to the oracle bound."""
    P = make_problem("N", "N", 256, 256, 256, seed=2024)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    flips = [(77, 200, 5, 56)]
    rc, rep, out, log = run_injected(ft, P, 1.0, 1.0, flips)
    assert rc == 0
    check_log_against_oracle(orc, P, flips, log)
    assert rep["detected"] == 1 and rep["corrected"] == 1
    assert rep["locs"][0][:2] == (77, 200) and rep["locs"][0][3] == 0
    assert_parity(orc, P, out, ref, E)


def test_every_bit_one_position(ft, orc):
    """Bits 0..62 at one position: clearly-above-threshold flips are detected
    and corrected, clearly-below ones leave the tile unflagged, and the
    oracle's scheme agrees on the counts."""
    P = make_problem("N", "T", 256, 256, 256, seed=7)
    alpha, beta = 1.5, 0.5
    ref, E = oracle_ref(orc, P, alpha, beta)
    i, j, s = 130, 5, 9
    tr, tc = tile_taus(orc, P, alpha, beta, i, j)
    opA = np_logical(P["A"], P["ar"]); opB = np_logical(P["B"], P["br"])
    part = orc.partial("N", "T", i, j, KSTEP * (s + 1), opA, opB)
    n_above = n_below = 0
    for bit in range(63):
        rc, rep, out, log = run_injected(ft, P, alpha, beta, [(i, j, s, bit)])
        assert rc == 0
        d = flip_value(part, bit) - part
        eff = abs(alpha * d) if math.isfinite(d) else math.inf
        if eff > 4 * max(tr, tc):
            n_above += 1
            assert rep["detected"] == 1, (bit, rep)
            assert rep["locs"][0][:2] == (i, j)
            assert_parity(orc, P, out, ref, E)
        elif eff < 0.25 * min(tr, tc):
            n_below += 1
            assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0 and rep["detected"] == 0
            extra = np.zeros_like(E); extra[i, j] = 2 * eff
            assert_parity(orc, P, out, ref, E, extra=extra)
        else:
            extra = np.zeros_like(E); extra[i, j] = 2 * eff
            assert_parity(orc, P, out, ref, E, extra=extra)
        # same flip through the oracle's scheme
        r = orc.ft_gemm("N", "T", alpha, opA, opB, beta, np_logical(P["C"], 256), BM=BM, BN=BN, BK=KSTEP,
                        flips=np.array([[i, j, s, bit]]))
        if eff > 4 * max(tr, tc) or eff < 0.25 * min(tr, tc):
            for k in ("detected", "flagged_rows", "flagged_cols", "checksum_only"):
                assert rep[k] == r.counts[k], (bit, k, rep[k], r.counts[k])
    assert n_above > 20 and n_below > 10


def test_multiple_flips_tiles_and_fallback(ft, orc):
    P = make_problem("T", "N", 300, 270, 180, seed=31)
    alpha, beta = 1.5, 0.5
    ref, E = oracle_ref(orc, P, alpha, beta)
    cases = [
        [(1, 2, 0, 55), (5, 6, 3, 58)],                       # one tile, distinct rows/cols
        [(3, 2, 0, 59), (3, 90, 5, 59)],                      # one tile, same row
        [(q, q, 2, 60) for q in range(9)],                    # 81 intersections > 64: segment fallback
        [(1, 1, 0, 61), (200, 260, 10, 61), (299, 269, 11, 57)],  # three tiles, ragged corner
    ]
    for flips in cases:
        rc, rep, out, log = run_injected(ft, P, alpha, beta, flips)
        assert rc == 0
        check_log_against_oracle(orc, P, flips, log)
        assert rep["detected"] == len(flips), (flips, rep)
        assert sorted(l[:2] for l in rep["locs"]) == sorted((i, j) for i, j, _, _ in flips)
        assert_parity(orc, P, out, ref, E)
        r = orc.ft_gemm("T", "N", alpha, np_logical(P["A"], P["ar"]), np_logical(P["B"], P["br"]), beta,
                        np_logical(P["C"], 300), BM=BM, BN=BN, BK=KSTEP, flips=np.array(flips))
        assert r.counts["detected"] == rep["detected"]
        assert sorted(l[3] for l in r.locs) == sorted(l[3] for l in rep["locs"])


def test_nonfinite_flips(ft, orc):
    P = make_problem("N", "N", 256, 256, 64, seed=41)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    for bit in (62, 61, 60, 52):
        flips = [(10, 20, 1, bit), (140, 150, 3, bit)]
        rc, rep, out, log = run_injected(ft, P, 1.0, 1.0, flips)
        assert rc == 0
        assert rep["detected"] == 2
        assert_parity(orc, P, out, ref, E)


def test_random_mode_matches_published_generator(ft, orc):
    M, N, K = 256, 384, 96
    P = make_problem("N", "N", M, N, K, seed=51)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    seed, count = 0xC0FFEE, 12
    assert ft.ftgemm_set_injection(mode=1, seed=seed, count=count) == 0
    try:
        rc, rep, out = run_gpu(ft, P, 1.0, 1.0)   # automatic k-split: kfirst may be > 0
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert rc == 0
    expect = orc.random_flips(seed, count, M, N, -(-K // KSTEP))
    got = np.array([[L["row"], L["col"], L["kstep"], L["bit"]] for L in log])
    np.testing.assert_array_equal(got, expect)
    check_log_against_oracle(orc, P, [tuple(x) for x in expect.tolist()], log)


def test_bounded_wait_times_out_and_context_survives(ft, orc):
    rc = ft.ftgemm_selftest_wait_timeout(2_000_000)  # 2 ms on a barrier nothing completes
    assert rc == ft.ERR_TIMEOUT
    P = make_problem("N", "N", 130, 140, 150, seed=61)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    rc, rep, out = run_gpu(ft, P, 1.0, 1.0)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)


def test_host_buffers_api(ft, orc):
    P = make_problem("T", "T", 200, 190, 180, seed=71, pad=(1, 2, 3))
    ref, E = oracle_ref(orc, P, 1.5, 0.5)
    A, B = P["A"].pin_memory(), P["B"].pin_memory()
    C = P["C"].clone().pin_memory()
    rc, rep = ft.ftgemm_d_host("T", "T", 200, 190, 180, 1.5, A, P["lda"], B, P["ldb"], 0.5, C, P["ldc"])
    assert rc == 0 and rep["detected"] == 0
    assert_parity(orc, P, C, ref, E)


def test_host_buffers_beta_zero_leaves_padding(ft, orc):
    """beta = 0 uploads no C, yet rows M..ldc-1 of the caller's C must come
    back as they were: a first call with finite padding and beta != 0 leaves
    that padding in the device workspace, which the second call (NaN
    padding, beta = 0) must not copy back."""
    P = make_problem("N", "N", 150, 70, 90, seed=73, pad=(0, 0, 5))
    A, B = P["A"].pin_memory(), P["B"].pin_memory()
    C1 = P["C"].clone()
    C1[:, P["M"]:] = 7.0
    rc, _ = ft.ftgemm_d_host("N", "N", 150, 70, 90, 1.0, A, P["lda"], B, P["ldb"], 0.5, C1.pin_memory(), P["ldc"])
    assert rc == 0
    ref, E = oracle_ref(orc, P, 1.5, 0.0)
    C = P["C"].clone().pin_memory()
    rc, rep = ft.ftgemm_d_host("N", "N", 150, 70, 90, 1.5, A, P["lda"], B, P["ldb"], 0.0, C, P["ldc"])
    assert rc == 0 and rep["detected"] == 0
    assert_parity(orc, P, C, ref, E)


# ------------------------------------------------------------------------------ split-K

@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("nsplit", [1, 2, 3, 7, 16])
def test_splitk_forced_parity(ft, orc, ta, tb, nsplit):
    """Forced k-splits (partial tiles + verifying reduction) match the oracle,
    FT and unprotected, ragged tiles, K not a multiple of the split."""
    P = make_problem(ta, tb, 300, 260, 700, seed=nsplit * 13 + 1)
    ref, E = oracle_ref(orc, P, 1.5, 0.5)
    with splitk(ft, nsplit):
        rc, rep, out = run_gpu(ft, P, 1.5, 0.5)
        assert rc == 0
        assert_parity(orc, P, out, ref, E)
        assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0
        rc, _, out = run_gpu(ft, P, 1.5, 0.5, noft=True)
        assert rc == 0
        assert_parity(orc, P, out, ref, E)


def test_splitk_auto_small_square(ft, orc):
    """1024^3 gives 64 tiles on 152 SMs: the automatic split is used."""
    P = make_problem("N", "N", 1024, 1024, 1024, seed=77)
    ref, E = oracle_ref(orc, P, 1.5, 0.5)
    n0 = ft.ftgemm_launch_count()
    rc, rep, out = run_gpu(ft, P, 1.5, 0.5)
    assert rc == 0
    # checksum pass (one kernel per operand); partials, with the C-side checksum sums beside them;
    # the partials' sum over the whole GPU; verifying reduction
    assert ft.ftgemm_launch_count() - n0 == 2 + 4
    assert_parity(orc, P, out, ref, E)
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0


@pytest.mark.parametrize("nsplit", [4, 32])
def test_splitk_injection(ft, orc, nsplit):
    """Flips in different k-splits: each flips the accumulator of its split
    (kfirst in the log); clearly-above-threshold ones are detected and
    corrected to the parity bound by the reduction's verification."""
    P = make_problem("N", "T", 256, 256, 512, seed=91)
    alpha, beta = 1.5, 0.5
    ref, E = oracle_ref(orc, P, alpha, beta)
    flips = [(3, 5, 0, 58), (100, 200, 9, 60), (200, 40, 17, 55), (255, 255, 31, 61), (130, 7, 22, 3)]
    rc, rep, out, log = run_injected(ft, P, alpha, beta, flips, nsplit=nsplit)
    assert rc == 0
    check_log_against_oracle(orc, P, flips, log)
    ks = -(-32 // nsplit) * KSTEP
    assert all(L["kfirst"] == (L["kstep"] * KSTEP // ks) * ks for L in log)
    opA = np_logical(P["A"], P["ar"]); opB = np_logical(P["B"], P["br"]).T
    expect_detected, extra = set(), np.zeros_like(E)
    for (i, j, s, bit), L in zip(flips, log):
        d = L["after"] - L["before"]
        eff = abs(alpha * d) if math.isfinite(d) else math.inf
        tr, tc = tile_taus(orc, P, alpha, beta, i, j)
        if eff > 4 * max(tr, tc):
            expect_detected.add((i, j))
        else:
            extra[i, j] = 2 * eff
    got = {l[:2] for l in rep["locs"]}
    assert expect_detected <= got
    assert_parity(orc, P, out, ref, E, extra=extra)


# ------------------------------------------------------------------------------ unfused ablation

@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("M,N,K,alpha,beta", [(300, 260, 200, 1.5, 0.5), (256, 384, 1000, -1.0, 0.0),
                                              (130, 140, 64, 2.0, -1.0), (1024, 512, 512, 1.0, 1.0)])
def test_unfused_ablation_parity(ft, orc, ta, tb, M, N, K, alpha, beta):
    """The unfused form (separate checksum passes, skinny GEMMs for the
    predicted checksums, unprotected GEMM, verify-only pass) gives the same
    result and a clean report."""
    P = make_problem(ta, tb, M, N, K, seed=M + N + K)
    ref, E = oracle_ref(orc, P, alpha, beta)
    dA, dB, dC = P["A"].cuda(), P["B"].cuda(), P["C"].cuda()
    rc, rep = ft.ftgemm_d_unfused(ta, tb, M, N, K, alpha, dA, P["lda"], dB, P["ldb"], beta, dC, P["ldc"])
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    assert_parity(orc, P, dC.cpu(), ref, E)
    for k in ("detected", "flagged_rows", "flagged_cols", "unverifiable", "checksum_only"):
        assert rep[k] == 0, (k, rep)


def test_unfused_requires_aligned_operands(ft):
    A = torch.zeros(9 * 8, dtype=torch.float64, device="cuda")
    rc, _ = ft.ftgemm_d_unfused("N", "N", 9, 8, 8, 1.0, A, 9, A, 8, 0.0, A, 10)
    assert rc == ft.ERR_UNALIGNED


# ------------------------------------------------------------------------------ per-k-panel verification

class panel:
    def __init__(self, ft, n):
        self.ft, self.n = ft, n

    def __enter__(self):
        assert self.ft.ftgemm_set_panel_check(self.n) == 0

    def __exit__(self, *a):
        self.ft.ftgemm_set_panel_check(0)


@pytest.mark.parametrize("dist", ["uniform", "normal", "loguniform"])
@pytest.mark.parametrize("ta,tb", [("N", "N"), ("T", "N"), ("N", "T"), ("T", "T")])
def test_panel_check_fault_free(ft, orc, dist, ta, tb):
    P = make_problem(ta, tb, 300, 260, 1500, seed=404, dist=dist)
    ref, E = oracle_ref(orc, P, 1.5, 0.5)
    with panel(ft, 4):
        rc, rep, out = run_gpu(ft, P, 1.5, 0.5)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)
    assert rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0 and rep["detected"] == 0


def test_panel_check_catches_faults_early_and_separately(ft, orc):
    """Panels of 8 k-slabs over K = 1024 (8 panels).  A fault in panel 0 is
    corrected at the first panel boundary (kind 2); a second fault in the same
    element in panel 3 is caught separately at its own boundary; a fault in
    the last panel is left to the end-of-tile verification (kind 0)."""
    P = make_problem("N", "N", 256, 256, 1024, seed=505)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    flips = [(10, 20, 3, 60), (10, 20, 27, 58), (200, 100, 5, 61), (130, 7, 62, 59)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        with panel(ft, 8), splitk(ft, 1):
            rc, rep, out = run_gpu(ft, P, 1.0, 1.0)
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert rc == 0
    assert_parity(orc, P, out, ref, E)
    assert rep["detected"] == 4 and rep["panel_detected"] == 3
    kinds = sorted((l[0], l[1], l[3]) for l in rep["locs"])
    assert kinds == [(10, 20, 2), (10, 20, 2), (130, 7, 0), (200, 100, 2)]


def test_panel_check_inside_k_splits(ft, orc):
    """The same problem split in two k-ranges of 32 k-slabs (the partial
    kernels check their own panels of 8 slabs, at local slabs 8, 16, 24): a
    fault in each split is corrected at the next panel boundary of its split
    (kind 2, over the split's own products), a fault after the last boundary
    of split 1 is left to the verifying reduction (kind 0); the log records
    the split's first product; the result is within the parity bound."""
    P = make_problem("N", "N", 256, 256, 1024, seed=505)
    ref, E = oracle_ref(orc, P, 1.0, 1.0)
    flips = [(10, 20, 3, 60), (10, 20, 40, 58), (200, 100, 5, 61), (130, 7, 62, 59)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        with panel(ft, 8), splitk(ft, 2):
            rc, rep, out = run_gpu(ft, P, 1.0, 1.0)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
    assert rc == 0
    check_log_against_oracle(orc, P, flips, log)
    assert [L["kfirst"] for L in log] == [0, 512, 0, 512]
    assert_parity(orc, P, out, ref, E)
    assert rep["detected"] == 4 and rep["panel_detected"] == 3
    kinds = sorted((l[0], l[1], l[3]) for l in rep["locs"])
    assert kinds == [(10, 20, 2), (10, 20, 2), (130, 7, 0), (200, 100, 2)]
