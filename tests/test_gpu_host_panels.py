"""ftgemm_d_host in column panels (copies overlapped with the compute),
through the C ABI: against the oracle, and against one ftgemm_d call on
device buffers bit for bit (output tiles are independent, so panels change
no arithmetic when K is not split), with seeded faults that fall in several
panels: the same faults, report, locations and injection log.
"""
from __future__ import annotations

import itertools

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
    yield ftgemm
    ftgemm.ftgemm_set_injection(mode=0)
    ftgemm.ftgemm_set_host_panels(0)
    ftgemm.ftgemm_set_splitk(0)


def _problem(ta, tb, M, N, K, seed, pad=(0, 0, 0)):
    from paper_2305_02444_gb300 import inputs
    ar, ac = (M, K) if ta == "N" else (K, M)
    br, bc = (K, N) if tb == "N" else (N, K)
    lda, ldb, ldc = ar + pad[0], br + pad[1], M + pad[2]
    return dict(ta=ta, tb=tb, M=M, N=N, K=K, ar=ar, br=br, lda=lda, ldb=ldb, ldc=ldc,
                A=inputs.matrix(ar, ac, seed, ld=lda), B=inputs.matrix(br, bc, seed + 1, ld=ldb),
                C=inputs.matrix(M, N, seed + 2, ld=ldc))


def _host(ft, P, alpha, beta, panels, C=None):
    assert ft.ftgemm_set_host_panels(panels) == 0
    try:
        hC = (P["C"] if C is None else C).clone().pin_memory()
        rc, rep = ft.ftgemm_d_host(P["ta"], P["tb"], P["M"], P["N"], P["K"], alpha, P["A"].pin_memory(), P["lda"],
                                   P["B"].pin_memory(), P["ldb"], beta, hC, P["ldc"], loc_cap=4096)
    finally:
        ft.ftgemm_set_host_panels(0)
    assert rc == 0, ft.ftgemm_strerror(rc)
    return hC, rep


def _device(ft, P, alpha, beta):
    dC = P["C"].cuda()
    rc, rep = ft.ftgemm_d(P["ta"], P["tb"], P["M"], P["N"], P["K"], alpha, P["A"].cuda(), P["lda"],
                          P["B"].cuda(), P["ldb"], beta, dC, P["ldc"], loc_cap=4096)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    return dC.cpu(), rep


def _oracle(orc, P, alpha, beta):
    opA = P["A"][:, :P["ar"]].T.numpy(); opB = P["B"][:, :P["br"]].T.numpy()
    return orc.gemm(P["ta"], P["tb"], alpha, opA, opB, beta, P["C"][:, :P["M"]].T.numpy(), want_E=True, k=P["K"])


@pytest.mark.parametrize("ta,tb", list(itertools.product("NT", "NT")))
@pytest.mark.parametrize("panels", [2, 3, 100])
def test_panels_match_the_oracle_and_one_call(ft, orc, ta, tb, panels):
    """300 x 700 x 200 with padded leading dimensions: 2, 3 and one panel per
    tile column (the last ragged); within the parity bound of the oracle, the
    padding rows of C untouched, and (K not split) equal bit for bit to
    ftgemm_d on device buffers."""
    P = _problem(ta, tb, 300, 700, 200, seed=11 + panels, pad=(1, 3, 2))
    alpha, beta = 1.5, 0.5
    ref, E = _oracle(orc, P, alpha, beta)
    with_pad = P["C"].clone()
    with_pad[:, P["M"]:] = float("nan")
    got, rep = _host(ft, P, alpha, beta, panels, C=with_pad)
    g = got[:, :P["M"]].T.numpy()
    assert np.all(np.abs(g - ref) <= orc.parity_tol(P["K"], E))
    assert torch.isnan(got[:, P["M"]:]).all()            # rows M..ldc-1 not written
    assert rep["detected"] == 0 and rep["flagged_rows"] == 0 and rep["flagged_cols"] == 0
    assert ft.ftgemm_set_splitk(1) == 0
    try:
        one, _ = _device(ft, P, alpha, beta)
        got, _ = _host(ft, P, alpha, beta, panels)
    finally:
        ft.ftgemm_set_splitk(0)
    np.testing.assert_array_equal(got[:, :P["M"]].numpy(), one[:, :P["M"]].numpy())


def test_panels_beta_zero_never_reads_c(ft, orc):
    P = _problem("N", "T", 260, 530, 96, seed=5, pad=(0, 0, 3))
    C = torch.full_like(P["C"], float("nan"))
    got, rep = _host(ft, P, 1.0, 0.0, 4, C=C)
    ref, E = _oracle(orc, P, 1.0, 0.0)
    assert np.all(np.abs(got[:, :P["M"]].T.numpy() - ref) <= orc.parity_tol(P["K"], E))
    assert torch.isnan(got[:, P["M"]:]).all()


@pytest.mark.parametrize("tb", ["N", "T"])
def test_panels_faults_report_and_log_as_one_call(ft, orc, tb):
    """40 seeded faults over a 384 x 900 problem in 4 panels: the injection
    log lists the same faults as the oracle's draw over the whole problem
    (global rows and columns, in draw order), with the values they changed
    equal to those of one ftgemm_d call; the report, the located elements
    (global coordinates and tile numbers) and C equal that call's."""
    P = _problem("N", tb, 384, 900, 256, seed=21)
    alpha, beta = 1.5, 0.5
    nks = -(-P["K"] // 16)
    want = orc.random_flips(77, 40, P["M"], P["N"], nks)
    assert len({(int(c) // 256) for c in want[:, 1]}) >= 3     # the faults span panels
    assert ft.ftgemm_set_splitk(1) == 0
    assert ft.ftgemm_set_injection(mode=1, seed=77, count=40) == 0
    try:
        one, rep1 = _device(ft, P, alpha, beta)
        log1 = ft.ftgemm_injection_log()
        got, rep = _host(ft, P, alpha, beta, 4)
        log = ft.ftgemm_injection_log()
    finally:
        ft.ftgemm_set_injection(mode=0)
        ft.ftgemm_set_splitk(0)
    assert [(L["row"], L["col"], L["kstep"], L["bit"]) for L in log] == [tuple(map(int, f)) for f in want]
    assert all(L["applied"] == 1 for L in log)
    for a, b in zip(log, log1):
        assert (a["before"], a["after"]) == (b["before"], b["after"])
    for k in ("detected", "corrected", "flagged_rows", "flagged_cols", "checksum_only", "unverifiable", "n_loc"):
        assert rep[k] == rep1[k], k
    assert rep["detected"] > 5
    assert sorted(l[:4] for l in rep["locs"]) == sorted(l[:4] for l in rep1["locs"])
    np.testing.assert_array_equal(got.numpy(), one.numpy())
    ref, E = _oracle(orc, P, alpha, beta)
    located = {(l[0], l[1]) for l in rep["locs"]}
    g = got[:, :P["M"]].T.numpy()
    for (i, j) in located:
        assert abs(g[i, j] - ref[i, j]) <= orc.parity_tol(P["K"], E)[i, j]
