"""ftgemm_d_noalloc, the entry point for callers that cannot allocate device
memory (framework-owned memory pools, latency-critical loops that cannot take
cudaMalloc's implicit synchronisation, out-of-memory recovery paths), checked
against ftgemm_d through the C ABI on two calls in a row.

It keeps all scratch in one static device array, so the second call also
checks that nothing left over from the first call leaks into the result.
This file is named to be collected last.
"""
from __future__ import annotations

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
    return ftgemm


def _problem(ta, tb, M, N, K, seed):
    from paper_2305_02444_gb300 import inputs
    ar, ac = (M, K) if ta == "N" else (K, M)
    br, bc = (K, N) if tb == "N" else (N, K)
    A = inputs.matrix(ar, ac, seed)
    B = inputs.matrix(br, bc, seed + 1)
    C = inputs.matrix(M, N, seed + 2)
    return A, B, C, ar, br


def _check(ft, orc, ta, tb, M, N, K, alpha, beta, seed):
    A, B, C, ar, br = _problem(ta, tb, M, N, K, seed)
    dA, dB = A.cuda(), B.cuda()
    c_ref, c_na = C.cuda(), C.cuda()
    rc, rep = ft.ftgemm_d(ta, tb, M, N, K, alpha, dA, ar, dB, br, beta, c_ref, M)
    assert rc == 0
    rc, rep_na = ft.ftgemm_d_noalloc(ta, tb, M, N, K, alpha, dA, ar, dB, br, beta, c_na, M)
    assert rc == 0, ft.ftgemm_strerror(rc)
    torch.cuda.synchronize()
    # the tolerance the parity tests use: max(4K, 2K+6) u E, E = |alpha||A||B| + |beta||C|
    _, E = orc.gemm(ta, tb, alpha, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), beta, C.T.numpy(),
                    want_E=True, k=K)
    tol = orc.parity_tol(K, E)
    got_ref = c_ref.cpu().T.numpy()
    got_na = c_na.cpu().T.numpy()
    assert np.all(np.abs(got_na - got_ref) <= tol)
    for k in ("detected", "flagged_rows", "flagged_cols", "unverifiable", "checksum_only"):
        assert rep_na[k] == rep[k] == 0, (k, rep_na, rep)


def test_noalloc_matches_ftgemm_d_two_calls(ft, orc):
    # first call: ragged 3x3 tiles, K a multiple of the 16-product k-step
    _check(ft, orc, "N", "N", 300, 260, 208, 1.5, 0.5, seed=101)
    # second call in a row: other layout, sizes and K with a partial k-step,
    # so the stale contents of the shared array would show if not cleared
    _check(ft, orc, "T", "N", 256, 384, 150, -0.75, 2.0, seed=202)


def test_noalloc_rejects_what_it_cannot_hold(ft):
    n = 16384  # needs more than the 32 MiB of static scratch; nothing is launched
    rc, _ = ft.ftgemm_d_noalloc("N", "N", n, n, n, 1.0, 0, n, 0, n, 0.0, 0, n, stream=0)
    assert rc == ft.ERR_SCRATCH
    A = torch.zeros(8 * 9, dtype=torch.float64, device="cuda")
    rc, _ = ft.ftgemm_d_noalloc("N", "N", 9, 8, 8, 1.0, A, 9, A, 8, 0.0, A, 9)  # odd lda
    assert rc == ft.ERR_UNALIGNED


def test_noalloc_refuses_a_report_inside_a_stream_capture(ft):
    """A report is read back by waiting for the stream, which a stream
    capture does not allow: the call returns ERR_CAPTURE and enqueues
    nothing (the captured graph stays empty)."""
    import warnings
    n = 128
    A = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    C = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    rc, _ = ft.ftgemm_d_noalloc("N", "N", n, n, n, 1.0, A, n, A, n, 0.0, C, n)   # set-up outside the capture
    assert rc == 0
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")      # the graph is empty by design
        with torch.cuda.graph(g, stream=side):
            rc, _ = ft.ftgemm_d_noalloc("N", "N", n, n, n, 1.0, A, n, A, n, 0.0, C, n, stream=side)
    assert rc == ft.ERR_CAPTURE
    assert "capture" in ft.ftgemm_strerror(rc)
