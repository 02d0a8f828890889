"""Batched FT-DGEMM (one persistent kernel per layout, CUDA graph) against
the oracle, per problem, within the parity bound of the single-problem tests."""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

BM = BN = 128
_REF = {}


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


def make_batch(shapes, seed, dist="uniform"):
    """shapes: (ta, tb, M, N, K, alpha, beta).  Even leading dimensions."""
    from paper_2305_02444_gb300 import inputs
    host, dev, probs = [], [], []
    for q, (ta, tb, m, n, k, alpha, beta) in enumerate(shapes):
        ar, ac = (m, k) if ta == "N" else (k, m)
        br, bc = (k, n) if tb == "N" else (n, k)
        lda, ldb, ldc = max(2, ar + (ar & 1)), max(2, br + (br & 1)), max(2, m + (m & 1))
        A = inputs.matrix(ar, ac, seed + 5 * q, dist, lda)
        B = inputs.matrix(br, bc, seed + 5 * q + 1, dist, ldb)
        C = inputs.matrix(m, n, seed + 5 * q + 2, dist, ldc)
        dA, dB, dC = A.cuda(), B.cuda(), C.cuda()
        host.append((A, B, C, ar, br))
        dev.append((dA, dB, dC))
        probs.append((ta, tb, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc))
    return host, dev, probs


def check_problem(orc, shape, host, dC, extra=None):
    ta, tb, m, n, k, alpha, beta = shape
    A, B, C, ar, br = host
    ref, E = orc.gemm(ta, tb, alpha, A[:, :ar].T.numpy(), B[:, :br].T.numpy(), beta, C[:, :m].T.numpy(),
                      want_E=True, k=k)
    got = dC.cpu()[:, :m].T.numpy()
    tol = orc.parity_tol(k, E)
    if extra is not None:
        tol = tol + extra
    assert np.all(np.abs(got - ref) <= tol), shape


def random_shapes(rng, count, lo=1, hi=300, layouts="NT", betas=(0.0, 1.0, 0.5), alphas=(1.0, 1.5, -0.5)):
    out = []
    for _ in range(count):
        m, n, k = (int(x) for x in rng.integers(lo, hi + 1, size=3))
        out.append((str(rng.choice(list(layouts))), str(rng.choice(list(layouts))), m, n, k,
                    float(rng.choice(alphas)), float(rng.choice(betas))))
    return out


def test_batched_mixed_layouts_ragged(ft, orc):
    rng = np.random.default_rng(1)
    shapes = random_shapes(rng, 24)
    host, dev, probs = make_batch(shapes, seed=100)
    rc, reps = ft.ftgemm_batched(probs)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    for q, sh in enumerate(shapes):
        check_problem(orc, sh, host[q], dev[q][2])
        assert reps[q]["detected"] == 0 and reps[q]["flagged_rows"] == 0 and reps[q]["flagged_cols"] == 0


def test_batched_quick_returns_inside_batch(ft, orc):
    shapes = [("N", "N", 100, 90, 0, 1.5, 0.5), ("N", "N", 64, 70, 33, 0.0, -2.0), ("N", "N", 128, 128, 64, 1.0, 1.0),
              ("T", "N", 5, 7, 9, 1.0, 0.0), ("N", "T", 200, 1, 300, 2.0, 1.0)]
    host, dev, probs = make_batch(shapes, seed=7)
    rc, reps = ft.ftgemm_batched(probs)
    torch.cuda.synchronize()
    assert rc == 0
    for q, sh in enumerate(shapes):
        check_problem(orc, sh, host[q], dev[q][2])


@pytest.mark.parametrize("schedule", [0, 1, 2, 16, 17, 33, 50])
def test_batched_schedules_and_relaunch(ft, orc, schedule):
    """Every schedule gives the same bits; a plan launched 3 times with beta = 0
    is idempotent (the graph resets its counters and reports)."""
    rng = np.random.default_rng(3)
    shapes = [(ta, tb, m, n, k, a, 0.0) for (ta, tb, m, n, k, a, _) in random_shapes(rng, 16, 20, 400, layouts="N")]
    host, dev, probs = make_batch(shapes, seed=55)
    plan = ft.BatchedPlan(probs, schedule=schedule)
    first = None
    for it in range(3):
        plan.launch()
        rc, reps = plan.report()
        assert rc == 0
        outs = [d[2].cpu()[:, :sh[2]].clone() for d, sh in zip(dev, shapes)]   # padding rows hold NaN
        if first is None:
            first = outs
        else:
            for a, b in zip(first, outs):
                assert torch.equal(a, b)
    plan.destroy()
    for q, sh in enumerate(shapes):
        check_problem(orc, sh, host[q], dev[q][2])
    if "outs" not in _REF:
        _REF["outs"] = [o.clone() for o in first]
    else:   # same inputs (same seed): every schedule gives the same bits
        for a, b in zip(_REF["outs"], first):
            assert torch.equal(a, b)


def test_batched_injection_ten_percent(ft, orc):
    """Config-4 style: flips in a random 10% of the problems (one each,
    exponent bits so every one is far above the threshold): each is detected
    and located in its own problem's report and corrected."""
    rng = np.random.default_rng(11)
    count = 40
    shapes = []
    for q in range(count):
        m, n, k = (int(round(math.exp(x))) for x in rng.uniform(math.log(32), math.log(512), size=3))
        shapes.append(("N", "N", m, n, k, 1.0, float(rng.choice([0.0, 1.0]))))
    host, dev, probs = make_batch(shapes, seed=900)
    hit = sorted(rng.choice(count, size=count // 10, replace=False).tolist())
    flips = []
    for q in hit:
        _, _, m, n, k, _, _ = shapes[q]
        flips.append((int(rng.integers(m)), int(rng.integers(n)), int(rng.integers(-(-k // 16))), 60, q))
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        plan = ft.BatchedPlan(probs)
    finally:
        ft.ftgemm_set_injection(mode=0)
    plan.launch()
    rc, reps = plan.report()
    log = plan.injection_log()
    plan.destroy()
    assert rc == 0
    assert [L["problem"] for L in log] == hit
    for L, (i, j, s, bit, q) in zip(log, flips):
        assert L["applied"] == 1 and (L["row"], L["col"], L["kstep"], L["bit"]) == (i, j, s, bit)
    for q, sh in enumerate(shapes):
        check_problem(orc, sh, host[q], dev[q][2])
        if q in hit:
            f = flips[hit.index(q)]
            assert reps[q]["detected"] == 1 and reps[q]["locs"][0][:2] == (f[0], f[1]), (q, reps[q])
        else:
            assert reps[q]["detected"] == 0


def test_batched_argument_codes(ft):
    probs = [("N", "N", 4, 4, 4, 1.0, 0, 4, 0, 4, 0.0, 0, 4), ("N", "N", 4, 4, 4, 1.0, 0, 3, 0, 4, 0.0, 0, 4)]
    rc, _ = ft.ftgemm_batched(probs)
    assert rc == -(100 * 1 + 8)


def test_batched_every_block_count_equals_single_calls(ft, orc):
    """The batched kernel computes a tile's valid rows and columns rounded up
    to 16 (any of 1..8 accumulator blocks each way, in binary pieces); every
    accumulator still gets the same FMAs in the same order as in ftgemm_d's
    whole-tile kernel, so each problem's output equals one ftgemm_d call (K
    not split) bit for bit.  Row and column extents 16r - 3 and 16c - 7 cover
    every block count; two problems span several tiles with ragged edges."""
    shapes = []
    for q in range(8):
        r, c = q + 1, 8 - q
        shapes.append(("N", "N", 16 * r - 3, 16 * c - 7, (1, 15, 17, 100)[q % 4], 1.5, (0.0, 0.5)[q % 2]))
        shapes.append(("T", "N", 16 * c - 3, 16 * r - 7, (33, 64, 5, 250)[q % 4], -0.75, (1.0, 0.0)[q % 2]))
    shapes += [("N", "T", 200, 333, 129, 1.0, 1.0), ("T", "T", 257, 144, 48, 2.0, 0.5)]
    host, dev, probs = make_batch(shapes, seed=4242)
    rc, reps = ft.ftgemm_batched(probs)
    torch.cuda.synchronize()
    assert rc == 0, ft.ftgemm_strerror(rc)
    assert ft.ftgemm_set_splitk(1) == 0
    try:
        for q, (ta, tb, m, n, k, alpha, beta) in enumerate(shapes):
            A, B, C, ar, br = host[q]
            dC = C.cuda()
            rc1, rep1 = ft.ftgemm_d(ta, tb, m, n, k, alpha, A.cuda(), A.shape[1], B.cuda(), B.shape[1], beta, dC,
                                    C.shape[1])
            torch.cuda.synchronize()
            assert rc1 == 0
            assert torch.equal(dev[q][2].cpu()[:, :m], dC.cpu()[:, :m]), shapes[q]
            check_problem(orc, shapes[q], host[q], dev[q][2])
            assert reps[q]["detected"] == 0 and reps[q]["unverifiable"] == 0
    finally:
        ft.ftgemm_set_splitk(0)


@pytest.mark.parametrize("layout", ["NN", "TT"])
def test_batched_checks_at_the_edges_of_the_fp32_range(ft, orc, layout):
    """The batched checksum pass keeps the operands' absolute sums in FP32
    (rounded upward) and takes them again in FP64 where FP32's range would
    overflow them or leave them loose.  Operands scaled by 2^140 / 2^-140
    (FP32 overflow) and by 2^-400 each (every |x| under FP32's smallest
    number, products near 2^-800) stay verifiable: no unverifiable count, no
    false positive, each problem's one exponent flip detected at its element
    and corrected, every output within the parity bound (in both layouts, so
    both shapes of the pass see both scales)."""
    ta, tb = layout
    shapes = [(ta, tb, 150, 170, 90, 1.0, 1.0), (ta, tb, 140, 60, 200, 1.0, 0.0), (ta, tb, 100, 100, 100, 1.5, 0.5)]
    scales = [(2.0 ** 140, 2.0 ** -140), (2.0 ** -400, 2.0 ** -400), (1.0, 1.0)]
    host, dev, probs = make_batch(shapes, seed=77)
    for q, (sa, sb) in enumerate(scales):
        A, B, C, ar, br = host[q]
        A.mul_(sa)
        B.mul_(sb)
        C.mul_(sa * sb)
        dev[q][0].copy_(A)
        dev[q][1].copy_(B)
        dev[q][2].copy_(C)
    flips = [(7, 11, 2, 60, 0), (100, 33, 5, 61, 1), (50, 50, 3, 60, 2)]
    assert ft.ftgemm_set_injection(mode=2, flips=flips) == 0
    try:
        plan = ft.BatchedPlan(probs)
    finally:
        ft.ftgemm_set_injection(mode=0)
    plan.launch()
    rc, reps = plan.report()
    plan.destroy()
    assert rc == 0
    for q, sh in enumerate(shapes):
        assert reps[q]["unverifiable"] == 0, (q, reps[q])
        assert reps[q]["detected"] == 1 and reps[q]["corrected"] == 1, (q, reps[q])
        assert reps[q]["locs"][0][:2] == flips[q][:2]
        check_problem(orc, sh, host[q], dev[q][2])


def test_tune_batched_picks_a_plan_that_matches_the_oracle(ft, orc, tmp_path):
    """The autotuner on a small mixed batch (every layout, ragged sizes): it
    times every candidate schedule, caches the choice (a second call returns
    it untimed), and a plan built with the chosen schedule matches the oracle
    problem by problem, with no check raised."""
    from paper_2305_02444_gb300 import autotune
    rng = np.random.default_rng(5)
    shapes = random_shapes(rng, 20, 8, 260)
    cache = str(tmp_path / "sched.json")
    tune_shapes = [(ta, tb, m, n, k) for (ta, tb, m, n, k, _, _) in shapes]
    best, times = autotune.tune_batched(tune_shapes, reps=2, cache_path=cache)
    assert set(times) == set(autotune.CANDIDATES) and best in autotune.CANDIDATES
    assert all(t > 0 for t in times.values()) and times[best] == min(times.values())
    again, cached = autotune.tune_batched(tune_shapes, reps=2, cache_path=cache)
    assert again == best and {int(k) for k in cached} == set(times)
    host, dev, probs = make_batch(shapes, seed=600)
    plan = ft.BatchedPlan(probs, schedule=best)
    plan.launch()
    rc, reps = plan.report()
    plan.destroy()
    assert rc == 0
    for q, sh in enumerate(shapes):
        check_problem(orc, sh, host[q], dev[q][2])
        assert reps[q]["detected"] == 0 and reps[q]["flagged_rows"] == 0 and reps[q]["flagged_cols"] == 0
