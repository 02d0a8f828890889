"""Benchmark of the GB300 fault-tolerant DGEMM (FT-GEMM, HPDC'23).

One step = one fault-tolerant DGEMM C = 1.5*A*B + 0.5*C at M = N = K = 8192
(FP64, column-major, entries U[-1,1], seeded), with one seeded bit flip per
64 output tiles (64 flips per call, random k-steps, bits 0..62), through the
C ABI (ftgemm_d).  Inputs (3 x 512 MiB) are larger than the 129 MB L2.

Printed (one JSON line, rank 0):
  value          TFLOP/s of the FT path with injection, inputs resident in HBM
                 (2*M*N*K per step; checksum work not counted)
  overhead       ABFT overhead vs the unprotected kernel of the same tiles
                 (fault-free and with injection)
  errors         detected / corrected / injected counts per step
  roofline       dominant kernel (the FT main kernel) against the FP64 FMA
                 pipe peak 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz
  e2e            the same metric through ftgemm_d_host with pinned host
                 buffers (copies in and out inside the timed region)
  cpu_baseline   the CPU oracle on a bounded row sample of the same workload
  clocks         nvidia-smi samples taken during the timed region

--impl reference times the CPU oracle (the reference arm of this build).
Multi-GPU (torchrun): every rank runs its own replica (independent problems,
weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M = N = K = 8192
ALPHA, BETA = 1.5, 0.5
SEED = 20230614
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # FP64 FMA pipe, max SM clock


def measured_peaks():
    """Measured copy bandwidth and cuBLAS bf16 throughput of this GPU model
    (MEASURED_PEAKS.json beside this file), else the fallback figures."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"bf16_tflops": float(d["bf16_tflops"]), "hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"bf16_tflops": 1900.0, "hbm_gbs": 6800.0, "source": "fallback"}


def set_size(n: int):
    global M, N, K, TILES, FLIPS, WORKLOAD
    M = N = K = n
    TILES = -(-M // 128) * -(-N // 128)
    FLIPS = math.ceil(TILES / 64)
    WORKLOAD = f"ftdgemm_nn_{M}x{N}x{K}_a{ALPHA}_b{BETA}_uniform_flips1per64tiles"


set_size(8192)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int, device) -> float:
    """Max of x over all ranks (host-level timing reduction, not a data-path
    collective); identity on one rank."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, ws: int, device) -> float:
    """Sum of x over all ranks (the whole job's fault counts: a host-level
    scalar reduction, not a data-path collective); identity on one rank."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_tflops(ws: int, flops_per_rank_step: float, steps: int, t_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank runs its own replica)."""
    return ws * flops_per_rank_step * steps / t_max / 1e12


def sample_clocks_start(dev_index: int, path: str):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    f = None
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), f"--query-gpu={q}",
                              "--format=csv,noheader,nounits", "-lms", "200"], stdout=f,
                             stderr=subprocess.DEVNULL)
        return p, f
    except OSError:   # no writable folder, or no nvidia-smi: no clock record
        if f is not None:
            f.close()
        return None, None


def sample_clocks_stop(proc, f, path: str):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    with open(path) as fh:
        lines = fh.read().splitlines()
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def read_traffic(kernel_tag: str):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = os.path.join(ROOT, "paper_2305_02444_gb300", "csrc", "ftgemm_kernel.cuh")
    with open(src, "rb") as fh:
        h = hashlib.sha256(fh.read()).hexdigest()[:16]
    with open(path) as fh:
        lines = fh.read().splitlines()
    for line in lines:
        if line.startswith("#") or not line.strip():
            continue
        tag, src_hash, nbytes = line.split()[:3]
        if tag == kernel_tag and src_hash == h:
            return float(nbytes)
    return None


_SAMPLE_INPUTS = {}


def _sample_inputs(rows: int, seed: int):
    key = (M, N, K, seed)
    if key not in _SAMPLE_INPUTS:
        from paper_2305_02444_gb300 import inputs
        _SAMPLE_INPUTS.clear()
        _SAMPLE_INPUTS[key] = (inputs.matrix(M, K, seed).T.numpy(), inputs.matrix(K, N, seed + 1).T.numpy(),
                               inputs.matrix(M, N, seed + 2).T.numpy())
    A, B, C = _SAMPLE_INPUTS[key]
    return A[:rows], B, C[:rows]                                 # first `rows` rows of A and C


def oracle_sample(rows: int, seed: int):
    """The oracle's FT-DGEMM on `rows` full rows of the workload (rows x N x K)."""
    import oracle
    A, B, C = _sample_inputs(rows, seed)
    nflips = max(1, round(FLIPS * rows / M))
    flips = oracle.random_flips(seed, nflips, rows, N, -(-K // 16))
    t0 = time.perf_counter()
    r = oracle.ft_gemm("N", "N", ALPHA, A, B, BETA, C, BM=128, BN=128, BK=16, flips=flips)
    dt = time.perf_counter() - t0
    return dt, r


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_cpu_baseline(target_s: float = 15.0):
    """Calibrated sample: grow the row count until one run takes ~target_s."""
    rows = 128
    dt, _ = oracle_sample(rows, SEED)
    if dt < target_s / 2:
        rows = int(min(M, max(128, 128 * round(rows * target_s / max(dt, 1e-3) / 128))))
        dt, _ = oracle_sample(rows, SEED)
    flops = 2.0 * rows * N * K
    return {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
            "sample": f"{rows} of {M} rows of C (full N={N}, K={K}), plain C FT-DGEMM oracle with "
                      f"per-tile encode/verify/correct, {dt:.1f} s"}


def _flip_bit(x: float, bit: int) -> float:
    import struct
    u = struct.unpack("<Q", struct.pack("<d", x))[0] ^ (1 << bit)
    return struct.unpack("<d", struct.pack("<Q", u))[0]


def flip_accounting(log, rep, A, B, Cin, out_at, tm: int = 128, tn: int = 128):
    """Classify the injected faults of one call by the oracle (CPU leg, after
    the timed regions): each fault's effect alpha * (flipped - true partial
    sum) against the oracle's row and column thresholds of its tile.  Above:
    more than 4x the larger threshold (must be detected, located and
    corrected); below: under a quarter of the smaller one (no checksum scheme
    sees it); the band between may go either way.  out_at(i, j) returns the
    call's output element, checked against the oracle's value within the
    parity bound for every located fault.  A, B, Cin: (M, K), (K, N), (M, N)
    numpy views of the call's inputs."""
    import oracle
    Mx, Kx = A.shape
    Nx = B.shape[1]
    enc = oracle.encode_operands("N", "N", Mx, Nx, Kx, A, B, tm, tn)
    above, band, below = [], [], []
    for L in log:
        i, j, s, bit, kf = L["row"], L["col"], L["kstep"], L["bit"], L["kfirst"]
        kend = min(Kx, 16 * (s + 1))
        part = oracle.partial("N", "N", i, j, kend, A, B) if kf == 0 else \
            float(A[i, kf:kend] @ B[kf:kend, j])
        d = _flip_bit(part, bit) - part
        eff = abs(ALPHA * d) if math.isfinite(d) else math.inf
        I, J = i // tm, j // tn
        cols = slice(J * tn, min(Nx, (J + 1) * tn))
        rows = slice(I * tm, min(Mx, (I + 1) * tm))
        tr = oracle.tau(Kx, cols.stop - cols.start, ALPHA, enc.arowabs[i], enc.babsmax[J], BETA,
                        float(abs(Cin[i, cols]).sum()))
        tc = oracle.tau(Kx, rows.stop - rows.start, ALPHA, enc.bcolabs[j], enc.aabsmax[I], BETA,
                        float(abs(Cin[rows, j]).sum()))
        (above if eff > 4 * max(tr, tc) else below if eff < 0.25 * min(tr, tc) else band).append((i, j))
    located = {(l[0], l[1]) for l in rep["locs"]}
    det_above = sum(1 for x in set(above) if x in located)
    det_band = sum(1 for x in set(band) if x in located)
    within = True
    for (i, j) in located:
        r, E = oracle.gemm("N", "N", ALPHA, A[i:i + 1], B[:, j:j + 1], BETA, Cin[i:i + 1, j:j + 1], want_E=True)
        within = within and bool(abs(out_at(i, j) - r[0, 0]) <= oracle.parity_tol(Kx, E)[0, 0])
    return {"checked_call": {"injected": len(log), "above_threshold": len(above), "in_guard_band": len(band),
                             "below_threshold": len(below), "detected": rep["detected"],
                             "corrected": rep["corrected"], "detected_above": det_above,
                             "detected_in_band": det_band,
                             "detected_elsewhere": rep["detected"] - det_above - det_band,
                             "every_above_threshold_fault_fixed": bool(det_above == len(set(above)) and
                                                                       rep["corrected"] == rep["detected"] and
                                                                       within),
                             "located_within_parity_bound": within,
                             "rule": "above: alpha*|flip effect| > 4 max(tau_row, tau_col) of the oracle; "
                                     "below: < min/4; corrected elements checked against the oracle"}}


SPLIT_ENGINES = {"tc": 2, "mma": 1, "tcp": 5, "i8": 7}   # ftgemm_set_split_engine codes
METRIC = "FT-GEMM TFLOP/s (FP64) & % FP64 peak; ABFT overhead % vs plain; errors fixed"


def main_config():
    """The workload of the default run (both arms report it)."""
    return {"workload": WORKLOAD, "M": M, "N": N, "K": K, "alpha": ALPHA, "beta": BETA,
            "layout": "column-major NN", "dist": "uniform[-1,1]", "tile": "128x128x16",
            "flips_per_call": FLIPS,
            "l2": f"inputs larger than L2 (3 x {M * N * 8 / 2**20:.0f} MiB vs 129 MB)"
            if 3 * M * N * 8 > 129e6 else "inputs smaller than L2"}


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    rows = 128
    dt0, _ = oracle_sample(rows, SEED)               # calibration (untimed)
    rows = int(min(M, max(128, 128 * round(rows * 6.0 / max(dt0, 1e-3) / 128))))
    for _ in range(args.warmup):
        oracle_sample(rows, SEED)
    times = [oracle_sample(rows, SEED)[0] for _ in range(args.steps)]
    t = sum(times) / len(times)
    v = 2.0 * rows * N * K / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": main_config(),
            "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": f"{rows} of {M} rows of C per step (full N, K)"},
            "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def sweep(args):
    """Square sweep M = N = K in {1024 .. 16384} plus the rank-k update
    8192^2 x 256 (alpha 1.5, beta 0.5, U[-1,1], one flip per 64 tiles): FT
    with injection, FT fault-free and the unprotected kernel, per size."""
    import torch
    from paper_2305_02444_gb300 import build, ftgemm, inputs
    build.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    rows = []
    shapes = [(1024,) * 3, (2048,) * 3, (4096,) * 3, (8192,) * 3, (16384,) * 3, (8192, 8192, 256)]
    if args.sweep_shapes:
        shapes = [tuple(int(x) for x in sh.split("x")) for sh in args.sweep_shapes.split(",")]
    for (m, n, k) in shapes:
        A = inputs.matrix(m, k, SEED, args.sweep_dist, device="cuda")
        B = inputs.matrix(k, n, SEED + 1, args.sweep_dist, device="cuda")
        C = inputs.matrix(m, n, SEED + 2, args.sweep_dist, device="cuda")
        tiles = -(-m // 128) * -(-n // 128)
        nfl = math.ceil(tiles / 64)
        reps = args.sweep_reps or max(2, min(10, int(2e12 / (2.0 * m * n * k))))

        def t(fn):
            for _ in range(args.sweep_warmup):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps / 1e3

        ft_call = lambda: ftgemm.ftgemm_d("N", "N", m, n, k, ALPHA, A, m, B, k, BETA, C, m, report=False)
        t_noft = t(lambda: ftgemm.ftgemm_d_noft("N", "N", m, n, k, ALPHA, A, m, B, k, BETA, C, m))
        t_ft = t(ft_call)
        t_unf = float("nan") if args.no_unfused else \
            t(lambda: ftgemm.ftgemm_d_unfused("N", "N", m, n, k, ALPHA, A, m, B, k, BETA, C, m, report=False))
        ftgemm.ftgemm_set_injection(mode=1, seed=SEED, count=nfl)
        t_inj = t(ft_call)
        rc, rep = ftgemm.ftgemm_d("N", "N", m, n, k, ALPHA, A, m, B, k, BETA, C, m, loc_cap=0)
        ftgemm.ftgemm_set_injection(mode=0)
        fl = 2.0 * m * n * k
        rows.append({"M": m, "N": n, "K": k, "tiles": tiles, "noft_tflops": fl / t_noft / 1e12,
                     "ft_tflops": fl / t_ft / 1e12, "ft_inj_tflops": fl / t_inj / 1e12,
                     "pct_fp64_peak_ft_inj": 100 * fl / t_inj / 1e12 / FP64_PEAK_TFLOPS,
                     "overhead_pct": 100 * (t_ft / t_noft - 1), "overhead_inj_pct": 100 * (t_inj / t_noft - 1),
                     "unfused_overhead_pct": 100 * (t_unf / t_noft - 1),
                     "flips": nfl, "detected": rep["detected"], "corrected": rep["corrected"]})
        print(json.dumps(rows[-1]), flush=True)
        del A, B, C
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": rows, "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS}), flush=True)


def panel_sweep(args):
    """Per-k-panel verification (ftgemm_set_panel_check): overhead of checking
    the accumulators every n k-slabs (n = 8, 32, 128) at 8192^3 and 1024^3
    (NN, alpha 1.5, beta 0.5, U[-1,1]; and n = 2, finer than the 4-slab k-splits
    of the 1024^3 grid), fault-free and with one flip per 64
    tiles, against the unprotected kernel and the end-of-tile check; then
    several faults in one element across panels at 8192^3 (three flips of
    each of 64 elements, at k-steps in panels 0, 5 and 10 of 32 slabs): with
    panel checks each fault is found in its panel, with the end-of-tile check
    alone they merge into one correction per element; the injected elements
    against the oracle either way (CPU, after the timed regions)."""
    import numpy as np
    import torch
    import oracle
    from paper_2305_02444_gb300 import build, ftgemm, inputs
    build.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    shapes = [int(x) for x in args.panel_sizes.split(",") if x]
    rows, multi = [], None
    for n in shapes:
        A = inputs.matrix(n, n, SEED, device="cuda")
        B = inputs.matrix(n, n, SEED + 1, device="cuda")
        C = inputs.matrix(n, n, SEED + 2, device="cuda")
        nfl = math.ceil((-(-n // 128)) ** 2 / 64)
        reps = max(2, min(10, int(2e12 / (2.0 * n ** 3))))

        def t(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                fn()
            e1.record(s)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps / 1e3

        ft_call = lambda: ftgemm.ftgemm_d("N", "N", n, n, n, ALPHA, A, n, B, n, BETA, C, n, report=False)
        t_noft = t(lambda: ftgemm.ftgemm_d_noft("N", "N", n, n, n, ALPHA, A, n, B, n, BETA, C, n))
        fl = 2.0 * n ** 3
        for kslabs in [0] + [int(x) for x in args.panel_slabs.split(",") if x]:
            ftgemm.ftgemm_set_panel_check(kslabs)
            t_ft = t(ft_call)
            ftgemm.ftgemm_set_injection(mode=1, seed=SEED, count=nfl)
            t_inj = t(ft_call)
            rc, rep = ftgemm.ftgemm_d("N", "N", n, n, n, ALPHA, A, n, B, n, BETA, C, n, loc_cap=0)
            ftgemm.ftgemm_set_injection(mode=0)
            ftgemm.ftgemm_set_panel_check(0)
            rows.append({"M": n, "N": n, "K": n, "panel_kslabs": kslabs, "ft_tflops": fl / t_ft / 1e12,
                         "ft_inj_tflops": fl / t_inj / 1e12, "pct_fp64_peak": 100 * fl / t_ft / 1e12 / FP64_PEAK_TFLOPS,
                         "overhead_vs_noft_pct": 100 * (t_ft / t_noft - 1),
                         "overhead_inj_vs_noft_pct": 100 * (t_inj / t_noft - 1),
                         "flips": nfl, "detected": rep["detected"], "panel_detected": rep["panel_detected"], "rc": rc})
            print(json.dumps(rows[-1]), flush=True)
        if n == max(shapes):
            # several faults in one element, in different panels of 32 slabs
            rng = np.random.default_rng(SEED)
            pos = [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(64)]
            flips = [(i, j, 32 * p + 7, bit) for (i, j) in pos for p, bit in ((0, 62), (5, 58), (10, 55))]
            Ah, Bh, Ch = A.cpu().T.numpy(), B.cpu().T.numpy(), C.cpu().T.numpy()
            multi = {}
            for kslabs in (32, 0):
                ftgemm.ftgemm_set_panel_check(kslabs)
                ftgemm.ftgemm_set_injection(mode=2, flips=flips)
                Cw = C.clone()
                rc, rep = ftgemm.ftgemm_d("N", "N", n, n, n, ALPHA, A, n, B, n, BETA, Cw, n, loc_cap=4096)
                ftgemm.ftgemm_set_injection(mode=0)
                ftgemm.ftgemm_set_panel_check(0)
                torch.cuda.synchronize()
                worst = 0.0
                for (i, j) in pos:
                    r, E = oracle.gemm("N", "N", ALPHA, Ah[i:i + 1], Bh[:, j:j + 1], BETA, Ch[i:i + 1, j:j + 1],
                                       want_E=True)
                    worst = max(worst, abs(float(Cw[j, i]) - r[0, 0]) / oracle.parity_tol(n, E)[0, 0])
                multi[f"panel_kslabs_{kslabs}"] = {"flips": len(flips), "elements": len(pos),
                                                  "detected": rep["detected"], "panel_detected": rep["panel_detected"],
                                                  "corrected": rep["corrected"], "rc": rc,
                                                  "max_err_over_parity_bound": worst}
                print(json.dumps({"several_faults_per_element": multi}), flush=True)
        del A, B, C
        torch.cuda.empty_cache()
    print(json.dumps({"metric": "per-k-panel verification: TFLOP/s and overhead", "rows": rows,
                      "several_faults_per_element": multi,
                      "peak": FP64_PEAK_TFLOPS}), flush=True)


def batched(args):
    """512 independent FT-DGEMMs, M, N, K each log-uniform in [32, 1024], NN,
    U[-1,1], alpha = 1, beta in {0, 1} per problem, one exponent-bit flip in
    each of a random 10% of the problems; one persistent launch captured in a
    CUDA graph, schedule picked by the autotuner."""
    import numpy as np
    import torch
    from paper_2305_02444_gb300 import autotune, build, ftgemm, inputs
    build.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    count = 512
    shapes = inputs.batched_sizes(count, SEED)
    rng = np.random.default_rng(SEED)
    betas = rng.integers(0, 2, size=count).astype(float)
    probs, keep = [], []
    useful = padded = 0.0
    for q, (m, n, k) in enumerate(shapes):
        lda, ldb, ldc = m + (m & 1), k + (k & 1), m + (m & 1)
        A = inputs.matrix(m, k, SEED + 3 * q, ld=lda, device="cuda", fill_pad=0.0)
        B = inputs.matrix(k, n, SEED + 3 * q + 1, ld=ldb, device="cuda", fill_pad=0.0)
        C = inputs.matrix(m, n, SEED + 3 * q + 2, ld=ldc, device="cuda", fill_pad=0.0)
        keep += [A, B, C]
        probs.append(("N", "N", m, n, k, 1.0, A, lda, B, ldb, float(betas[q]), C, ldc))
        useful += 2.0 * m * n * k
        padded += 2.0 * (-(-m // 128) * 128) * (-(-n // 128) * 128) * (-(-k // 16) * 16)
    hit = sorted(rng.choice(count, size=count // 10, replace=False).tolist())
    flips = [(int(rng.integers(shapes[q][0])), int(rng.integers(shapes[q][1])),
              int(rng.integers(-(-shapes[q][2] // 16))), int(rng.integers(52, 63)), q) for q in hit]
    sched, tune_ms = autotune.tune_batched([("N", "N", m, n, k) for (m, n, k) in shapes])
    ftgemm.ftgemm_set_injection(mode=2, flips=flips)
    plan_ft = ftgemm.BatchedPlan(probs, ft=True, schedule=sched)
    ftgemm.ftgemm_set_injection(mode=0)
    plan_noft = ftgemm.BatchedPlan(probs, ft=False, schedule=sched)

    def t(plan, steps):
        for _ in range(args.warmup):
            plan.launch()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            plan.launch()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps / 1e3

    steps = max(args.steps, 10)
    t_ft = t(plan_ft, steps)
    rc, reps = plan_ft.report()
    t_noft = t(plan_noft, steps)
    det = sum(r["detected"] for r in reps)
    cor = sum(r["corrected"] for r in reps)
    hit_det = sum(1 for q in hit if reps[q]["detected"] >= 1)
    line = {"metric": "batched FT-DGEMM TFLOP/s (FP64)", "value": useful / t_ft / 1e12, "unit": "TFLOP/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": t_ft * 1e3,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "batched_512_loguniform32to1024_NN_alpha1_beta01_flips10pct",
                       "problems": count, "useful_flop": useful, "padded_flop_128x128x16": padded,
                       "schedule": sched, "graph": True},
            "pct_fp64_peak": 100.0 * useful / t_ft / 1e12 / FP64_PEAK_TFLOPS,
            "padded_tflops": padded / t_ft / 1e12,
            "noft_tflops": useful / t_noft / 1e12,
            "overhead_pct": 100.0 * (t_ft / t_noft - 1.0),
            "errors": {"problems_with_flip": len(hit), "detected": det, "corrected": cor,
                       "flipped_problems_detected": hit_det, "rc": rc},
            "autotune_ms": tune_ms}
    plan_ft.destroy()
    plan_noft.destroy()
    print(json.dumps(line), flush=True)


def split(args):
    """Split precision at M = N = K = 8192 (or --size), entries sign-random with
    |x| log-uniform in [1e-3, 1e3]: FP64 emulated with S BF16 slices and the
    plain BF16 form, FP32 checksums / FP64 verify, one flip per 64 tiles (top
    exponent bit of the FP64 accumulator after a random slice pair; exponent
    bit 9 of the plain form's accumulator); against
    the DFMA FP64 path on the same inputs; max error vs the FP64 oracle on
    sampled rows."""
    import numpy as np
    import torch
    import oracle
    from paper_2305_02444_gb300 import build, ftgemm, inputs
    build.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    n = M
    A = inputs.matrix(n, n, SEED, "loguniform", device="cuda")
    B = inputs.matrix(n, n, SEED + 1, "loguniform", device="cuda")
    C0 = inputs.matrix(n, n, SEED + 2, "loguniform", device="cuda")
    C = C0.clone()
    flops = 2.0 * n ** 3
    tiles = (-(-n // 128)) ** 2
    rng = np.random.default_rng(SEED)
    rows = np.sort(rng.choice(n, size=args.split_rows, replace=False))
    Ah, Bh, C0h = A.cpu().T.numpy(), B.cpu().T.numpy(), C0.cpu().T.numpy()
    refs = [oracle.gemm("N", "N", 1.0, Ah[i:i + 1], Bh, 1.0, C0h[i:i + 1])[0][0] for i in rows]

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps / 1e3

    def err_of(fn):
        C.copy_(C0)
        fn()
        torch.cuda.synchronize()
        out = C.cpu().T.numpy()
        return max(float(np.abs(out[i] - r).max() / np.abs(r).max()) for i, r in zip(rows, refs))

    res = {}
    engines = [e for e in args.split_engine.split(",") if e]
    forms = [("fp64_dfma", None, 1, None)]
    for eng in engines:
        sfx = {"tc": "", "mma": "_mma", "tcp": "_tcp", "i8": "_i8"}[eng]
        forms += [(f"emulated_S{S}_fp64ck{sfx}", S, 2, eng) for S in args.split_slices]
        if eng not in ("mma", "i8"):    # the plain form with FP32-carried checksums on the tcgen05 engines
            forms += [(f"bf16_plain_fp32ck{sfx}", 0, 1, eng)]
    forms += [(f"emulated_S{S}_fp32ck_mma", S, 1, "mma") for S in args.split_slices] + \
        [("bf16_plain_fp32ck_mma", 0, 1, "mma")]
    if args.split_forms:
        keep = set(x for x in args.split_forms.split(",") if x)
        forms = [f for f in forms if f[0] in keep]
    peaks = measured_peaks()
    for name, S, ck, eng in forms:
        if eng is not None:
            ftgemm.ftgemm_set_split_engine(SPLIT_ENGINES[eng])
        if S is None:
            ft_fn = lambda: ftgemm.ftgemm_d("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, report=False)
            no_fn = lambda: ftgemm.ftgemm_d_noft("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n)
            steps = 2
        else:
            ft_fn = lambda S=S, ck=ck: ftgemm.ftgemm_d_split("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n,
                                                             nslices=S, ft=ck, report=False)
            no_fn = lambda S=S: ftgemm.ftgemm_d_split("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, nslices=S,
                                                      ft=False, report=False)
            steps = max(3, args.steps)
        t_ft = timed(ft_fn, steps)
        ftgemm.ftgemm_timing(True)
        t_no = timed(no_fn, steps)
        k_ms, k_n, _ = ftgemm.ftgemm_timing_read()
        ftgemm.ftgemm_timing(False)
        kms = k_ms / max(1, k_n)   # event-timed product kernel of the unprotected calls
        err = err_of(ft_fn)
        npairs = 1 if S in (None, 0) else S * (S + 1) // 2
        nflip = math.ceil(tiles / 64)
        if S is None:
            ftgemm.ftgemm_set_injection(mode=1, seed=SEED, count=nflip)
        else:
            # emulated forms: the top exponent bit of the FP64 accumulator after a
            # random slice pair; plain form: exponent bit 9 (the value times 2^512
            # for accumulators in [2, 2^513)), since clearing the top bit only
            # zeroes an element, which at K = 8192 lies below the FP32-carried
            # threshold (about 2^-8 of the column's absolute checksum)
            bit = 61 if S == 0 else 62
            flips = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(npairs)), bit) for _ in range(nflip)]
            ftgemm.ftgemm_set_injection(mode=2, flips=flips)
        C.copy_(C0)
        if S is None:
            rc, rep = ftgemm.ftgemm_d("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, loc_cap=0)
        else:
            rc, rep = ftgemm.ftgemm_d_split("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, nslices=S, ft=ck,
                                            loc_cap=0)
        ftgemm.ftgemm_set_injection(mode=0)
        torch.cuda.synchronize()
        out = C.cpu().T.numpy()
        err_inj = max(float(np.abs(out[i] - r).max() / np.abs(r).max()) for i, r in zip(rows, refs))
        res[name] = {"tflops_fp64_equiv": flops / t_ft / 1e12, "unprotected_tflops": flops / t_no / 1e12,
                     "ft_overhead_pct": 100.0 * (t_ft / t_no - 1.0), "ms": t_ft * 1e3,
                     "max_rel_err_vs_oracle": err, "max_rel_err_injected_run": err_inj,
                     "flips": nflip, "detected": rep["detected"], "rc": rc,
                     "slices": S, "pairs": npairs if S else (1 if S == 0 else None),
                     "checksums": "fp64" if (S is None or ck == 2) else ("fp32" if ck == 1 else "none"),
                     "engine": "dfma" if S is None else ("mma.sync_int8" if eng == "i8" else
                                                         "mma.sync" if (eng == "mma" or (ck == 1 and S != 0))
                                                         else "tcgen05" if eng == "tc" else "tcgen05_persistent"),
                     "unprotected_kernel_ms": kms}
        if S is not None:
            # tensor work of the unprotected kernel: every kept pair is a 2MNK bf16 (or int8) product
            tf = npairs * flops / (kms / 1e3) / 1e12
            if eng == "i8":
                res[name]["kernel_int8_tops"] = tf
            else:
                res[name]["kernel_bf16_tflops"] = tf
                res[name]["kernel_frac_of_bf16_peak"] = tf / peaks["bf16_tflops"]
        print(json.dumps({name: res[name]}), flush=True)
    base = res["fp64_dfma"]["tflops_fp64_equiv"] if "fp64_dfma" in res else float("nan")
    line = {"metric": "split-precision FT-GEMM TFLOP/s (FP64-equivalent, 2MNK) and max error vs FP64 oracle",
            "config": {"workload": f"split_{n}cubed_loguniform1e-3to1e3_flips1per64tiles", "rows_checked": len(rows)},
            "results": res, "speedup_vs_fp64_dfma": {k: v["tflops_fp64_equiv"] / base for k, v in res.items()},
            "mma_sync_bf16_peak_tflops_measured": 595, "bf16_peak_tflops": peaks["bf16_tflops"], "peak_source": peaks["source"]}
    print(json.dumps(line), flush=True)


def config5(args):
    """32768^3, normal(0,1), alpha 1, beta 1: the FP64 FT-DGEMM timed
    fault-free and unprotected, then one call with flips at a rate of
    --flip-rate per minute of the fault-free time (seeded positions, k-steps
    and bits 0..62); the same inputs through the emulated FP64 forms on the
    tensor cores (S = 7 and 11, FP64 checksums, one exponent-bit flip per 64
    tiles).  Checked against the FP64 oracle on sampled rows and on every
    injected element."""
    import numpy as np
    import torch
    import oracle
    from paper_2305_02444_gb300 import build, ftgemm, inputs
    build.build()
    torch.cuda.set_device(0)
    s = torch.cuda.current_stream()
    n = args.size
    A = inputs.matrix(n, n, SEED, "normal", device="cuda")
    B = inputs.matrix(n, n, SEED + 1, "normal", device="cuda")
    C0 = inputs.matrix(n, n, SEED + 2, "normal", device="cuda")
    C = C0.clone()
    flops = 2.0 * n ** 3
    tiles = (-(-n // 128)) ** 2
    rng = np.random.default_rng(SEED)
    rows = np.sort(rng.choice(n, size=args.split_rows, replace=False))
    Ah, Bh, C0h = A.cpu().T.numpy(), B.cpu().T.numpy(), C0.cpu().T.numpy()
    refs = []
    for i in rows:
        r, E = oracle.gemm("N", "N", 1.0, Ah[i:i + 1], Bh, 1.0, C0h[i:i + 1], want_E=True)
        refs.append((r[0], E[0]))

    def one(fn):
        C.copy_(C0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        out = fn()
        e1.record(s)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, out

    def row_errors(tol_scale):
        out = C.cpu().T.numpy()
        worst_rel, within = 0.0, True
        for i, (r, E) in zip(rows, refs):
            worst_rel = max(worst_rel, float(np.abs(out[i] - r).max() / np.abs(r).max()))
            within = within and bool(np.all(np.abs(out[i] - r) <= tol_scale(E)))
        return out, worst_rel, within

    res = {}
    # FP64 FT-DGEMM
    t_no, _ = one(lambda: ftgemm.ftgemm_d_noft("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n))
    t_ft, _ = one(lambda: ftgemm.ftgemm_d("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, loc_cap=0))
    nflip = max(1, int(round(args.flip_rate * t_ft / 60.0)))
    assert ftgemm.ftgemm_set_injection(mode=1, seed=SEED, count=nflip) == 0
    try:
        t_inj, (rc, rep) = one(lambda: ftgemm.ftgemm_d("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n,
                                                       loc_cap=65536))
        log = ftgemm.ftgemm_injection_log()
    finally:
        ftgemm.ftgemm_set_injection(mode=0)
    out, rel, within = row_errors(lambda E: oracle.parity_tol(n, E))
    # every injected element against the oracle (faults below the threshold
    # stay, within their own effect)
    inj_ok = 0
    for L in log:
        i, j = L["row"], L["col"]
        r, E = oracle.gemm("N", "N", 1.0, Ah[i:i + 1], Bh[:, j:j + 1], 1.0, C0h[i:i + 1, j:j + 1], want_E=True)
        d = L["after"] - L["before"]
        eff = abs(d) if np.isfinite(d) else float("inf")
        # above-threshold faults are corrected; below-threshold ones stay
        err = abs(out[i, j] - r[0, 0])
        if err <= oracle.parity_tol(n, E)[0, 0] or (np.isfinite(eff) and err <= 2 * eff + oracle.parity_tol(n, E)[0, 0]):
            inj_ok += 1
    res["fp64_dfma"] = {"tflops": flops / t_ft / 1e12, "unprotected_tflops": flops / t_no / 1e12,
                        "pct_fp64_peak": 100.0 * flops / t_ft / 1e12 / FP64_PEAK_TFLOPS,
                        "ft_overhead_pct": 100.0 * (t_ft / t_no - 1.0), "s": t_ft,
                        "injected_call_tflops": flops / t_inj / 1e12, "flip_rate_per_min": args.flip_rate,
                        "flips": nflip, "detected": rep["detected"], "corrected": rep["corrected"],
                        "checksum_only": rep["checksum_only"], "rc": rc,
                        "injected_elements_within_bound": inj_ok, "sampled_rows_within_parity_bound": within,
                        "max_rel_err_sampled_rows": rel}
    print(json.dumps({"fp64_dfma": res["fp64_dfma"]}), flush=True)
    # emulated FP64 on the tensor cores
    w = 5  # slice width at this K
    for S in (7, 11):
        npairs = S * (S + 1) // 2
        t_no, _ = one(lambda: ftgemm.ftgemm_d_split("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, nslices=S,
                                                    ft=0, report=False))
        t_ft, _ = one(lambda: ftgemm.ftgemm_d_split("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n, nslices=S,
                                                    ft=2, report=False))
        nf = math.ceil(tiles / 64)
        flips = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(npairs)), 62) for _ in range(nf)]
        assert ftgemm.ftgemm_set_injection(mode=2, flips=flips) == 0
        try:
            _, (rc, rep) = one(lambda: ftgemm.ftgemm_d_split("N", "N", n, n, n, 1.0, A, n, B, n, 1.0, C, n,
                                                             nslices=S, ft=2, loc_cap=0))
        finally:
            ftgemm.ftgemm_set_injection(mode=0)
        _, rel, _ = row_errors(lambda E: oracle.parity_tol(n, E))
        res[f"emulated_S{S}_fp64ck"] = {"tflops_fp64_equiv": flops / t_ft / 1e12,
                                        "unprotected_tflops": flops / t_no / 1e12,
                                        "ft_overhead_pct": 100.0 * (t_ft / t_no - 1.0), "s": t_ft,
                                        "bits_kept": w * S, "flips": nf, "detected": rep["detected"], "rc": rc,
                                        "max_rel_err_sampled_rows": rel}
        print(json.dumps({f"emulated_S{S}_fp64ck": res[f"emulated_S{S}_fp64ck"]}), flush=True)
    print(json.dumps({"metric": "config 5: FT-GEMM at 32768^3, normal(0,1), beta 1, flips at a rate",
                      "config": {"workload": f"ftdgemm_{n}cubed_normal_a1_b1_rate{args.flip_rate:g}perminute",
                                 "rows_checked": len(rows)}, "results": res}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ftgemm", choices=["ftgemm", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=8192, help="M = N = K (default 8192)")
    ap.add_argument("--sweep", action="store_true", help="per-size results of the square sweep")
    ap.add_argument("--sweep-shapes", default="", help="comma list of MxNxK for --sweep")
    ap.add_argument("--sweep-warmup", type=int, default=3)
    ap.add_argument("--sweep-reps", type=int, default=0, help="timed calls per path (0: by size)")
    ap.add_argument("--sweep-dist", default="uniform", help="input distribution for --sweep")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--batched", action="store_true", help="the batched workload (512 small problems)")
    ap.add_argument("--panel-sweep", action="store_true", help="per-k-panel verification: overhead and faults")
    ap.add_argument("--panel-sizes", default="8192,1024", help="M = N = K of --panel-sweep")
    ap.add_argument("--panel-slabs", default="2,8,32,128", help="k-slabs per panel check for --panel-sweep")
    ap.add_argument("--split", action="store_true", help="split-precision forms (BF16 tensor cores)")
    ap.add_argument("--split-slices", default="7,9,11", help="slice counts for --split")
    ap.add_argument("--split-rows", type=int, default=4, help="rows checked against the oracle")
    ap.add_argument("--split-engine", default="tc,mma",
                    help="split engines: tc (tcgen05, one CTA per tile), tcp (persistent tcgen05), "
                         "mma (mma.sync), i8 (mma.sync with INT8 slices)")
    ap.add_argument("--split-forms", default="", help="comma list of form names to run (default: all)")
    ap.add_argument("--config5", action="store_true", help="32768^3 normal(0,1), beta 1, flips at a rate")
    ap.add_argument("--flip-rate", type=float, default=360.0, help="flips per minute for --config5")
    args = ap.parse_args()
    if args.config5 and args.size == 8192:
        args.size = 32768
    set_size(args.size)
    if args.config5:
        return config5(args)
    if args.sweep:
        return sweep(args)
    if args.panel_sweep:
        return panel_sweep(args)
    if args.split:
        if args.warmup < 3:
            args.warmup = 3
        args.split_slices = [int(x) for x in args.split_slices.split(",") if x]
        return split(args)
    if args.batched:
        if args.warmup < 3:
            args.warmup = 3
        return batched(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)

    ws, rank, local = dist_env()
    import torch
    import torch.distributed as dist
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, ws, "cuda")

    from paper_2305_02444_gb300 import build, ftgemm, inputs
    build.build()
    lib = ftgemm.lib()
    s = torch.cuda.current_stream()
    seed = SEED + 1000 * rank
    A = inputs.matrix(M, K, seed, device="cuda")
    B = inputs.matrix(K, N, seed + 1, device="cuda")
    C = inputs.matrix(M, N, seed + 2, device="cuda")
    C0 = C.clone()
    flops = 2.0 * M * N * K

    def ft_call(rep=True):
        rc, r = ftgemm.ftgemm_d("N", "N", M, N, K, ALPHA, A, M, B, K, BETA, C, M, report=rep, loc_cap=0)
        if rc:
            raise RuntimeError(f"ftgemm_d: {ftgemm.ftgemm_strerror(rc)}")
        return r

    def noft_call():
        rc = ftgemm.ftgemm_d_noft("N", "N", M, N, K, ALPHA, A, M, B, K, BETA, C, M)
        if rc:
            raise RuntimeError(f"ftgemm_d_noft: {ftgemm.ftgemm_strerror(rc)}")

    def timed(fn, steps, with_report=False):
        reps = []
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(steps):
            r = fn()
            if with_report:
                reps.append(r)
        e1.record(s)
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1) / 1e3), reps

    # warm-up (all three paths)
    ftgemm.ftgemm_set_injection(mode=1, seed=seed, count=FLIPS)
    for _ in range(args.warmup):
        ft_call()
    ftgemm.ftgemm_set_injection(mode=0)
    for _ in range(args.warmup):
        noft_call()
    ft_call()

    # 1) headline: FT path with injection, inputs resident in HBM
    clk_path = os.path.join(os.environ.get("FTGEMM_BENCH_DIR", tempfile.gettempdir()), f"bench_clocks_r{rank}.csv")
    proc, fh = sample_clocks_start(local, clk_path)
    ftgemm.ftgemm_set_injection(mode=1, seed=seed, count=FLIPS)
    l0 = ftgemm.ftgemm_launch_count()
    ftgemm.ftgemm_timing(True)
    t_inj, reps = timed(lambda: ft_call(True), args.steps, with_report=True)
    main_ms, main_n, aux_ms = ftgemm.ftgemm_timing_read()
    ftgemm.ftgemm_timing(False)
    launches = ftgemm.ftgemm_launch_count() - l0
    ftgemm.ftgemm_set_injection(mode=0)
    # 2) unprotected kernel and fault-free FT path (overhead)
    ftgemm.ftgemm_timing(True)
    t_noft, _ = timed(noft_call, args.steps)
    noft_ms, noft_n, _ = ftgemm.ftgemm_timing_read()
    ftgemm.ftgemm_timing(True)
    t_ft, _ = timed(lambda: ft_call(False), args.steps)
    ft_ms, ft_n, ft_aux = ftgemm.ftgemm_timing_read()
    ftgemm.ftgemm_timing(False)

    def unfused_call():
        rc, _ = ftgemm.ftgemm_d_unfused("N", "N", M, N, K, ALPHA, A, M, B, K, BETA, C, M, report=False)
        if rc:
            raise RuntimeError(f"ftgemm_d_unfused: {ftgemm.ftgemm_strerror(rc)}")
    unfused_call()
    t_unf, _ = timed(unfused_call, max(2, args.steps // 2))
    t_unf = t_unf / max(2, args.steps // 2) * args.steps
    clocks = sample_clocks_stop(proc, fh, clk_path)

    # 3) end to end through the host-buffer entry point (pinned host memory)
    hA, hB = A.cpu().pin_memory(), B.cpu().pin_memory()
    hC0 = C0.cpu()
    hC = hC0.pin_memory()
    ftgemm.ftgemm_set_injection(mode=1, seed=seed, count=FLIPS)
    rc, _ = ftgemm.ftgemm_d_host("N", "N", M, N, K, ALPHA, hA, M, hB, K, BETA, hC, M, loc_cap=0)
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        rc, _ = ftgemm.ftgemm_d_host("N", "N", M, N, K, ALPHA, hA, M, hB, K, BETA, hC, M, loc_cap=0)
        if rc:
            raise RuntimeError(ftgemm.ftgemm_strerror(rc))
    torch.cuda.synchronize()
    barrier()
    t_e2e = max_over_ranks((time.perf_counter() - te0) / args.e2e_steps)
    ftgemm.ftgemm_set_injection(mode=0)

    # the whole job's fault counts: every rank's reports summed (all ranks
    # take part before rank 0 alone reports)
    det = [r["detected"] for r in reps]
    cor = [r["corrected"] for r in reps]
    job_counts = [int(round(reduce_sum(float(x), ws, "cuda")))
                  for x in (det[-1] if det else 0, cor[-1] if cor else 0, sum(det), sum(cor))]

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    value = job_tflops(ws, flops, args.steps, t_inj)
    avg_main = main_ms / max(1, main_n) / 1e3
    achieved = flops / avg_main / 1e12
    line = {
        "metric": METRIC,
        "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_inj / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": main_config(),
        "pct_fp64_peak": 100.0 * value / ws / FP64_PEAK_TFLOPS,
        "overhead_pct": {"ft_vs_noft": 100.0 * (t_ft / t_noft - 1.0),
                         "ft_injected_vs_noft": 100.0 * (t_inj / t_noft - 1.0),
                         "noft_tflops": flops * args.steps / t_noft / 1e12,
                         "ft_tflops": flops * args.steps / t_ft / 1e12,
                         "main_kernel_ft_vs_noft": 100.0 * ((ft_ms / max(1, ft_n)) / (noft_ms / max(1, noft_n)) - 1.0),
                         "unfused_vs_noft": 100.0 * (t_unf / t_noft - 1.0)},
        "checksum_pass": {"ms": ft_aux / max(1, ft_n), "bytes_read": 8 * (M * K + K * N),
                          "gbs": 8 * (M * K + K * N) / (max(1e-9, ft_aux / max(1, ft_n)) / 1e3) / 1e9,
                          "what": "operand checksum vectors (and the report reset) before each fault-free call"},
        "errors": {"injected_per_step": FLIPS * ws, "detected_per_step": job_counts[0] if det else None,
                   "corrected_per_step": job_counts[1] if cor else None,
                   "detected_total": job_counts[2], "corrected_total": job_counts[3],
                   "per_minute": 60.0 * FLIPS * ws / (t_inj / args.steps)},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": read_traffic(f"ftdgemm_nn_ft_inj_{M}") if M == N == K else None,
                     "kernel": "ftdgemm_kernel<N,N,FT,INJ> (main FT-DGEMM kernel)",
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.070 GHz",
                     "pre_kernel_ms_per_step": aux_ms / max(1, main_n)},
        "e2e": {"value": job_tflops(ws, flops, 1, t_e2e), "unit": "TFLOP/s",
                "h2d_bytes_per_step": 3 * M * N * 8, "d2h_bytes_per_step": M * N * 8,
                "steps": args.e2e_steps},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = run_cpu_baseline()
        # the fault accounting of one call, classified by the oracle on the CPU
        C.copy_(C0)
        ftgemm.ftgemm_set_injection(mode=1, seed=seed, count=FLIPS)
        try:
            rc, rep = ftgemm.ftgemm_d("N", "N", M, N, K, ALPHA, A, M, B, K, BETA, C, M, loc_cap=4 * FLIPS + 64)
            log = ftgemm.ftgemm_injection_log()
        finally:
            ftgemm.ftgemm_set_injection(mode=0)
        torch.cuda.synchronize()
        if rc == 0:
            line["errors"].update(flip_accounting(log, rep, hA.T.numpy(), hB.T.numpy(), hC0.T.numpy(),
                                                  lambda i, j: float(C[j, i])))
    print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
