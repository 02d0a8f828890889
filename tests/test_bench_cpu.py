"""bench.py's host-side logic on CPU: the clock record of the timed region,
the DRAM-traffic record that is only used while the kernel source it was
taken on is unchanged, and the whole-job throughput arithmetic."""
from __future__ import annotations

import hashlib
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

pytest.importorskip("torch")
import bench  # noqa: E402


class _Proc:
    """Stands in for the nvidia-smi sampler process."""

    def __init__(self):
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def _clocks(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    proc, fh = _Proc(), open(tmp_path / "unused", "w")
    out = bench.sample_clocks_stop(proc, fh, str(path))
    assert proc.terminated
    return out


def test_clock_record_median_max_and_reasons(tmp_path):
    """Median SM clock under load, the maximum clock, and every throttle
    reason seen Active in any sample (nvidia-smi csv, noheader, nounits);
    malformed lines are skipped."""
    row = "0, {sm}, 2070, 1200.5, 0x{act:x}, {hw}, Not Active, Not Active, {pc}"
    lines = [row.format(sm=s, act=0, hw="Not Active", pc="Not Active") for s in (1900, 1950, 2000)]
    lines += [row.format(sm=1600, act=4, hw="Not Active", pc="Active"),
              row.format(sm=1700, act=8, hw="Active", pc="Not Active"),
              "garbage", "0, [N/A], 2070, 1, 0, Not Active, Not Active, Not Active, Not Active"]
    out = _clocks(tmp_path, lines)
    assert out["sm_mhz"] == 1900 and out["sm_max_mhz"] == 2070 and out["samples"] == 5
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    clean = _clocks(tmp_path, [row.format(sm=2070, act=0, hw="Not Active", pc="Not Active")] * 3)
    assert clean["reasons"] == [] and clean["sm_mhz"] == 2070


def test_clock_record_absent_without_sampler(tmp_path):
    assert bench.sample_clocks_stop(None, None, str(tmp_path / "none.csv")) is None
    assert _clocks(tmp_path, ["not a sample"]) is None


def test_traffic_only_for_the_kernel_source_it_was_taken_on(tmp_path, monkeypatch):
    """roofline.traffic comes from profiles/traffic.txt only while the
    recorded hash equals that of the current kernel source; any edit of the
    kernel, an unknown tag or a missing record gives null."""
    src_rel = os.path.join("paper_2305_02444_gb300", "csrc", "ftgemm_kernel.cuh")
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / os.path.dirname(src_rel))
    shutil.copy(os.path.join(ROOT, src_rel), tmp_path / src_rel)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic("k") is None                       # no record
    h = hashlib.sha256(open(tmp_path / src_rel, "rb").read()).hexdigest()[:16]
    (tmp_path / "profiles" / "traffic.txt").write_text(f"# header\n\nk {h} 12345\nother {h} 7\n")
    assert bench.read_traffic("k") == 12345.0
    assert bench.read_traffic("missing") is None
    with open(tmp_path / src_rel, "a") as f:
        f.write("// edited\n")
    assert bench.read_traffic("k") is None


def test_committed_traffic_record_is_well_formed():
    """Every record line: tag, 16 hex digits of the source hash, a byte count."""
    for line in open(os.path.join(ROOT, "profiles", "traffic.txt")):
        if line.startswith("#") or not line.strip():
            continue
        tag, h, nbytes = line.split()[:3]
        assert len(h) == 16 and int(h, 16) >= 0 and int(nbytes) > 0 and tag


def test_whole_job_throughput():
    """value = units of all ranks / the slowest rank's time (weak scaling)."""
    assert bench.job_tflops(1, 2.0e12, 4, 8.0) == pytest.approx(1.0)
    assert bench.job_tflops(4, 2.0e12, 4, 8.0) == pytest.approx(4.0)


def test_fp64_peak_from_unit_counts():
    """152 SMs x 2 FP64 FMAs per clock each x 2 flops per FMA x 2070 MHz; the
    measured peaks (or the stated fallback) carry both roofline denominators."""
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12)
    peaks = bench.measured_peaks()
    assert peaks["source"] in ("measured", "fallback") and peaks["hbm_gbs"] > 0 and peaks["bf16_tflops"] > 0


def test_main_assembles_the_line_with_fakes(monkeypatch, capsys):
    """bench.main() end to end on the CPU with the device and the library
    replaced by stand-ins: the JSON line carries every key of the contract,
    the fault counts of all timed steps, and no traffic figure for a size the
    DRAM capture was not taken at."""
    import json
    import torch
    from paper_2305_02444_gb300 import build as b, ftgemm, inputs

    class Stream:
        cuda_stream = 0

    class Event:
        def __init__(self, enable_timing=False):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 100.0

    real_matrix = inputs.matrix
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: Stream())
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self, *a, **k: self)
    monkeypatch.setattr(inputs, "matrix", lambda r, c, seed, dist="uniform", ld=None, device="cpu",
                        fill_pad=float("nan"): real_matrix(r, c, seed, dist, ld, "cpu", fill_pad))
    monkeypatch.setattr(b, "build", lambda *a, **k: None)
    monkeypatch.setattr(ftgemm, "lib", lambda: object())
    monkeypatch.setattr(ftgemm, "ftgemm_d", lambda *a, report=True, **k: (0, {"detected": 3, "corrected": 3}
                                                                         if report else None))
    monkeypatch.setattr(ftgemm, "ftgemm_d_noft", lambda *a, **k: 0)
    monkeypatch.setattr(ftgemm, "ftgemm_d_unfused", lambda *a, **k: (0, None))
    monkeypatch.setattr(ftgemm, "ftgemm_d_host", lambda *a, **k: (0, {"detected": 3, "corrected": 3}))
    monkeypatch.setattr(ftgemm, "ftgemm_set_injection", lambda **k: 0)
    count = iter(range(0, 10 ** 6, 6))
    monkeypatch.setattr(ftgemm, "ftgemm_launch_count", lambda: next(count))
    monkeypatch.setattr(ftgemm, "ftgemm_timing", lambda on: 0)
    monkeypatch.setattr(ftgemm, "ftgemm_timing_read", lambda: (90.0, 4, 1.0))
    monkeypatch.setattr(bench, "sample_clocks_start", lambda dev, path: (None, None))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--size", "256", "--steps", "4", "--warmup", "3",
                                      "--no-cpu-baseline"])
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    try:
        bench.main()
    finally:
        bench.set_size(8192)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches",
                "clocks", "errors"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 4 and line["config"]["M"] == 256
    assert line["errors"]["detected_per_step"] == 3 and line["errors"]["detected_total"] == 12
    assert line["errors"]["injected_per_step"] == 1
    assert line["roofline"]["traffic"] is None and line["roofline"]["bound"] == "alu"
    assert line["e2e"]["h2d_bytes_per_step"] == 3 * 256 * 256 * 8
    assert line["gpu_launches"] == 6


def test_clock_sampler_absent_tool(tmp_path, monkeypatch):
    """Without nvidia-smi the sampler reports no clock record (and leaves no
    open file); the bench line then carries "clocks": null."""
    monkeypatch.setenv("PATH", str(tmp_path))
    proc, fh = bench.sample_clocks_start(0, str(tmp_path / "c.csv"))
    assert proc is None and fh is None
    assert bench.sample_clocks_stop(proc, fh, str(tmp_path / "c.csv")) is None


def test_flip_accounting_against_the_oracles_own_call():
    """The bench's fault accounting of one call, fed with the oracle's own
    FT-DGEMM (256 x 256 x 512, the bench's alpha and beta, 40 seeded faults
    over every bit range): the classification counts add up, every fault
    above the threshold band is found among the located elements, and each
    located element is checked against the oracle's value.  A planted wrong
    output element makes the check fail."""
    import numpy as np
    oracle = pytest.importorskip("oracle")
    from paper_2305_02444_gb300 import inputs
    M_, N_, K_ = 256, 256, 512
    A = inputs.matrix(M_, K_, 5).T.numpy()
    B = inputs.matrix(K_, N_, 6).T.numpy()
    C = inputs.matrix(M_, N_, 7).T.numpy()
    flips = oracle.random_flips(99, 40, M_, N_, K_ // 16)
    r = oracle.ft_gemm("N", "N", bench.ALPHA, A, B, bench.BETA, C, flips=flips)
    log = [{"row": int(i), "col": int(j), "kstep": int(s), "bit": int(b), "kfirst": 0} for i, j, s, b in flips]
    rep = {"detected": r.counts["detected"], "corrected": r.counts["corrected"], "locs": r.locs}
    out = bench.flip_accounting(log, rep, A, B, C, lambda i, j: float(r.C[i, j]))
    import json
    json.dumps(out)                                   # goes into the bench's JSON line as it is
    acc = out["checked_call"]
    assert acc["injected"] == 40
    assert acc["above_threshold"] + acc["in_guard_band"] + acc["below_threshold"] == 40
    assert acc["above_threshold"] >= 10 and acc["below_threshold"] >= 5      # bits 0..62 span both sides
    assert acc["detected_above"] == acc["above_threshold"] and acc["detected_elsewhere"] == 0
    assert acc["every_above_threshold_fault_fixed"] and acc["located_within_parity_bound"]
    i, j = r.locs[0][:2]
    bad = bench.flip_accounting(log, rep, A, B, C, lambda a, b: float(r.C[a, b]) + (1.0 if (a, b) == (i, j) else 0))
    assert not bad["checked_call"]["located_within_parity_bound"]
    assert not bad["checked_call"]["every_above_threshold_fault_fixed"]
