"""GPU probes behind two design decisions, compiled with nvcc when the test
runs (tests/probes/*.cu):

- fp64_rate.cu: the FP64 pipe's rate with DFMA and with the legacy FP64
  tensor instruction (mma.sync m8n8k4 f64).  The FT-DGEMM mainloop uses DFMA
  because the FP64 tensor path shares the same pipe and delivers less; the
  roofline peak of the FP64 kernels is SMs x 2 DFMA/clk x 2 flop x clock.
- umma_issue.cu: tcgen05.mma issue rate when the issuing thread also polls an
  mbarrier versus when another warp polls and hands over at a named barrier
  (the split kernel's waiter warp).
- bit_tricks.cu: the integer shortcuts that keep conversions and scalings
  off the FP64 pipe give the same bits as the CUDA conversions and FP64
  operations they replace.

The assertions are loose bounds on what the designs rely on; `-s` prints the
measured figures."""
from __future__ import annotations

import json
import os
import subprocess
import tempfile

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def build_and_run(name):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_02444_gb300 import build
    src = os.path.join(HERE, "probes", name + ".cu")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, name)
        subprocess.run([build.nvcc()] + build.ARCH + ["-O3", "-std=c++17", "-I" + build.CSRC,
                       "-I" + os.path.join(build.ROOT, "include"), src, "-o", exe, "-lcuda"],
                       check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    print(name, json.dumps(d))
    return d


def test_fp64_pipe_rates():
    d = build_and_run("fp64_rate")
    derived = d["sms"] * 2 * 2 * d["max_clock_mhz"] * 1e6 / 1e12
    assert 0.8 * derived <= d["dfma_tflops"] <= 1.02 * derived
    assert d["dmma_m8n8k4_tflops"] < d["dfma_tflops"]


def test_tcgen05_issue_with_and_without_polling():
    d = build_and_run("umma_issue")
    c = d["cycles_per_mma"]
    # 128 x 128 x 16 BF16 MMA = 262144 FMAs at 4096 FMA/clk/SM = 64 cycles
    assert c["plain"] <= 72 and c["handoff"] <= 72
    assert c["poll"] >= 1.3 * c["handoff"]


def test_integer_shortcuts_match_the_conversions():
    """FP32 round-up of |x|, bf16 rounding, power-of-two scaling, FP32 -> FP64
    and the scaled exact pair products: bit-identical to the conversions and
    FP64 operations on 2^26 inputs (ties, range edges, subnormals, Inf, NaN)."""
    d = build_and_run("bit_tricks")
    assert d["inputs"] == 1 << 26
    assert all(v == 0 for v in d["mismatch"].values()), d
