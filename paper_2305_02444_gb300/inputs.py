"""Seeded synthetic inputs (no method arithmetic here).

The paper evaluates square random matrices (§3: 2048^2..10240^2 serial,
512^2..20480^2 parallel); these generators stand in for them.  Both the GPU
path (bench) and the tests draw from here; the oracle never imports it.

A column-major matrix of `rows` x `cols` with leading dimension `ld` is held
as a torch tensor of shape (cols, ld) in row-major order: element (r, c) is
storage[c, r].  `logical(storage, rows)` returns the (rows, cols) view.
"""
from __future__ import annotations

import math

import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & ((1 << 63) - 1))
    return g


def matrix(rows: int, cols: int, seed: int, dist: str = "uniform", ld: int | None = None,
           device="cpu", fill_pad: float = float("nan")) -> torch.Tensor:
    """Column-major fp64 storage (cols, ld) with entries drawn from `dist`:
    'uniform' U[-1,1]; 'normal' N(0,1); 'loguniform' sign-random with |x|
    log-uniform in [1e-3, 1e3].  Padding rows (ld > rows) hold fill_pad."""
    ld = max(1, rows) if ld is None else ld
    g = _gen(seed, device)
    st = torch.full((cols, ld), fill_pad, dtype=torch.float64, device=device)
    if rows == 0 or cols == 0:
        return st
    if dist == "uniform":
        v = torch.rand((cols, rows), generator=g, dtype=torch.float64, device=device) * 2 - 1
    elif dist == "normal":
        v = torch.randn((cols, rows), generator=g, dtype=torch.float64, device=device)
    elif dist == "loguniform":
        e = torch.rand((cols, rows), generator=g, dtype=torch.float64, device=device) * 6 - 3
        s = torch.randint(0, 2, (cols, rows), generator=g, device=device).to(torch.float64) * 2 - 1
        v = s * torch.pow(10.0, e)
    else:
        raise ValueError(dist)
    st[:, :rows] = v
    return st


def logical(storage: torch.Tensor, rows: int) -> torch.Tensor:
    """(rows, cols) view of column-major storage (cols, ld)."""
    return storage[:, :rows].T


def batched_sizes(count: int, seed: int, lo: int = 32, hi: int = 1024):
    """(M, N, K) triples, each log-uniform in [lo, hi] (batched workload)."""
    g = _gen(seed, "cpu")
    u = torch.rand((count, 3), generator=g, dtype=torch.float64)
    v = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))).round().to(torch.int64)
    return [tuple(int(x) for x in row) for row in v]
