"""Seeded synthetic inputs for the biquaternion matrix product.

This module is shared by the CPU oracle tests and the CUDA path; it holds none
of the method's arithmetic (no products, no ops, no pre- or post-additions):
only random draws, shapes and zero patterns.

Every generator returns an 8 x rows x cols float64 torch tensor (component-
major, the storage order [M1..M8] of the paper's Sec. III), drawn from a
``torch.Generator`` seeded with ``seed`` on ``device``.  A CPU and a CUDA
generator give different streams for the same seed; each test draws its input
once and hands copies of the same tensor to both sides.

Workload recipes (the paper benchmarks seeded random host matrices, Sec. IV;
it ships no data set, so these stand in for its Fock/Kohn-Sham matrices):
  * ``uniform``:   iid U[-1, 1] in every active component.
  * ``fock_like``: N(0,1) * exp(-|i-j|/200) (a banded, exponentially decaying
    matrix such as a Fock matrix in a localised basis), optionally with
    per-row scales 10**U(-6, 0) shared by the eight components of a row.
  * ``small_int``: integers in [-8, 8]; every FP64 step of the product is then
    exact for inner dimensions up to a few thousand, so results are compared
    bit for bit.
  * ``batch_shapes``: (m, n, k) drawn log-uniformly in [32, 1024].
Zero patterns (component activity flags, bit c-1 = component c stored):
  REAL = 0x01, COMPLEX = 0x11, TRS = 0x0F (real quaternion), TRA = 0xF0
  (i times a real quaternion), BQ = 0xFF (paper's Tables I-II notation
  [1,0,0,0,0,0,0,0] ... [1,1,1,1,1,1,1,1]).
"""
from __future__ import annotations

import math

import torch

REAL, COMPLEX, TRS, TRA, BQ = 0x01, 0x11, 0x0F, 0xF0, 0xFF
FLAG_NAMES = {"REAL": REAL, "COMPLEX": COMPLEX, "TRS": TRS, "TRA": TRA, "BQ": BQ}


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def apply_flags(X: torch.Tensor, flags: int) -> torch.Tensor:
    """Zero the components whose flag bit is clear (in place); returns X."""
    for c in range(8):
        if not (flags >> c) & 1:
            X[c].zero_()
    return X


def uniform(seed: int, rows: int, cols: int, flags: int = BQ, device="cpu") -> torch.Tensor:
    g = _gen(seed, device)
    X = torch.rand((8, rows, cols), generator=g, device=device, dtype=torch.float64)
    X.mul_(2.0).sub_(1.0)
    return apply_flags(X, flags)


def small_int(seed: int, rows: int, cols: int, flags: int = BQ, lo: int = -8, hi: int = 8,
              device="cpu") -> torch.Tensor:
    g = _gen(seed, device)
    X = torch.randint(lo, hi + 1, (8, rows, cols), generator=g, device=device).to(torch.float64)
    return apply_flags(X, flags)


def fock_like(seed: int, rows: int, cols: int, flags: int = BQ, decay: float = 200.0,
              row_scale: bool = False, device="cpu") -> torch.Tensor:
    """N(0,1) * exp(-|i-j|/decay); with row_scale, row i is multiplied by 10**U(-6,0)."""
    g = _gen(seed, device)
    X = torch.randn((8, rows, cols), generator=g, device=device, dtype=torch.float64)
    i = torch.arange(rows, device=device, dtype=torch.float64).view(rows, 1)
    j = torch.arange(cols, device=device, dtype=torch.float64).view(1, cols)
    # build the envelope in row blocks to bound temporary memory at large sizes
    blk = max(1, (1 << 26) // max(cols, 1))
    for r0 in range(0, rows, blk):
        r1 = min(rows, r0 + blk)
        env = torch.exp(-(i[r0:r1] - j).abs() / decay)
        X[:, r0:r1, :].mul_(env)
    if row_scale:
        u = torch.rand((rows,), generator=g, device=device, dtype=torch.float64)
        s = torch.pow(10.0, -6.0 * u)        # 10**U(-6, 0)
        X.mul_(s.view(1, rows, 1))
    return apply_flags(X, flags)


def batch_shapes(seed: int, count: int = 512, lo: int = 32, hi: int = 1024):
    """count (m, n, k) triples, each drawn independently log-uniform in [lo, hi]."""
    g = _gen(seed, "cpu")
    u = torch.rand((count, 3), generator=g, dtype=torch.float64)
    v = torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))
    dims = torch.round(v).to(torch.int64).clamp_(lo, hi)
    return [tuple(int(x) for x in row) for row in dims]


def complex_scalar(seed: int):
    """A seeded complex scalar with both parts in [-1, 1]."""
    g = _gen(seed, "cpu")
    u = torch.rand((2,), generator=g, dtype=torch.float64) * 2 - 1
    return complex(float(u[0]), float(u[1]))
