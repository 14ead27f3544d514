"""Device-side (torch) copy of the counter-based generators of ``synth``.

Same SplitMix64 hashing of (seed, row, column) in int64 arithmetic with
wrap-around, so block presence and uniform entries are bit-identical to the
numpy generators (tested on the CPU); only input creation lives here.  Used
for large batched workloads whose host generation would take minutes.
"""
from __future__ import annotations

import numpy as np
import torch

from . import BlockCOO, batched_specs


def _s64(u: int) -> int:
    """uint64 constant as the int64 with the same bits."""
    return u - (1 << 64) if u >= (1 << 63) else u


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_C1 = _s64(0xBF58476D1CE4E5B9)
_C2 = _s64(0x94D049BB133111EB)


def _shr(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bits."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def splitmix64(x: torch.Tensor) -> torch.Tensor:
    z = x + _GOLDEN
    z = (z ^ _shr(z, 30)) * _C1
    z = (z ^ _shr(z, 27)) * _C2
    return z ^ _shr(z, 31)


def hash3(seed: int, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    s = splitmix64(torch.tensor(_s64(seed & 0xFFFFFFFFFFFFFFFF), dtype=torch.int64,
                                device=a.device))
    return splitmix64(splitmix64(s ^ a) ^ b)


def uniform01(h: torch.Tensor) -> torch.Tensor:
    return _shr(h, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def random_blocks(n: int, bs: int, p: float, seed: int, device, ncols: int | None = None):
    """Device tensors (brow, bcol, vals) of synth.random_blocks(..., dist="uniform")."""
    ncols = n if ncols is None else ncols
    mb, nb = -(-n // bs), -(-ncols // bs)
    I = torch.arange(mb, dtype=torch.int64, device=device)[:, None].expand(mb, nb)
    J = torch.arange(nb, dtype=torch.int64, device=device)[None, :].expand(mb, nb)
    keep = uniform01(hash3(seed ^ 0x5BD1E995, I, J)) < p
    brow = I[keep].contiguous()
    bcol = J[keep].contiguous()
    r = torch.arange(bs, dtype=torch.int64, device=device)
    gi = brow[:, None, None] * bs + r[None, :, None]
    gj = bcol[:, None, None] * bs + r[None, None, :]
    vals = 2.0 * uniform01(hash3(seed, gi, gj)) - 1.0
    vals = torch.where((gi < n) & (gj < ncols), vals, torch.zeros_like(vals))
    nz = (vals != 0).flatten(1).any(1)
    return brow[nz].to(torch.int32), bcol[nz].to(torch.int32), vals[nz].contiguous()


def batched(nprod: int, seed: int, device, bs: int = 32, **kw):
    """Device tensors of synth.batched(..., ) with uniform entries: a list of
    ((n, brow, bcol, vals) for A, same for B)."""
    out = []
    for t, (n, dens) in enumerate(batched_specs(nprod, seed, bs=bs, **kw)):
        a = random_blocks(n, bs, dens, seed * 1000003 + 2 * t + 1, device)
        b = random_blocks(n, bs, dens, seed * 1000003 + 2 * t + 2, device)
        out.append(((n,) + a, (n,) + b))
    return out


def to_host(n: int, bs: int, brow, bcol, vals) -> BlockCOO:
    return BlockCOO(n, n, bs, brow.cpu().numpy(), bcol.cpu().numpy(), vals.cpu().numpy())
