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


def decay(npoints: int, bs: int, seed: int, device, nfun: int = 5, alpha: float = 0.5,
          cutoff: float = 1e-6, density: float = 0.1, chunk_blocks: int | None = None,
          cross: tuple[int, int] | None = None, keep=None, points=None, blocks=None):
    """Device tensors (n, brow, bcol, vals) of the decay-type matrix of
    synth.decay: points from synth.decay_points (host, recursive bisection
    order), blocks whose bounding boxes come within the cutoff radius, entries
    s_ij exp(-alpha r_ij) below `cutoff` set to zero.  Entries may differ from
    the numpy generator in the last bit (exp on the device).  cross=(lo, hi):
    only the blocks whose block row or block column lies in [lo, hi) (the
    operands of the C blocks [lo, hi)^2 of A*A).  keep=(row_mask, col_mask),
    boolean device tensors over the block rows / columns: only the blocks
    whose row is in row_mask or whose column is in col_mask (the operands of
    the C blocks of those rows and columns).  points: the host array of
    decay_points(npoints, seed, density), if already made."""
    from . import decay_points

    pts_np = decay_points(npoints, seed, density) if points is None else points
    pts = torch.from_numpy(pts_np).to(device)
    n = npoints * nfun
    if blocks is None:
        brow, bcol = decay_blocks(npoints, bs, seed, device, nfun, alpha, cutoff, density,
                                  cross, keep, pts_np)
    else:   # the candidate blocks of decay_blocks, filtered by `keep`
        brow, bcol = blocks
        if keep is not None:
            sel = keep[0][brow] | keep[1][bcol]
            brow, bcol = brow[sel], bcol[sel]
    return n, brow.to(torch.int32), bcol.to(torch.int32), decay_values(
        pts, brow, bcol, bs, n, npoints, seed, nfun, alpha, cutoff, chunk_blocks)


def decay_blocks(npoints: int, bs: int, seed: int, device, nfun: int = 5, alpha: float = 0.5,
                 cutoff: float = 1e-6, density: float = 0.1, cross=None, keep=None, points=None):
    """Candidate blocks (brow, bcol: int64 device tensors, row-major) of the
    decay-type matrix: block pairs whose point groups' bounding boxes come
    within the cutoff radius (their entries may still all fall below it)."""
    import math

    from . import decay_points

    pts_np = decay_points(npoints, seed, density) if points is None else points
    pts = torch.from_numpy(pts_np).to(device)
    n = npoints * nfun
    nbk = -(-n // bs)
    rcut = -math.log(cutoff) / alpha
    ptidx = torch.clamp(torch.arange(nbk * bs, device=device) // nfun, max=npoints - 1).view(nbk, bs)
    bp = pts[ptidx]                      # [nbk, bs, 3]
    lo, hi = bp.min(1).values, bp.max(1).values
    rows, cols = [], []
    step = max(1, (1 << 24) // nbk)
    if cross is not None:
        incross = torch.zeros(nbk, dtype=torch.bool, device=device)
        incross[cross[0]:cross[1]] = True
    for r0 in range(0, nbk, step):
        r1 = min(nbk, r0 + step)
        gap = torch.clamp(torch.maximum(lo[r0:r1, None, :] - hi[None, :, :],
                                        lo[None, :, :] - hi[r0:r1, None, :]), min=0.0)
        near = (gap * gap).sum(-1).sqrt() <= rcut
        if cross is not None:
            near &= incross[r0:r1, None] | incross[None, :]
        if keep is not None:
            near &= keep[0][r0:r1, None] | keep[1][None, :]
        bi, bj = torch.nonzero(near, as_tuple=True)
        rows.append(bi + r0)
        cols.append(bj)
    return torch.cat(rows).to(torch.int64), torch.cat(cols).to(torch.int64)


def decay_values(pts, brow, bcol, bs: int, n: int, npoints: int, seed: int, nfun: int = 5,
                 alpha: float = 0.5, cutoff: float = 1e-6, chunk_blocks: int | None = None):
    """Entries s_ij exp(-alpha r_ij) of the given blocks (dropped below
    `cutoff`), pts the device tensor of the points."""
    device = pts.device
    brow = brow.to(torch.int64)
    bcol = bcol.to(torch.int64)
    if chunk_blocks is None:
        chunk_blocks = max(1, (1 << 27) // (bs * bs))  # 2^27 entries per chunk
    nb_ = brow.numel()
    vals = torch.empty((nb_, bs, bs), dtype=torch.float64, device=device)
    r = torch.arange(bs, dtype=torch.int64, device=device)
    sseed = seed ^ 0x2545F491
    for t0 in range(0, nb_, chunk_blocks):
        t1 = min(nb_, t0 + chunk_blocks)
        gi = brow[t0:t1, None, None] * bs + r[None, :, None]
        gj = bcol[t0:t1, None, None] * bs + r[None, None, :]
        pi = torch.clamp(gi // nfun, max=npoints - 1)
        pj = torch.clamp(gj // nfun, max=npoints - 1)
        d = pts[pi] - pts[pj]
        rr = (d * d).sum(-1).sqrt()
        lo_i, hi_i = torch.minimum(gi, gj), torch.maximum(gi, gj)
        sgn = torch.where((hash3(sseed, lo_i, hi_i) & 1) == 1, -1.0, 1.0).to(torch.float64)
        sgn = torch.where(gi == gj, torch.ones_like(sgn), sgn)
        v = sgn * torch.exp(-alpha * rr)
        v = torch.where(v.abs() < cutoff, torch.zeros_like(v), v)
        v = torch.where((gi < n) & (gj < n), v, torch.zeros_like(v))
        vals[t0:t1] = v
    return vals
