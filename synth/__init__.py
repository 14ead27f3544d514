"""Seeded synthetic inputs for block-sparse C = A*B.

This module only produces inputs: COO lists of dense bs x bs leaf blocks whose
entries are pure functions of (seed, global row, global column).  It holds no
part of the product itself, so both the CPU oracle and the CUDA path can take
their inputs from here without sharing any of the method's arithmetic.

Randomness is counter based (SplitMix64, Steele/Lea/Flood 2014): any entry or
block-presence decision can be regenerated anywhere from its coordinates.

Workload families follow the paper's test matrices:
  * banded matrices with half-bandwidth d (Sec. 5.1, Eq. 5; Sec. 6.1 weak
    scaling runs),
  * uniformly random placement of nonzero blocks (Sec. 6.1, leaf library
    benchmark "randomly uniformly distributed" blocks),
  * distance-decay matrices of particles ordered by recursive spatial
    bisection (Sec. 5.1 overlap-type matrices; Sec. 6.2 Ergo overlap
    matrices, for which this is a synthetic stand-in),
  * small-integer blocks for exact-cancellation tests.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

BASE_SEED = 1501078000


@dataclasses.dataclass
class BlockCOO:
    """A matrix given as its list of stored bs x bs blocks.

    brow, bcol: int32 block coordinates; vals: float64 [nblk, bs, bs], each
    block row-major.  Entries of edge blocks that fall outside nrows x ncols
    are zero (the quadtree pads the matrix to a power-of-two block count).
    """

    nrows: int
    ncols: int
    bs: int
    brow: np.ndarray
    bcol: np.ndarray
    vals: np.ndarray

    @property
    def nblk(self) -> int:
        return int(self.brow.shape[0])

    @property
    def mb(self) -> int:
        return -(-self.nrows // self.bs)

    @property
    def nb(self) -> int:
        return -(-self.ncols // self.bs)

    def to_dense(self) -> np.ndarray:
        """Dense float64 copy (small matrices only)."""
        bs = self.bs
        d = np.zeros((self.mb * bs, self.nb * bs))
        for t in range(self.nblk):
            i, j = int(self.brow[t]), int(self.bcol[t])
            d[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = self.vals[t]
        return d[: self.nrows, : self.ncols]

    def transpose(self) -> "BlockCOO":
        return BlockCOO(self.ncols, self.nrows, self.bs, self.bcol.copy(),
                        self.brow.copy(),
                        np.ascontiguousarray(self.vals.transpose(0, 2, 1)))

    def sorted(self) -> "BlockCOO":
        """Copy with blocks in canonical row-major (I, J) order."""
        o = np.lexsort((self.bcol, self.brow))
        return BlockCOO(self.nrows, self.ncols, self.bs, self.brow[o].copy(),
                        self.bcol[o].copy(), self.vals[o].copy())


def from_dense(d: np.ndarray, bs: int, keep_zero_blocks: bool = False) -> BlockCOO:
    """Cut a dense matrix into bs x bs blocks; all-zero blocks are omitted."""
    n, m = d.shape
    mb, nb = -(-n // bs), -(-m // bs)
    p = np.zeros((mb * bs, nb * bs))
    p[:n, :m] = d
    t = p.reshape(mb, bs, nb, bs).transpose(0, 2, 1, 3)
    nz = np.any(t != 0.0, axis=(2, 3)) | keep_zero_blocks
    bi, bj = np.nonzero(nz)
    return BlockCOO(n, m, bs, bi.astype(np.int32), bj.astype(np.int32),
                    np.ascontiguousarray(t[bi, bj]))


# ---------------------------------------------------------------- hashing
def upper_blocks(m: BlockCOO) -> BlockCOO:
    """The blocks with I <= J: upper-triangle storage of a symmetric matrix."""
    k = m.brow <= m.bcol
    return BlockCOO(m.nrows, m.ncols, m.bs, m.brow[k].copy(), m.bcol[k].copy(),
                    np.ascontiguousarray(m.vals[k]))


def random_upper(n: int, bs: int, p: float, seed: int) -> BlockCOO:
    """Upper-triangle storage of a random symmetric matrix: random blocks with
    I < J, and diagonal blocks made symmetric (x + x^T) where present."""
    m = upper_blocks(random_blocks(n, bs, p, seed))
    d = m.brow == m.bcol
    v = m.vals.copy()
    v[d] = v[d] + v[d].transpose(0, 2, 1)
    return BlockCOO(m.nrows, m.ncols, m.bs, m.brow, m.bcol, v)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied to x + golden gamma (vectorised, uint64)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _GOLDEN) & _M64
        z = ((z ^ (z >> np.uint64(30))) * _C1) & _M64
        z = ((z ^ (z >> np.uint64(27))) * _C2) & _M64
        return z ^ (z >> np.uint64(31))


def hash3(seed: int, a, b) -> np.ndarray:
    """Counter-based hash of (seed, a, b) -> uint64."""
    s = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
    h = splitmix64(s ^ np.asarray(a, dtype=np.uint64))
    return splitmix64(h ^ np.asarray(b, dtype=np.uint64))


def uniform01(h: np.ndarray) -> np.ndarray:
    """Top 53 bits of a uint64 hash as a double in [0, 1)."""
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _elem_coords(brow, bcol, bs):
    r = np.arange(bs, dtype=np.int64)
    gi = brow.astype(np.int64)[:, None, None] * bs + r[None, :, None]
    gj = bcol.astype(np.int64)[:, None, None] * bs + r[None, None, :]
    return np.broadcast_to(gi, (len(brow), bs, bs)), np.broadcast_to(gj, (len(brow), bs, bs))


def _entries(seed, gi, gj, dist):
    h = hash3(seed, gi, gj)
    if dist == "uniform":  # uniform[-1, 1)
        return 2.0 * uniform01(h) - 1.0
    if dist == "normal":  # Box-Muller on two hash streams
        u1 = uniform01(h)
        u2 = uniform01(splitmix64(h))
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    if dist.startswith("int"):  # small integers in [-k, k]
        k = int(dist[3:] or 8)
        return ((h % np.uint64(2 * k + 1)).astype(np.int64) - k).astype(np.float64)
    raise ValueError(dist)


def _mask_outside(vals, gi, gj, nrows, ncols):
    vals[(gi >= nrows) | (gj >= ncols)] = 0.0
    return vals


def _drop_zero_blocks(coo: BlockCOO) -> BlockCOO:
    nz = np.any(coo.vals != 0.0, axis=(1, 2))
    return BlockCOO(coo.nrows, coo.ncols, coo.bs, coo.brow[nz], coo.bcol[nz],
                    np.ascontiguousarray(coo.vals[nz]))


# ------------------------------------------------------------ generators
def banded(n: int, d: int, bs: int, seed: int, dist: str = "uniform",
           ncols: int | None = None) -> BlockCOO:
    """A_ij nonzero iff |i - j| <= d (bandwidth 2d+1, Sec. 5.1); entries from dist."""
    ncols = n if ncols is None else ncols
    mb, nb = -(-n // bs), -(-ncols // bs)
    reach = -(-d // bs) if d > 0 else 0
    bi, bj = [], []
    for i in range(mb):
        lo, hi = max(0, i - reach - 1), min(nb - 1, i + reach + 1)
        for j in range(lo, hi + 1):
            # block (i, j) intersects the band iff the closest element pair is within d
            dmin = max(0, (j - i) * bs - (bs - 1), (i - j) * bs - (bs - 1))
            if dmin <= d:
                bi.append(i)
                bj.append(j)
    brow = np.array(bi, dtype=np.int32)
    bcol = np.array(bj, dtype=np.int32)
    gi, gj = _elem_coords(brow, bcol, bs)
    vals = _entries(seed, gi, gj, dist)
    vals[np.abs(gi - gj) > d] = 0.0
    vals = _mask_outside(vals, gi, gj, n, ncols)
    return _drop_zero_blocks(BlockCOO(n, ncols, bs, brow, bcol, vals))


def random_blocks(n: int, bs: int, p: float, seed: int, dist: str = "normal",
                  ncols: int | None = None, max_blocks: int | None = None) -> BlockCOO:
    """Each block position independently nonzero with probability p (uniform
    placement, Sec. 6.1); nonzero blocks are dense with entries from dist."""
    ncols = n if ncols is None else ncols
    mb, nb = -(-n // bs), -(-ncols // bs)
    bi_all, bj_all = [], []
    rows_per = max(1, (1 << 22) // max(nb, 1))
    for r0 in range(0, mb, rows_per):
        r1 = min(mb, r0 + rows_per)
        I, J = np.meshgrid(np.arange(r0, r1, dtype=np.uint64),
                           np.arange(nb, dtype=np.uint64), indexing="ij")
        keep = uniform01(hash3(seed ^ 0x5BD1E995, I, J)) < p
        bi_all.append(I[keep].astype(np.int32))
        bj_all.append(J[keep].astype(np.int32))
    brow = np.concatenate(bi_all) if bi_all else np.zeros(0, np.int32)
    bcol = np.concatenate(bj_all) if bj_all else np.zeros(0, np.int32)
    if max_blocks is not None:
        brow, bcol = brow[:max_blocks], bcol[:max_blocks]
    gi, gj = _elem_coords(brow, bcol, bs)
    vals = _entries(seed, gi, gj, dist)
    vals = _mask_outside(vals, gi, gj, n, ncols)
    return _drop_zero_blocks(BlockCOO(n, ncols, bs, brow, bcol, vals))


def identity(n: int, bs: int) -> BlockCOO:
    return from_dense(np.eye(n), bs)


def block_permutation(nbk: int, bs: int, seed: int) -> tuple[BlockCOO, np.ndarray]:
    """Block permutation matrix P with P[i, perm[i]] = I_bs."""
    perm = np.argsort(uniform01(hash3(seed, np.arange(nbk, dtype=np.uint64), 7)))
    vals = np.broadcast_to(np.eye(bs), (nbk, bs, bs)).copy()
    return BlockCOO(nbk * bs, nbk * bs, bs, np.arange(nbk, dtype=np.int32),
                    perm.astype(np.int32), vals), perm


# ------------------------------------- decay-type (overlap-like) matrices
def bisection_order(pts: np.ndarray) -> np.ndarray:
    """Recursive spatial bisection: split at the median along the longest axis
    of the bounding box, lower half first; returns the point order."""
    order = np.empty(len(pts), dtype=np.int64)
    stack = [(np.arange(len(pts)), 0)]
    while stack:
        idx, out = stack.pop()
        if len(idx) <= 1:
            order[out:out + len(idx)] = idx
            continue
        p = pts[idx]
        ax = int(np.argmax(p.max(0) - p.min(0)))
        srt = idx[np.argsort(p[:, ax], kind="stable")]
        h = len(srt) // 2
        stack.append((srt[h:], out + h))
        stack.append((srt[:h], out))
    return order


def decay_points(npoints: int, seed: int, density: float = 0.1) -> np.ndarray:
    """npoints uniform in a cube of side (npoints/density)^(1/3) Angstrom,
    returned in recursive-bisection order."""
    side = (npoints / density) ** (1.0 / 3.0)
    k = np.arange(npoints, dtype=np.uint64)
    pts = np.stack([uniform01(hash3(seed, k, 11 + a)) for a in range(3)], axis=1) * side
    return pts[bisection_order(pts)]


def decay(npoints: int, bs: int, seed: int, nfun: int = 5, alpha: float = 0.5,
          cutoff: float = 1e-6, density: float = 0.1) -> BlockCOO:
    """Symmetric A_ij = s_ij * exp(-alpha * r_ij) over nfun basis functions per
    point (consecutive indices), s_ii = +1, s_ij = s_ji = +-1 from the hash of
    (min, max), entries with |A_ij| < cutoff dropped.  Small sizes only: the
    block list is built with a dense distance test per block pair."""
    pts = decay_points(npoints, seed, density)
    n = npoints * nfun
    nbk = -(-n // bs)
    rcut = -math.log(cutoff) / alpha
    # block bounding boxes over the points they touch
    ptidx = np.minimum(np.arange(nbk * bs) // nfun, npoints - 1).reshape(nbk, bs)
    lo = pts[ptidx].min(axis=1)
    hi = pts[ptidx].max(axis=1)
    gap = np.maximum(0.0, np.maximum(lo[:, None, :] - hi[None, :, :], lo[None, :, :] - hi[:, None, :]))
    near = np.sqrt((gap ** 2).sum(-1)) <= rcut
    bi, bj = np.nonzero(near)
    brow = bi.astype(np.int32)
    bcol = bj.astype(np.int32)
    gi, gj = _elem_coords(brow, bcol, bs)
    pi = np.minimum(gi // nfun, npoints - 1)
    pj = np.minimum(gj // nfun, npoints - 1)
    r = np.sqrt(((pts[pi] - pts[pj]) ** 2).sum(-1))
    lo_, hi_ = np.minimum(gi, gj), np.maximum(gi, gj)
    sgn = np.where((hash3(seed ^ 0x2545F491, lo_, hi_) & np.uint64(1)) == 1, -1.0, 1.0)
    sgn[gi == gj] = 1.0
    vals = sgn * np.exp(-alpha * r)
    vals[np.abs(vals) < cutoff] = 0.0
    vals = _mask_outside(vals, gi, gj, n, n)
    return _drop_zero_blocks(BlockCOO(n, n, bs, brow, bcol, vals))


# ------------------------------------------------------------ R-MAT graphs
def rmat_edges(scale: int, a: float, nnz_per_row: int, seed: int):
    """Distinct (row, col) pairs of an R-MAT graph (Chakrabarti, Zhan and
    Faloutsos, SDM 2004) on 2^scale nodes with nnz_per_row * 2^scale edge
    draws: each draw picks one quadrant per bit level with probabilities
    a (top-left), b = c = d = (1 - a) / 3 (top-right, bottom-left,
    bottom-right); repeated edges collapse to one entry."""
    n = 1 << scale
    m = nnz_per_row * n
    e = np.arange(m, dtype=np.uint64)
    b = (1.0 - a) / 3.0
    row = np.zeros(m, np.int64)
    col = np.zeros(m, np.int64)
    for lvl in range(scale):
        u = uniform01(hash3(seed, e, 1000 + lvl))
        bottom = u >= a + b                              # quadrants c, d
        right = ((u >= a) & (u < a + b)) | (u >= a + 2 * b)  # quadrants b, d
        row = 2 * row + bottom
        col = 2 * col + right
    key = np.unique(row * n + col)
    return key // n, key % n


def rmat(scale: int, a: float, bs: int, seed: int, nnz_per_row: int = 5) -> BlockCOO:
    """R-MAT graph matrix (entries 1.0) cut into bs x bs blocks."""
    n = 1 << scale
    row, col = rmat_edges(scale, a, nnz_per_row, seed)
    nb = -(-n // bs)
    bkey, inv = np.unique((row // bs) * nb + col // bs, return_inverse=True)
    vals = np.zeros((bkey.size, bs, bs))
    vals[inv, row % bs, col % bs] = 1.0
    return BlockCOO(n, n, bs, (bkey // nb).astype(np.int32), (bkey % nb).astype(np.int32), vals)


# ------------------------------------------------------ batched workload
def batched_specs(nprod: int, seed: int, nmin: int = 2048, nmax: int = 32768,
                  dmin: float = 0.005, dmax: float = 0.10, bs: int = 32):
    """Sizes and block densities for a batch of independent products:
    N = bs * round(exp(U[ln nmin, ln nmax]) / bs), density U[dmin, dmax]."""
    k = np.arange(nprod, dtype=np.uint64)
    u = uniform01(hash3(seed, k, 101))
    v = uniform01(hash3(seed, k, 202))
    n = np.maximum(bs, bs * np.round(np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin))) / bs))
    dens = dmin + v * (dmax - dmin)
    return [(int(a), float(b)) for a, b in zip(n, dens)]


def batched(nprod: int, seed: int, bs: int = 32, **kw):
    """List of (A, B) pairs for a batch of independent random block-sparse products."""
    out = []
    for t, (n, dens) in enumerate(batched_specs(nprod, seed, bs=bs, **kw)):
        a = random_blocks(n, bs, dens, seed * 1000003 + 2 * t + 1)
        b = random_blocks(n, bs, dens, seed * 1000003 + 2 * t + 2)
        out.append((a, b))
    return out
