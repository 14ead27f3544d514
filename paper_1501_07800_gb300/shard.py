"""C = A*B split over ranks by contiguous Morton ranges of C's block keys.

A contiguous Morton range of C is a union of quadtree subtrees, so disjoint
ranges partition C: every C block has one owner, no partial sums cross
ranks, and the data-path exchange is one step -- each rank needs the A
blocks of the block rows its range touches and the B blocks (the "halo") of
the block columns it touches that meet those rows' inner indices.  Ranges are
balanced by an estimate of the block products per coarse C node (the product
of coarse block-count matrices).  Host logic only (numpy); the product of a
shard is `bsm_multiply_range` on the shard's GPU.
"""
from __future__ import annotations

import numpy as np


def morton(I, J) -> np.ndarray:
    """Morton keys of block coordinates (bit 2b+1 = bit b of I, bit 2b = bit b of J)."""
    I = np.asarray(I, np.uint64)
    J = np.asarray(J, np.uint64)
    k = np.zeros(np.broadcast(I, J).shape, np.uint64)
    for b in range(32):
        k |= ((I >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
        k |= ((J >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
    return k


def unmorton(k):
    k = np.asarray(k, np.uint64)
    I = np.zeros(k.shape, np.uint64)
    J = np.zeros(k.shape, np.uint64)
    for b in range(32):
        I |= ((k >> np.uint64(2 * b + 1)) & np.uint64(1)) << np.uint64(b)
        J |= ((k >> np.uint64(2 * b)) & np.uint64(1)) << np.uint64(b)
    return I.astype(np.int64), J.astype(np.int64)


def depth(*sides: int) -> int:
    """Tree depth L with 2^L >= every block count."""
    m = max(max(sides), 1)
    return int(m - 1).bit_length()


def balanced_ranges(a_rows, a_cols, b_rows, b_cols, nparts: int, L: int, coarse: int = 6):
    """Split the key space [0, 4^L) of C into `nparts` contiguous ranges of
    about equal estimated work.  Work of a coarse C node (2^coarse per side, or
    the full depth if smaller) = sum_k nA(i, k) nB(k, j) over coarse block
    counts -- an upper bound proportional to its block products.  Returns a
    list of (lo, hi) key pairs covering the space in order."""
    g = min(coarse, L)
    h = L - g                      # height of the coarse nodes above the blocks
    n = 1 << g
    nA = np.zeros((n, n))
    nB = np.zeros((n, n))
    np.add.at(nA, (np.asarray(a_rows) >> h, np.asarray(a_cols) >> h), 1.0)
    np.add.at(nB, (np.asarray(b_rows) >> h, np.asarray(b_cols) >> h), 1.0)
    w = nA @ nB                    # coarse work estimate, indexed (i, j)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    keys = morton(ii.ravel(), jj.ravel())
    order = np.argsort(keys, kind="stable")
    cum = np.cumsum(w.ravel()[order])
    total = cum[-1] if cum.size else 0.0
    bounds = [0]
    for r in range(1, nparts):
        # first coarse node whose cumulative work passes r/nparts of the total
        t = np.searchsorted(cum, total * r / nparts, side="right") if total > 0 else 0
        bounds.append(max(bounds[-1], int(t)))
    bounds.append(n * n)
    sh = np.uint64(2 * h)
    sorted_keys = keys[order]
    def key_at(pos):
        return int(sorted_keys[pos]) << int(sh) if pos < n * n else 1 << (2 * L)
    return [(key_at(bounds[r]), key_at(bounds[r + 1])) for r in range(nparts)]


def range_rows_cols(lo: int, hi: int, L: int):
    """Block rows and columns that C blocks with keys in [lo, hi) can have,
    as boolean masks over 0 .. 2^L - 1 (a range is a union of aligned
    subtrees; each contributes its row and column interval)."""
    n = 1 << L
    rows = np.zeros(n, bool)
    cols = np.zeros(n, bool)
    k = lo
    while k < hi:
        # largest aligned subtree starting at k that fits in [k, hi)
        s = 0
        while s < L and k % (1 << (2 * (s + 1))) == 0 and k + (1 << (2 * (s + 1))) <= hi:
            s += 1
        I, J = unmorton(np.array([k >> (2 * s)], np.uint64))
        r0, c0 = int(I[0]) << s, int(J[0]) << s
        rows[r0:r0 + (1 << s)] = True
        cols[c0:c0 + (1 << s)] = True
        k += 1 << (2 * s)
    return rows, cols


def shard_operands(a_rows, a_cols, b_rows, b_cols, lo: int, hi: int, L: int):
    """Index masks of the A and B blocks a shard [lo, hi) needs: A blocks in
    the rows the range touches; B blocks in the columns it touches whose row
    index K is an inner index of those A blocks (the B halo)."""
    rows, cols = range_rows_cols(lo, hi, L)
    a_rows = np.asarray(a_rows)
    a_cols = np.asarray(a_cols)
    b_rows = np.asarray(b_rows)
    b_cols = np.asarray(b_cols)
    amask = rows[a_rows]
    kset = np.zeros(1 << L, bool)
    kset[a_cols[amask]] = True
    bmask = cols[b_cols] & kset[b_rows]
    return amask, bmask


def run_sharded(A, B, rank: int, world: int, compute, gather=None, coarse: int = 6):
    """This rank's part of C = A*B (A, B: objects with nrows, ncols, bs, brow,
    bcol, vals).  `compute(A_part, B_part, lo, hi)` returns the rank's C blocks
    as (brow, bcol, vals) for keys in [lo, hi); `gather(obj)` (optional, e.g.
    torch.distributed.all_gather_object) collects every rank's part.  Returns
    (lo, hi, part) or, with gather, all parts merged in key order."""
    L = depth(-(-A.nrows // A.bs), -(-A.ncols // A.bs), -(-B.ncols // B.bs))
    ranges = balanced_ranges(A.brow, A.bcol, B.brow, B.bcol, world, L, coarse)
    lo, hi = ranges[rank]
    amask, bmask = shard_operands(A.brow, A.bcol, B.brow, B.bcol, lo, hi, L)
    part = compute(_subset(A, amask), _subset(B, bmask), lo, hi)
    if gather is None:
        return lo, hi, part
    parts = gather((lo, hi, part))
    parts.sort(key=lambda x: x[0])
    r = np.concatenate([p[2][0] for p in parts])
    c = np.concatenate([p[2][1] for p in parts])
    v = np.concatenate([p[2][2] for p in parts])
    return r, c, v


def _subset(M, mask):
    sub = type(M).__new__(type(M))
    sub.__dict__.update(M.__dict__)
    sub.brow = np.ascontiguousarray(M.brow[mask])
    sub.bcol = np.ascontiguousarray(M.bcol[mask])
    sub.vals = np.ascontiguousarray(M.vals[mask])
    return sub
