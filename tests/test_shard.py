"""Host logic of C-range sharding (CPU): Morton ranges, their row/column
spans, the operand subsets (B halo) a shard needs, and the two-rank driver
over gloo with the oracle as the per-shard compute."""
import os

import numpy as np
import pytest

import oracle
import synth
from paper_1501_07800_gb300 import shard


def restrict(C, lo, hi):
    k = shard.morton(C.brow, C.bcol)
    m = (k >= np.uint64(lo)) & (k < np.uint64(hi))
    return C.brow[m], C.bcol[m], C.vals[m]


def oracle_range(A, B, lo, hi):
    """The oracle's C blocks with keys in [lo, hi) (full product, filtered)."""
    return restrict(oracle.multiply(A, B).C, lo, hi)


def test_morton_round_trip():
    rng = np.random.default_rng(1)
    I = rng.integers(0, 1 << 20, 1000)
    J = rng.integers(0, 1 << 20, 1000)
    k = shard.morton(I, J)
    I2, J2 = shard.unmorton(k)
    assert np.array_equal(I, I2) and np.array_equal(J, J2)
    assert int(shard.morton([1], [0])[0]) == 2 and int(shard.morton([0], [1])[0]) == 1


@pytest.mark.parametrize("nparts", [1, 2, 3, 8])
def test_ranges_partition_and_balance(nparts):
    A = synth.random_blocks(2000, 16, 0.05, 11)
    B = synth.random_blocks(2000, 16, 0.05, 12)
    L = shard.depth(-(-2000 // 16))
    ranges = shard.balanced_ranges(A.brow, A.bcol, B.brow, B.bcol, nparts, L)
    assert ranges[0][0] == 0 and ranges[-1][1] == 4 ** L
    assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
    # actual block products per range (brute force over C's structure)
    C = oracle.multiply(A, B)
    tri = {}
    for I, K in zip(A.brow, A.bcol):
        for K2, J in zip(B.brow, B.bcol):
            if K == K2:
                tri[(int(I), int(J))] = tri.get((int(I), int(J)), 0) + 1
    keys = shard.morton([i for i, _ in tri], [j for _, j in tri])
    cnt = np.array(list(tri.values()))
    work = [int(cnt[(keys >= np.uint64(lo)) & (keys < np.uint64(hi))].sum()) for lo, hi in ranges]
    assert sum(work) == C.triples
    assert max(work) <= 1.35 * C.triples / nparts + 64 * 16   # balanced up to coarse granularity


def test_range_rows_cols_cover_every_key():
    L = 5
    rng = np.random.default_rng(2)
    for _ in range(50):
        lo, hi = sorted(rng.integers(0, 4 ** L, 2))
        if lo == hi:
            continue
        rows, cols = shard.range_rows_cols(int(lo), int(hi), L)
        I, J = shard.unmorton(np.arange(lo, hi, dtype=np.uint64))
        assert rows[I].all() and cols[J].all()
        # and nothing outside: every marked row holds some key of the range
        assert set(np.flatnonzero(rows)) == set(I.tolist())
        assert set(np.flatnonzero(cols)) == set(J.tolist())


@pytest.mark.parametrize("nparts", [2, 5])
def test_shard_operands_suffice(nparts):
    """A shard's product from only its A rows and B halo equals the full
    product on its range, bit for bit; the parts cover the product."""
    A = synth.random_blocks(1500, 16, 0.06, 21, ncols=1300)
    B = synth.random_blocks(1300, 16, 0.06, 22, ncols=1700)
    L = shard.depth(-(-1500 // 16), -(-1300 // 16), -(-1700 // 16))
    ranges = shard.balanced_ranges(A.brow, A.bcol, B.brow, B.bcol, nparts, L)
    full = oracle.multiply(A, B).C
    got = 0
    for lo, hi in ranges:
        am, bm = shard.shard_operands(A.brow, A.bcol, B.brow, B.bcol, lo, hi, L)
        sa = synth.BlockCOO(A.nrows, A.ncols, 16, A.brow[am], A.bcol[am], A.vals[am])
        sb = synth.BlockCOO(B.nrows, B.ncols, 16, B.brow[bm], B.bcol[bm], B.vals[bm])
        r1, c1, v1 = oracle_range(sa, sb, lo, hi)
        r2, c2, v2 = restrict(full, lo, hi)
        assert np.array_equal(r1, r2) and np.array_equal(c1, c2) and np.array_equal(v1, v2)
        assert am.sum() <= A.nblk and bm.sum() <= B.nblk
        got += r1.size
    assert got == full.nblk


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = synth.random_blocks(1200, 16, 0.08, 31)
    B = synth.random_blocks(1200, 16, 0.08, 32)

    def compute(sa, sb, lo, hi):
        return oracle_range(sa, sb, lo, hi)

    def gather(obj):
        objs = [None] * world
        dist.all_gather_object(objs, obj)
        return objs

    r, c, v = shard.run_sharded(A, B, rank, world, compute, gather)
    if rank == 0:
        np.savez(out, r=r, c=c, v=v)
    dist.destroy_process_group()


def test_two_rank_driver_over_gloo(tmp_path):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "c.npz")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    d = np.load(out)
    A = synth.random_blocks(1200, 16, 0.08, 31)
    B = synth.random_blocks(1200, 16, 0.08, 32)
    full = oracle.multiply(A, B).C
    o = np.argsort(shard.morton(full.brow, full.bcol), kind="stable")
    g = np.argsort(shard.morton(d["r"], d["c"]), kind="stable")
    assert np.array_equal(d["r"][g], full.brow[o]) and np.array_equal(d["c"][g], full.bcol[o])
    assert np.array_equal(d["v"][g], full.vals[o])
