"""The allocation-free entry point bsm_block_products_fp64_noalloc.

Some callers cannot allocate device memory on their own path: a process whose
device memory is reserved in full up front by another allocator (any new
cudaMalloc fails there), or a loop that cannot take an allocation's implicit
synchronisation.  This entry point serves them: the caller passes the task
list, the operand blocks and every output buffer, and the only other device
memory it touches is a static scratch array set up by the first call on the
device.

The tests build a task list on the host and call the entry point through the
C ABI, twice in a row, checking both results against the oracle (C's
structure: the blocks with an entry != 0.0 are exactly the oracle's; values
within the FP64 tolerance of the other tests, 1e-12 relative Frobenius) and
against the existing entry point bsm_multiply.  They also check that exactly
zero C blocks are left out of the count, that an out-of-range block index
gives nnz_out = -1 without disturbing the other C blocks, the size limit, the
binding's argument checks, and that a call after the set-up allocates
nothing.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import relerr, to_bsm

pytestmark = pytest.mark.gpu
TOL = 1e-12


def task_list(A, B):
    """C blocks in row-major order with their (A index, B index) products, K ascending."""
    a_at = {(int(i), int(k)): t for t, (i, k) in enumerate(zip(A.brow, A.bcol))}
    b_by_row = {}
    for t, (k, j) in enumerate(zip(B.brow, B.bcol)):
        b_by_row.setdefault(int(k), []).append((int(j), t))
    prods = {}
    for (i, k), ta in a_at.items():
        for j, tb in b_by_row.get(k, []):
            prods.setdefault((i, j), []).append((k, ta, tb))
    keys = sorted(prods)
    seg, ta, tb = [0], [], []
    for key in keys:
        for _, x, y in sorted(prods[key]):
            ta.append(x)
            tb.append(y)
        seg.append(len(ta))
    return keys, np.array(seg, np.int32), np.array(ta, np.int32), np.array(tb, np.int32)


class Call:
    """Device copies of one task list and its operands; run() calls the entry
    point into freshly poisoned output buffers."""

    def __init__(self, A, B, bs):
        import torch
        self.torch = torch
        self.bs = bs
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.keys, seg, ta, tb = task_list(A, B)
        self.seg, self.ta, self.tb = (torch.from_numpy(x).to(self.dev) for x in (seg, ta, tb))
        self.a = torch.from_numpy(A.vals).to(self.dev)
        self.b = torch.from_numpy(B.vals).to(self.dev)

    def buffers(self):
        t = self.torch
        out = t.full((len(self.keys), self.bs, self.bs), float("nan"), dtype=t.float64,
                     device=self.dev)
        nnz = t.full((1,), -7, dtype=t.int64, device=self.dev)
        return out, nnz

    def run(self, out, nnz, ta=None):
        bsm.bsm_block_products_fp64_noalloc(self.bs, self.seg, self.ta if ta is None else ta,
                                            self.tb, self.a, self.b, out, nnz)
        self.torch.cuda.synchronize()
        return out.cpu().numpy(), int(nnz.item())


def warm_up(bs):
    """The first call on the device (nc = 0) does the one-time set-up."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    e32 = torch.zeros(1, dtype=torch.int32, device=dev)
    e64 = torch.zeros((0, bs, bs), dtype=torch.float64, device=dev)
    nnz = torch.full((1,), -7, dtype=torch.int64, device=dev)
    bsm.bsm_block_products_fp64_noalloc(bs, e32, e32[:0], e32[:0], e64, e64, e64, nnz)
    torch.cuda.synchronize()
    assert int(nnz.item()) == 0


def check_against_oracle(call, got, nnz, P):
    """Blocks of the oracle's C: within TOL; every other block exactly zero."""
    ref = {(int(i), int(j)): t for t, (i, j) in enumerate(zip(P.C.brow, P.C.bcol))}
    assert nnz == P.C.nblk
    idx = [t for t, k in enumerate(call.keys) if k in ref]
    zero = [t for t, k in enumerate(call.keys) if k not in ref]
    assert len(idx) == P.C.nblk
    assert relerr(got[idx], P.C.vals[[ref[call.keys[t]] for t in idx]]) < TOL
    assert np.all(got[zero] == 0.0)


@pytest.mark.parametrize("bs", [16, 32, 64])
def test_noalloc_matches_oracle_twice(bs):
    import torch
    torch.cuda.init()
    bsm.load()
    warm_up(bs)
    n = 1536 if bs < 64 else 2048 + 40   # bs 64: a ragged last block row and column
    A = synth.random_blocks(n, bs, 0.06 if bs < 64 else 0.12, 9001 + bs)
    B = synth.random_blocks(n, bs, 0.06 if bs < 64 else 0.12, 9101 + bs)
    P = oracle.multiply(A, B)
    # the existing entry point, for comparison
    r, c, v = bsm.bsm_to_blocks(bsm.bsm_multiply(to_bsm(A), to_bsm(B)))
    mine = {(int(i), int(j)): t for t, (i, j) in enumerate(zip(r, c))}
    call = Call(A, B, bs)
    for k in range(2):
        out, nnz = call.buffers()
        torch.cuda.synchronize()
        free0, inuse0 = torch.cuda.mem_get_info()[0], bsm.bsm_memory_in_use()
        got, count = call.run(out, nnz)
        free1, inuse1 = torch.cuda.mem_get_info()[0], bsm.bsm_memory_in_use()
        check_against_oracle(call, got, count, P)
        idx = np.array([mine[key] for key in call.keys if key in mine])
        sel = [t for t, key in enumerate(call.keys) if key in mine]
        assert relerr(got[sel], v[idx]) < TOL, f"call {k}"
        if k == 1:   # after the set-up and a first call, nothing is allocated
            assert free1 == free0 and inuse1 == inuse0


def test_noalloc_counts_exact_zero_blocks():
    import torch
    bs = 16
    bsm.load()
    warm_up(bs)
    x = synth.random_blocks(2 * bs, bs, 1.0, 61, dist="int8").to_dense()
    y = synth.random_blocks(2 * bs, bs, 1.0, 62, dist="int8").to_dense()
    z = synth.random_blocks(2 * bs, bs, 1.0, 63, dist="int8").to_dense()
    # C = [X X; Z 0] [Y; -Y] = [0; Z Y]: the top block row cancels exactly
    A = synth.from_dense(np.block([[x, x], [z, np.zeros_like(z)]]), bs)
    B = synth.from_dense(np.vstack([y, -y]), bs)
    P = oracle.multiply(A, B)
    call = Call(A, B, bs)
    assert len(call.keys) > P.C.nblk   # some task-list blocks cancel
    for _ in range(2):
        out, nnz = call.buffers()
        got, count = call.run(out, nnz)
        check_against_oracle(call, got, count, P)
        # small integers: every partial sum is exact, so the values are too
        ref = {(int(i), int(j)): t for t, (i, j) in enumerate(zip(P.C.brow, P.C.bcol))}
        for t, key in enumerate(call.keys):
            if key in ref:
                assert np.array_equal(got[t], P.C.vals[ref[key]])
    torch.cuda.synchronize()


def test_noalloc_out_of_range_index():
    import torch
    bs = 32
    bsm.load()
    warm_up(bs)
    A = synth.random_blocks(1024, bs, 0.1, 9201)
    B = synth.random_blocks(1024, bs, 0.1, 9202)
    call = Call(A, B, bs)
    out, nnz = call.buffers()
    good, count = call.run(out, nnz)
    assert count > 0
    # one product of C block c names A block index na (one past the end)
    c = len(call.keys) // 2
    seg = call.seg.cpu().numpy()
    bad = call.ta.clone()
    bad[int(seg[c])] = A.nblk
    out, nnz = call.buffers()
    got, count = call.run(out, nnz, ta=bad)
    assert count == -1
    others = np.arange(len(call.keys)) != c
    assert np.array_equal(got[others], good[others])   # other C blocks untouched by the error
    # the next call starts clean: the error word is cleared at every call
    out, nnz = call.buffers()
    again, count2 = call.run(out, nnz)
    assert count2 > 0 and np.array_equal(again, good)
    torch.cuda.synchronize()


def test_noalloc_argument_checks():
    import torch
    lib = bsm.load()
    n = ctypes.c_int64(0)
    code = lib.bsm_block_products_fp64_noalloc(32, bsm.BSM_NOALLOC_MAX_CBLOCKS + 1, 1, 1, 1, 1, 1,
                                               1, 1, 1, ctypes.byref(n), None)
    assert bsm.STATUS[code] == "BSM_ERR_UNSUPPORTED"
    assert lib.bsm_block_products_fp64_noalloc(17, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                               ctypes.byref(n), None) == -3
    # the binding checks, and does not convert (a conversion would allocate)
    dev = torch.device("cuda", torch.cuda.current_device())
    seg = torch.zeros(2, dtype=torch.int32, device=dev)   # one C block with no products
    t = torch.zeros(1, dtype=torch.int32, device=dev)     # (index arrays must not be empty)
    blk = torch.zeros((1, 32, 32), dtype=torch.float64, device=dev)
    nnz = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(ValueError):
        bsm.bsm_block_products_fp64_noalloc(32, seg.long(), t, t, blk, blk, blk, nnz)
    with pytest.raises(ValueError):
        bsm.bsm_block_products_fp64_noalloc(32, seg, t, t, blk, blk, blk.transpose(1, 2), nnz)
    with pytest.raises(ValueError):
        bsm.bsm_block_products_fp64_noalloc(32, seg, t, t, blk.cpu(), blk, blk, nnz)
    with pytest.raises(ValueError):
        bsm.bsm_block_products_fp64_noalloc(16, seg, t, t, blk, blk, blk, nnz)
    bsm.bsm_block_products_fp64_noalloc(32, seg, t, t, blk, blk, blk, nnz)
    torch.cuda.synchronize()
    assert int(nnz.item()) == 0
