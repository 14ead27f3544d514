"""The allocation-free entry point bsm_block_products_fp64_noalloc.

It serves callers that must not allocate device memory on their own path
(memory reserved in full by another allocator, or loops that cannot take an
allocation's implicit synchronisation).  The test builds a task list on the
host, calls the entry point twice in a row through the C ABI, and checks both
results against bsm_multiply's output within the FP64 tolerance of the other
tests (1e-12 relative Frobenius).  This file is collected last on purpose.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("bs", [16, 32])
def test_noalloc_matches_bsm_multiply_twice(bs):
    import torch
    torch.cuda.init()
    bsm.load()
    A = synth.random_blocks(1536, bs, 0.06, 9001 + bs)
    B = synth.random_blocks(1536, bs, 0.06, 9101 + bs)
    # existing entry point
    C = bsm.bsm_multiply(to_bsm(A), to_bsm(B))
    r, c, v = bsm.bsm_to_blocks(C)
    ref = {(int(i), int(j)): t for t, (i, j) in enumerate(zip(r, c))}
    keys, seg, ta, tb = task_list(A, B)
    dev = torch.device("cuda", torch.cuda.current_device())
    d_seg, d_ta, d_tb = (torch.from_numpy(x).to(dev) for x in (seg, ta, tb))
    d_a = torch.from_numpy(A.vals).to(dev)
    d_b = torch.from_numpy(B.vals).to(dev)
    for call in range(2):
        out = torch.full((len(keys), bs, bs), float("nan"), dtype=torch.float64, device=dev)
        nnz = torch.full((1,), -7, dtype=torch.int64, device=dev)
        bsm.bsm_block_products_fp64_noalloc(bs, d_seg, d_ta, d_tb, d_a, d_b, out, nnz)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert int(nnz.item()) == len(ref), f"call {call}"
        idx = np.array([ref[k] for k in keys])
        assert relerr(got, v[idx]) < TOL, f"call {call}"


def test_noalloc_rejects_sizes_beyond_scratch():
    import ctypes
    lib = bsm.load()
    n = ctypes.c_int64(0)
    code = lib.bsm_block_products_fp64_noalloc(32, bsm.BSM_NOALLOC_MAX_CBLOCKS + 1, 1, 1, 1, 1, 1,
                                               1, 1, 1, ctypes.byref(n), None)
    assert bsm.STATUS[code] == "BSM_ERR_UNSUPPORTED"
    assert lib.bsm_block_products_fp64_noalloc(17, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                               ctypes.byref(n), None) == -3
