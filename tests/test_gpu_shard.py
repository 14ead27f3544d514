"""GPU: products restricted to Morton ranges of C (bsm_multiply_range) and the
sharded driver emulated rank by rank in one process.  Every C block is
computed as by the full product, so the union of the shards equals it bit for
bit."""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm
from paper_1501_07800_gb300 import shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


def union(parts):
    r = np.concatenate([p.brow for p in parts])
    c = np.concatenate([p.bcol for p in parts])
    v = np.concatenate([p.vals for p in parts])
    o = np.lexsort((c, r))
    return r[o], c[o], v[o]


@pytest.mark.parametrize("prec", [bsm.BSM_FP64, bsm.BSM_SPLIT_BF16])
@pytest.mark.parametrize("nparts", [2, 7])
def test_ranges_union_is_the_product(prec, nparts):
    A = synth.random_blocks(3000, 32, 0.04, 700, ncols=2600)
    B = synth.random_blocks(2600, 32, 0.04, 701, ncols=3300)
    ga, gb = to_bsm(A), to_bsm(B)
    full = from_bsm(bsm.bsm_multiply(ga, gb, prec=prec))
    L = shard.depth(-(-3000 // 32), -(-2600 // 32), -(-3300 // 32))
    ranges = shard.balanced_ranges(A.brow, A.bcol, B.brow, B.bcol, nparts, L)
    parts = []
    for lo, hi in ranges:
        P = from_bsm(bsm.bsm_multiply_range(ga, gb, lo, hi, prec=prec))
        k = shard.morton(P.brow, P.bcol)
        assert np.all((k >= np.uint64(lo)) & (k < np.uint64(hi)))
        parts.append(P)
    r, c, v = union(parts)
    assert np.array_equal(r, full.brow) and np.array_equal(c, full.bcol)
    assert np.array_equal(v, full.vals)


def test_range_split_bs64_recut():
    A = synth.random_blocks(40 * 64, 64, 0.08, 710)
    B = synth.random_blocks(40 * 64, 64, 0.08, 711)
    ga, gb = to_bsm(A), to_bsm(B)
    full = from_bsm(bsm.bsm_multiply(ga, gb, prec=bsm.BSM_SPLIT_BF16))
    L = shard.depth(40)
    ranges = shard.balanced_ranges(A.brow, A.bcol, B.brow, B.bcol, 3, L)
    parts = [from_bsm(bsm.bsm_multiply_range(ga, gb, lo, hi, prec=bsm.BSM_SPLIT_BF16))
             for lo, hi in ranges]
    r, c, v = union(parts)
    assert np.array_equal(r, full.brow) and np.array_equal(c, full.bcol)
    assert np.array_equal(v, full.vals)


def test_emulated_ranks_with_halo_operands():
    """Each emulated rank builds only its A rows and B halo on the GPU."""
    A = synth.random_blocks(2500, 32, 0.05, 720)
    B = synth.random_blocks(2500, 32, 0.05, 721)
    world = 4

    def compute(sa, sb, lo, hi):
        P = from_bsm(bsm.bsm_multiply_range(to_bsm(sa), to_bsm(sb), lo, hi))
        return P.brow, P.bcol, P.vals

    outs = [shard.run_sharded(A, B, r, world, compute) for r in range(world)]
    r = np.concatenate([o[2][0] for o in outs])
    c = np.concatenate([o[2][1] for o in outs])
    v = np.concatenate([o[2][2] for o in outs])
    o = np.lexsort((c, r))
    E = oracle.multiply(A, B).C
    assert np.array_equal(r[o], E.brow) and np.array_equal(c[o], E.bcol)
    assert relerr(v[o], E.vals) < 1e-12


def test_range_errors():
    A = to_bsm(synth.random_blocks(512, 32, 0.2, 730))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply_range(A, A, 10, 10)
    assert e.value.name == "BSM_ERR_INVALID_ARG"
    C = from_bsm(bsm.bsm_multiply_range(A, A, 1 << 40, 1 << 41))   # beyond the key space
    assert C.nblk == 0
