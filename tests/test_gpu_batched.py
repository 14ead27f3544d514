"""Batched products: one persistent numeric launch over a longest-first work
list of (product, C block) items from many independent products.

Each C block's arithmetic is the same as in a single bsm_multiply, so batched
results must equal the single-product results bit for bit (FP64 and split),
and both must match the oracle (structure exact, values within tolerance).
"""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


def small_batch(nprod=12, seed=5, bs=32):
    return synth.batched(nprod, seed, bs=bs, nmin=256, nmax=3000, dmin=0.01, dmax=0.2)


@pytest.mark.parametrize("prec", [bsm.BSM_FP64, bsm.BSM_SPLIT_BF16])
def test_batched_equals_single_bit_exact(prec):
    pairs = small_batch()
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    Cb = bsm.bsm_multiply_batched(As, Bs, prec=prec)
    for (a, b), ga, gb, gc in zip(pairs, As, Bs, Cb):
        single = from_bsm(bsm.bsm_multiply(ga, gb, prec=prec))
        got = from_bsm(gc)
        assert_same_structure(got, single)
        assert np.array_equal(got.vals, single.vals)


@pytest.mark.parametrize("prec,tol", [(bsm.BSM_FP64, 1e-12), (bsm.BSM_SPLIT_BF16, 1e-11)])
def test_batched_matches_oracle(prec, tol):
    pairs = small_batch(nprod=10, seed=9)
    Cb = bsm.bsm_multiply_batched([to_bsm(a) for a, _ in pairs], [to_bsm(b) for _, b in pairs],
                                  prec=prec)
    for (a, b), gc in zip(pairs, Cb):
        E = oracle.multiply(a, b).C
        got = from_bsm(gc)
        assert_same_structure(got, E)
        if E.nblk:
            assert relerr(got.vals, E.vals) < tol


def test_batched_mixed_block_sizes_and_empty_products():
    a16 = synth.random_blocks(700, 16, 0.1, 1)
    b16 = synth.random_blocks(700, 16, 0.1, 2)
    a64 = synth.random_blocks(900, 64, 0.3, 3)
    b64 = synth.random_blocks(900, 64, 0.3, 4)
    z = synth.BlockCOO(512, 512, 32, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, 32, 32)))
    a32 = synth.random_blocks(512, 32, 0.2, 5)
    # left half times bottom half: no overlapping K, empty result
    L = synth.from_dense(np.hstack([np.ones((256, 128)), np.zeros((256, 128))]), 32)
    R = synth.from_dense(np.vstack([np.zeros((128, 256)), np.ones((128, 256))]), 32)
    pairs = [(a16, b16), (z, a32), (a64, b64), (a32, z), (L, R), (a32, a32)]
    Cb = bsm.bsm_multiply_batched([to_bsm(a) for a, _ in pairs], [to_bsm(b) for _, b in pairs])
    for (a, b), gc in zip(pairs, Cb):
        E = oracle.multiply(a, b).C
        got = from_bsm(gc)
        assert_same_structure(got, E)
        if E.nblk:
            assert relerr(got.vals, E.vals) < 1e-12
    assert from_bsm(Cb[4]).nblk == 0


def test_batched_error_leaves_no_results():
    good = synth.random_blocks(256, 32, 0.2, 1)
    bad = synth.random_blocks(256, 32, 0.2, 2, ncols=320)
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply_batched([to_bsm(good), to_bsm(bad)], [to_bsm(good), to_bsm(bad)])
    assert e.value.name == "BSM_ERR_DIM_MISMATCH"
    assert bsm.bsm_multiply_batched([], []) == []


def test_batched_stats_sum_over_products():
    pairs = small_batch(nprod=6, seed=21)
    bsm.bsm_multiply_batched([to_bsm(a) for a, _ in pairs], [to_bsm(b) for _, b in pairs])
    _, triples, ncs = bsm.bsm_last_stats()
    assert triples == sum(oracle.multiply(a, b).triples for a, b in pairs)
