"""Chunked symbolic phase: with a tiny per-level pair budget the product is
expanded and computed in consecutive Morton ranges of C; results must equal
the one-pass results bit for bit and match the oracle."""
import os

import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _budget():
    import torch
    torch.cuda.init()
    bsm.load()
    yield
    os.environ.pop("BSM_SYM_BUDGET", None)


CASES = {
    "random": lambda: (synth.random_blocks(3000, 32, 0.05, 1), synth.random_blocks(3000, 32, 0.05, 2)),
    "banded": lambda: (synth.banded(4096, 64, 32, 3), synth.banded(4096, 96, 32, 4)),
    "rect": lambda: (synth.random_blocks(900, 16, 0.2, 5, ncols=2000),
                     synth.random_blocks(2000, 16, 0.2, 6, ncols=700)),
    "dense_node": lambda: (synth.random_blocks(512, 32, 1.0, 7), synth.random_blocks(512, 32, 1.0, 8)),
    # a dense corner (long product lists: sibling-pair items in split mode)
    # in a sparse matrix (short lists: one C block per item), so that one
    # product's chunks use both operand layouts
    "mixed": lambda: (dense_corner(3000, 32, 0.03, 9), dense_corner(3000, 32, 0.03, 10)),
}


def dense_corner(n, bs, p, seed, corner=24):
    """Random blocks of density p plus every block of the top-left corner x corner blocks."""
    M = synth.random_blocks(n, bs, p, seed)
    keep = ~((M.brow < corner) & (M.bcol < corner))
    I, J = np.meshgrid(np.arange(corner, dtype=np.int32), np.arange(corner, dtype=np.int32),
                       indexing="ij")
    rng = np.random.default_rng(seed)
    vals = rng.standard_normal((corner * corner, bs, bs))
    return synth.BlockCOO(M.nrows, M.ncols, bs, np.concatenate([M.brow[keep], I.ravel()]),
                          np.concatenate([M.bcol[keep], J.ravel()]),
                          np.concatenate([M.vals[keep], vals]))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [bsm.BSM_FP64, bsm.BSM_SPLIT_BF16])
def test_chunked_equals_one_pass(case, prec):
    A, B = CASES[case]()
    ga, gb = to_bsm(A), to_bsm(B)
    os.environ.pop("BSM_SYM_BUDGET", None)
    one = from_bsm(bsm.bsm_multiply(ga, gb, prec=prec))
    assert bsm.bsm_last_chunks() == 1
    tasks1, trip1, _ = bsm.bsm_last_stats()
    os.environ["BSM_SYM_BUDGET"] = "64"
    got = from_bsm(bsm.bsm_multiply(ga, gb, prec=prec))
    assert bsm.bsm_last_chunks() > 1
    tasks2, trip2, _ = bsm.bsm_last_stats()
    assert np.array_equal(tasks1, tasks2) and trip1 == trip2   # every pair counted once
    assert_same_structure(got, one)
    assert np.array_equal(got.vals, one.vals)
    E = oracle.multiply(A, B).C
    assert_same_structure(got, E)
    assert relerr(got.vals, E.vals) < (1e-12 if prec == bsm.BSM_FP64 else 1e-11)
