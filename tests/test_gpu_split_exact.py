"""The split-precision kernels against the split oracle (oracle/split.py), bit
for bit: scales, digits, exact diagonal sums and the single rounding are the
same definitions on both sides, so the GPU result equals the oracle's exactly
for every slice count and leaf size, including rows and columns of wide
dynamic range (decay-type entries from 1 down to 1e-6)."""
import numpy as np
import pytest

import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, to_bsm
from oracle import split as osplit

pytestmark = pytest.mark.gpu

PREC = {"bf16": bsm.BSM_SPLIT_BF16, "fp8": bsm.BSM_SPLIT_FP8}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


@pytest.mark.parametrize("fmt,slices,bs", [("bf16", 3, 32), ("bf16", 7, 32), ("bf16", 7, 16),
                                           ("fp8", 6, 32), ("fp8", 12, 32),
                                           # one pipeline (its shared memory fits no two)
                                           ("bf16", 8, 32),
                                           ("bf16", 2, 32), ("bf16", 5, 16), ("fp8", 2, 32)])
def test_random_equals_split_oracle_bit_for_bit(fmt, slices, bs):
    A = synth.random_blocks(3 * bs + 5, bs, 0.4, 801 + bs)
    B = synth.random_blocks(3 * bs + 5, bs, 0.4, 802 + bs)
    got = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), prec=PREC[fmt], slices=slices))
    want = osplit.multiply(A, B, fmt, slices)
    assert_same_structure(got, want)
    assert np.array_equal(got.vals, want.vals)


@pytest.mark.parametrize("fmt,slices", [("bf16", 7), ("fp8", 12)])
def test_decay_equals_split_oracle_bit_for_bit(fmt, slices):
    A = synth.decay(60, 32, 811)
    got = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(A), prec=PREC[fmt], slices=slices))
    want = osplit.multiply(A, A, fmt, slices)
    assert_same_structure(got, want)
    assert np.array_equal(got.vals, want.vals)
