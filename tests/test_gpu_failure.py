"""Failure detection without a GPU fault: a device wait that can never
complete gives up after its time limit and surfaces as BSM_ERR_TIMEOUT, and
the context stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    import torch
    torch.cuda.init()
    bsm.load()
    t0 = time.time()
    assert bsm.bsm_selftest_wait_timeout(200) == "BSM_ERR_TIMEOUT"
    assert time.time() - t0 < 30
    # the same process keeps working on the GPU
    A = synth.random_blocks(512, 32, 0.2, 1)
    B = synth.random_blocks(512, 32, 0.2, 2)
    C = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B)))
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < 1e-12
    assert bsm.bsm_selftest_wait_timeout(0) == "BSM_ERR_INVALID_ARG"
