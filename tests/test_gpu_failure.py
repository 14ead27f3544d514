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


def _cap_sweep(base, run):
    """Run `run` under caps of base + 1 KiB, x1.6, ... until it succeeds; every
    failing run must return OOM and leave nothing allocated.  Returns the
    successful run's result and the number of failing caps."""
    extra, fails = 1024, 0
    try:
        while True:
            bsm.bsm_set_memory_limit(base + extra)
            try:
                out = run()
            except bsm.BsmError as e:
                assert e.name == "BSM_ERR_OOM", e.name
                bsm.bsm_set_memory_limit(0)
                assert bsm.bsm_memory_in_use() == base, "memory left allocated after OOM"
                fails += 1
                extra = int(extra * 1.6) + 1
                continue
            return out, fails
    finally:
        bsm.bsm_set_memory_limit(0)


@pytest.mark.parametrize("prec", [bsm.BSM_FP64, bsm.BSM_SPLIT_BF16, bsm.BSM_SPLIT_FP8])
def test_memory_cap_gives_oom_at_every_allocation_and_frees_everything(prec):
    """Fault injection on the host: a cap on the library's pool makes an
    allocation fail at a different point of the call for each cap; the call
    returns OOM and frees all it had allocated, and the first cap that is
    large enough gives the normal result."""
    import torch
    torch.cuda.init()
    bsm.load()
    A = synth.random_blocks(40 * 32 + 5, 32, 0.15, 901)
    B = synth.random_blocks(40 * 32 + 5, 32, 0.15, 902)
    ga, gb = to_bsm(A), to_bsm(B)
    want = from_bsm(bsm.bsm_multiply(ga, gb, prec=prec))
    base = bsm.bsm_memory_in_use()
    C, fails = _cap_sweep(base, lambda: bsm.bsm_multiply(ga, gb, prec=prec))
    assert fails >= 5
    got = from_bsm(C)
    del C
    assert_same_structure(got, want)
    assert np.array_equal(got.vals, want.vals)
    # the batched call and plan creation clean up the same way
    Cs, fails = _cap_sweep(base, lambda: bsm.bsm_multiply_batched([ga, ga], [gb, ga], prec=prec))
    assert fails >= 5
    assert np.array_equal(from_bsm(Cs[0]).vals, want.vals)
    del Cs
    plan, fails = _cap_sweep(base, lambda: bsm.bsm_plan_create([ga], [gb], prec=prec))
    assert fails >= 5
    bsm.bsm_plan_execute(plan)
    assert np.array_equal(from_bsm(bsm.bsm_plan_results(plan)[0]).vals, want.vals)
    del plan
    assert bsm.bsm_memory_in_use() == base
