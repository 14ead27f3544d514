"""Plans: symbolic work once, numeric phase replayed from a CUDA graph, with
an optional measuring autotuner; bsm_update_values changes operand values under
a fixed structure."""
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


def batch(nprod=8, seed=31):
    return synth.batched(nprod, seed, nmin=256, nmax=2500, dmin=0.02, dmax=0.2)


@pytest.mark.parametrize("prec", [bsm.BSM_FP64, bsm.BSM_SPLIT_BF16])
@pytest.mark.parametrize("autotune", [False, True])
def test_plan_equals_batched_and_replays(prec, autotune):
    pairs = batch()
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    ref = [from_bsm(c) for c in bsm.bsm_multiply_batched(As, Bs, prec=prec)]
    plan = bsm.bsm_plan_create(As, Bs, prec=prec, autotune=autotune)
    order, chunk, ctas, nitems = bsm.bsm_plan_info(plan)
    assert order in (0, 1) and 1 <= chunk <= 32 and ctas >= 0
    assert nitems == sum(r.nblk for r in ref)   # generic data: nothing cancels
    form, tm, tn = bsm.bsm_plan_tile(plan)
    bs = pairs[0][0].bs
    if prec == bsm.BSM_FP64:   # a thread's DFMA tile covers the C block among 128 threads
        assert form == 1 and tm * tn * 128 == bs * bs and tn in (bs // 16, bs // 8, bs // 4)
    else:
        assert form == 2 and tm == 128 and tn in (bs, 2 * bs)
    for _ in range(2):                           # graph replays are idempotent
        bsm.bsm_plan_execute(plan)
        got = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
        for g, r in zip(got, ref):
            assert_same_structure(g, r)
            assert np.array_equal(g.vals, r.vals)   # every thread tile sums in one order


@pytest.mark.parametrize("autotune", [False, True])
def test_plan_item_shape_bs16(autotune):
    """At bs 16 the split item shape (grouped or single C blocks) is a tuned
    parameter: whichever the plan picks, its results are the batched call's
    bits, and bsm_plan_tile reports it (3: grouped, 2: single)."""
    pairs = synth.batched(6, 37, bs=16, nmin=256, nmax=2500, dmin=0.02, dmax=0.2)
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    ref = [from_bsm(c) for c in bsm.bsm_multiply_batched(As, Bs, prec=bsm.BSM_SPLIT_BF16)]
    plan = bsm.bsm_plan_create(As, Bs, prec=bsm.BSM_SPLIT_BF16, autotune=autotune)
    assert bsm.bsm_plan_block_size(plan) == 16
    form, tm, tn = bsm.bsm_plan_tile(plan)
    assert form in (2, 3) and tm == 128 and tn == 16
    if not autotune:
        assert form == 3   # the default: grouped items where compiled
    bsm.bsm_plan_execute(plan)
    got = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
    for g, r in zip(got, ref):
        assert_same_structure(g, r)
        assert np.array_equal(g.vals, r.vals)
    bsm.bsm_plan_destroy(plan)


@pytest.mark.parametrize("prec,tol", [(bsm.BSM_FP64, 1e-12), (bsm.BSM_SPLIT_BF16, 1e-11)])
def test_plan_after_value_update(prec, tol):
    pairs = batch(nprod=5, seed=41)
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    plan = bsm.bsm_plan_create(As, Bs, prec=prec)
    # new values on the same blocks (shuffled COO order), then replay
    rng = np.random.default_rng(7)
    new_pairs = []
    for (a, b), ga in zip(pairs, As):
        perm = rng.permutation(a.nblk)
        vals = a.vals * -1.5 + 0.25
        vals[a.vals == 0.0] = 0.0  # padding outside the matrix stays zero
        bsm.bsm_update_values(ga, a.brow[perm], a.bcol[perm], vals[perm])
        new_pairs.append((synth.BlockCOO(a.nrows, a.ncols, a.bs, a.brow, a.bcol, vals), b))
    bsm.bsm_plan_execute(plan)
    got = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
    for (a, b), g in zip(new_pairs, got):
        fresh = from_bsm(bsm.bsm_multiply(to_bsm(a), to_bsm(b), prec=prec))
        assert_same_structure(g, fresh)
        assert np.array_equal(g.vals, fresh.vals)
        E = oracle.multiply(a, b).C
        assert_same_structure(g, E)
        assert relerr(g.vals, E.vals) < tol


def test_update_values_rejects_other_block_sets():
    a = synth.random_blocks(512, 32, 0.2, 3)
    M = to_bsm(a)
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_update_values(M, a.brow[1:], a.bcol[1:], a.vals[1:])
    assert e.value.name == "BSM_ERR_INVALID_ARG"
    bcol = a.bcol.copy()
    free = next(j for j in range(16) if not np.any((a.brow == a.brow[0]) & (a.bcol == j)))
    bcol[0] = free
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_update_values(M, a.brow, bcol, a.vals)
    assert e.value.name == "BSM_ERR_INVALID_ARG"
    # the handle is unchanged
    r = from_bsm(M)
    assert np.array_equal(r.vals, a.sorted().vals)


@pytest.mark.parametrize("prec,tol", [(bsm.BSM_FP64, 1e-12), (bsm.BSM_SPLIT_BF16, 1e-11)])
def test_plan_chooses_leaf_size(prec, tol):
    """With leaf-size tuning the plan may compute at another block side on
    re-blocked copies; results come back at the operands' block size with the
    oracle's structure, also after the operand values change."""
    pairs = batch(nprod=4, seed=51)
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    plan = bsm.bsm_plan_create(As, Bs, prec=prec, autotune=True, autotune_bs=True)
    cb = bsm.bsm_plan_block_size(plan)
    assert cb in (16, 32)  # FP64: the operands' size or finer; split: 16 or 32
    bsm.bsm_plan_execute(plan)
    got = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
    for (a, b), g in zip(pairs, got):
        E = oracle.multiply(a, b).C
        assert_same_structure(g, E)
        assert relerr(g.vals, E.vals) < tol
    # new values, same blocks: the re-blocked copies are refreshed on execute
    new_pairs = []
    for (a, b), ga in zip(pairs, As):
        vals = a.vals * 0.5 - 0.125
        vals[a.vals == 0.0] = 0.0
        bsm.bsm_update_values(ga, a.brow, a.bcol, vals)
        new_pairs.append((synth.BlockCOO(a.nrows, a.ncols, a.bs, a.brow, a.bcol, vals), b))
    bsm.bsm_plan_execute(plan)
    got = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
    for (a, b), g in zip(new_pairs, got):
        E = oracle.multiply(a, b).C
        assert_same_structure(g, E)
        assert relerr(g.vals, E.vals) < tol


@pytest.mark.parametrize("cb", [16, 64])
def test_plan_at_forced_leaf_sizes_matches(cb):
    """Each leaf size the tuner may pick gives the oracle's result (the tuner
    is bypassed by re-blocking by hand and planning at that size)."""
    pairs = batch(nprod=3, seed=61)
    ra = [bsm.bsm_reblock(to_bsm(a), cb) for a, _ in pairs]
    rb = [bsm.bsm_reblock(to_bsm(b), cb) for _, b in pairs]
    plan = bsm.bsm_plan_create(ra, rb)
    bsm.bsm_plan_execute(plan)
    got = [from_bsm(bsm.bsm_reblock(c, 32)) for c in bsm.bsm_plan_results(plan)]
    for (a, b), g in zip(pairs, got):
        E = oracle.multiply(a, b).C
        assert_same_structure(g, E)
        assert relerr(g.vals, E.vals) < 1e-12


def test_plan_fp8_equals_batched():
    pairs = batch(nprod=4, seed=71)
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    ref = [from_bsm(c) for c in bsm.bsm_multiply_batched(As, Bs, prec=bsm.BSM_SPLIT_FP8,
                                                         slices=12)]
    plan = bsm.bsm_plan_create(As, Bs, prec=bsm.BSM_SPLIT_FP8, slices=12, autotune=True)
    bsm.bsm_plan_execute(plan)
    for g, r, (a, b) in zip(bsm.bsm_plan_results(plan), ref, pairs):
        g = from_bsm(g)
        assert_same_structure(g, r)
        assert np.array_equal(g.vals, r.vals)
        E = oracle.multiply(a, b).C
        assert relerr(g.vals, E.vals) < 1e-11


def test_plan_with_sibling_pairs():
    """Plans whose split numeric phase runs on pairs of sibling C blocks give
    the bits of single-block items, also after a value update (the pair-slot
    slices are recomputed in the replayed graph)."""
    import os
    pairs = [(synth.decay(200, 32, 90 + k), None) for k in range(3)]
    pairs = [(a, synth.random_blocks(a.ncols, 32, 0.4, 95 + k, ncols=a.ncols - 40))
             for k, (a, _) in enumerate(pairs)]
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]

    def run(flag):
        os.environ["BSM_SPLIT_PAIRS"] = flag
        try:
            plan = bsm.bsm_plan_create(As, Bs, prec=bsm.BSM_SPLIT_BF16, autotune=True)
            bsm.bsm_plan_execute(plan)
            return plan, [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
        finally:
            os.environ.pop("BSM_SPLIT_PAIRS", None)

    plan1, one = run("0")
    plan2, two = run("1")
    assert bsm.bsm_plan_info(plan2)[3] < bsm.bsm_plan_info(plan1)[3]   # fewer items: pairs
    for a, b in zip(one, two):
        assert_same_structure(b, a)
        assert np.array_equal(b.vals, a.vals)
    # new values of A, same blocks: replay both plans
    for (a, b), ga in zip(pairs, As):
        bsm.bsm_update_values(ga, a.brow, a.bcol, a.vals * 0.75)
    for plan in (plan1, plan2):
        bsm.bsm_plan_execute(plan)
    one = [from_bsm(c) for c in bsm.bsm_plan_results(plan1)]
    two = [from_bsm(c) for c in bsm.bsm_plan_results(plan2)]
    for (a, b), x, y in zip(pairs, one, two):
        assert np.array_equal(x.vals, y.vals)
        E = oracle.multiply(synth.BlockCOO(a.nrows, a.ncols, a.bs, a.brow, a.bcol, a.vals * 0.75),
                            b).C
        assert_same_structure(y, E)
        assert relerr(y.vals, E.vals) < 1e-11
