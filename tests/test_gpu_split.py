"""GPU parity of the split-precision mode (BF16 slices on tcgen05) vs the oracle.

Structure must match the oracle exactly.  Values: small-integer inputs are
represented exactly by one slice, so every digit product and every
accumulation is exact and the result equals the FP64 oracle bit for bit, for
any slice count.  For real-valued inputs the error bound is set by the 7s-bit
fixed point of each operand row/column: with the default s = 7 (49 bits) the
relative Frobenius error stays far below the 1e-11 target, and it must shrink
as s grows.
"""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm
from oracle import split as osplit

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


def split_product(A, B, slices=0):
    return from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), prec=bsm.BSM_SPLIT_BF16,
                                     slices=slices))


@pytest.mark.parametrize("bs", [32, 16])
def test_single_block_integers_exact(bs):
    A = synth.random_blocks(bs, bs, 1.0, 1, dist="int8")
    B = synth.random_blocks(bs, bs, 1.0, 2, dist="int8")
    C = split_product(A, B, slices=1)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


@pytest.mark.parametrize("bs", [16, 32])
@pytest.mark.parametrize("slices", [1, 3, 7])
def test_integers_exact_any_slice_count(bs, slices):
    A = synth.random_blocks(40 * bs + 5, bs, 0.3, 3, dist="int8")
    B = synth.random_blocks(40 * bs + 5, bs, 0.3, 4, dist="int8")
    C = split_product(A, B, slices=slices)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


def test_integer_cancellation_removed():
    bs = 32
    x = synth.random_blocks(2 * bs, bs, 1.0, 61, dist="int8").to_dense()
    y = synth.random_blocks(2 * bs, bs, 1.0, 62, dist="int8").to_dense()
    z = synth.random_blocks(2 * bs, bs, 1.0, 63, dist="int8").to_dense()
    a = np.block([[x, x], [z, np.zeros_like(z)]])
    b = np.vstack([y, -y])
    A, B = synth.from_dense(a, bs), synth.from_dense(b, bs)
    C = split_product(A, B)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


@pytest.mark.parametrize("bs", [16, 32])
def test_random_normal_default_slices(bs):
    A = synth.random_blocks(2048, bs, 0.05, 100 + bs)
    B = synth.random_blocks(2048, bs, 0.05, 200 + bs)
    C = split_product(A, B)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


def test_error_decreases_with_slices():
    A = synth.random_blocks(1024, 32, 0.1, 7)
    B = synth.random_blocks(1024, 32, 0.1, 8)
    E = oracle.multiply(A, B).C
    errs = []
    for s in range(2, 9):
        C = split_product(A, B, slices=s)
        assert_same_structure(C, E)
        errs.append(relerr(C.vals, E.vals))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < TOL_SPLIT


def test_banded_4096_split():
    A = synth.banded(4096, 64, 32, synth.BASE_SEED)
    B = synth.banded(4096, 64, 32, synth.BASE_SEED + 100)
    C = split_product(A, B)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert C.nblk == 1132
    assert relerr(C.vals, E.vals) < TOL_SPLIT


def test_long_k_lists_split():
    """Hundreds of products per C block: many exact-accumulation flushes."""
    A = synth.random_blocks(256, 32, 1.0, 34, ncols=32 * 200)
    B = synth.random_blocks(32 * 200, 32, 1.0, 35, ncols=256)
    C = split_product(A, B)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


@pytest.mark.parametrize("bs,nk", [(32, 1600), (32, 5000), (16, 3600), (16, 8000)])
def test_fold_of_very_long_k_lists_exact(bs, nk):
    """C blocks whose product lists exceed the 511 flushes that the 32-bit
    diagonal sums hold: the sums are folded into 64-bit pairs (one to several
    times) and the integer result stays bit-exact."""
    A = synth.random_blocks(2 * bs, bs, 1.0, 36, dist="int8", ncols=bs * nk)
    B = synth.random_blocks(bs * nk, bs, 1.0, 37, dist="int8", ncols=2 * bs)
    C = split_product(A, B)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


@pytest.mark.parametrize("slices", [1, 7])
def test_fold_prevents_32bit_overflow(slices):
    """All entries 127: every diagonal-0 product term is 127^2, the 32-bit sum
    of a C entry would pass 2^31 after ~1330 flushes; with 5000 products
    (1667 flushes) the exact result 127^2 * 32 * 5000 needs the folds."""
    bs, nk = 32, 5000
    ones = np.full((nk, bs, bs), 127.0)
    A = synth.BlockCOO(bs, bs * nk, bs, np.zeros(nk, np.int32), np.arange(nk, dtype=np.int32),
                       ones)
    B = synth.BlockCOO(bs * nk, bs, bs, np.arange(nk, dtype=np.int32), np.zeros(nk, np.int32),
                       ones.copy())
    C = split_product(A, B, slices=slices)
    assert C.nblk == 1
    assert np.all(C.vals == 127.0 ** 2 * bs * nk)


def test_fold_real_values_and_batched_and_plan():
    bs, nk = 32, 2100
    A = synth.random_blocks(bs, bs, 1.0, 38, ncols=bs * nk)
    B = synth.random_blocks(bs * nk, bs, 1.0, 39, ncols=bs)
    E = oracle.multiply(A, B).C
    C = split_product(A, B)
    assert relerr(C.vals, E.vals) < TOL_SPLIT
    ga, gb = to_bsm(A), to_bsm(B)
    Cb = from_bsm(bsm.bsm_multiply_batched([ga, ga], [gb, gb], prec=bsm.BSM_SPLIT_BF16)[1])
    assert np.array_equal(Cb.vals, C.vals)
    plan = bsm.bsm_plan_create([ga], [gb], prec=bsm.BSM_SPLIT_BF16)
    bsm.bsm_plan_execute(plan)
    Cp = from_bsm(bsm.bsm_plan_results(plan)[0])
    assert np.array_equal(Cp.vals, C.vals)


def test_decay_square_split():
    A = synth.decay(300, 16, 33)
    C = split_product(A, A)
    E = oracle.multiply(A, A).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


def test_rectangular_ragged_split():
    A = synth.random_blocks(1000, 32, 0.15, 31, ncols=777)
    B = synth.random_blocks(777, 32, 0.15, 32, ncols=1234)
    C = split_product(A, B)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


def test_split_is_deterministic():
    A = synth.random_blocks(1500, 32, 0.1, 41)
    B = synth.random_blocks(1500, 32, 0.1, 42)
    C1 = split_product(A, B)
    C2 = split_product(A, B)
    assert np.array_equal(C1.vals, C2.vals)


def test_split_bs64_equals_bs32_recut():
    """bs 64 runs as the bs-32 product of the re-cut operands: identical bits
    to splitting the same matrices cut at 32, and the oracle's structure."""
    A = synth.random_blocks(40 * 64 + 17, 64, 0.1, 5)
    B = synth.random_blocks(40 * 64 + 17, 64, 0.1, 6)
    C = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), prec=bsm.BSM_SPLIT_BF16))
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT
    a32 = synth.from_dense(A.to_dense(), 32)
    b32 = synth.from_dense(B.to_dense(), 32)
    C32 = from_bsm(bsm.bsm_reblock(bsm.bsm_multiply(to_bsm(a32), to_bsm(b32),
                                                    prec=bsm.BSM_SPLIT_BF16), 64))
    assert_same_structure(C, C32)
    assert np.array_equal(C.vals, C32.vals)


def test_split_bs64_symmetric_square():
    A = synth.decay(300, 64, 19)
    U = synth.upper_blocks(A)
    C = from_bsm(bsm.bsm_sym_square(to_bsm(U), prec=bsm.BSM_SPLIT_BF16))
    E = oracle.sym_square(U)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


# ------------------------------------------------------------ E4M3 digits
FP8_SLICES = [2, 3, 4, 6, 8, 12]


def fp8_product(A, B, slices=0):
    return from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), prec=bsm.BSM_SPLIT_FP8, slices=slices))


@pytest.mark.parametrize("slices", FP8_SLICES)
def test_fp8_integers_exact(slices):
    """|entries| <= 8 need one base-16 digit: every product and sum is exact."""
    A = synth.random_blocks(40 * 32 + 5, 32, 0.3, 600, dist="int8")
    B = synth.random_blocks(40 * 32 + 5, 32, 0.3, 601, dist="int8")
    C = fp8_product(A, B, slices)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


def test_fp8_error_decreases_with_slices():
    A = synth.random_blocks(1024, 32, 0.1, 602)
    B = synth.random_blocks(1024, 32, 0.1, 603)
    E = oracle.multiply(A, B).C
    errs = []
    for s in FP8_SLICES:
        C = fp8_product(A, B, s)
        assert_same_structure(C, E)
        errs.append(relerr(C.vals, E.vals))
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[FP8_SLICES.index(6)] < 1e-5     # 24-bit fixed point per row / column
    assert errs[-1] < TOL_SPLIT                # 48 bits


@pytest.mark.parametrize("bs", [16, 64])
def test_fp8_other_widths_equal_bs32_recut(bs):
    """E4M3 runs on 32-wide blocks; other widths are re-cut exactly, so the
    result equals the bs-32 product of the same matrices, re-cut."""
    A = synth.random_blocks(37 * bs + 9, bs, 0.1, 610 + bs)
    B = synth.random_blocks(37 * bs + 9, bs, 0.1, 611 + bs)
    C = fp8_product(A, B, 12)
    a32 = synth.from_dense(A.to_dense(), 32)
    b32 = synth.from_dense(B.to_dense(), 32)
    R = from_bsm(bsm.bsm_reblock(bsm.bsm_multiply(to_bsm(a32), to_bsm(b32),
                                                  prec=bsm.BSM_SPLIT_FP8, slices=12), bs))
    assert_same_structure(C, R)
    assert np.array_equal(C.vals, R.vals)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


@pytest.mark.parametrize("bs", [16, 32])
def test_fp8_symmetric_square(bs):
    A = synth.decay(240, bs, 620 + bs)
    U = synth.upper_blocks(A)
    C = from_bsm(bsm.bsm_sym_square(to_bsm(U), prec=bsm.BSM_SPLIT_FP8, slices=12))
    E = oracle.sym_square(U)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


def test_fp8_batched_equals_single():
    pairs = synth.batched(5, 630, nmin=256, nmax=2000, dmin=0.02, dmax=0.2)
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    got = bsm.bsm_multiply_batched(As, Bs, prec=bsm.BSM_SPLIT_FP8, slices=8)
    for ga, gb, c in zip(As, Bs, got):
        one = from_bsm(bsm.bsm_multiply(ga, gb, prec=bsm.BSM_SPLIT_FP8, slices=8))
        g = from_bsm(c)
        assert_same_structure(g, one)
        assert np.array_equal(g.vals, one.vals)


def test_fp8_rejects_uncompiled_slice_counts():
    A = to_bsm(synth.random_blocks(256, 32, 0.3, 640))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(A, A, prec=bsm.BSM_SPLIT_FP8, slices=5)
    assert e.value.name == "BSM_ERR_UNSUPPORTED"
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(A, A, prec=bsm.BSM_SPLIT_FP8, slices=13)
    assert e.value.name == "BSM_ERR_INVALID_ARG"


@pytest.mark.parametrize("prec,x,slices", [(bsm.BSM_SPLIT_FP8, 15 / 16, 2),
                                           (bsm.BSM_SPLIT_BF16, 127 / 128, 2)])
def test_accumulator_exact_near_its_bound(prec, x, slices):
    """Every entry x has one large top digit (15 in base 16, 127 in base 128)
    and zero below it, so each flush sums digit products of one sign up to
    just under 2^22: the tensor-core accumulation must be exact there."""
    bs, nk = 32, 2000
    vals = np.full((nk, bs, bs), x)
    A = synth.BlockCOO(bs, bs * nk, bs, np.zeros(nk, np.int32), np.arange(nk, dtype=np.int32),
                       vals)
    B = synth.BlockCOO(bs * nk, bs, bs, np.arange(nk, dtype=np.int32), np.zeros(nk, np.int32),
                       vals.copy())
    C = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), prec=prec, slices=slices))
    assert C.nblk == 1
    assert np.all(C.vals == x * x * bs * nk)   # exactly representable


@pytest.mark.parametrize("e", [-531, 510])
def test_results_beyond_the_normal_range(e):
    """Operands scaled by 2^e (exact): products far below the smallest normal
    double round to subnormals and products far above the largest overflow to
    infinity, like the scaled exact result (the out-of-line rounding path)."""
    A = synth.random_blocks(256, 32, 0.5, 650)
    B = synth.random_blocks(256, 32, 0.5, 651)
    E = oracle.multiply(A, B).C
    A.vals = np.ldexp(A.vals, e)
    B.vals = np.ldexp(B.vals, e)
    C = split_product(A, B)
    assert_same_structure(C, E)
    with np.errstate(over="ignore"):
        want = np.ldexp(E.vals, 2 * e)
    if e < 0:
        assert np.all(np.abs(C.vals) < 2.3e-308)
        assert np.max(np.abs(C.vals - want)) <= 2 * 4.95e-324      # two subnormal ulps
        assert np.count_nonzero(C.vals) > 0.9 * np.count_nonzero(want)
    else:
        inf = np.isinf(C.vals)
        assert inf.any() and np.isfinite(C.vals).any()
        assert np.mean(inf != np.isinf(want)) < 1e-3                # only at the threshold
        both = inf & np.isinf(want)
        assert np.array_equal(np.sign(C.vals[both]), np.sign(want[both]))
        fin = ~inf & np.isfinite(want)
        # compare scaled back down (norms of values near 1e308 overflow)
        assert relerr(np.ldexp(C.vals[fin], -2 * e), np.ldexp(want[fin], -2 * e)) < TOL_SPLIT


# ------------------------------------------------- pairs of sibling C blocks
def with_pairs(flag, fn):
    import os
    old = os.environ.get("BSM_SPLIT_PAIRS")
    os.environ["BSM_SPLIT_PAIRS"] = flag
    try:
        return fn()
    finally:
        if old is None:
            os.environ.pop("BSM_SPLIT_PAIRS", None)
        else:
            os.environ["BSM_SPLIT_PAIRS"] = old


PAIR_MODES = [(bsm.BSM_SPLIT_BF16, s) for s in (3, 4, 5, 6, 7, 8)] + \
             [(bsm.BSM_SPLIT_FP8, s) for s in (4, 6, 8, 12)]


@pytest.mark.parametrize("prec,slices,bs", [m + (32,) for m in PAIR_MODES] +
                         [(bsm.BSM_SPLIT_BF16, s, 16) for s in (3, 7, 8)])
def test_pairs_equal_single_blocks(prec, slices, bs):
    """Two sibling C blocks per MMA (N = 2 bs) give the same bits as one block
    per MMA: the same exact digit sums, rounded once."""
    A = synth.decay(260, bs, 660)
    B = synth.random_blocks(A.ncols, bs, 0.3, 661, ncols=A.ncols + 70)  # odd block columns
    ga, gb = to_bsm(A), to_bsm(B)
    run = lambda: from_bsm(bsm.bsm_multiply(ga, gb, prec=prec, slices=slices))
    one = with_pairs("0", run)
    two = with_pairs("1", run)
    assert_same_structure(two, one)
    assert np.array_equal(two.vals, one.vals)
    bits = slices * (7 if prec == bsm.BSM_SPLIT_BF16 else 4)
    if bits >= 40:  # with fewer bits tiny blocks may round to exact zero
        E = oracle.multiply(A, B).C
        assert_same_structure(two, E)
        assert relerr(two.vals, E.vals) < max(TOL_SPLIT, 2.0 ** -(bits - 8))


def test_pairs_long_lists_fold_and_chunks():
    """Pairs with folded accumulations (2000 products per C block) and with the
    symbolic phase cut into many Morton chunks (siblings in different chunks)."""
    import os
    bs, nk = 32, 2000
    A = synth.random_blocks(bs, bs, 1.0, 670, dist="int8", ncols=bs * nk)
    B = synth.random_blocks(bs * nk, bs, 1.0, 671, dist="int8", ncols=3 * bs)
    E = oracle.multiply(A, B).C
    C = with_pairs("1", lambda: from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B),
                                                          prec=bsm.BSM_SPLIT_BF16)))
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)
    A2 = synth.random_blocks(2000, 32, 0.2, 672)
    B2 = synth.random_blocks(2000, 32, 0.2, 673)
    ga, gb = to_bsm(A2), to_bsm(B2)
    base = with_pairs("0", lambda: from_bsm(bsm.bsm_multiply(ga, gb, prec=bsm.BSM_SPLIT_BF16)))
    os.environ["BSM_SYM_BUDGET"] = "500"
    try:
        got = with_pairs("1", lambda: from_bsm(bsm.bsm_multiply(ga, gb, prec=bsm.BSM_SPLIT_BF16)))
        assert bsm.bsm_last_chunks() > 1
    finally:
        os.environ.pop("BSM_SYM_BUDGET", None)
    assert_same_structure(got, base)
    assert np.array_equal(got.vals, base.vals)


def test_pairs_symmetric_square():
    A = synth.decay(300, 32, 680)
    U = to_bsm(synth.upper_blocks(A))
    one = with_pairs("0", lambda: from_bsm(bsm.bsm_sym_square(U, prec=bsm.BSM_SPLIT_BF16)))
    two = with_pairs("1", lambda: from_bsm(bsm.bsm_sym_square(U, prec=bsm.BSM_SPLIT_BF16)))
    assert_same_structure(two, one)
    assert np.array_equal(two.vals, one.vals)


def test_batched_with_sibling_pairs():
    prods = [(synth.decay(180 + 20 * k, 32, 690 + k), synth.decay(180 + 20 * k, 32, 690 + k))
             for k in range(3)]
    As = [to_bsm(a) for a, _ in prods]
    Bs = [to_bsm(b) for _, b in prods]
    one = with_pairs("0", lambda: [from_bsm(c) for c in
                                   bsm.bsm_multiply_batched(As, Bs, prec=bsm.BSM_SPLIT_BF16)])
    two = with_pairs("1", lambda: [from_bsm(c) for c in
                                   bsm.bsm_multiply_batched(As, Bs, prec=bsm.BSM_SPLIT_BF16)])
    for (a, b), x, y in zip(prods, one, two):
        assert_same_structure(y, x)
        assert np.array_equal(y.vals, x.vals)
        E = oracle.multiply(a, b).C
        assert_same_structure(y, E)
        assert relerr(y.vals, E.vals) < TOL_SPLIT


@pytest.mark.parametrize("prec,slices,bs", [(bsm.BSM_SPLIT_BF16, 7, 64), (bsm.BSM_SPLIT_FP8, 12, 64),
                                            (bsm.BSM_SPLIT_FP8, 12, 16)])
def test_recut_batched_and_plan_equal_single(prec, slices, bs):
    """Batched products and plans at a leaf size the split kernels do not take
    run on re-cut operands and give the bits of single products (which are
    tested against the bs-32 product of the same matrices above)."""
    pairs = synth.batched(4, 650 + bs, bs=bs, nmin=8 * bs, nmax=40 * bs, dmin=0.05, dmax=0.3)
    As = [to_bsm(a) for a, _ in pairs]
    Bs = [to_bsm(b) for _, b in pairs]
    As.append(As[0])  # a handle used twice, and a square
    Bs.append(As[0])
    single = [from_bsm(bsm.bsm_multiply(a, b, prec=prec, slices=slices)) for a, b in zip(As, Bs)]
    batched = [from_bsm(c) for c in bsm.bsm_multiply_batched(As, Bs, prec=prec, slices=slices)]
    plan = bsm.bsm_plan_create(As, Bs, prec=prec, slices=slices)
    assert bsm.bsm_plan_block_size(plan) == 32
    bsm.bsm_plan_execute(plan)
    planned = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
    for one, b, p in zip(single, batched, planned):
        assert one.bs == b.bs == p.bs == bs
        assert_same_structure(b, one)
        assert np.array_equal(b.vals, one.vals)
        assert_same_structure(p, one)
        assert np.array_equal(p.vals, one.vals)
    E = oracle.multiply(*pairs[0]).C
    assert_same_structure(single[0], E)
    assert relerr(single[0].vals, E.vals) < TOL_SPLIT


# ------------------------------------------------ grouped items (bs 16)
def with_env(name, flag, fn):
    import os
    old = os.environ.get(name)
    os.environ[name] = flag
    try:
        return fn()
    finally:
        if old is None:
            os.environ.pop(name, None)
        else:
            os.environ[name] = old


def grouped_and_single(fn):
    """fn() with grouped items (the default at bs 16) and without; pair items off."""
    run = lambda flag: with_env("BSM_SPLIT_PAIRS", "0",
                                lambda: with_env("BSM_SPLIT_GROUPS", flag, fn))
    return run("1"), run("0")


@pytest.mark.parametrize("slices", [3, 5, 7, 8])
def test_groups_equal_single_blocks(slices):
    """Up to four C blocks of short product lists per work item, each list in
    its own TMEM columns, give the bits of one C block per item: on a product
    of short lists only (one product per C block for most) and on one that
    mixes short lists with lists longer than one narrow flush."""
    bs = 16
    short = (synth.random_blocks(1000, bs, 0.06, 670 + slices),
             synth.random_blocks(1000, bs, 0.06, 680 + slices, ncols=1000 + 37))
    A = synth.decay(260, bs, 690)
    mixed = (A, synth.random_blocks(A.ncols, bs, 0.3, 691, ncols=A.ncols + 70))
    for a, b in (short, mixed):
        ga, gb = to_bsm(a), to_bsm(b)
        g, one = grouped_and_single(lambda: from_bsm(
            bsm.bsm_multiply(ga, gb, prec=bsm.BSM_SPLIT_BF16, slices=slices)))
        assert_same_structure(g, one)
        assert np.array_equal(g.vals, one.vals)
    # and the split oracle's bits on a small product of short lists
    a = synth.random_blocks(12 * bs + 7, bs, 0.25, 700 + slices)
    b = synth.random_blocks(12 * bs + 7, bs, 0.25, 710 + slices)
    want = osplit.multiply(a, b, "bf16", slices)
    g, _ = grouped_and_single(lambda: from_bsm(
        bsm.bsm_multiply(to_bsm(a), to_bsm(b), prec=bsm.BSM_SPLIT_BF16, slices=slices)))
    assert_same_structure(g, want)
    assert np.array_equal(g.vals, want.vals)


def test_groups_batched_and_plan_equal_single():
    """Batched products and plans at bs 16: groups never span two products
    (the work list interleaves them), and the bits equal single products."""
    bs = 16
    prods = synth.batched(5, 720, bs=bs, nmin=8 * bs, nmax=60 * bs, dmin=0.02, dmax=0.3)
    As = [to_bsm(a) for a, _ in prods]
    Bs = [to_bsm(b) for _, b in prods]

    def run():
        single = [from_bsm(bsm.bsm_multiply(a, b, prec=bsm.BSM_SPLIT_BF16))
                  for a, b in zip(As, Bs)]
        batched = [from_bsm(c) for c in
                   bsm.bsm_multiply_batched(As, Bs, prec=bsm.BSM_SPLIT_BF16)]
        plan = bsm.bsm_plan_create(As, Bs, prec=bsm.BSM_SPLIT_BF16)
        bsm.bsm_plan_execute(plan)
        planned = [from_bsm(c) for c in bsm.bsm_plan_results(plan)]
        bsm.bsm_plan_destroy(plan)
        return single, batched, planned

    (gs, gb, gp), (os_, _, _) = grouped_and_single(run)
    for i, one in enumerate(os_):
        for x in (gs[i], gb[i], gp[i]):
            assert_same_structure(x, one)
            assert np.array_equal(x.vals, one.vals)
    E = oracle.multiply(*prods[0]).C
    assert_same_structure(gb[0], E)
    assert relerr(gb[0].vals, E.vals) < TOL_SPLIT
