"""GPU parity of the remaining task types of Sec. 3.2: transposition, the
transposed products C = A^T B, A B^T, A^T B^T, and C = A + B (Algorithm 2).

Transposition and addition are bit-exact (data movement, and one rounding per
entry).  Transposed products: structure bit-exact against the oracle's
transposed recursion; values within 1e-12 relative Frobenius error in FP64 and
1e-11 in the split mode, as for the plain product.
"""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL_SPLIT = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


@pytest.mark.parametrize("bs", [16, 32, 64])
def test_transpose_bit_exact(bs):
    A = synth.random_blocks(40 * bs + 7, bs, 0.2, 300 + bs, ncols=23 * bs + 3)
    T = from_bsm(bsm.bsm_transpose(to_bsm(A)))
    E = A.transpose().sorted()
    assert_same_structure(T, E)
    assert np.array_equal(T.vals, E.vals)


def test_transpose_levels_and_involution():
    A = synth.random_blocks(3000, 32, 0.05, 311, ncols=1700)
    M = to_bsm(A)
    T = bsm.bsm_transpose(M)
    TT = from_bsm(bsm.bsm_transpose(T))
    assert_same_structure(TT, A.sorted())
    assert np.array_equal(TT.vals, A.sorted().vals)
    # the level arrays of the transposed handle are those of a fresh build
    F = to_bsm(A.transpose())
    assert np.array_equal(bsm.bsm_level_counts(T), bsm.bsm_level_counts(F))


def test_transpose_empty():
    Z = synth.BlockCOO(100, 60, 16, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, 16, 16)))
    T = bsm.bsm_transpose(to_bsm(Z))
    assert bsm.bsm_info(T) == (60, 100, 16, 0)


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("n,k,m,bs", [(1000, 777, 1234, 32), (520, 300, 410, 16),
                                      (640, 640, 640, 64)])
def test_transposed_products_fp64(ta, tb, n, k, m, bs):
    A = synth.random_blocks(k if ta else n, bs, 0.15, 320 + n, ncols=n if ta else k)
    B = synth.random_blocks(m if tb else k, bs, 0.15, 321 + m, ncols=k if tb else m)
    C = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), trans_a=bool(ta), trans_b=bool(tb)))
    E = oracle.multiply(A, B, trans_a=bool(ta), trans_b=bool(tb)).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL


@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
def test_transposed_products_split(ta, tb):
    A = synth.random_blocks(1500, 32, 0.1, 330, ncols=900)
    B = synth.random_blocks(1500 if not tb else 1100, 32, 0.1, 331,
                            ncols=1100 if not tb else 1500)
    if not ta:
        A = A.transpose()          # op(A) = A must be 900 x 1500
    C = from_bsm(bsm.bsm_multiply(to_bsm(A), to_bsm(B), prec=bsm.BSM_SPLIT_BF16,
                                  trans_a=bool(ta), trans_b=bool(tb)))
    E = oracle.multiply(A, B, trans_a=bool(ta), trans_b=bool(tb)).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


def test_gram_matrices_same_handle():
    """A^T A and A A^T with one handle passed twice."""
    A = synth.random_blocks(1200, 32, 0.1, 340, ncols=800)
    M = to_bsm(A)
    for ta, tb in [(1, 0), (0, 1)]:
        C = from_bsm(bsm.bsm_multiply(M, M, trans_a=bool(ta), trans_b=bool(tb)))
        E = oracle.multiply(A, A, trans_a=bool(ta), trans_b=bool(tb)).C
        assert_same_structure(C, E)
        assert relerr(C.vals, E.vals) < TOL


def test_transposed_dimension_check():
    M = to_bsm(synth.random_blocks(640, 32, 0.2, 350, ncols=320))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(M, M)
    assert e.value.name == "BSM_ERR_DIM_MISMATCH"
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(M, M, trans_a=True, trans_b=True)
    assert e.value.name == "BSM_ERR_DIM_MISMATCH"


@pytest.mark.parametrize("bs", [16, 32, 64])
def test_add_bit_exact(bs):
    A = synth.random_blocks(50 * bs + 9, bs, 0.2, 360 + bs, ncols=31 * bs + 5)
    B = synth.random_blocks(50 * bs + 9, bs, 0.2, 361 + bs, ncols=31 * bs + 5)
    C = from_bsm(bsm.bsm_add(to_bsm(A), to_bsm(B)))
    E = oracle.add(A, B)
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


def test_add_cancellation_and_empty():
    A = synth.random_blocks(2000, 32, 0.05, 370)
    S = A.sorted()
    neg = synth.BlockCOO(A.nrows, A.ncols, A.bs, S.brow.copy(), S.bcol.copy(), -S.vals)
    assert bsm.bsm_info(bsm.bsm_add(to_bsm(A), to_bsm(neg)))[3] == 0
    part = synth.BlockCOO(A.nrows, A.ncols, A.bs, S.brow[::3].copy(), S.bcol[::3].copy(),
                          -S.vals[::3])
    C = from_bsm(bsm.bsm_add(to_bsm(A), to_bsm(part)))
    E = oracle.add(A, part)
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)
    Z = synth.BlockCOO(2000, 2000, 32, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, 32, 32)))
    C = from_bsm(bsm.bsm_add(to_bsm(Z), to_bsm(A)))
    assert_same_structure(C, S)
    assert np.array_equal(C.vals, S.vals)
    assert bsm.bsm_info(bsm.bsm_add(to_bsm(Z), to_bsm(Z)))[3] == 0


def test_add_then_multiply_levels_valid():
    """The sum is a complete handle: its product matches the oracle's."""
    A = synth.random_blocks(1500, 32, 0.05, 380)
    B = synth.random_blocks(1500, 32, 0.05, 381)
    S = bsm.bsm_add(to_bsm(A), to_bsm(B))
    C = from_bsm(bsm.bsm_multiply(S, S))
    s = oracle.add(A, B)
    E = oracle.multiply(s, s).C
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL


def test_add_errors():
    A = to_bsm(synth.random_blocks(640, 32, 0.2, 390))
    B = to_bsm(synth.random_blocks(640, 32, 0.2, 391, ncols=320))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_add(A, B)
    assert e.value.name == "BSM_ERR_DIM_MISMATCH"
    C = to_bsm(synth.random_blocks(640, 16, 0.2, 392))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_add(A, C)
    assert e.value.name == "BSM_ERR_BLOCKSIZE"


def recut(m: synth.BlockCOO, bs: int) -> synth.BlockCOO:
    """The dense matrix cut into bs x bs blocks, all-zero blocks omitted."""
    return synth.from_dense(m.to_dense(), bs).sorted()


@pytest.mark.parametrize("obs,nbs", [(32, 16), (64, 16), (64, 32), (16, 32), (16, 64), (32, 64),
                                     (32, 32)])
def test_reblock_bit_exact(obs, nbs):
    A = synth.random_blocks(20 * obs + 13, obs, 0.2, 450 + obs + nbs, ncols=17 * obs + 5)
    # make some sub-blocks exactly zero so that splitting must drop them
    A.vals[::3, : obs // 2, : obs // 2] = 0.0
    R = from_bsm(bsm.bsm_reblock(to_bsm(A), nbs))
    E = recut(A, nbs)
    assert_same_structure(R, E)
    assert np.array_equal(R.vals, E.vals)


def test_reblock_round_trip_and_product():
    A = synth.random_blocks(3000, 32, 0.03, 460)
    B = synth.random_blocks(3000, 32, 0.03, 461)
    M = to_bsm(A)
    back = from_bsm(bsm.bsm_reblock(bsm.bsm_reblock(M, 64), 32))
    assert_same_structure(back, A.sorted())
    assert np.array_equal(back.vals, A.sorted().vals)
    # the product at bs 64 is the product at bs 32, re-cut
    C64 = from_bsm(bsm.bsm_reblock(bsm.bsm_multiply(bsm.bsm_reblock(M, 64),
                                                     bsm.bsm_reblock(to_bsm(B), 64)), 32))
    E = oracle.multiply(A, B).C
    assert_same_structure(C64, E)
    assert relerr(C64.vals, E.vals) < TOL


# ---------------------------------------------------- leaf-size override
def _recut(m: synth.BlockCOO, bs: int) -> synth.BlockCOO:
    return synth.from_dense(m.to_dense(), bs)


@pytest.mark.parametrize("abs_,bbs,cbs", [(32, 16, 32), (16, 16, 64), (64, 32, 16)])
def test_bs_override_equals_product_of_recut_operands(abs_, bbs, cbs):
    """opts.bs: operands of any sizes are re-cut exactly to the requested
    size; the product equals, bit for bit, the product of operands built at
    that size, and C has that size."""
    n = 23 * 16 + 5
    A = synth.random_blocks(n, abs_, 0.25, 700 + abs_)
    B = synth.random_blocks(n, bbs, 0.25, 701 + bbs)
    ga, gb = to_bsm(A), to_bsm(B)
    want = from_bsm(bsm.bsm_multiply(to_bsm(_recut(A, cbs)), to_bsm(_recut(B, cbs))))
    got = from_bsm(bsm.bsm_multiply(ga, gb, bs=cbs))
    assert got.bs == cbs
    assert_same_structure(got, want)
    assert np.array_equal(got.vals, want.vals)
    E = oracle.multiply(_recut(A, cbs), _recut(B, cbs)).C
    assert_same_structure(got, E)
    assert relerr(got.vals, E.vals) < 1e-12
    # transposed, split, batched and planned forms take the same override
    gt = from_bsm(bsm.bsm_multiply(gb, ga, trans_a=True, trans_b=True, bs=cbs))
    wt = from_bsm(bsm.bsm_multiply(to_bsm(_recut(B, cbs)), to_bsm(_recut(A, cbs)),
                                   trans_a=True, trans_b=True))
    assert_same_structure(gt, wt)
    assert np.array_equal(gt.vals, wt.vals)
    ws = from_bsm(bsm.bsm_multiply(to_bsm(_recut(A, cbs)), to_bsm(_recut(B, cbs)),
                                   prec=bsm.BSM_SPLIT_BF16))
    gs = from_bsm(bsm.bsm_multiply(ga, gb, prec=bsm.BSM_SPLIT_BF16, bs=cbs))
    assert_same_structure(gs, ws)
    assert np.array_equal(gs.vals, ws.vals)
    for prec, w in ((bsm.BSM_FP64, want), (bsm.BSM_SPLIT_BF16, ws)):
        gbt = [from_bsm(c) for c in bsm.bsm_multiply_batched([ga, ga], [gb, gb], prec=prec,
                                                             bs=cbs)]
        plan = bsm.bsm_plan_create([ga], [gb], prec=prec, bs=cbs)
        bsm.bsm_plan_execute(plan)
        gp = from_bsm(bsm.bsm_plan_results(plan)[0])
        for g in gbt + [gp]:
            assert g.bs == cbs
            assert_same_structure(g, w)
            assert np.array_equal(g.vals, w.vals)


def test_different_block_sizes_need_the_override():
    A = to_bsm(synth.random_blocks(256, 32, 0.3, 710))
    B = to_bsm(synth.random_blocks(256, 16, 0.3, 711))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(A, B)
    assert e.value.name == "BSM_ERR_BLOCKSIZE"
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(A, A, bs=24)
    assert e.value.name == "BSM_ERR_BLOCKSIZE"
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply_batched([A], [B])
    assert e.value.name == "BSM_ERR_BLOCKSIZE"


def test_calls_without_the_override_reject_it():
    import ctypes
    A = to_bsm(synth.random_blocks(256, 32, 0.3, 712))
    lib = bsm.load()
    out = ctypes.c_void_p()
    opts = bsm.bsm_mult_opts(bsm.BSM_FP64, 0, 0, 16)
    assert lib.bsm_multiply_range(A.handle, A.handle, 0, 1 << 20, ctypes.byref(out),
                                  ctypes.byref(opts), None) == -1
    assert lib.bsm_sym_square(A.handle, ctypes.byref(out), ctypes.byref(opts), None) == -1
    assert out.value is None
