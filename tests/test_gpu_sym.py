"""GPU parity of the symmetric task types (upper-triangle storage): the full
matrix from its upper triangle, the symmetric square, the symmetric rank-k
products and the symmetric multiply, against the oracle's definitions.

Mirroring is data movement and must be bit-exact.  Products: structure
bit-exact, values within 1e-12 (FP64) / 1e-11 (split) relative Frobenius
error, as for the plain product.
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
def test_sym_to_full_bit_exact(bs):
    U = synth.random_upper(45 * bs + 11, bs, 0.15, 400 + bs)
    F = from_bsm(bsm.bsm_sym_to_full(to_bsm(U)))
    E = oracle.sym_full(U)
    assert_same_structure(F, E)
    assert np.array_equal(F.vals, E.vals)


@pytest.mark.parametrize("bs", [16, 32, 64])
def test_sym_square_fp64(bs):
    U = synth.random_upper(40 * bs + 5, bs, 0.15, 410 + bs)
    C = from_bsm(bsm.bsm_sym_square(to_bsm(U)))
    E = oracle.sym_square(U)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL


def test_sym_square_decay_halves_the_work():
    A = synth.decay(400, 32, 17)
    U = synth.upper_blocks(A)
    C = from_bsm(bsm.bsm_sym_square(to_bsm(U)))
    sym_triples = bsm.bsm_last_stats()[1]
    E = oracle.sym_square(U)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL
    bsm.bsm_multiply(to_bsm(A), to_bsm(A))
    full_triples = bsm.bsm_last_stats()[1]
    assert sym_triples < 0.6 * full_triples


def test_sym_square_split():
    A = synth.decay(400, 32, 18)
    U = synth.upper_blocks(A)
    C = from_bsm(bsm.bsm_sym_square(to_bsm(U), prec=bsm.BSM_SPLIT_BF16))
    E = oracle.sym_square(U)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL_SPLIT


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("bs", [16, 32])
def test_syrk(trans, bs):
    n, k = 37 * bs + 3, 23 * bs + 9
    A = synth.random_blocks(k if trans else n, bs, 0.15, 420 + bs, ncols=n if trans else k)
    C = from_bsm(bsm.bsm_syrk(to_bsm(A), trans=trans))
    E = oracle.syrk(A, trans)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL


@pytest.mark.parametrize("side", [bsm.BSM_SYM_LEFT, bsm.BSM_SYM_RIGHT])
def test_sym_multiply(side):
    U = synth.random_upper(1500, 32, 0.08, 430)
    G = synth.random_blocks(1500, 32, 0.08, 431, ncols=900) if side == 0 else \
        synth.random_blocks(900, 32, 0.08, 431, ncols=1500)
    a, b = (U, G) if side == 0 else (G, U)
    C = from_bsm(bsm.bsm_sym_multiply(to_bsm(a), to_bsm(b), side))
    E = oracle.sym_multiply(a, b, side)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < TOL


def test_sym_storage_errors():
    A = to_bsm(synth.random_blocks(640, 32, 0.3, 440))     # blocks below the diagonal
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_sym_square(A)
    assert e.value.name == "BSM_ERR_OUT_OF_RANGE"
    R = to_bsm(synth.upper_blocks(synth.random_blocks(640, 32, 0.3, 441, ncols=320)))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_sym_square(R)
    assert e.value.name == "BSM_ERR_DIM_MISMATCH"
    Z = synth.BlockCOO(640, 640, 32, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, 32, 32)))
    assert bsm.bsm_info(bsm.bsm_sym_square(to_bsm(Z)))[3] == 0
