"""GPU parity of the Frobenius node norms and the truncation (bit-exact: both
sides sum in the same fixed order and decide the truncation in integers), and
of the per-level task counts on R-MAT graph matrices of increasing locality."""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, to_bsm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


@pytest.mark.parametrize("bs", [16, 32, 64])
def test_node_norms_bit_exact(bs):
    A = synth.random_blocks(30 * bs + 7, bs, 0.2, 500 + bs)
    A.vals *= np.exp(np.linspace(-20, 5, A.nblk))[:, None, None]
    M = to_bsm(A)
    depth = bsm.bsm_level_counts(M).size - 1
    for h in range(depth + 1):
        I, J, v = bsm.bsm_node_norms2(M, h)
        oI, oJ, ov = oracle.node_norms2(A, h)
        assert np.array_equal(I, oI) and np.array_equal(J, oJ)
        assert np.array_equal(v, ov)


@pytest.mark.parametrize("frac", [0.0, 1e-8, 1e-3, 0.3, 1.0, 2.0])
def test_truncate_bit_exact(frac):
    A = synth.random_blocks(1500, 32, 0.05, 510)
    A.vals *= np.exp(np.linspace(-25, 3, A.nblk))[:, None, None]
    tau = float(np.sqrt(np.sum(A.vals ** 2) * frac))
    R, removed, bound = bsm.bsm_truncate(to_bsm(A), tau)
    E, oremoved, obound = oracle.truncate(A, tau)
    assert removed == oremoved and bound == obound
    G = from_bsm(R)
    assert_same_structure(G, E)
    assert np.array_equal(G.vals, E.vals)


def test_truncate_limits():
    A = synth.random_blocks(800, 16, 0.1, 520)
    M = to_bsm(A)
    assert bsm.bsm_truncate(M, 0.0)[1] == 0
    assert bsm.bsm_truncate(M, float("inf"))[1] == A.nblk
    R, removed, _ = bsm.bsm_truncate(M, 1e300)
    assert removed == A.nblk and bsm.bsm_info(R)[3] == 0


@pytest.mark.parametrize("a", [0.25, 0.55, 0.8, 0.95])
def test_rmat_task_counts_and_product(a):
    """Fig. 5 (right) quantity: multiply tasks per level of A*A for R-MAT
    matrices, N = 8192, 5 edge draws per row; GPU counts equal the oracle's."""
    A = synth.rmat(13, a, 16, synth.BASE_SEED + 40)
    M = to_bsm(A)
    C = from_bsm(bsm.bsm_multiply(M, M))
    tasks, triples, _ = bsm.bsm_last_stats()
    P = oracle.multiply(A, A, leaf_dim=16)
    assert np.array_equal(tasks, P.tasks) and triples == P.triples
    assert_same_structure(C, P.C)
    assert np.array_equal(C.vals, P.C.vals)   # small integer sums: exact
