"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each check uses something other than the oracle itself: dense brute force
(numpy A @ B), closed forms of banded products, identity and permutation
invariants, associativity / transposition, brute-force task counts per level,
and the task-count formulas and bounds printed in Sec. 5.1.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth
from synth import metrics

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_bounds.json")))


def relerr(x, y):
    n = np.linalg.norm(y)
    return np.linalg.norm(x - y) / (n if n > 0 else 1.0)


def dense_product_blocks(A, B):
    """Brute force: dense A @ B cut into blocks, all-zero blocks omitted."""
    return synth.from_dense(A.to_dense() @ B.to_dense(), A.bs).sorted()


def assert_same_structure(C, E):
    assert C.nblk == E.nblk
    assert np.array_equal(C.brow, E.brow) and np.array_equal(C.bcol, E.bcol)


# ----------------------------------------------------------- brute force
@pytest.mark.parametrize("n,m,k,bs,p,leaf", [
    (256, 256, 256, 16, 0.15, 4096),
    (300, 200, 250, 16, 0.3, 64),     # ragged, rectangular, several leaves
    (128, 128, 128, 4, 0.1, 16),
    (97, 131, 77, 8, 0.5, 8),         # leaf = single block
    (512, 512, 512, 32, 0.05, 4096),
    (64, 64, 64, 64, 1.0, 4096),
    (33, 33, 33, 32, 1.0, 32),
])
def test_dense_bruteforce(n, m, k, bs, p, leaf):
    A = synth.random_blocks(n, bs, p, 11 + n, ncols=k)
    B = synth.random_blocks(k, bs, p, 12 + m, ncols=m)
    P = oracle.multiply(A, B, leaf_dim=leaf)
    E = dense_product_blocks(A, B)
    assert_same_structure(P.C, E)
    assert relerr(P.C.vals, E.vals) < 1e-14
    assert P.C.nrows == n and P.C.ncols == m


def test_structure_is_symbolic_product():
    """S_C = {(I,J): exists K with A_IK, B_KJ stored} for generic data."""
    A = synth.random_blocks(640, 32, 0.1, 3)
    B = synth.random_blocks(640, 32, 0.1, 4)
    P = oracle.multiply(A, B, leaf_dim=128)
    pa = np.zeros((20, 20), bool); pa[A.brow, A.bcol] = True
    pb = np.zeros((20, 20), bool); pb[B.brow, B.bcol] = True
    pc = (pa.astype(int) @ pb.astype(int)) > 0
    bi, bj = np.nonzero(pc)
    assert np.array_equal(P.C.brow, bi) and np.array_equal(P.C.bcol, bj)
    assert P.triples == int((pa.astype(int) @ pb.astype(int)).sum())


def test_leaf_dim_does_not_change_result():
    A = synth.random_blocks(1000, 16, 0.05, 21)
    B = synth.random_blocks(1000, 16, 0.05, 22)
    r = [oracle.multiply(A, B, leaf_dim=ld) for ld in (16, 64, 256, 4096)]
    for q in r[1:]:
        assert_same_structure(q.C, r[0].C)
        assert relerr(q.C.vals, r[0].C.vals) < 1e-14
        assert q.triples == r[0].triples


# ------------------------------------------------------- C0 (banded 4096)
def test_banded_4096_counts():
    """Banded 4096 x 4096, half-bandwidth 64, bs 32: |I-J| <= 2 block pattern."""
    A = synth.banded(4096, 64, 32, synth.BASE_SEED)
    B = synth.banded(4096, 64, 32, synth.BASE_SEED + 100)
    assert A.nblk == 128 * 5 - 6 == 634
    P = oracle.multiply(A, B)
    assert P.triples == 3150
    assert P.C.nblk == 128 * 9 - 20 == 1132
    assert np.all(np.abs(P.C.brow - P.C.bcol) <= 4)


# ---------------------------------------------------- banded closed forms
@pytest.mark.parametrize("n,da,db,bs", [(200, 5, 7, 16), (256, 16, 16, 32), (130, 0, 3, 8)])
def test_banded_product_closed_form(n, da, db, bs):
    A = synth.banded(n, da, bs, 31)
    B = synth.banded(n, db, bs, 32)
    C = oracle.multiply(A, B, leaf_dim=64).C.to_dense()
    a, b = A.to_dense(), B.to_dense()
    i, j = np.indices(C.shape)
    assert np.all(C[np.abs(i - j) > da + db] == 0.0)        # bandwidth adds
    assert np.all(C[np.abs(i - j) == da + db] != 0.0)
    for r in range(n - da - db):                              # corners: one product, exact
        assert C[r, r + da + db] == a[r, r + da] * b[r + da, r + da + db]
        assert C[r + da + db, r] == a[r + da + db, r + db] * b[r + db, r]


@pytest.mark.parametrize("n,d", [(10, 1), (64, 4), (100, 7), (33, 16)])
def test_banded_flop_formula(n, d):
    """Sec. 6.1 flop count = 2 x brute-force count of multiply-adds (n > 2d)."""
    i, k, j = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    count = np.count_nonzero((np.abs(i - k) <= d) & (np.abs(k - j) <= d))
    assert metrics.banded_element_flops(n, d) == pytest.approx(2 * count, rel=0, abs=1e-6)


# ------------------------------------------------------------ invariants
def test_identity_bit_exact():
    A = synth.random_blocks(300, 16, 0.2, 41)
    I = synth.identity(300, 16)
    for C in (oracle.multiply(A, I).C, oracle.multiply(I, A).C):
        assert_same_structure(C, A.sorted())
        assert np.array_equal(C.vals, A.sorted().vals)


def test_block_permutation_bit_exact():
    nbk, bs = 24, 8
    A = synth.random_blocks(nbk * bs, bs, 0.3, 43)
    P, perm = synth.block_permutation(nbk, bs, 44)
    C = oracle.multiply(P, A, leaf_dim=32).C       # (P A) block row i = A block row perm[i]
    inv = np.argsort(perm)
    exp = synth.BlockCOO(A.nrows, A.ncols, bs, inv[A.brow].astype(np.int32), A.bcol.copy(),
                         A.vals.copy()).sorted()
    assert_same_structure(C, exp)
    assert np.array_equal(C.vals, exp.vals)


def test_associativity_and_transpose():
    A = synth.random_blocks(256, 16, 0.15, 51, ncols=192)
    B = synth.random_blocks(192, 16, 0.15, 52, ncols=320)
    C = synth.random_blocks(320, 16, 0.15, 53, ncols=128)
    ab = oracle.multiply(A, B).C
    abc1 = oracle.multiply(ab, C).C
    bc = oracle.multiply(B, C).C
    abc2 = oracle.multiply(A, bc).C
    d1, d2 = abc1.to_dense(), abc2.to_dense()
    assert relerr(d1, d2) < 1e-13
    btat = oracle.multiply(B.transpose(), A.transpose()).C
    assert relerr(btat.to_dense(), ab.to_dense().T) < 1e-14
    assert_same_structure(btat, ab.transpose().sorted())


# ------------------------------------- transposed task types and C = A + B
@pytest.mark.parametrize("ta,tb", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("n,k,m,bs,leaf", [(300, 200, 250, 16, 64), (97, 131, 77, 8, 8),
                                           (256, 256, 256, 32, 4096)])
def test_transposed_products_bruteforce(ta, tb, n, k, m, bs, leaf):
    """op(A) op(B) against the dense product of the transposed dense arrays."""
    A = synth.random_blocks(k if ta else n, bs, 0.25, 91 + n, ncols=n if ta else k)
    B = synth.random_blocks(m if tb else k, bs, 0.25, 92 + m, ncols=k if tb else m)
    P = oracle.multiply(A, B, leaf_dim=leaf, trans_a=bool(ta), trans_b=bool(tb))
    a = A.to_dense().T if ta else A.to_dense()
    b = B.to_dense().T if tb else B.to_dense()
    E = synth.from_dense(a @ b, bs).sorted()
    assert_same_structure(P.C, E)
    assert relerr(P.C.vals, E.vals) < 1e-14
    assert (P.C.nrows, P.C.ncols) == (n, m)
    # the transposed recursion visits the same products in the same order as
    # the plain recursion on explicitly transposed operands: identical bits
    Q = oracle.multiply(A.transpose() if ta else A, B.transpose() if tb else B, leaf_dim=leaf)
    assert_same_structure(P.C, Q.C)
    assert np.array_equal(P.C.vals, Q.C.vals)
    assert np.array_equal(P.tasks, Q.tasks) and P.triples == Q.triples


def test_transposed_dimension_check():
    A = synth.random_blocks(64, 16, 0.5, 1, ncols=48)
    with pytest.raises(oracle.OracleError) as e:
        oracle.multiply(A, A, trans_a=False, trans_b=False)
    assert e.value.code == -2
    assert oracle.multiply(A, A, trans_a=True).C.nrows == 48      # A^T A: 48 x 48
    assert oracle.multiply(A, A, trans_b=True).C.nrows == 64      # A A^T: 64 x 64


@pytest.mark.parametrize("n,m,bs,p,leaf", [(300, 200, 16, 0.3, 64), (97, 131, 8, 0.5, 8),
                                           (512, 512, 32, 0.05, 4096)])
def test_add_bruteforce(n, m, bs, p, leaf):
    A = synth.random_blocks(n, bs, p, 101 + n, ncols=m)
    B = synth.random_blocks(n, bs, p, 102 + m, ncols=m)
    C = oracle.add(A, B, leaf_dim=leaf)
    # one rounding per entry: the sum is bit-exact against the dense sum
    E = synth.from_dense(A.to_dense() + B.to_dense(), bs).sorted()
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)
    keys = set(zip(A.brow.tolist(), A.bcol.tolist())) | set(zip(B.brow.tolist(), B.bcol.tolist()))
    assert set(zip(C.brow.tolist(), C.bcol.tolist())) == keys   # generic data: no cancellation
    D = oracle.add(B, A, leaf_dim=leaf)
    assert np.array_equal(C.vals, D.vals)


def test_add_cancellation_and_identity():
    A = synth.random_blocks(200, 16, 0.3, 111)
    neg = synth.BlockCOO(A.nrows, A.ncols, A.bs, A.brow.copy(), A.bcol.copy(), -A.vals)
    assert oracle.add(A, neg).nblk == 0
    Z = synth.BlockCOO(200, 200, 16, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, 16, 16)))
    S = oracle.add(A, Z)
    assert_same_structure(S, A.sorted())
    assert np.array_equal(S.vals, A.sorted().vals)
    # partial cancellation: one block of the sum cancels, the others stay
    half = A.sorted()
    part = synth.BlockCOO(A.nrows, A.ncols, A.bs, half.brow[:1].copy(), half.bcol[:1].copy(),
                          -half.vals[:1])
    T = oracle.add(half, part)
    assert T.nblk == A.nblk - 1
    B = synth.random_blocks(200, 16, 0.3, 112, ncols=120)
    with pytest.raises(oracle.OracleError) as e:
        oracle.add(A, B)
    assert e.value.code == -2


# ------------------------------------------------- symmetric task types
def dense_sym(U):
    """Dense symmetric matrix of upper-triangle storage, by numpy: the stored
    blocks, plus every strictly-upper block transposed into the mirror."""
    bs, nb = U.bs, -(-U.nrows // U.bs)
    d = np.zeros((nb * bs, nb * bs))
    for I, J, v in zip(U.brow, U.bcol, U.vals):
        d[I * bs:(I + 1) * bs, J * bs:(J + 1) * bs] = v
        if I < J:
            d[J * bs:(J + 1) * bs, I * bs:(I + 1) * bs] = v.T
    return d[:U.nrows, :U.ncols]


def upper_of_dense(d, bs):
    return synth.upper_blocks(synth.from_dense(d, bs)).sorted()


@pytest.mark.parametrize("n,bs,p,leaf", [(300, 16, 0.2, 64), (97, 8, 0.4, 8), (512, 32, 0.1, 4096)])
def test_sym_full_and_square_bruteforce(n, bs, p, leaf):
    U = synth.random_upper(n, bs, p, 121 + n)
    S = dense_sym(U)
    assert np.array_equal(S, S.T)
    F = oracle.sym_full(U, leaf_dim=leaf)
    assert np.array_equal(F.to_dense(), S)
    C = oracle.sym_square(U, leaf_dim=leaf)
    E = upper_of_dense(S @ S, bs)
    assert_same_structure(C, E)
    assert np.all(C.brow <= C.bcol)
    assert relerr(C.vals, E.vals) < 1e-14


def test_sym_square_of_exactly_symmetric_matrix():
    """For an exactly symmetric A, the upper storage mirrors back to A bit for
    bit, and A^2 from it equals the upper triangle of the plain product."""
    A = synth.decay(120, 16, 9)
    U = synth.upper_blocks(A)
    F = oracle.sym_full(U)
    assert_same_structure(F, A.sorted())
    assert np.array_equal(F.vals, A.sorted().vals)
    C = oracle.sym_square(U)
    E = synth.upper_blocks(oracle.multiply(A, A).C)
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)
    # the upper triangle holds a little over half of the product's blocks
    full = oracle.multiply(A, A).C.nblk
    assert C.nblk == (full + np.sum(oracle.multiply(A, A).C.brow == oracle.multiply(A, A).C.bcol)) // 2


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("n,k,bs", [(300, 170, 16), (97, 131, 8)])
def test_syrk_bruteforce(trans, n, k, bs):
    A = synth.random_blocks(k if trans else n, bs, 0.3, 131 + n, ncols=n if trans else k)
    a = A.to_dense()
    g = a.T @ a if trans else a @ a.T
    C = oracle.syrk(A, trans)
    E = upper_of_dense(g, bs)
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < 1e-14
    assert (C.nrows, C.ncols) == (n, n)


@pytest.mark.parametrize("side", [0, 1])
def test_sym_multiply_bruteforce(side):
    bs = 16
    U = synth.random_upper(280, bs, 0.2, 141)
    G = synth.random_blocks(280, bs, 0.2, 142, ncols=200) if side == 0 else \
        synth.random_blocks(200, bs, 0.2, 142, ncols=280)
    S = dense_sym(U)
    if side == 0:
        C, d = oracle.sym_multiply(U, G, 0), S @ G.to_dense()
    else:
        C, d = oracle.sym_multiply(G, U, 1), G.to_dense() @ S
    E = synth.from_dense(d, bs).sorted()
    assert_same_structure(C, E)
    assert relerr(C.vals, E.vals) < 1e-14


def test_sym_storage_errors():
    A = synth.random_blocks(128, 16, 0.5, 151)          # has blocks below the diagonal
    with pytest.raises(oracle.OracleError) as e:
        oracle.sym_square(A)
    assert e.value.code == -4
    R = synth.upper_blocks(synth.random_blocks(128, 16, 0.5, 152, ncols=96))
    with pytest.raises(oracle.OracleError) as e:
        oracle.sym_square(R)
    assert e.value.code == -2


def test_symmetric_square_structure_symmetric():
    A = synth.decay(60, 16, 7)
    C = oracle.multiply(A, A).C
    k1 = set(zip(C.brow.tolist(), C.bcol.tolist()))
    assert k1 == set(zip(C.bcol.tolist(), C.brow.tolist()))


# ------------------------------------------------------- zero detection
def test_exact_cancellation_dropped():
    bs = 8
    x = synth.random_blocks(2 * bs, bs, 1.0, 61, dist="int8").to_dense()
    # A = [X X], B = [Y; -Y]  =>  C = XY - XY = 0 exactly (small integers)
    y = synth.random_blocks(2 * bs, bs, 1.0, 62, dist="int8").to_dense()
    a = np.hstack([x, x])
    b = np.vstack([y, -y])
    P = oracle.multiply(synth.from_dense(a, bs), synth.from_dense(b, bs))
    assert P.triples > 0 and P.C.nblk == 0


def test_partial_cancellation_keeps_other_blocks():
    bs = 4
    a = np.zeros((8, 8)); b = np.zeros((8, 8))
    a[0:4, 0:4] = 1.0; a[0:4, 4:8] = 1.0; a[4:8, 0:4] = 2.0
    b[0:4, 0:4] = 3.0; b[4:8, 0:4] = -3.0; b[0:4, 4:8] = 1.0
    C = oracle.multiply(synth.from_dense(a, bs), synth.from_dense(b, bs)).C
    keys = set(zip(C.brow.tolist(), C.bcol.tolist()))
    assert keys == {(0, 1), (1, 0), (1, 1)}  # block (0,0) cancels to exactly zero
    assert np.array_equal(C.to_dense(), a @ b)


def test_zero_rules_on_input():
    bs = 2
    vals = np.zeros((3, bs, bs))
    vals[1, 0, 0] = -0.0          # -0.0 is zero: dropped
    vals[2, 1, 1] = np.nan        # NaN is not zero: kept
    m = synth.BlockCOO(4, 4, bs, np.array([0, 1, 1], np.int32), np.array([0, 0, 1], np.int32), vals)
    t = oracle.tree(m)
    assert t.nblocks() == 1


def test_errors():
    bs = 4
    one = np.ones((1, bs, bs))
    with pytest.raises(oracle.OracleError) as e:
        oracle.tree(synth.BlockCOO(8, 8, bs, np.array([2], np.int32), np.array([0], np.int32), one))
    assert e.value.code == -4
    with pytest.raises(oracle.OracleError) as e:
        oracle.tree(synth.BlockCOO(8, 8, bs, np.array([1, 1], np.int32), np.array([0, 0], np.int32),
                                   np.ones((2, bs, bs))))
    assert e.value.code == -5
    A = synth.random_blocks(8, 4, 1.0, 1, ncols=12)
    with pytest.raises(oracle.OracleError) as e:
        oracle.multiply(A, A)
    assert e.value.code == -2


def test_empty_and_one_sided():
    bs = 16
    A = synth.random_blocks(128, bs, 0.2, 71)
    Z = synth.BlockCOO(128, 128, bs, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, bs, bs)))
    assert oracle.multiply(A, Z).C.nblk == 0
    assert oracle.multiply(Z, A).C.nblk == 0
    # A nonzero only in the left half, B only in the bottom half: no K overlaps
    L = synth.from_dense(np.hstack([np.ones((128, 64)), np.zeros((128, 64))]), bs)
    R = synth.from_dense(np.vstack([np.zeros((64, 128)), np.ones((64, 128))]), bs)
    P = oracle.multiply(L, R, leaf_dim=bs)
    assert P.C.nblk == 0 and P.triples == 0
    one = synth.random_blocks(1, 1, 1.0, 5)
    assert oracle.multiply(one, one).C.vals[0, 0, 0] == one.vals[0, 0, 0] ** 2


def test_block_product_by_definition():
    A = synth.random_blocks(512, 32, 0.2, 81)
    B = synth.random_blocks(512, 32, 0.2, 82)
    L = oracle.common_depth(A, B)
    ta, tb = oracle.tree(A, L), oracle.tree(B, L)
    E = dense_product_blocks(A, B)
    for t in range(0, E.nblk, 7):
        found, blk = oracle.block_product(ta, tb, E.brow[t], E.bcol[t])
        assert found and relerr(blk, E.vals[t]) < 1e-14


def test_block_product_from_restricted_operands():
    """The sampled checks compute C_IJ from A restricted to the sampled block
    rows and B to the sampled block columns: the same bits as from the whole
    operands, since C_IJ only reads row I of A and column J of B."""
    A = synth.random_blocks(700, 32, 0.15, 83)
    B = synth.random_blocks(700, 32, 0.15, 84)
    L = oracle.common_depth(A, B)
    ta, tb = oracle.tree(A, L), oracle.tree(B, L)
    rows, cols = np.array([1, 5, 9, 12, 16, 20]), np.array([0, 3, 5, 11, 17, 21])
    ka, kb = np.isin(A.brow, rows), np.isin(B.bcol, cols)
    left = synth.BlockCOO(A.nrows, A.ncols, 32, A.brow[ka], A.bcol[ka], A.vals[ka])
    right = synth.BlockCOO(B.nrows, B.ncols, 32, B.brow[kb], B.bcol[kb], B.vals[kb])
    tl, tr = oracle.tree(left, L), oracle.tree(right, L)
    E = dense_product_blocks(A, B)
    n = 0
    for i in rows:
        for j in cols:
            f1, b1 = oracle.block_product(ta, tb, i, j)
            f2, b2 = oracle.block_product(tl, tr, i, j)
            assert f1 == f2 and np.array_equal(b1, b2)
            hit = (E.brow == i) & (E.bcol == j)
            if hit.any():
                n += 1
                assert relerr(b1, E.vals[hit][0]) < 1e-14
            else:
                assert not np.any(b1)
    assert n > 5


def test_pattern_product_helper_is_the_oracle_structure():
    """The block-pattern product the full-size GPU tests use as C's
    definition equals the oracle's structure (no exact cancellation with
    N(0,1) entries), rectangular and ragged included."""
    from helpers import pattern_product
    for (m, k, n, bs, p, seed) in [(900, 700, 500, 32, 0.05, 91), (333, 333, 333, 16, 0.2, 92)]:
        A = synth.random_blocks(m, bs, p, seed, ncols=k)
        B = synth.random_blocks(k, bs, p, seed + 1, ncols=n)
        E = oracle.multiply(A, B).C
        r, c = pattern_product(A.brow, A.bcol, B.brow, B.bcol, A.mb, A.nb, B.nb)
        assert np.array_equal(r, E.brow) and np.array_equal(c, E.bcol)


# ------------------------------------------------- task counts (Sec. 5.1)
def brute_force_level_counts(A, B, L):
    """Count (A node (I,K), B node (K,J)) pairs at every level of a block quadtree."""
    out = []
    for level in range(L + 1):
        s = L - level
        an = set(zip((A.brow >> s).tolist(), (A.bcol >> s).tolist()))
        bn = set(zip((B.brow >> s).tolist(), (B.bcol >> s).tolist()))
        ca, cb = {}, {}
        for (_, k) in an:
            ca[k] = ca.get(k, 0) + 1
        for (k, _) in bn:
            cb[k] = cb.get(k, 0) + 1
        out.append(sum(v * cb.get(k, 0) for k, v in ca.items()))
    return np.array(out)


@pytest.mark.parametrize("kind", ["random", "banded", "rect"])
def test_task_counts_match_brute_force(kind):
    if kind == "random":
        A = synth.random_blocks(2048, 16, 0.03, 91); B = synth.random_blocks(2048, 16, 0.03, 92)
    elif kind == "banded":
        A = synth.banded(2000, 40, 16, 93); B = synth.banded(2000, 24, 16, 94)
    else:
        A = synth.random_blocks(700, 16, 0.1, 95, ncols=1500)
        B = synth.random_blocks(1500, 16, 0.1, 96, ncols=300)
    L = oracle.common_depth(A, B)
    t = oracle.task_counts(A, B)
    assert np.array_equal(t, brute_force_level_counts(A, B, L))


def test_eq1_random_expectation_and_bounds():
    """Blocksize-1 quadtree, random pattern: mean C_l vs Eq. 1, bounds Eq. 2/3 and total."""
    L, delta, reps = 8, 0.02, 12
    N = 1 << L
    acc = np.zeros(L + 1)
    for r in range(reps):
        A = synth.random_blocks(N, 1, delta, 1000 + 2 * r)
        B = synth.random_blocks(N, 1, delta, 1001 + 2 * r)
        t = oracle.task_counts(A, B)
        assert np.all(t <= 8.0 ** np.arange(L + 1))                    # Eq. 2, always
        acc += t
    mean = acc / reps
    l = np.arange(L + 1)
    expect = 2.0 ** (3 * l) * (1 - (1 - delta) ** (2.0 ** (2 * (L - l)))) ** 2   # Eq. 1
    assert np.allclose(mean, expect, rtol=0.06)
    assert np.all(expect <= 16.0 ** L * delta ** 2 / 2.0 ** l + 1e-9)          # Eq. 3
    fac = GOLD["random_total_bound_factor"]["value"]
    assert mean.sum() < fac * (delta * N * N) ** 1.5


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_eq5_banded_bounds(k):
    """Blocksize-1 quadtree, banded with d = 2^k: per-level bound Eq. 5 and total bound."""
    L = 9
    N, d = 1 << L, 1 << k
    A = synth.banded(N, d, 1, 2000 + k)
    B = synth.banded(N, d, 1, 3000 + k)
    t = oracle.task_counts(A, B)
    l = np.arange(L + 1)
    dl = np.where(l < L - k, 1, 2.0 ** (l - (L - k)))
    assert np.all(t < 2.0 ** l * (2 * dl + 1) ** 2)
    c2, c1, c0, cm1 = GOLD["banded_total_bound_coeffs"]["value"]
    assert t.sum() < (c2 * d * d + c1 * d + c0 + cm1 / d) * N
    # leaf-level task count equals the element multiply-add count of the product
    assert 2 * t[-1] == metrics.banded_element_flops(N, d)
