"""Pins of the oracle's Frobenius norms and truncation, and of the R-MAT
generator (CPU only).

Norms: against numpy sums (to rounding) and exactly for integer data; node
norms against the blocks of each node's region.  Truncation: against the
properties the rule must have, in exact rational arithmetic -- the removed
squared norm never exceeds tau^2, the removed blocks are the smallest ones,
the run is maximal up to the integer rounding slack, and the limit cases.
"""
import fractions

import numpy as np
import pytest

import oracle
import synth


def exact_norm2(block) -> fractions.Fraction:
    return sum((fractions.Fraction(float(x)) ** 2 for x in np.ravel(block)), fractions.Fraction(0))


def morton(I, J):
    k = 0
    for b in range(32):
        k |= ((I >> b) & 1) << (2 * b + 1) | ((J >> b) & 1) << (2 * b)
    return k


def test_block_norm2_against_numpy_and_integers():
    rng = np.random.default_rng(3)
    for bs in (4, 16, 32, 64):
        x = rng.standard_normal((bs, bs))
        assert abs(oracle.block_norm2(x) - np.sum(x * x)) <= 1e-14 * np.sum(x * x)
        z = rng.integers(-1000, 1000, (bs, bs)).astype(np.float64)
        assert oracle.block_norm2(z) == float(np.sum(z.astype(np.int64) ** 2))
    # the fixed order (row sums first, then the rows): row 0 = 2^54 + 1 rounds
    # to 2^54, row 1 = 3, total 2^54 + 3 rounds to 2^54 + 4; one running sum
    # over all entries would lose every +1 and give 2^54
    b = np.array([[2.0 ** 27, 1, 0], [1, 1, 1], [0, 0, 0]])
    assert oracle.block_norm2(b) == 2.0 ** 54 + 4


@pytest.mark.parametrize("height", [0, 1, 2, 3])
def test_node_norms_are_region_sums(height):
    A = synth.random_blocks(40 * 16 + 3, 16, 0.2, 71, dist="int8")   # exact integer sums
    I, J, v = oracle.node_norms2(A, height)
    f = 1 << height
    expect = {}
    for r, c, blk in zip(A.brow, A.bcol, A.vals):
        k = (int(r) // f, int(c) // f)
        expect[k] = expect.get(k, 0) + int(np.sum(blk.astype(np.int64) ** 2))
    assert len(v) == len(expect)
    for i, j, x in zip(I, J, v):
        assert x == float(expect[(int(i), int(j))])
    # depth-first child order is Morton order
    keys = [morton(int(i), int(j)) for i, j in zip(I, J)]
    assert keys == sorted(keys)


def test_root_norm_is_frobenius_norm():
    A = synth.random_blocks(300, 16, 0.3, 72)
    depth = oracle.tree(A, None, leaf_dim=16).depth
    _, _, v = oracle.node_norms2(A, depth)
    assert v.size == 1
    assert abs(v[0] - np.sum(A.vals ** 2)) <= 1e-13 * v[0]


def truncation_case(seed=81, n=600, bs=16, p=0.3, spread=True):
    A = synth.random_blocks(n, bs, p, seed)
    if spread:   # norms over many magnitudes
        A.vals *= np.exp(np.linspace(-12, 2, A.nblk))[:, None, None]
    return A


@pytest.mark.parametrize("frac", [1e-6, 1e-3, 0.1, 0.5, 0.999])
def test_truncation_properties(frac):
    A = truncation_case()
    total = exact_norm2(A.vals)
    tau = float(np.sqrt(float(total) * frac))
    T, removed, bound = oracle.truncate(A, tau)
    keep = set(zip(T.brow.tolist(), T.bcol.tolist()))
    gone = [(int(r), int(c), b) for r, c, b in zip(A.brow, A.bcol, A.vals)
            if (int(r), int(c)) not in keep]
    assert len(gone) == removed == A.nblk - T.nblk
    t2 = fractions.Fraction(tau) ** 2
    # the computed squared norms of the removed blocks sum to at most tau^2,
    # decided exactly (rational arithmetic here)
    comp = sum((fractions.Fraction(oracle.block_norm2(b)) for _, _, b in gone),
               fractions.Fraction(0))
    assert comp <= t2
    # each computed norm is within bs^2 rounding errors of the true one
    rem = sum((exact_norm2(b) for _, _, b in gone), fractions.Fraction(0))
    assert rem <= t2 * (1 + fractions.Fraction(2 * A.bs ** 2, 2 ** 53))
    # the reported bound: the integer sum as a double, between the two
    assert fractions.Fraction(bound) <= t2
    assert fractions.Fraction(bound) >= comp * (1 - fractions.Fraction(1, 2 ** 52))
    # the removed blocks are the smallest ones
    kept_norms = [oracle.block_norm2(b) for b in T.vals]
    gone_norms = [oracle.block_norm2(b) for _, _, b in gone]
    if gone_norms and kept_norms:
        assert max(gone_norms) <= min(kept_norms)
        # maximal up to the rounding slack (< 2^e per block, 2^e <= tau^2 2^-63)
        nxt = min(kept_norms)
        slack = t2 * A.nblk / fractions.Fraction(2 ** 63)
        assert comp + fractions.Fraction(nxt) > t2 - slack
    # kept blocks are unchanged
    S = A.sorted()
    lookup = {(int(r), int(c)): b for r, c, b in zip(S.brow, S.bcol, S.vals)}
    for r, c, b in zip(T.brow, T.bcol, T.vals):
        assert np.array_equal(b, lookup[(int(r), int(c))])


def test_truncation_limits_and_ties():
    A = truncation_case(spread=False)
    assert oracle.truncate(A, 0.0)[1] == 0
    assert oracle.truncate(A, -1.0)[1] == 0
    assert oracle.truncate(A, float("inf"))[1] == A.nblk
    total = float(exact_norm2(A.vals))
    assert oracle.truncate(A, np.sqrt(total) * (1 + 1e-9))[1] == A.nblk
    # equal norms: removed in Morton order
    bs = 4
    vals = np.ones((6, bs, bs))
    brow = np.array([3, 0, 2, 1, 0, 2], np.int32)
    bcol = np.array([0, 3, 2, 1, 0, 0], np.int32)
    E = synth.BlockCOO(16, 16, bs, brow, bcol, vals)
    T, removed, _ = oracle.truncate(E, np.sqrt(3 * 16.0) * (1 + 1e-12))  # room for three
    assert removed == 3
    order = sorted(zip(brow.tolist(), bcol.tolist()), key=lambda ij: morton(*ij))
    assert set(zip(T.brow.tolist(), T.bcol.tolist())) == set(order[3:])


def test_rmat_generator():
    r, c = synth.rmat_edges(13, 0.25, 5, 7)
    n = 1 << 13
    assert r.size <= 5 * n and r.size > 0.99 * 5 * n      # few repeats at a = 0.25
    assert np.all((0 <= r) & (r < n) & (0 <= c) & (c < n))
    key = r * n + c
    assert np.unique(key).size == key.size and np.all(np.diff(key) > 0)
    # a = 0.25 is uniform: each top-level quadrant holds about a quarter
    q = (r >= n // 2) * 2 + (c >= n // 2)
    assert np.all(np.abs(np.bincount(q, minlength=4) / r.size - 0.25) < 0.02)
    # larger a concentrates entries toward the top-left corner and repeats more
    # (where draws repeat, the distinct entries fall below the draw share a)
    prev, prev_tl = None, 0.0
    for a in (0.25, 0.5, 0.75, 0.95):
        r, c = synth.rmat_edges(13, a, 5, 7)
        top_left = np.mean((r < n // 2) & (c < n // 2))
        assert top_left > prev_tl and top_left <= a + 0.01
        if a <= 0.5:
            assert abs(top_left - a) < 0.02
        if prev is not None:
            assert r.size < prev
        prev, prev_tl = r.size, top_left
    M = synth.rmat(13, 0.6, 16, 7)
    assert np.array_equal(np.sort(np.argwhere(M.to_dense() != 0) @ [n, 1]),
                          np.sort(np.array(synth.rmat_edges(13, 0.6, 5, 7)).T @ [n, 1]))
