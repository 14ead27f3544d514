"""Pins of the split-precision oracle (oracle/split.py) on the CPU: the digit
decomposition reconstructs its integer, small-integer data come out equal to
the FP64 oracle, the error against the FP64 oracle stays within the bound of
the fixed point and shrinks with the slice count, and the result is
symmetric under transposition and exact under power-of-two row scaling."""
import math

import numpy as np
import pytest

import oracle
import synth
from helpers import assert_same_structure, relerr
from oracle import split as osplit


@pytest.mark.parametrize("B,S", [(7, 1), (7, 3), (7, 7), (7, 8), (4, 2), (4, 6), (4, 12)])
def test_digits_reconstruct_and_stay_balanced(B, S):
    rng = np.random.default_rng(5 + B * S)
    lim = 1 << (B * S)
    for X in list(rng.integers(-lim, lim, 200)) + [0, lim, -lim, lim - 1, 1 - lim]:
        X = int(X)
        d = osplit.digits(X, B, S)
        assert sum(di << (B * (S - 1 - i)) for i, di in enumerate(d)) == X
        assert all(-(1 << (B - 1)) <= di < (1 << (B - 1)) for di in d[1:])
        assert abs(d[0]) <= (1 << B)  # |X| <= 2^(BS)


def test_scale_exponent_definition():
    for x in [1.0, 0.75, 2.0, 3.0, 1e300, -0.5, 2.0 ** -1022, 1.5 * 2.0 ** -1000]:
        E = osplit.scale_exponent(x)
        assert abs(x) < 2.0 ** E and abs(x) >= 2.0 ** (E - 1)
    assert osplit.scale_exponent(5e-324) == -1022  # subnormal: counts as 2^-1022
    assert osplit.scale_exponent(0.0) is None


def test_fixed_point_rounds_ties_away_from_zero():
    assert osplit.fixed_point(2.5 * 2.0 ** -14, 0, 7, 2) == 3
    assert osplit.fixed_point(-2.5 * 2.0 ** -14, 0, 7, 2) == -3
    assert osplit.fixed_point(0.3, 0, 7, 7) == round(0.3 * 2 ** 49)


@pytest.mark.parametrize("fmt,slices", [("bf16", 1), ("bf16", 2), ("fp8", 2)])
def test_small_integers_equal_fp64(fmt, slices):
    """Integers |a| <= 8 take at most 4 bits from the row's scale: the first
    digit holds them exactly, every digit product and sum is exact, so the
    split result is the exact product, which the FP64 oracle also gets."""
    A = synth.random_blocks(2 * 32 + 5, 32, 0.6, 31, dist="int8")
    B = synth.random_blocks(2 * 32 + 5, 32, 0.6, 32, dist="int8")
    C = osplit.multiply(A, B, fmt, slices)
    E = oracle.multiply(A, B).C
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


def test_error_bound_and_monotone_in_slices():
    A = synth.random_blocks(2 * 16 + 3, 16, 0.7, 41)
    B = synth.random_blocks(2 * 16 + 3, 16, 0.7, 42)
    E = oracle.multiply(A, B).C
    prev = math.inf
    for S in (2, 3, 5, 7):
        C = osplit.multiply(A, B, "bf16", S)
        assert_same_structure(C, E)
        err = relerr(C.vals, E.vals)
        # each operand carries 7S bits against its row / column scale; the
        # dropped digit pairs and the rounding of both operands stay below a
        # few units of 2^-7S relative to the scales (entries are N(0,1))
        assert err < 2.0 ** (-7 * S + 10), (S, err)
        assert err < prev
        prev = err


def test_transpose_symmetry_bit_exact():
    """Row scales of A are column scales of A^T, and every digit pair (i, j)
    of C_rc is the pair (j, i) of (C^T)_cr: the two products agree bit for
    bit."""
    A = synth.random_blocks(3 * 16 + 2, 16, 0.5, 51, ncols=2 * 16 + 9)
    B = synth.random_blocks(2 * 16 + 9, 16, 0.5, 52, ncols=3 * 16 + 7)

    def t(m):
        return synth.BlockCOO(m.ncols, m.nrows, m.bs, m.bcol.copy(), m.brow.copy(),
                              np.ascontiguousarray(m.vals.transpose(0, 2, 1)))
    C = osplit.multiply(A, B, "bf16", 4)
    CT = osplit.multiply(t(B), t(A), "bf16", 4)
    assert CT.nblk == C.nblk > 0
    assert np.array_equal(CT.to_dense(), C.to_dense().T)


def test_power_of_two_row_scaling_is_exact():
    A = synth.random_blocks(2 * 16 + 1, 16, 0.8, 61)
    B = synth.random_blocks(2 * 16 + 1, 16, 0.8, 62)
    C = osplit.multiply(A, B, "fp8", 6)
    As = synth.BlockCOO(A.nrows, A.ncols, A.bs, A.brow, A.bcol, A.vals.copy())
    As.vals[As.brow == 1] *= 2.0 ** 40  # block row 1 of A, exactly
    Cs = osplit.multiply(As, B, "fp8", 6)
    want = C.to_dense()
    want[16:32] *= 2.0 ** 40
    assert np.array_equal(Cs.to_dense(), want)


def test_one_slice_is_the_rounded_product_of_the_rounded_operands():
    """With one slice nothing is dropped: C_rc is the correctly rounded exact
    sum of products of the operands rounded to B bits against their row /
    column scales, a_rk = round(A_rk 2^(B-E_r)) 2^(E_r-B) -- an independent
    check of the scales, the fixed point and the final exponent."""
    from fractions import Fraction
    Bb = 7
    A = synth.random_blocks(2 * 16 + 3, 16, 0.8, 71)
    B = synth.random_blocks(2 * 16 + 3, 16, 0.8, 72)
    C = osplit.multiply(A, B, "bf16", 1)
    Ad, Bd = A.to_dense(), B.to_dense()
    n = Ad.shape[0]
    er = [max((osplit.scale_exponent(v) for v in Ad[r] if v != 0), default=0) for r in range(n)]
    fc = [max((osplit.scale_exponent(v) for v in Bd[:, c] if v != 0), default=0) for c in range(n)]

    def rnd(x, E):  # x rounded to B bits below 2^E, ties away from zero
        v = Fraction(float(x)) * Fraction(2) ** (Bb - E)
        q = int(abs(v) + Fraction(1, 2))
        return Fraction(-q if v < 0 else q) * Fraction(2) ** (E - Bb)
    Ar = [[rnd(Ad[r, k], er[r]) for k in range(n)] for r in range(n)]
    Br = [[rnd(Bd[k, c], fc[c]) for c in range(n)] for k in range(n)]
    Cd = C.to_dense()
    rng = np.random.default_rng(73)
    for r, c in zip(rng.integers(0, n, 60), rng.integers(0, n, 60)):
        exact = sum((Ar[r][k] * Br[k][c] for k in range(n)), Fraction(0))
        assert Cd[r, c] == float(exact)
