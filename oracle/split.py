"""Exact result of the split-precision product (test infrastructure).

Only the tests may import this module; it shares no code with the CUDA
library.  The split modes are not in Rubensson & Rudberg's paper: they follow
the error-free splitting of matrix products into low-precision slices of
Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012), with a per-row /
per-column power-of-two scale.  This module writes the scheme's result out by
its definition, in exact integers, step by step:

1. Scales.  Row r of A gets the exponent E_r, the largest over the row of
   the smallest E with |A_rk| < 2^E (a subnormal entry counts as 2^-1022);
   column c of B gets F_c the same way.
2. Fixed point.  X = A_rk 2^(BS - E_r), rounded to the nearest integer, ties
   away from zero (B bits per digit, S digits: B = 7 for BF16, 4 for E4M3).
3. Digits.  X is cut into S balanced base-2^B digits, lowest first: digit =
   ((X + 2^(B-1)) mod 2^B) - 2^(B-1), X <- (X - digit) / 2^B; the last
   quotient is the leading digit a_0, so X = sum_i a_i 2^(B(S-1-i)).
4. Diagonal sums.  D_d = sum_k sum_{i+j=d} a_i(r,k) b_j(k,c) for d < S (the
   digit pairs beyond the last diagonal are dropped).
5. Result.  C_rc = D 2^(E_r + F_c - B(S+1)) with D = sum_{d<S} D_d
   2^(B(S-1-d)), rounded once to the nearest double, ties to even.
6. A C block whose entries are all zero is dropped.

Exact Python integers throughout (numpy int64 where the magnitudes are
bounded), so the result depends on nothing but these definitions.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

from synth import BlockCOO

FORMATS = {"bf16": 7, "fp8": 4}


def _smallest_e(x: float) -> int:
    """Smallest integer E with |x| < 2^E (x != 0), by exact comparison."""
    num, den = abs(float(x)).as_integer_ratio()
    e = num.bit_length() - den.bit_length() - 1
    while Fraction(num, den) >= Fraction(2) ** e:
        e += 1
    return e


def scale_exponent(x: float) -> int | None:
    """Step 1 for one entry: the smallest E with |x| < 2^E, at least -1022
    (a subnormal entry counts as 2^-1022); None for zero."""
    if x == 0.0:
        return None
    return max(_smallest_e(x), -1022)


def fixed_point(x: float, E: int, B: int, S: int) -> int:
    """round(x 2^(BS - E)), ties away from zero, exactly."""
    v = Fraction(float(x)) * Fraction(2) ** (B * S - E)
    mag = abs(v)
    q = int(mag + Fraction(1, 2))  # floor(|v| + 1/2): ties away from zero
    return -q if v < 0 else q


def digits(X: int, B: int, S: int) -> list[int]:
    """Balanced base-2^B digits, leading digit first."""
    out = [0] * S
    half, mask = 1 << (B - 1), (1 << B) - 1
    for i in range(S - 1, 0, -1):
        d = ((X + half) & mask) - half
        out[i] = d
        X = (X - d) >> B
    out[0] = X
    return out


def _row_exponents(m: BlockCOO, axis: int) -> dict[int, int]:
    """Exponent per global row (axis 0) or column (axis 1)."""
    out: dict[int, int] = {}
    bs = m.bs
    for t in range(m.nblk):
        blk = m.vals[t]
        base = (m.brow[t] if axis == 0 else m.bcol[t]) * bs
        for u in range(bs):
            line = blk[u, :] if axis == 0 else blk[:, u]
            es = [scale_exponent(v) for v in line if v != 0.0]
            if es:
                g = int(base + u)
                out[g] = max(out.get(g, -10**9), max(es))
    return out


def _slices(m: BlockCOO, exps: dict[int, int], axis: int, B: int, S: int) -> np.ndarray:
    """Digits of every entry: int64 [nblk][S][bs][bs]."""
    bs = m.bs
    out = np.zeros((m.nblk, S, bs, bs), dtype=np.int64)
    for t in range(m.nblk):
        for r in range(bs):
            for c in range(bs):
                x = float(m.vals[t, r, c])
                if x == 0.0:
                    continue
                g = int((m.brow[t] * bs + r) if axis == 0 else (m.bcol[t] * bs + c))
                ds = digits(fixed_point(x, exps[g], B, S), B, S)
                out[t, :, r, c] = ds
    return out


def multiply(A: BlockCOO, B_: BlockCOO, fmt: str = "bf16", slices: int = 7) -> BlockCOO:
    """The split-precision product C = A*B by the definition above."""
    assert A.bs == B_.bs and A.ncols == B_.nrows
    Bb, S, bs = FORMATS[fmt], slices, A.bs
    er = _row_exponents(A, 0)
    fc = _row_exponents(B_, 1)
    sa = _slices(A, er, 0, Bb, S)
    sb = _slices(B_, fc, 1, Bb, S)
    a_by_row: dict[int, list[int]] = {}
    for t in range(A.nblk):
        a_by_row.setdefault(int(A.brow[t]), []).append(t)
    b_by_key = {(int(B_.brow[t]), int(B_.bcol[t])): t for t in range(B_.nblk)}
    b_cols = sorted({int(j) for j in B_.bcol})
    rows, cols, vals = [], [], []
    for I in sorted(a_by_row):
        for J in b_cols:
            D = np.zeros((S, bs, bs), dtype=np.int64)
            hit = False
            for ta in a_by_row[I]:
                tb = b_by_key.get((int(A.bcol[ta]), J))
                if tb is None:
                    continue
                hit = True
                for i in range(S):
                    for j in range(S - i):
                        D[i + j] += sa[ta, i] @ sb[tb, j]
            if not hit:
                continue
            blk = np.zeros((bs, bs))
            for r in range(bs):
                for c in range(bs):
                    V = sum(int(D[d, r, c]) << (Bb * (S - 1 - d)) for d in range(S))
                    if V == 0:
                        continue
                    X = er[I * bs + r] + fc[J * bs + c] - Bb * (S + 1)
                    blk[r, c] = float(Fraction(V) * Fraction(2) ** X)
            if np.any(blk != 0.0):
                rows.append(I)
                cols.append(J)
                vals.append(blk)
    vals_a = np.stack(vals) if vals else np.zeros((0, bs, bs))
    return BlockCOO(A.nrows, B_.ncols, bs, np.array(rows, np.int32), np.array(cols, np.int32),
                    vals_a)
