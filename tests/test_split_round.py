"""The split kernel's exact recombination and single rounding, built for the
host from the header the kernel includes (csrc/bsm_split_round.cuh) and
checked against exact rational arithmetic.

For every output the kernel holds S diagonal sums D_d as FP32 bit patterns
D_d + 1.5 * 2^23 and needs RN(V 2^X), V = sum_d D_d 2^(B (S-1-d)) (the
digit expansion of the split product, base 2^B, B = 7 for BF16 and 4 for
E4M3 digits).  Checked here:
  - V is recombined exactly from the bit patterns (against Python integers),
    for diagonal sums up to the bounds of the largest fast-path flush;
  - V 2^X is rounded to the nearest double, ties to even (against
    float(Fraction), which rounds correctly), and +0.0 for V = 0;
  - the fast rounding declines exactly outside the normal range (the kernel
    then takes its general path);
  - the fast-path flush sizes: the largest block-product count per narrow
    flush whose worst-case |V| stays below 2^63 and whose diagonal sums stay
    below 2^22.
"""
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "split_round_check.cpp")
FORMATS = [(7, 7), (6, 7), (3, 7), (6, 4), (12, 4)]   # (S, B)


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("round") / "split_round_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-o", exe, SRC], check=True)
    return exe


def run(exe, cases):
    inp = "".join(f"{S} {B} {X} " + " ".join(map(str, D)) + "\n" for S, B, X, D in cases)
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True)
    lines = r.stdout.strip().split("\n")
    return lines[0], [ln.split() for ln in lines[1:]]


def max_products(S, B, bs):
    """Largest k with n = k bs inner elements: |D_0| <= n 2^(2B) and the last
    diagonal's n (S+2) 2^(2B-2) at most 2^22 (D + 1.5 2^23 is exact, with bit
    pattern 0x4B400000 + D, for every |D| <= 2^22: the ends are 2^23 and
    2^24), and sum_d |D_d| 2^(B(S-1-d)) < 2^63 with |D_d| <= n (d+3) 2^(2B-2)
    for d >= 1 (leading digits up to 2^B, the others up to 2^(B-1)), counted
    here as n (2d+2) 2^(2B-2) with a margin of 2^63 - 9e18 as in the header."""
    k = 0
    while True:
        n = (k + 1) * bs
        d0 = n * 4 ** B
        dl = n * (S + 2) * 2 ** (2 * B - 2)
        bound = d0 * 2 ** (B * (S - 1)) + sum(n * (2 * d + 2) * 2 ** (2 * B - 2) * 2 ** (B * (S - 1 - d))
                                              for d in range(1, S))
        if d0 > 2 ** 22 or dl > 2 ** 22 or bound >= 9.0e18:
            return k
        k += 1


def test_fast_path_flush_sizes(harness):
    head, _ = run(harness, [])
    got = list(map(int, head.split()))
    want = [max_products(7, 7, 32), max_products(7, 7, 16), max_products(6, 7, 32),
            max_products(3, 7, 32), max_products(12, 4, 32), max_products(6, 4, 32)]
    assert got == want
    assert got[0] >= 1 and got[4] >= 1   # BF16 x 7 and E4M3 x 12 at bs 32 use it


def digit_sums(rng, S, B, n):
    """Diagonal sums of one output for n inner elements, up to the bounds."""
    if rng.random() < 0.15:
        return [rng.randint(-50, 50) for _ in range(S)]
    if rng.random() < 0.05:   # every diagonal at its bound
        sg = rng.choice([-1, 1])
        return [sg * min(n * 4 ** B, 2 ** 22)] + \
               [sg * min(n * (d + 3) * 2 ** (2 * B - 2), 2 ** 22) for d in range(1, S)]
    return [rng.randint(-n * 4 ** B, n * 4 ** B)] + \
           [rng.randint(-n * (d + 3) * 2 ** (2 * B - 2), n * (d + 3) * 2 ** (2 * B - 2))
            for d in range(1, S)]


@pytest.mark.parametrize("S,B", FORMATS)
def test_recombination_and_rounding_exact(harness, S, B):
    rng = random.Random(1000 * S + B)
    n = max(1, max_products(S, B, 32)) * 32
    cases = []
    for _ in range(6000):
        D = digit_sums(rng, S, B, n)
        if rng.random() < 0.05:
            D = [0] * S
        X = rng.randint(-1150, 1000) if rng.random() < 0.1 else rng.randint(-140, 20)
        cases.append((S, B, X, D))
    # ties and near-ties: V = q 2^m + {0, 1/2, 1/2 +- 1} 2^m, q of 53 bits
    for _ in range(1500):
        q = rng.getrandbits(53) | (1 << 52)
        m = rng.randint(1, 9)
        V = (q << m) + rng.choice([0, 1, -1, 0]) + ((1 << (m - 1)) if rng.random() < 0.7 else 0)
        V = -V if rng.random() < 0.5 else V
        D, rest = [0] * S, V            # base-2^B digits of V, the leading one taking the rest
        for d in range(S - 1, 0, -1):
            D[d] = rest % (1 << B)
            rest //= 1 << B
        D[0] = rest
        if abs(D[0]) < 2 ** 22:
            cases.append((S, B, rng.randint(-60, 0), D))
    _, out = run(harness, cases)
    assert len(out) == len(cases)
    declined = 0
    for (S_, B_, X, D), (v, ok, bits) in zip(cases, out):
        V = sum(D[d] << (B_ * (S_ - 1 - d)) for d in range(S_))
        assert int(v) == V, (D, v, V)
        got = struct.unpack(">d", bytes.fromhex(bits))[0]
        if V == 0:
            assert ok == "1" and bits == "0000000000000000"
            continue
        be = abs(V).bit_length() - 1 + X + 1023       # biased exponent before rounding
        if ok == "0":
            declined += 1
            assert be < 1 or be > 2045, (V, X)
            continue
        assert 1 <= be <= 2045
        assert got == float(Fraction(V) * Fraction(2) ** X), (V, X)
    assert declined < len(cases) // 5
