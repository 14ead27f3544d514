"""Flop conventions used to report throughput (no part of the product itself).

* Block-useful flops: 2 * bs^3 per nonzero (A_IK, B_KJ) block pair, the
  convention of the paper's leaf library runs (2 b^3 per b x b product,
  Sec. 6.1, Table 2; dense products counted as 2 N^3, Sec. 6).
* Element-level flops of a banded product with bandwidth 2d+1 (Sec. 6.1):
  2 (N (2d+1)^2 - (5/3) d (d+1) (2d+1)).
"""


def block_flops(bs: int, triples: int) -> float:
    return 2.0 * bs ** 3 * triples


def banded_element_flops(n: int, d: int) -> float:
    return 2.0 * (n * (2 * d + 1) ** 2 - (5.0 / 3.0) * d * (d + 1) * (2 * d + 1))
