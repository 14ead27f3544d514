"""CPU oracle for block-sparse C = A*B over a sparse quadtree (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline
may import this package.  It wraps ``bsm_oracle.c`` -- a plain, single-threaded
pointer quadtree that follows Algorithm 1 (multiply), Algorithm 2 (add) and the
block-sparse leaf multiply of Sec. 4.1 / Fig. 3 of Rubensson & Rudberg -- and
shares no code with the CUDA library.

Functions here are argument marshalling only; all arithmetic is in the C file.
``oracle/split.py`` (exact Python integers) defines the split-precision modes'
result, which the paper does not cover.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np

from synth import BlockCOO

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

ERRORS = {0: "ok", -1: "invalid argument", -2: "dimension mismatch", -3: "block size",
          -4: "out of range", -5: "duplicate block", -6: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle: {ERRORS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no vectorisation flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.orc_build.restype = P
    lib.orc_build.argtypes = [I64, I64, I32, I32, I32, I64, P, P, P, ctypes.POINTER(I32)]
    lib.orc_multiply.restype = P
    lib.orc_multiply.argtypes = [P, P, P, P, ctypes.POINTER(I32)]
    lib.orc_multiply_t.restype = P
    lib.orc_multiply_t.argtypes = [P, I32, P, I32, P, P, ctypes.POINTER(I32)]
    lib.orc_add.restype = P
    lib.orc_add.argtypes = [P, P, ctypes.POINTER(I32)]
    lib.orc_node_norms2.restype = I64
    lib.orc_node_norms2.argtypes = [P, I32, P, P, P]
    lib.orc_truncate.restype = P
    lib.orc_truncate.argtypes = [P, ctypes.c_double, ctypes.POINTER(I64),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(I32)]
    lib.orc_block_norm2.restype = ctypes.c_double
    lib.orc_block_norm2.argtypes = [P, I32]
    lib.orc_sym_full.restype = P
    lib.orc_sym_full.argtypes = [P, ctypes.POINTER(I32)]
    lib.orc_sym_square.restype = P
    lib.orc_sym_square.argtypes = [P, ctypes.POINTER(I32)]
    lib.orc_syrk.restype = P
    lib.orc_syrk.argtypes = [P, I32, ctypes.POINTER(I32)]
    lib.orc_symm.restype = P
    lib.orc_symm.argtypes = [P, P, I32, ctypes.POINTER(I32)]
    lib.orc_nblocks.restype = I64
    lib.orc_nblocks.argtypes = [P]
    lib.orc_depth.restype = I32
    lib.orc_depth.argtypes = [P]
    lib.orc_to_blocks.restype = I32
    lib.orc_to_blocks.argtypes = [P, P, P, P]
    lib.orc_free.restype = None
    lib.orc_free.argtypes = [P]
    lib.orc_block_product.restype = I32
    lib.orc_block_product.argtypes = [P, P, I64, I64, P]
    _lib = lib
    return lib


def ceil_log2(x: int) -> int:
    return max(0, int(x - 1).bit_length()) if x > 1 else 0


def common_depth(*ms: BlockCOO) -> int:
    """Tree depth L (in blocks) shared by the operands of one product."""
    return max(ceil_log2(max(m.mb, m.nb, 1)) for m in ms)


class Tree:
    """An oracle quadtree (owns the C-side object)."""

    def __init__(self, ptr, nrows, ncols, bs, L, leaf_nb):
        self._p = ptr
        self.nrows, self.ncols, self.bs, self.L, self.leaf_nb = nrows, ncols, bs, L, leaf_nb

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.orc_free(self._p)
            self._p = None

    @property
    def depth(self) -> int:
        return _load().orc_depth(self._p)

    def nblocks(self) -> int:
        return int(_load().orc_nblocks(self._p))

    def to_coo(self) -> BlockCOO:
        n = self.nblocks()
        bs = self.bs
        brow = np.zeros(n, np.int32)
        bcol = np.zeros(n, np.int32)
        vals = np.zeros((n, bs, bs), np.float64)
        rc = _load().orc_to_blocks(self._p, brow.ctypes.data, bcol.ctypes.data, vals.ctypes.data)
        if rc:
            raise OracleError(rc)
        return BlockCOO(self.nrows, self.ncols, bs, brow, bcol, vals)


def tree(m: BlockCOO, L: int | None = None, leaf_dim: int = 4096) -> Tree:
    """Build an oracle quadtree.  leaf_dim is the leaf matrix side in elements
    (4096 in the paper's runs, Sec. 6); it is rounded to whole blocks."""
    lib = _load()
    L = common_depth(m) if L is None else L
    leaf_nb = max(1, leaf_dim // m.bs)
    leaf_nb = 1 << (leaf_nb.bit_length() - 1)
    st = ctypes.c_int(0)
    brow = np.ascontiguousarray(m.brow, np.int32)
    bcol = np.ascontiguousarray(m.bcol, np.int32)
    vals = np.ascontiguousarray(m.vals, np.float64)
    p = lib.orc_build(m.nrows, m.ncols, m.bs, L, leaf_nb, m.nblk, brow.ctypes.data,
                      bcol.ctypes.data, vals.ctypes.data, ctypes.byref(st))
    if st.value:
        raise OracleError(st.value)
    return Tree(p, m.nrows, m.ncols, m.bs, L, min(leaf_nb, 1 << L))


@dataclasses.dataclass
class Product:
    C: BlockCOO
    tasks: np.ndarray  # multiply tasks per level, root level 0 first
    triples: int       # leaf block products (nonzero A_IK, B_KJ pairs)


def multiply(A: BlockCOO, B: BlockCOO, leaf_dim: int = 4096, trans_a: bool = False,
             trans_b: bool = False) -> Product:
    """C = op(A)*op(B) by the quadtree recursion (Algorithm 1/2, and the
    transposed task types of Sec. 3.2), zero blocks dropped."""
    L = common_depth(A, B)
    ta, tb = tree(A, L, leaf_dim), tree(B, L, leaf_dim)
    return multiply_trees(ta, tb, trans_a, trans_b)


def multiply_trees(ta: Tree, tb: Tree, trans_a: bool = False, trans_b: bool = False) -> Product:
    lib = _load()
    tasks = np.zeros(ta.depth + 1, np.int64)
    trip = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    p = lib.orc_multiply_t(ta._p, int(trans_a), tb._p, int(trans_b), tasks.ctypes.data,
                           ctypes.byref(trip), ctypes.byref(st))
    if st.value:
        raise OracleError(st.value)
    nrows = ta.ncols if trans_a else ta.nrows
    ncols = tb.nrows if trans_b else tb.ncols
    tc = Tree(p, nrows, ncols, ta.bs, ta.L, ta.leaf_nb)
    return Product(tc.to_coo(), tasks, int(trip.value))


def add(A: BlockCOO, B: BlockCOO, leaf_dim: int = 4096) -> BlockCOO:
    """C = A + B by Algorithm 2 (leaf add where both have a block), exactly
    zero sums dropped."""
    lib = _load()
    L = common_depth(A, B)
    ta, tb = tree(A, L, leaf_dim), tree(B, L, leaf_dim)
    st = ctypes.c_int(0)
    p = lib.orc_add(ta._p, tb._p, ctypes.byref(st))
    if st.value:
        raise OracleError(st.value)
    return Tree(p, ta.nrows, ta.ncols, ta.bs, ta.L, ta.leaf_nb).to_coo()


def task_counts(A: BlockCOO, B: BlockCOO) -> np.ndarray:
    """Multiply tasks per level of a quadtree whose leaves are single blocks
    (the per-level counts C_l of Sec. 5.1 at block granularity)."""
    return multiply(A, B, leaf_dim=A.bs).tasks


def block_product(ta: Tree, tb: Tree, I: int, J: int) -> tuple[bool, np.ndarray]:
    """C_IJ = sum_K A_IK B_KJ by definition (for sampled checks)."""
    out = np.zeros((ta.bs, ta.bs), np.float64)
    any_ = _load().orc_block_product(ta._p, tb._p, int(I), int(J), out.ctypes.data)
    return bool(any_), out


# ------------------------------------------------------- symmetric storage
# A symmetric matrix is passed as its upper triangle of blocks (I <= J), the
# diagonal blocks in full; symmetric results come back the same way.
def _call(fn, *args):
    st = ctypes.c_int(0)
    p = fn(*args, ctypes.byref(st))
    if st.value:
        raise OracleError(st.value)
    return p


def sym_full(U: BlockCOO, leaf_dim: int = 4096) -> BlockCOO:
    """The full matrix of an upper-triangle-stored symmetric matrix."""
    t = tree(U, None, leaf_dim)
    p = _call(_load().orc_sym_full, t._p)
    return Tree(p, U.nrows, U.ncols, U.bs, t.L, t.leaf_nb).to_coo()


def sym_square(U: BlockCOO, leaf_dim: int = 4096) -> BlockCOO:
    """Upper triangle of S*S, S the symmetric matrix U stores."""
    t = tree(U, None, leaf_dim)
    p = _call(_load().orc_sym_square, t._p)
    return Tree(p, U.nrows, U.ncols, U.bs, t.L, t.leaf_nb).to_coo()


def syrk(A: BlockCOO, trans: bool = False, leaf_dim: int = 4096) -> BlockCOO:
    """Upper triangle of A A^T (trans False) or A^T A (trans True)."""
    t = tree(A, None, leaf_dim)
    p = _call(_load().orc_syrk, t._p, int(bool(trans)))
    n = A.ncols if trans else A.nrows
    return Tree(p, n, n, A.bs, t.L, t.leaf_nb).to_coo()


def sym_multiply(A: BlockCOO, B: BlockCOO, side: int = 0, leaf_dim: int = 4096) -> BlockCOO:
    """S B (side 0, A stores S) or A S (side 1, B stores S)."""
    L = common_depth(A, B)
    ta, tb = tree(A, L, leaf_dim), tree(B, L, leaf_dim)
    p = _call(_load().orc_symm, ta._p, tb._p, int(side))
    return Tree(p, A.nrows, B.ncols, A.bs, L, ta.leaf_nb).to_coo()


# ---------------------------------------------------------- Frobenius norms
def block_norm2(block: np.ndarray) -> float:
    """Squared Frobenius norm of one block in the fixed summation order (rows
    ascending, each row's squares summed in ascending column order)."""
    b = np.ascontiguousarray(block, np.float64)
    return float(_load().orc_block_norm2(b.ctypes.data, b.shape[0]))


def node_norms2(A: BlockCOO, height: int):
    """(I, J, squared norm) of the quadtree nodes `height` levels above the
    blocks (0 = the blocks), in depth-first child order."""
    t = tree(A, None, leaf_dim=A.bs)
    lib = _load()
    n = lib.orc_node_norms2(t._p, int(height), None, None, None)
    if n < 0:
        raise OracleError(-1)
    I = np.zeros(n, np.int32)
    J = np.zeros(n, np.int32)
    v = np.zeros(n, np.float64)
    lib.orc_node_norms2(t._p, int(height), I.ctypes.data, J.ctypes.data, v.ctypes.data)
    return I, J, v


def truncate(A: BlockCOO, tau: float, leaf_dim: int = 4096):
    """(truncated matrix, blocks removed, bound on the removed squared norm)."""
    t = tree(A, None, leaf_dim)
    rem, bound = ctypes.c_int64(0), ctypes.c_double(0.0)
    p = _call(_load().orc_truncate, t._p, float(tau), ctypes.byref(rem), ctypes.byref(bound))
    return Tree(p, A.nrows, A.ncols, A.bs, t.L, t.leaf_nb).to_coo(), rem.value, bound.value
