"""CPU oracle for block-sparse C = A*B over a sparse quadtree (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline
may import this package.  It wraps ``bsm_oracle.c`` -- a plain, single-threaded
pointer quadtree that follows Algorithm 1 (multiply), Algorithm 2 (add) and the
block-sparse leaf multiply of Sec. 4.1 / Fig. 3 of Rubensson & Rudberg -- and
shares no code with the CUDA library.

Functions here are argument marshalling only; all arithmetic is in the C file.
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
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC])
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


def multiply(A: BlockCOO, B: BlockCOO, leaf_dim: int = 4096) -> Product:
    """C = A*B by the quadtree recursion (Algorithm 1/2), zero blocks dropped."""
    lib = _load()
    L = common_depth(A, B)
    ta, tb = tree(A, L, leaf_dim), tree(B, L, leaf_dim)
    return multiply_trees(ta, tb)


def multiply_trees(ta: Tree, tb: Tree) -> Product:
    lib = _load()
    tasks = np.zeros(ta.depth + 1, np.int64)
    trip = ctypes.c_int64(0)
    st = ctypes.c_int(0)
    p = lib.orc_multiply(ta._p, tb._p, tasks.ctypes.data, ctypes.byref(trip), ctypes.byref(st))
    if st.value:
        raise OracleError(st.value)
    tc = Tree(p, ta.nrows, tb.ncols, ta.bs, ta.L, ta.leaf_nb)
    return Product(tc.to_coo(), tasks, int(trip.value))


def task_counts(A: BlockCOO, B: BlockCOO) -> np.ndarray:
    """Multiply tasks per level of a quadtree whose leaves are single blocks
    (the per-level counts C_l of Sec. 5.1 at block granularity)."""
    return multiply(A, B, leaf_dim=A.bs).tasks


def block_product(ta: Tree, tb: Tree, I: int, J: int) -> tuple[bool, np.ndarray]:
    """C_IJ = sum_K A_IK B_KJ by definition (for sampled checks)."""
    out = np.zeros((ta.bs, ta.bs), np.float64)
    any_ = _load().orc_block_product(ta._p, tb._p, int(I), int(J), out.ctypes.data)
    return bool(any_), out
