"""Python binding of libbsm: block-sparse C = A*B over a sparse quadtree on GB300.

Argument marshalling only: every step of the product runs in the CUDA library
(``csrc/``), declared in ``include/bsm.h``.  Function names match the C ABI.
Host inputs are numpy arrays; device inputs and outputs are torch CUDA tensors
(PyTorch supplies device memory and streams, nothing else).  If libbsm.so is
missing the import fails: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbsm.so")

BSM_FP64 = 0
BSM_SPLIT_BF16 = 1
BSM_SPLIT_FP8 = 2
BSM_FLAG_AUTOTUNE = 1
BSM_FLAG_TRANS_A = 2
BSM_FLAG_TRANS_B = 4
BSM_FLAG_AUTOTUNE_BS = 8
BSM_SYM_LEFT = 0
BSM_SYM_RIGHT = 1

STATUS = {
    0: "BSM_OK", -1: "BSM_ERR_INVALID_ARG", -2: "BSM_ERR_DIM_MISMATCH", -3: "BSM_ERR_BLOCKSIZE",
    -4: "BSM_ERR_OUT_OF_RANGE", -5: "BSM_ERR_DUPLICATE", -6: "BSM_ERR_OOM", -7: "BSM_ERR_CUDA",
    -8: "BSM_ERR_TIMEOUT", -9: "BSM_ERR_BUFFER_TOO_SMALL", -10: "BSM_ERR_UNSUPPORTED",
}

# function name -> (restype, argtypes)
_P, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
_PROTOS = {
    "bsm_build": (_I32, [_I64, _I64, _I32, _I64, _P, _P, _P, _I32, _P, _P]),
    "bsm_multiply": (_I32, [_P, _P, _P, _P, _P]),
    "bsm_transpose": (_I32, [_P, _P, _P]),
    "bsm_multiply_range": (_I32, [_P, _P, ctypes.c_uint64, ctypes.c_uint64, _P, _P, _P]),
    "bsm_add": (_I32, [_P, _P, _P, _P]),
    "bsm_sym_square": (_I32, [_P, _P, _P, _P]),
    "bsm_syrk": (_I32, [_P, _I32, _P, _P, _P]),
    "bsm_sym_multiply": (_I32, [_P, _P, _I32, _P, _P, _P]),
    "bsm_sym_to_full": (_I32, [_P, _P, _P]),
    "bsm_reblock": (_I32, [_P, _I32, _P, _P]),
    "bsm_node_norms2": (_I32, [_P, _I32, _P, _P, _P, _P, _I32, _P]),
    "bsm_truncate": (_I32, [_P, ctypes.c_double, _P, _P, _P, _P]),
    "bsm_multiply_batched": (_I32, [_I32, _P, _P, _P, _P, _P]),
    "bsm_to_blocks": (_I32, [_P, _P, _P, _P, _P, _I32, _P]),
    "bsm_info": (_I32, [_P, _P, _P, _P, _P]),
    "bsm_level_counts": (_I32, [_P, _P, _I32, _P]),
    "bsm_last_stats": (_I32, [_P, _I32, _P, _P, _P]),
    "bsm_last_chunks": (_I32, [_P]),
    "bsm_set_timing": (_I32, [_I32]),
    "bsm_release_memory": (_I32, []),
    "bsm_set_memory_limit": (_I32, [ctypes.c_uint64]),
    "bsm_memory_in_use": (_I32, [_P]),
    "bsm_last_phase_ms": (_I32, [_P, _I32, _P, _P]),
    "bsm_block_products_fp64_noalloc": (_I32, [_I32, _I64, _P, _P, _P, _P, _I64, _P, _I64, _P,
                                                _P, _P]),
    "bsm_selftest_wait_timeout": (_I32, [_I32, _P]),
    "bsm_probe_fp64": (_I32, [_I32, _I64, _P, _P, _P]),
    "bsm_probe_tcgen05": (_I32, [_I32, _I32, _I32, _I32, _I64, _P, _P, _P]),
    "bsm_probe_bulk_copy": (_I32, [_I64, _I32, _I32, _P, _P, _P]),
    "bsm_update_values": (_I32, [_P, _I64, _P, _P, _P, _I32, _P]),
    "bsm_plan_create": (_I32, [_I32, _P, _P, _P, _P, _P]),
    "bsm_plan_execute": (_I32, [_P, _P]),
    "bsm_plan_results": (_I32, [_P, _P, _P]),
    "bsm_plan_info": (_I32, [_P, _P, _P, _P, _P]),
    "bsm_plan_block_size": (_I32, [_P, _P]),
    "bsm_plan_tile": (_I32, [_P, _P, _P, _P]),
    "bsm_plan_destroy": (_I32, [_P]),
    "bsm_destroy": (_I32, [_P]),
    "bsm_status_string": (ctypes.c_char_p, [_I32]),
}

_lib = None


class BsmError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        name = STATUS.get(code, str(code))
        super().__init__(f"{what}: {name}" if what else name)
        self.code = code
        self.name = name


class bsm_mult_opts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("slices", ctypes.c_int), ("flags", ctypes.c_int),
                ("bs", ctypes.c_int)]


def load(path: str | None = None):
    """Load libbsm.so (built by ``build.build()``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libbsm.so not built ({path}); run paper_1501_07800_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(code: int, what: str):
    if code != 0:
        raise BsmError(code, what)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and x.is_cuda


class Matrix:
    """Owning wrapper of a bsm_matrix handle (freed with bsm_destroy)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.bsm_destroy(h)
            self.handle = None

    def destroy(self):
        self.__del__()

    def info(self):
        return bsm_info(self)

    @property
    def nblk(self) -> int:
        return bsm_info(self)[3]


def bsm_status_string(code: int) -> str:
    return load().bsm_status_string(code).decode()


def bsm_build(nrows: int, ncols: int, bs: int, brow, bcol, vals, stream=None) -> Matrix:
    """Build from COO blocks: numpy (host) or torch CUDA tensors (device)."""
    lib = load()
    out = ctypes.c_void_p()
    if _is_torch_cuda(vals):
        import torch
        brow = brow.to(torch.int32).contiguous()
        bcol = bcol.to(torch.int32).contiguous()
        vals = vals.to(torch.float64).contiguous()
        n = int(brow.numel())
        code = lib.bsm_build(nrows, ncols, bs, n, brow.data_ptr(), bcol.data_ptr(),
                             vals.data_ptr(), 1, _stream_ptr(stream), ctypes.byref(out))
    else:
        brow = np.ascontiguousarray(brow, np.int32)
        bcol = np.ascontiguousarray(bcol, np.int32)
        vals = np.ascontiguousarray(vals, np.float64)
        n = int(brow.shape[0])
        code = lib.bsm_build(nrows, ncols, bs, n, brow.ctypes.data, bcol.ctypes.data,
                             vals.ctypes.data, 0, _stream_ptr(stream), ctypes.byref(out))
    _check(code, "bsm_build")
    return Matrix(out.value)


def _opts(prec: int, slices: int, flags: int = 0, bs: int = 0):
    if prec == BSM_FP64 and slices == 0 and flags == 0 and bs == 0:
        return None
    return ctypes.byref(bsm_mult_opts(prec, slices, flags, bs))


def bsm_multiply(A: Matrix, B: Matrix, prec: int = BSM_FP64, slices: int = 0,
                 stream=None, trans_a: bool = False, trans_b: bool = False,
                 bs: int = 0) -> Matrix:
    """C = op(A) op(B); op(X) = X^T when trans_x is set.  bs: leaf size to
    compute at (operands re-cut to it; 0 = theirs)."""
    lib = load()
    out = ctypes.c_void_p()
    flags = (BSM_FLAG_TRANS_A if trans_a else 0) | (BSM_FLAG_TRANS_B if trans_b else 0)
    code = lib.bsm_multiply(A.handle, B.handle, ctypes.byref(out),
                            _opts(prec, slices, flags, bs), _stream_ptr(stream))
    _check(code, "bsm_multiply")
    return Matrix(out.value)


def bsm_multiply_range(A: Matrix, B: Matrix, key_lo: int, key_hi: int, prec: int = BSM_FP64,
                       slices: int = 0, stream=None) -> Matrix:
    """The C blocks of A*B with Morton keys in [key_lo, key_hi)."""
    out = ctypes.c_void_p()
    _check(load().bsm_multiply_range(A.handle, B.handle, int(key_lo), int(key_hi),
                                     ctypes.byref(out), _opts(prec, slices), _stream_ptr(stream)),
           "bsm_multiply_range")
    return Matrix(out.value)


def bsm_transpose(A: Matrix, stream=None) -> Matrix:
    out = ctypes.c_void_p()
    _check(load().bsm_transpose(A.handle, ctypes.byref(out), _stream_ptr(stream)),
           "bsm_transpose")
    return Matrix(out.value)


def bsm_add(A: Matrix, B: Matrix, stream=None) -> Matrix:
    out = ctypes.c_void_p()
    _check(load().bsm_add(A.handle, B.handle, ctypes.byref(out), _stream_ptr(stream)), "bsm_add")
    return Matrix(out.value)


def bsm_sym_square(A: Matrix, prec: int = BSM_FP64, slices: int = 0, stream=None) -> Matrix:
    """Upper triangle of A*A; A symmetric in upper-triangle storage."""
    out = ctypes.c_void_p()
    _check(load().bsm_sym_square(A.handle, ctypes.byref(out), _opts(prec, slices),
                                 _stream_ptr(stream)), "bsm_sym_square")
    return Matrix(out.value)


def bsm_syrk(A: Matrix, trans: bool = False, prec: int = BSM_FP64, slices: int = 0,
             stream=None) -> Matrix:
    """Upper triangle of A A^T (trans False) or A^T A (trans True)."""
    out = ctypes.c_void_p()
    _check(load().bsm_syrk(A.handle, int(bool(trans)), ctypes.byref(out), _opts(prec, slices),
                           _stream_ptr(stream)), "bsm_syrk")
    return Matrix(out.value)


def bsm_sym_multiply(A: Matrix, B: Matrix, side: int = BSM_SYM_LEFT, prec: int = BSM_FP64,
                     slices: int = 0, stream=None) -> Matrix:
    """A B with A (side BSM_SYM_LEFT) or B (BSM_SYM_RIGHT) symmetric in
    upper-triangle storage."""
    out = ctypes.c_void_p()
    _check(load().bsm_sym_multiply(A.handle, B.handle, int(side), ctypes.byref(out),
                                   _opts(prec, slices), _stream_ptr(stream)), "bsm_sym_multiply")
    return Matrix(out.value)


def bsm_sym_to_full(A: Matrix, stream=None) -> Matrix:
    out = ctypes.c_void_p()
    _check(load().bsm_sym_to_full(A.handle, ctypes.byref(out), _stream_ptr(stream)),
           "bsm_sym_to_full")
    return Matrix(out.value)


def bsm_reblock(A: Matrix, bs: int, stream=None) -> Matrix:
    out = ctypes.c_void_p()
    _check(load().bsm_reblock(A.handle, int(bs), ctypes.byref(out), _stream_ptr(stream)),
           "bsm_reblock")
    return Matrix(out.value)


def bsm_node_norms2(M: Matrix, height: int = 0, stream=None):
    """(I, J, squared norm) of the nodes `height` levels above the blocks."""
    lib = load()
    n = ctypes.c_int64(0)
    _check(lib.bsm_node_norms2(M.handle, int(height), None, None, None, ctypes.byref(n), 0,
                               _stream_ptr(stream)), "bsm_node_norms2")
    v = np.zeros(n.value, np.float64)
    I = np.zeros(n.value, np.int32)
    J = np.zeros(n.value, np.int32)
    _check(lib.bsm_node_norms2(M.handle, int(height), v.ctypes.data, I.ctypes.data, J.ctypes.data,
                               ctypes.byref(n), 0, _stream_ptr(stream)), "bsm_node_norms2")
    return I, J, v


def bsm_truncate(M: Matrix, tau: float, stream=None):
    """(truncated handle, blocks removed, bound on the removed squared norm)."""
    out = ctypes.c_void_p()
    rem, bound = ctypes.c_int64(0), ctypes.c_double(0.0)
    _check(load().bsm_truncate(M.handle, float(tau), ctypes.byref(out), ctypes.byref(rem),
                               ctypes.byref(bound), _stream_ptr(stream)), "bsm_truncate")
    return Matrix(out.value), rem.value, bound.value


def bsm_multiply_batched(As, Bs, prec: int = BSM_FP64, slices: int = 0, stream=None,
                         bs: int = 0):
    lib = load()
    n = len(As)
    if len(Bs) != n:
        raise ValueError("As and Bs differ in length")
    ha = (ctypes.c_void_p * max(n, 1))(*[a.handle for a in As])
    hb = (ctypes.c_void_p * max(n, 1))(*[b.handle for b in Bs])
    hc = (ctypes.c_void_p * max(n, 1))()
    code = lib.bsm_multiply_batched(n, ha, hb, hc, _opts(prec, slices, 0, bs),
                                    _stream_ptr(stream))
    _check(code, "bsm_multiply_batched")
    return [Matrix(hc[i]) for i in range(n)]


def bsm_info(M: Matrix):
    """(nrows, ncols, bs, nblk)."""
    nr, nc, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    bs = ctypes.c_int()
    _check(load().bsm_info(M.handle, ctypes.byref(nr), ctypes.byref(nc), ctypes.byref(bs),
                           ctypes.byref(nb)), "bsm_info")
    return nr.value, nc.value, bs.value, nb.value


def bsm_to_blocks(M: Matrix, device: bool = False, stream=None, out=None,
                  asynchronous: bool = False):
    """Stored blocks in row-major (I, J) order: (brow, bcol, vals).

    device=False: numpy arrays (the call synchronises the stream);
    device=True: torch CUDA tensors on the current device.  `out` may supply
    preallocated (brow, bcol, vals) buffers of either kind.  asynchronous=True
    (host output into page-locked `out` buffers): the copy is queued on the
    stream and the call returns at once; synchronise the stream before reading
    the buffers, and keep M alive until then.
    """
    if asynchronous and (device or out is None):
        raise ValueError("asynchronous output needs page-locked host buffers in `out`")
    lib = load()
    nr, nc, bs, n = bsm_info(M)
    if out is not None:
        # capacity = the smallest caller buffer, in blocks
        caps = [int(out[0].shape[0]), int(out[1].shape[0]), int(out[2].shape[0])]
        if tuple(out[2].shape[1:]) != (bs, bs):
            raise ValueError("vals buffer must be [n, bs, bs]")
        want = ("int32", "int32", "float64")
        for o, w in zip(out, want):
            if str(o.dtype).replace("torch.", "") != w:
                raise ValueError(f"buffer dtype {o.dtype}, expected {w}")
        cnt = ctypes.c_int64(min(caps))
    else:
        cnt = ctypes.c_int64(n)
    if device:
        import torch
        if out is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            out = (torch.empty(n, dtype=torch.int32, device=dev),
                   torch.empty(n, dtype=torch.int32, device=dev),
                   torch.empty((n, bs, bs), dtype=torch.float64, device=dev))
        ptrs = [t.data_ptr() for t in out]
        code = lib.bsm_to_blocks(M.handle, ctypes.byref(cnt), *ptrs, 1, _stream_ptr(stream))
    else:
        if out is None:
            out = (np.empty(n, np.int32), np.empty(n, np.int32), np.empty((n, bs, bs), np.float64))
        ptrs = [o.data_ptr() if hasattr(o, "data_ptr") else o.ctypes.data for o in out]
        code = lib.bsm_to_blocks(M.handle, ctypes.byref(cnt), *ptrs, 2 if asynchronous else 0,
                                 _stream_ptr(stream))
    _check(code, "bsm_to_blocks")
    return out


def bsm_level_counts(M: Matrix) -> np.ndarray:
    lib = load()
    nlev = ctypes.c_int()
    _check(lib.bsm_level_counts(M.handle, None, 0, ctypes.byref(nlev)), "bsm_level_counts")
    c = np.zeros(nlev.value, np.int64)
    _check(lib.bsm_level_counts(M.handle, c.ctypes.data, nlev.value, ctypes.byref(nlev)),
           "bsm_level_counts")
    return c


def bsm_last_stats():
    """(tasks per level root first, triples, C blocks before zero removal)."""
    lib = load()
    nlev, trip, ncs = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
    t = np.zeros(64, np.int64)
    _check(lib.bsm_last_stats(t.ctypes.data, 64, ctypes.byref(nlev), ctypes.byref(trip),
                              ctypes.byref(ncs)), "bsm_last_stats")
    return t[: nlev.value].copy(), trip.value, ncs.value


def bsm_last_chunks() -> int:
    n = ctypes.c_int()
    _check(load().bsm_last_chunks(ctypes.byref(n)), "bsm_last_chunks")
    return n.value


def bsm_set_timing(on: bool):
    _check(load().bsm_set_timing(1 if on else 0), "bsm_set_timing")


def bsm_set_memory_limit(nbytes: int):
    """Cap the library's device pool usage (0: no cap); allocations beyond it
    make the call return BSM_ERR_OOM."""
    _check(load().bsm_set_memory_limit(int(nbytes)), "bsm_set_memory_limit")


def bsm_memory_in_use() -> int:
    """Bytes of the library's device pool held by live allocations."""
    v = ctypes.c_uint64()
    _check(load().bsm_memory_in_use(ctypes.byref(v)), "bsm_memory_in_use")
    return v.value


def bsm_release_memory():
    """Give the library's cached device memory back to the driver (after a
    device synchronisation), e.g. before a large PyTorch allocation."""
    _check(load().bsm_release_memory(), "bsm_release_memory")


def bsm_last_phase_ms():
    """([symbolic, numeric, finish] ms of the last timed product, kernel launches)."""
    ms = np.zeros(3, np.float64)
    n, launches = ctypes.c_int(), ctypes.c_int64()
    _check(load().bsm_last_phase_ms(ms.ctypes.data, 3, ctypes.byref(n), ctypes.byref(launches)),
           "bsm_last_phase_ms")
    return ms, launches.value


BSM_NOALLOC_MAX_CBLOCKS = 1 << 20


def bsm_block_products_fp64_noalloc(bs: int, seg, ta, tb, a_vals, b_vals, c_vals, nnz_out,
                                    stream=None):
    """FP64 block products of a caller-supplied task list into caller buffers,
    with no allocation (all arguments are torch CUDA tensors; see bsm.h).

    The tensors are checked, not converted (a conversion would allocate):
    seg, ta, tb int32; a_vals, b_vals, c_vals float64 [n, bs, bs]; nnz_out
    int64 with one element; all contiguous and on the current CUDA device.
    """
    import torch
    dev = torch.cuda.current_device()
    want = (("seg", seg, torch.int32), ("ta", ta, torch.int32), ("tb", tb, torch.int32),
            ("a_vals", a_vals, torch.float64), ("b_vals", b_vals, torch.float64),
            ("c_vals", c_vals, torch.float64), ("nnz_out", nnz_out, torch.int64))
    for name, t, dt in want:
        if not _is_torch_cuda(t) or t.device.index != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device (cuda:{dev})")
        if t.dtype != dt:
            raise ValueError(f"{name} has dtype {t.dtype}, expected {dt}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    for name, t in (("a_vals", a_vals), ("b_vals", b_vals), ("c_vals", c_vals)):
        if t.dim() != 3 or tuple(t.shape[1:]) != (bs, bs):
            raise ValueError(f"{name} must have shape [n, {bs}, {bs}]")
    if seg.dim() != 1 or seg.numel() < 1:
        raise ValueError("seg must be a 1-D tensor of nc + 1 offsets")
    if ta.shape != tb.shape or ta.dim() != 1:
        raise ValueError("ta and tb must be 1-D tensors of the same length")
    if nnz_out.numel() != 1:
        raise ValueError("nnz_out must hold one element")
    nc = int(seg.numel()) - 1
    if int(c_vals.shape[0]) != nc:
        raise ValueError(f"c_vals holds {int(c_vals.shape[0])} blocks, seg describes {nc}")
    code = load().bsm_block_products_fp64_noalloc(
        bs, nc, seg.data_ptr(), ta.data_ptr(), tb.data_ptr(), a_vals.data_ptr(),
        int(a_vals.shape[0]), b_vals.data_ptr(), int(b_vals.shape[0]), c_vals.data_ptr(),
        nnz_out.data_ptr(), _stream_ptr(stream))
    _check(code, "bsm_block_products_fp64_noalloc")


BSM_PROBE_DMMA_M8N8K4 = 0
BSM_PROBE_DMMA_M16N8K4 = 1
BSM_PROBE_DMMA_M16N8K8 = 2
BSM_PROBE_DMMA_M16N8K16 = 3
BSM_PROBE_DFMA = 4
BSM_PROBE_MIXED = 5


def bsm_probe_fp64(kind: int, iters: int, stream=None):
    """(flops, ms) of one FP64 probe launch (include/bsm_probe.h)."""
    f, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().bsm_probe_fp64(int(kind), int(iters), ctypes.byref(f), ctypes.byref(ms),
                                 _stream_ptr(stream)), "bsm_probe_fp64")
    return f.value, ms.value


def bsm_probe_tcgen05(fmt: int, n: int, iters: int, tiles: int = 1, issuers: int = 1,
                      stream=None):
    """(flops, ms) of one tcgen05.mma probe launch: fmt 0 BF16, 1 E4M3; M = 128;
    consecutive instructions cycle through `tiles` distinct operand pairs;
    `issuers` threads per SM issue concurrently."""
    f, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().bsm_probe_tcgen05(int(fmt), int(n), int(tiles), int(issuers), int(iters),
                                    ctypes.byref(f), ctypes.byref(ms), _stream_ptr(stream)),
           "bsm_probe_tcgen05")
    return f.value, ms.value


def bsm_probe_bulk_copy(nbytes: int, stage_bytes: int = 32768, stages: int = 4, stream=None):
    """(bytes, ms) of one bulk-copy streaming launch."""
    f, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().bsm_probe_bulk_copy(int(nbytes), int(stage_bytes), int(stages),
                                      ctypes.byref(f), ctypes.byref(ms), _stream_ptr(stream)),
           "bsm_probe_bulk_copy")
    return f.value, ms.value


def bsm_selftest_wait_timeout(limit_ms: int, stream=None) -> str:
    """Status name the bounded-wait self test returns (expected BSM_ERR_TIMEOUT)."""
    return STATUS.get(load().bsm_selftest_wait_timeout(limit_ms, _stream_ptr(stream)), "?")


def bsm_update_values(M: Matrix, brow, bcol, vals, stream=None):
    """New values for exactly the blocks M stores (numpy host or torch CUDA arrays)."""
    lib = load()
    if _is_torch_cuda(vals):
        import torch
        brow = brow.to(torch.int32).contiguous()
        bcol = bcol.to(torch.int32).contiguous()
        vals = vals.to(torch.float64).contiguous()
        code = lib.bsm_update_values(M.handle, int(brow.numel()), brow.data_ptr(),
                                     bcol.data_ptr(), vals.data_ptr(), 1, _stream_ptr(stream))
    else:
        brow = np.ascontiguousarray(brow, np.int32)
        bcol = np.ascontiguousarray(bcol, np.int32)
        vals = np.ascontiguousarray(vals, np.float64)
        code = lib.bsm_update_values(M.handle, int(brow.shape[0]), brow.ctypes.data,
                                     bcol.ctypes.data, vals.ctypes.data, 0, _stream_ptr(stream))
    _check(code, "bsm_update_values")


class Plan:
    """Owning wrapper of a bsm_plan (freed with bsm_plan_destroy).  Keeps the
    operand handles alive as long as the plan."""

    def __init__(self, handle: int, As, Bs):
        self.handle = handle
        self._operands = (list(As), list(Bs))
        self.n = len(As)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.bsm_plan_destroy(h)
            self.handle = None


def bsm_plan_create(As, Bs, prec: int = BSM_FP64, slices: int = 0, autotune: bool = False,
                    stream=None, autotune_bs: bool = False, bs: int = 0) -> Plan:
    lib = load()
    n = len(As)
    ha = (ctypes.c_void_p * max(n, 1))(*[a.handle for a in As])
    hb = (ctypes.c_void_p * max(n, 1))(*[b.handle for b in Bs])
    flags = (BSM_FLAG_AUTOTUNE if autotune else 0) | (BSM_FLAG_AUTOTUNE_BS if autotune_bs else 0)
    opts = bsm_mult_opts(prec, slices, flags, bs)
    out = ctypes.c_void_p()
    code = lib.bsm_plan_create(n, ha, hb, ctypes.byref(opts), _stream_ptr(stream),
                               ctypes.byref(out))
    _check(code, "bsm_plan_create")
    return Plan(out.value, As, Bs)


def bsm_plan_execute(plan: Plan, stream=None):
    _check(load().bsm_plan_execute(plan.handle, _stream_ptr(stream)), "bsm_plan_execute")


def bsm_plan_results(plan: Plan, stream=None):
    hc = (ctypes.c_void_p * max(plan.n, 1))()
    _check(load().bsm_plan_results(plan.handle, hc, _stream_ptr(stream)), "bsm_plan_results")
    return [Matrix(hc[i]) for i in range(plan.n)]


def bsm_plan_info(plan: Plan):
    """(order, chunk, ctas_per_sm, work items)."""
    o, c, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    n = ctypes.c_int64()
    _check(load().bsm_plan_info(plan.handle, ctypes.byref(o), ctypes.byref(c), ctypes.byref(k),
                                ctypes.byref(n)), "bsm_plan_info")
    return o.value, c.value, k.value, n.value


def bsm_plan_tile(plan: Plan):
    """(form, tile_m, tile_n): 1 = FP64 DFMA, a thread's tile_m x tile_n
    outputs; 0 = FP64 mma.sync 8 x 8 tiles; 2 = split, tcgen05 M x N."""
    f, m, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().bsm_plan_tile(plan.handle, ctypes.byref(f), ctypes.byref(m), ctypes.byref(n)),
           "bsm_plan_tile")
    return f.value, m.value, n.value


def bsm_plan_block_size(plan: Plan) -> int:
    b = ctypes.c_int()
    _check(load().bsm_plan_block_size(plan.handle, ctypes.byref(b)), "bsm_plan_block_size")
    return b.value


def bsm_plan_destroy(plan: Plan):
    plan.__del__()


def bsm_destroy(M: Matrix):
    M.destroy()
