"""GPU parity at the workloads' full sizes, through the calls the benchmark
times (bsm_multiply with its default launch configuration, bsm_sym_square,
bsm_multiply_batched).

The oracle cannot compute these products whole within a test, so each test
checks:
- C's block structure against its definition: the block-pattern product of
  the operands' stored blocks (SciPy sparse, on the host).  Every stored C
  block must be in it; a block of the definition may be missing from C only
  when all of its entries vanish.
- On a grid of sampled block rows x block columns, every block of the
  definition: its presence in C against the oracle's block-by-block
  definition C_IJ = sum_K A_IK B_KJ (zero iff every entry compares equal to
  0.0), and the relative Frobenius error of the values over the sampled
  blocks (1e-12 in FP64, 1e-11 in the split modes).  The oracle works on the
  operands restricted to the sampled block rows (left) and block columns
  (right), which is exact for these blocks.

Workloads: the random block-sparse product (N = 65536, p = 0.02, N(0,1)
entries) at leaf sizes 32, 16 and 64; the decay-type product with 20,000
points (N = 100,000), full and symmetric square; 64 batched products with N
log-uniform in [2048, 32768] and block density U[0.5%, 10%].
"""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import pattern_product, relerr
from paper_1501_07800_gb300 import shard

pytestmark = pytest.mark.gpu
TOL_FP64, TOL_SPLIT = 1e-12, 1e-11


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()
    yield
    # hand the large products' memory back for the tests that follow
    import gc
    gc.collect()
    bsm.bsm_release_memory()
    torch.cuda.empty_cache()


def host(x) -> np.ndarray:
    return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)


def stored_pattern(M):
    """Block rows and columns of a handle's stored blocks (row-major)."""
    import ctypes
    nblk = bsm.bsm_info(M)[3]
    r = np.zeros(max(nblk, 1), np.int32)
    c = np.zeros(max(nblk, 1), np.int32)
    cnt = ctypes.c_int64(nblk)
    assert bsm.load().bsm_to_blocks(M.handle, ctypes.byref(cnt), r.ctypes.data, c.ctypes.data,
                                    None, 0, None) == 0
    return r[:nblk], c[:nblk]


def grid(lo: int, hi: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(np.arange(lo, hi), size=min(k, hi - lo), replace=False))


class Reference:
    """Oracle values of the definition's blocks on a grid of block rows x
    block columns, from operands restricted to those rows / columns."""

    def __init__(self, n, bs, a, b, rows, cols):
        # a, b: (brow, bcol, vals) of the operands (host or device arrays)
        keep_a = np.isin(host(a[0]), rows)
        keep_b = np.isin(host(b[1]), cols)
        ka = np.flatnonzero(keep_a)
        kb = np.flatnonzero(keep_b)
        va, vb = a[2], b[2]
        if hasattr(va, "cpu"):
            import torch
            va = va[torch.from_numpy(ka).to(va.device)].cpu().numpy()
            vb = vb[torch.from_numpy(kb).to(vb.device)].cpu().numpy()
        else:
            va, vb = va[ka], vb[kb]
        self.left = synth.BlockCOO(n, n, bs, host(a[0])[ka], host(a[1])[ka], va)
        self.right = synth.BlockCOO(n, n, bs, host(b[0])[kb], host(b[1])[kb], vb)
        self.rows, self.cols = rows, cols
        self._memo = None

    def blocks(self, di, dj, nb):
        """The definition's blocks (di, dj) inside the grid: keys, nonzero
        flags and values."""
        if self._memo is None:
            self._memo = self._blocks(di, dj, nb)
        return self._memo

    def _blocks(self, di, dj, nb):
        inside = np.isin(di, self.rows) & np.isin(dj, self.cols)
        I, J = di[inside], dj[inside]
        bs = self.left.bs
        if len(I) == 0:
            return np.zeros(0, np.int64), np.zeros(0, bool), np.zeros((0, bs, bs))
        L = oracle.common_depth(self.left, self.right)
        tl, tr = oracle.tree(self.left, L), oracle.tree(self.right, L)
        vals = np.stack([oracle.block_product(tl, tr, i, j)[1] for i, j in zip(I, J)])
        nz = np.array([bool(np.any(v != 0.0)) for v in vals])
        return I * nb + J, nz, vals

    def upper_view(self, nb):
        """The same grid's blocks with I <= J (after blocks() has run)."""
        key, nz, vals = self._memo
        keep = key // nb <= key % nb
        view = Reference.__new__(Reference)
        view._memo = (key[keep], nz[keep], vals[keep])
        return view


def check(C, nb, di, dj, ref: Reference, tol):
    """Structure against the definition (di, dj), presence and values on the
    reference grid.  Returns (relative error, blocks compared, blocks of C,
    blocks of the definition)."""
    import torch
    # the library's cached pool memory is not available to PyTorch's allocator
    bsm.bsm_release_memory()
    r, c, v = bsm.bsm_to_blocks(C, device=True)
    gkey = host(r).astype(np.int64) * nb + host(c).astype(np.int64)
    dkey = di * nb + dj
    assert np.all(np.diff(gkey) > 0), "C blocks not in row-major order"
    pos = np.searchsorted(dkey, gkey)
    assert np.all(pos < len(dkey)) and np.array_equal(dkey[pos], gkey), \
        "C holds blocks outside the definition's structure"
    skey, snz, svals = ref.blocks(di, dj, nb)
    if len(skey) == 0:
        return 0.0, 0, len(gkey), len(dkey)
    gi = np.searchsorted(gkey, skey)
    present = (gi < len(gkey)) & (gkey[np.minimum(gi, len(gkey) - 1)] == skey)
    assert np.array_equal(present, snz), \
        f"presence differs from the oracle on {int((present != snz).sum())} sampled blocks"
    got = v[torch.from_numpy(gi[present]).to(v.device)].cpu().numpy()
    err = relerr(got, svals[present])
    assert err <= tol, err
    return err, int(present.sum()), len(gkey), len(dkey)


# ------------------------------------------------------------ random product
@pytest.fixture(scope="module", params=[32, 16, 64])
def random_65536(request):
    bs, n, p = request.param, 65536, 0.02
    A = synth.random_blocks(n, bs, p, synth.BASE_SEED + 1)
    B = synth.random_blocks(n, bs, p, synth.BASE_SEED + 1 + 7919)
    nb = -(-n // bs)
    di, dj = pattern_product(A.brow, A.bcol, B.brow, B.bcol, nb, nb, nb)
    ref = Reference(n, bs, (A.brow, A.bcol, A.vals), (B.brow, B.bcol, B.vals),
                    grid(0, nb, 48, 11), grid(0, nb, 48, 12))
    ga = bsm.bsm_build(n, n, bs, A.brow, A.bcol, A.vals)
    gb = bsm.bsm_build(n, n, bs, B.brow, B.bcol, B.vals)
    yield bs, nb, ga, gb, di, dj, ref
    del ga, gb


@pytest.mark.parametrize("prec,slices", [(bsm.BSM_FP64, 0), (bsm.BSM_SPLIT_BF16, 7),
                                         (bsm.BSM_SPLIT_FP8, 12)],
                         ids=["fp64", "bf16x7", "fp8x12"])
def test_random_65536_full_size(random_65536, prec, slices):
    bs, nb, ga, gb, di, dj, ref = random_65536
    C = bsm.bsm_multiply(ga, gb, prec=prec, slices=slices)
    err, ncmp, nc, nd = check(C, nb, di, dj, ref, TOL_FP64 if prec == bsm.BSM_FP64 else TOL_SPLIT)
    # N(0,1) entries: no C block of the definition vanishes
    assert nc == nd
    assert ncmp > 100


# ------------------------------------------------------------- decay product
def test_decay_20000_full_size():
    import torch

    from synth import device as sd
    dev = torch.device("cuda", torch.cuda.current_device())
    bs = 32
    n, r, c, v = sd.decay(20000, bs, synth.BASE_SEED + 2, dev)
    nb = -(-n // bs)
    A = bsm.bsm_build(n, n, bs, r, c, v)
    up = r <= c
    U = bsm.bsm_build(n, n, bs, r[up].contiguous(), c[up].contiguous(), v[up].contiguous())
    del up
    # the definition's structure from A's stored blocks (the generator's
    # blocks whose entries all fall below the cutoff are not stored)
    ar, ac = stored_pattern(A)
    di, dj = pattern_product(ar, ac, ar, ac, nb, nb, nb)
    del ar, ac
    # grid 1: uniform over C; grid 2: inside the diagonal node [1024, 1536)^2
    rows1, cols1 = grid(0, nb, 24, 21), grid(0, nb, 24, 22)
    rows2, cols2 = grid(1024, 1536, 24, 23), grid(1024, 1536, 24, 24)
    ops = (r, c, v)
    ref1 = Reference(n, bs, ops, ops, rows1, cols1)
    ref2 = Reference(n, bs, ops, ops, rows2, cols2)
    del r, c, v, ops
    torch.cuda.empty_cache()

    # full product, split BF16 x 7 (the benchmark's split leg)
    C = bsm.bsm_multiply(A, A, prec=bsm.BSM_SPLIT_BF16, slices=7)
    err, ncmp, nc, nd = check(C, nb, di, dj, ref1, TOL_SPLIT)
    assert nd - nc > 0  # blocks of point groups beyond twice the cutoff vanish
    assert ncmp > 200
    del C
    torch.cuda.empty_cache()

    # symmetric square in upper-triangle storage, split BF16 x 7
    upper = di <= dj
    CU = bsm.bsm_sym_square(U, prec=bsm.BSM_SPLIT_BF16, slices=7)
    err, ncmp, _, _ = check(CU, nb, di[upper], dj[upper], ref1.upper_view(nb), TOL_SPLIT)
    assert ncmp > 100
    del CU, U
    torch.cuda.empty_cache()

    # FP64 on the C blocks of one quadtree node (a Morton range), same kernels
    lo = int(shard.morton(1024, 1024))
    hi = lo + 512 * 512
    CR = bsm.bsm_multiply_range(A, A, lo, hi)
    inr = (di >= 1024) & (di < 1536) & (dj >= 1024) & (dj < 1536)
    err, ncmp, _, _ = check(CR, nb, di[inr], dj[inr], ref2, TOL_FP64)
    assert ncmp > 100


# ----------------------------------------------------------- batched products
def test_batched_64_full_size():
    import torch

    from synth import device as sd
    dev = torch.device("cuda", torch.cuda.current_device())
    gen = sd.batched(64, synth.BASE_SEED + 3, dev)
    As = [bsm.bsm_build(n, n, 32, r, c, v) for (n, r, c, v), _ in gen]
    Bs = [bsm.bsm_build(n, n, 32, r, c, v) for _, (n, r, c, v) in gen]
    defs, refs = [], []
    for t, ((n, ar, ac, av), (_, br, bc, bv)) in enumerate(gen):
        nb = -(-n // 32)
        di, dj = pattern_product(ar, ac, br, bc, nb, nb, nb)
        defs.append((nb, di, dj))
        # grid: the rows and columns of 8 blocks drawn from the definition
        pick = np.random.default_rng(100 + t).choice(len(di), size=min(8, len(di)), replace=False)
        refs.append(Reference(n, 32, (ar, ac, av), (br, bc, bv),
                              np.unique(di[pick]), np.unique(dj[pick])))
    del gen
    torch.cuda.empty_cache()
    for prec, tol in ((bsm.BSM_FP64, TOL_FP64), (bsm.BSM_SPLIT_BF16, TOL_SPLIT)):
        Cs = bsm.bsm_multiply_batched(As, Bs, prec=prec)
        ncmp = 0
        for C, (nb, di, dj), ref in zip(Cs, defs, refs):
            err, k, nc, nd = check(C, nb, di, dj, ref, tol)
            assert nc == nd  # uniform entries: no C block vanishes
            ncmp += k
        assert ncmp > 200
        del Cs
