"""GPU parity: tree builder, symbolic phase and FP64 numeric phase vs the oracle.

Structure must match the oracle bit-exactly; values within 1e-12 relative
Frobenius error (FP64 summation-order differences are ~sqrt(K) u ~ 1e-14 for
the inner lengths here, so 1e-12 leaves a wide margin without hiding a wrong
term, which would show up as O(1) error).
"""
import numpy as np
import pytest

import oracle
import paper_1501_07800_gb300 as bsm
import synth
from helpers import assert_same_structure, from_bsm, relerr, to_bsm

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    torch.cuda.init()
    bsm.load()


def gpu_product(A, B, device_inputs=False, **kw):
    ga, gb = to_bsm(A, device_inputs), to_bsm(B, device_inputs)
    gc = bsm.bsm_multiply(ga, gb, **kw)
    return from_bsm(gc)


# ------------------------------------------------------------- tree builder
@pytest.mark.parametrize("device", [False, True])
def test_build_roundtrip(device):
    A = synth.random_blocks(1000, 32, 0.1, 5)
    M = to_bsm(A, device)
    R = from_bsm(M)
    E = A.sorted()
    assert_same_structure(R, E)
    assert np.array_equal(R.vals, E.vals)


def test_build_from_pinned_host_inputs():
    """Pinned host COO arrays are read in place by the build kernels: the same
    matrix as from pageable arrays (exactly-zero blocks dropped), the same
    errors, and the caller may overwrite its buffers once the call returns.
    A pinned values array the device sees misaligned goes through the staged
    copy."""
    import torch
    A = synth.random_blocks(2000, 32, 0.08, 31)
    A.vals[::7] = 0.0                                  # some exactly-zero blocks

    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
        t.numpy()[...] = a
        return t, t.numpy()

    keep = [pinned(x) for x in (A.brow, A.bcol, A.vals)]
    r, c, v = (x for _, x in keep)
    M = bsm.bsm_build(A.nrows, A.ncols, 32, r, c, v)
    v[...] = np.nan                                    # after the call: no effect on M
    R, E = from_bsm(M), from_bsm(to_bsm(A))
    assert R.nblk == E.nblk < A.nblk
    assert_same_structure(R, E)
    assert np.array_equal(R.vals, E.vals)
    v[...] = A.vals
    bad = r.copy()
    r[3] = r[5]
    c[3] = c[5]                                        # a duplicate coordinate
    with pytest.raises(bsm.BsmError, match="DUPLICATE"):
        bsm.bsm_build(A.nrows, A.ncols, 32, r, c, v)
    r[...] = bad
    c[...] = A.bcol
    r[0] = 10 ** 6                                     # out of range
    with pytest.raises(bsm.BsmError, match="OUT_OF_RANGE"):
        bsm.bsm_build(A.nrows, A.ncols, 32, r, c, v)
    r[...] = A.brow
    # values starting 8 bytes into a pinned buffer: staged
    tv = torch.empty(A.vals.size + 1, dtype=torch.float64, pin_memory=True)
    v8 = tv.numpy()[1:].reshape(A.vals.shape)
    v8[...] = A.vals
    R8 = from_bsm(bsm.bsm_build(A.nrows, A.ncols, 32, r, c, v8))
    assert_same_structure(R8, E)
    assert np.array_equal(R8.vals, E.vals)


def test_to_blocks_into_pinned_host_buffers():
    """Pinned host buffers are written directly by the gather kernels; the
    result equals the staged copy into pageable buffers."""
    import torch
    A = synth.random_blocks(3000, 32, 0.05, 8)
    M = to_bsm(A)
    n = M.nblk
    pinned = (torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
              torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
              torch.empty((n, 32, 32), dtype=torch.float64, pin_memory=True).numpy())
    r, c, v = bsm.bsm_to_blocks(M, out=pinned)
    E = A.sorted()
    assert np.array_equal(r, E.brow) and np.array_equal(c, E.bcol)
    assert np.array_equal(v, E.vals)
    # values only, into a pinned buffer; coordinates into pageable ones
    mixed = (np.empty(n, np.int32), np.empty(n, np.int32), pinned[2])
    mixed[2][...] = 0
    r2, c2, v2 = bsm.bsm_to_blocks(M, out=mixed)
    assert np.array_equal(r2, E.brow) and np.array_equal(v2, E.vals)


def test_to_blocks_asynchronous_into_pinned_buffers():
    """on_device = 2: the copy into page-locked buffers is queued on the stream
    and the call returns at once; after a synchronisation the buffers equal the
    synchronous result.  Pageable buffers are refused before any work."""
    import torch
    A = synth.random_blocks(3000, 32, 0.05, 18)
    M = to_bsm(A)
    n = M.nblk
    s = torch.cuda.Stream()
    pinned = (torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
              torch.empty(n, dtype=torch.int32, pin_memory=True).numpy(),
              torch.empty((n, 32, 32), dtype=torch.float64, pin_memory=True).numpy())
    bsm.bsm_to_blocks(M, out=pinned, stream=s, asynchronous=True)
    s.synchronize()
    E = A.sorted()
    assert np.array_equal(pinned[0], E.brow) and np.array_equal(pinned[1], E.bcol)
    assert np.array_equal(pinned[2], E.vals)
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_to_blocks(M, out=(np.empty(n, np.int32), np.empty(n, np.int32),
                                  np.empty((n, 32, 32))), asynchronous=True)
    assert e.value.name == "BSM_ERR_INVALID_ARG"


def test_to_blocks_asynchronous_in_several_chunks():
    """An asynchronous download larger than one 512 MB staging chunk (16384
    blocks of 64 x 64): two full chunks and a ragged tail, each gathered and
    copied in turn on the library's own stream.  An event recorded on the
    caller's stream right after the call completes only once every chunk has
    landed; the buffers then hold the input blocks in row-major order."""
    import torch
    import synth.device as sd
    n, bs = 25600, 64
    brow, bcol, vals = sd.random_blocks(n, bs, 0.25, 23, "cuda")
    m = brow.shape[0]
    assert m > 2 * 16384 and m % 16384 != 0
    M = bsm.bsm_build(n, n, bs, brow, bcol, vals)
    assert bsm.bsm_info(M)[3] == m
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    out = (torch.empty(m, dtype=torch.int32, pin_memory=True).numpy(),
           torch.empty(m, dtype=torch.int32, pin_memory=True).numpy(),
           torch.empty((m, bs, bs), dtype=torch.float64, pin_memory=True).numpy())
    out[2][...] = np.nan  # every block must be overwritten
    bsm.bsm_to_blocks(M, out=out, stream=s, asynchronous=True)
    ev = torch.cuda.Event()
    ev.record(s)
    ev.synchronize()
    r, c = brow.cpu().numpy(), bcol.cpu().numpy()
    order = np.lexsort((c, r))
    assert np.array_equal(out[0], r[order]) and np.array_equal(out[1], c[order])
    assert np.array_equal(out[2], vals.cpu().numpy()[order])


def test_build_drops_zero_blocks_and_rejects_bad_input():
    bs = 16
    A = synth.random_blocks(200, bs, 0.3, 6)
    vals = A.vals.copy()
    vals[0] = 0.0
    vals[1] = -0.0
    vals[2] = 0.0
    vals[2, 3, 4] = np.nan  # NaN is not zero: kept
    M = bsm.bsm_build(A.nrows, A.ncols, bs, A.brow, A.bcol, vals)
    assert bsm.bsm_info(M)[3] == A.nblk - 2
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_build(200, 200, bs, np.array([0, 0], np.int32), np.array([1, 1], np.int32),
                      np.ones((2, bs, bs)))
    assert e.value.name == "BSM_ERR_DUPLICATE"
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_build(200, 200, bs, np.array([13], np.int32), np.array([0], np.int32),
                      np.ones((1, bs, bs)))
    assert e.value.name == "BSM_ERR_OUT_OF_RANGE"


def test_level_counts_match_brute_force():
    A = synth.random_blocks(4096, 16, 0.02, 7, ncols=3000)
    M = to_bsm(A)
    counts = bsm.bsm_level_counts(M)
    L = oracle.common_depth(A)
    assert len(counts) == L + 1
    for level in range(L + 1):
        s = L - level
        nodes = set(zip((A.brow >> s).tolist(), (A.bcol >> s).tolist()))
        assert counts[level] == len(nodes)


# ---------------------------------------------------------- symbolic phase
@pytest.mark.parametrize("kind", ["random", "banded", "rect", "deep_vs_shallow"])
def test_symbolic_task_counts_match_oracle(kind):
    if kind == "random":
        A = synth.random_blocks(4096, 16, 0.03, 11); B = synth.random_blocks(4096, 16, 0.03, 12)
    elif kind == "banded":
        A = synth.banded(3000, 40, 16, 13); B = synth.banded(3000, 24, 16, 14)
    elif kind == "rect":
        A = synth.random_blocks(700, 16, 0.1, 15, ncols=1500)
        B = synth.random_blocks(1500, 16, 0.1, 16, ncols=300)
    else:  # A has far fewer levels than B
        A = synth.random_blocks(32, 16, 1.0, 17, ncols=2000)
        B = synth.random_blocks(2000, 16, 0.2, 18, ncols=4000)
    bsm.bsm_multiply(to_bsm(A), to_bsm(B))
    tasks, triples, ncs = bsm.bsm_last_stats()
    ref = oracle.task_counts(A, B)
    assert np.array_equal(tasks, ref)
    P = oracle.multiply(A, B)
    assert triples == P.triples
    # C blocks before zero removal = the block-pattern product
    pa = np.zeros((A.mb, A.nb), np.int64); pa[A.brow, A.bcol] = 1
    pb = np.zeros((B.mb, B.nb), np.int64); pb[B.brow, B.bcol] = 1
    assert ncs == int(np.count_nonzero(pa @ pb))
    assert ncs >= P.C.nblk


# ----------------------------------------------------------- FP64 parity
def check_fp64(A, B, **kw):
    C = gpu_product(A, B, **kw)
    P = oracle.multiply(A, B)
    assert_same_structure(C, P.C)
    if P.C.nblk:
        assert relerr(C.vals, P.C.vals) < TOL
    return C, P


def test_banded_4096_fp64():
    """Banded 4096, half-bandwidth 64, bs 32: 634 blocks, 3150 triples, 1132 C blocks."""
    A = synth.banded(4096, 64, 32, synth.BASE_SEED)
    B = synth.banded(4096, 64, 32, synth.BASE_SEED + 100)
    C, P = check_fp64(A, B)
    assert C.nblk == 1132 and P.triples == 3150
    _, triples, _ = bsm.bsm_last_stats()
    assert triples == 3150


@pytest.mark.parametrize("bs", [16, 32, 64])
@pytest.mark.parametrize("n,p", [(2048, 0.05), (1500, 0.2)])
def test_random_fp64(bs, n, p):
    A = synth.random_blocks(n, bs, p, 100 + bs)
    B = synth.random_blocks(n, bs, p, 200 + bs)
    check_fp64(A, B)


def test_rectangular_ragged_fp64():
    A = synth.random_blocks(1000, 32, 0.15, 31, ncols=777)
    B = synth.random_blocks(777, 32, 0.15, 32, ncols=1234)
    C, _ = check_fp64(A, B, device_inputs=True)
    assert (C.nrows, C.ncols) == (1000, 1234)


def test_decay_square_fp64():
    A = synth.decay(300, 16, 33)
    check_fp64(A, A)


def test_long_k_lists_fp64():
    """Dense-ish inner dimension: hundreds of products per C block."""
    A = synth.random_blocks(256, 32, 1.0, 34, ncols=32 * 200)
    B = synth.random_blocks(32 * 200, 32, 1.0, 35, ncols=256)
    check_fp64(A, B)


def test_identity_and_permutation_bit_exact():
    A = synth.random_blocks(1024, 32, 0.1, 41)
    I = synth.identity(1024, 32)
    for C in (gpu_product(A, I), gpu_product(I, A)):
        assert_same_structure(C, A.sorted())
        assert np.array_equal(C.vals, A.sorted().vals)
    P, perm = synth.block_permutation(32, 32, 42)
    C = gpu_product(P, A)
    inv = np.argsort(perm)
    E = synth.BlockCOO(A.nrows, A.ncols, 32, inv[A.brow].astype(np.int32), A.bcol.copy(),
                       A.vals.copy()).sorted()
    assert_same_structure(C, E)
    assert np.array_equal(C.vals, E.vals)


def test_exact_cancellation_removed():
    bs = 16
    x = synth.random_blocks(2 * bs, bs, 1.0, 61, dist="int8").to_dense()
    y = synth.random_blocks(2 * bs, bs, 1.0, 62, dist="int8").to_dense()
    z = synth.random_blocks(2 * bs, bs, 1.0, 63, dist="int8").to_dense()
    # C = [X X; Z 0] [Y; -Y] = [0; Z Y]: the top block row cancels exactly
    a = np.block([[x, x], [z, np.zeros_like(z)]])
    b = np.vstack([y, -y])
    A, B = synth.from_dense(a, bs), synth.from_dense(b, bs)
    C = gpu_product(A, B)
    P = oracle.multiply(A, B)
    assert_same_structure(C, P.C)
    assert np.array_equal(C.vals, P.C.vals)   # small integers: every partial sum exact
    _, triples, ncs = bsm.bsm_last_stats()
    assert ncs > C.nblk


def test_empty_and_single_block():
    bs = 32
    A = synth.random_blocks(256, bs, 0.2, 71)
    Z = synth.BlockCOO(256, 256, bs, np.zeros(0, np.int32), np.zeros(0, np.int32),
                       np.zeros((0, bs, bs)))
    assert gpu_product(A, Z).nblk == 0
    assert gpu_product(Z, A).nblk == 0
    one = synth.random_blocks(20, bs, 1.0, 72)   # 1x1 blocks, ragged 20x20
    C, _ = check_fp64(one, one)
    assert C.nblk == 1
    L = synth.from_dense(np.hstack([np.ones((128, 64)), np.zeros((128, 64))]), bs)
    R = synth.from_dense(np.vstack([np.zeros((64, 128)), np.ones((64, 128))]), bs)
    assert gpu_product(L, R).nblk == 0


def test_errors_from_multiply():
    A = to_bsm(synth.random_blocks(64, 32, 1.0, 81, ncols=96))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(A, A)
    assert e.value.name == "BSM_ERR_DIM_MISMATCH"
    B16 = to_bsm(synth.random_blocks(96, 16, 1.0, 82))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_multiply(A, B16)
    assert e.value.name == "BSM_ERR_BLOCKSIZE"


def test_chained_products_use_device_results():
    A = synth.random_blocks(1024, 16, 0.05, 91)
    B = synth.random_blocks(1024, 16, 0.05, 92)
    C = synth.random_blocks(1024, 16, 0.05, 93)
    g = bsm.bsm_multiply(bsm.bsm_multiply(to_bsm(A), to_bsm(B)), to_bsm(C))
    R = from_bsm(g)
    E = oracle.multiply(oracle.multiply(A, B).C, C).C
    assert_same_structure(R, E)
    assert relerr(R.vals, E.vals) < TOL


def test_to_blocks_device_and_small_buffer():
    import torch
    A = synth.random_blocks(512, 32, 0.2, 95)
    M = to_bsm(A)
    r, c, v = bsm.bsm_to_blocks(M, device=True)
    E = A.sorted()
    assert np.array_equal(r.cpu().numpy(), E.brow) and np.array_equal(v.cpu().numpy(), E.vals)
    small = (np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros((1, 32, 32)))
    with pytest.raises(bsm.BsmError) as e:
        bsm.bsm_to_blocks(M, out=small)
    assert e.value.name == "BSM_ERR_BUFFER_TOO_SMALL"
