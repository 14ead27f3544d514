"""The torch generator reproduces the numpy generator bit for bit (CPU)."""
import numpy as np
import torch

import synth
from synth import device as sd


def test_hash_and_uniform_match_numpy():
    a = np.arange(1000, dtype=np.uint64) * np.uint64(7919)
    b = np.arange(1000, dtype=np.uint64)[::-1].copy()
    h_np = synth.hash3(synth.BASE_SEED, a, b)
    h_t = sd.hash3(synth.BASE_SEED, torch.from_numpy(a.astype(np.int64)),
                   torch.from_numpy(b.astype(np.int64)))
    assert np.array_equal(h_np.view(np.int64), h_t.numpy())
    assert np.array_equal(synth.uniform01(h_np), sd.uniform01(h_t).numpy())


def test_random_blocks_match_numpy():
    for n, bs, p, seed in [(700, 32, 0.1, 5), (333, 16, 0.3, 9)]:
        ref = synth.random_blocks(n, bs, p, seed, dist="uniform")
        r, c, v = sd.random_blocks(n, bs, p, seed, "cpu")
        assert np.array_equal(r.numpy(), ref.brow) and np.array_equal(c.numpy(), ref.bcol)
        assert np.array_equal(v.numpy(), ref.vals)


def test_decay_matches_numpy_structure_and_values():
    ref = synth.decay(120, 16, 7)
    n, r, c, v = sd.decay(120, 16, 7, "cpu")
    nz = (v != 0).flatten(1).any(1)
    r, c, v = r[nz].numpy(), c[nz].numpy(), v[nz].numpy()
    o = np.lexsort((c, r))
    E = ref.sorted()
    assert n == ref.nrows
    assert np.array_equal(r[o], E.brow) and np.array_equal(c[o], E.bcol)
    assert np.allclose(v[o], E.vals, rtol=1e-15, atol=0)


def test_decay_cross_is_the_filtered_matrix():
    """cross=(lo, hi) keeps exactly the blocks with a row or a column in
    [lo, hi): the operands of the C blocks [lo, hi)^2 of A*A."""
    n, r, c, v = sd.decay(400, 32, 5, "cpu")
    n2, r2, c2, v2 = sd.decay(400, 32, 5, "cpu", cross=(10, 20), chunk_blocks=97)
    keep = ((r >= 10) & (r < 20)) | ((c >= 10) & (c < 20))
    assert n2 == n and 0 < int(keep.sum()) < len(r)
    assert torch.equal(r[keep], r2) and torch.equal(c[keep], c2) and torch.equal(v[keep], v2)
