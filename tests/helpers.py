"""Shared helpers for the GPU parity tests (marshalling and comparison only)."""
import numpy as np

import paper_1501_07800_gb300 as bsm
import synth


def to_bsm(m: synth.BlockCOO, device: bool = False) -> bsm.Matrix:
    if device:
        import torch
        return bsm.bsm_build(m.nrows, m.ncols, m.bs, torch.from_numpy(m.brow).cuda(),
                             torch.from_numpy(m.bcol).cuda(), torch.from_numpy(m.vals).cuda())
    return bsm.bsm_build(m.nrows, m.ncols, m.bs, m.brow, m.bcol, m.vals)


def from_bsm(M: bsm.Matrix) -> synth.BlockCOO:
    nr, nc, bs, n = bsm.bsm_info(M)
    r, c, v = bsm.bsm_to_blocks(M)
    return synth.BlockCOO(nr, nc, bs, r, c, v)


def relerr(x, y) -> float:
    n = np.linalg.norm(y)
    return float(np.linalg.norm(np.asarray(x) - np.asarray(y)) / (n if n > 0 else 1.0))


def assert_same_structure(C: synth.BlockCOO, E: synth.BlockCOO):
    assert (C.nrows, C.ncols, C.bs) == (E.nrows, E.ncols, E.bs)
    assert C.nblk == E.nblk, (C.nblk, E.nblk)
    assert np.array_equal(C.brow, E.brow) and np.array_equal(C.bcol, E.bcol)


def pattern_product(ar, ac, br, bc, mb, kb, nb):
    """(I, J) of C's structure by definition, row-major: some K has A_IK and
    B_KJ stored (SciPy sparse product of the block patterns, on the host)."""
    import scipy.sparse as sp

    def host(x):
        return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    PA = sp.csr_matrix((np.ones(len(ar), np.int32), (host(ar), host(ac))), shape=(mb, kb))
    PB = sp.csr_matrix((np.ones(len(br), np.int32), (host(br), host(bc))), shape=(kb, nb))
    C = (PA @ PB).tocsr()
    C.sort_indices()
    rows = np.repeat(np.arange(mb, dtype=np.int64), np.diff(C.indptr))
    return rows, C.indices.astype(np.int64)
