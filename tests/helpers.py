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
