"""The paper's CPU restriction of the buffer decisions (Sec. 3.1): only the particles in the
cell-linked-list cells that overlap a buffer's candidate region are tested.

Test infrastructure and a timed CPU baseline (bench.py), not part of the product.  Its
decisions equal ``buffer.decide``'s over every particle (tests/test_oracle_local_cell.py):
the candidate cells are a conservative superset of the cells that can hold a particle the
plain definition would act on.

Candidate cells of buffer k (host, once): a cell is kept when its centre lies within the box
dilated by 2 cs (the outflow candidate margin cs, plus one cell of movement within the step:
the cell list is the one of the step's start, |v| dt < cs) plus the cell's own half-extent
projected on each local axis.
"""
from __future__ import annotations

import numpy as np

from .buffer import BIDIR, INFLOW, OUTFLOW, Buffer


def candidate_cells(b: Buffer, lo, cs: float, dims, dim: int) -> np.ndarray:
    """Linear indices (ascending) of the cells that can hold a candidate of buffer ``b``."""
    half = 0.5 * np.asarray(b.extent[:dim], dtype=np.float64)
    R = b.R
    reach = half + 2.0 * cs + 0.5 * cs * np.abs(R).sum(axis=1)
    # axis-aligned bounds of the dilated box, then the exact test on each cell centre
    ext = np.abs(R).T @ reach
    lo_c = np.maximum(0, np.floor((b.origin[:dim] - ext - np.asarray(lo[:dim])) / cs).astype(np.int64))
    hi_c = np.minimum(np.asarray(dims[:dim]) - 1,
                      np.floor((b.origin[:dim] + ext - np.asarray(lo[:dim])) / cs).astype(np.int64))
    axes = [np.arange(lo_c[a], hi_c[a] + 1) for a in range(dim)]
    grid = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    centre = np.asarray(lo[:dim]) + (grid + 0.5) * cs
    X = (centre - b.origin[:dim]) @ R.T
    keep = np.all(np.abs(X) <= reach[None, :], axis=1)
    g = grid[keep]
    nx, ny = dims[0], dims[1]
    lin = g[:, 0] + nx * g[:, 1]
    if dim == 3:
        lin = lin + nx * ny * g[:, 2]
    return np.sort(lin)


def candidates(cell_start: np.ndarray, cells: np.ndarray) -> np.ndarray:
    """Indices of the particles (sorted by cell) in the given cells."""
    s0, s1 = cell_start[cells], cell_start[cells + 1]
    n = s1 - s0
    if n.sum() == 0:
        return np.zeros(0, dtype=np.int64)
    rep = np.repeat(s0 - np.concatenate([[0], np.cumsum(n)[:-1]]), n)
    return np.arange(int(n.sum()), dtype=np.int64) + rep


def decide_local(buffers, pos, label, cs: float, cell_start, cand_cells):
    """Algorithms 1-3 over the candidate cells only; same results as ``buffer.decide``."""
    inj, dels = [], []
    for b, cells in zip(buffers, cand_cells):
        idx = candidates(cell_start, cells)
        Xp = b.local(pos[idx])
        lab = label[idx]
        ha = 0.5 * b.extent[0]
        if b.bc in INFLOW:
            inj += [(b.k, int(i)) for i in idx[(lab == b.label) & (Xp[:, 0] > ha)]]
        elif b.bc in OUTFLOW:
            cand = (np.abs(Xp[:, 0]) < ha + cs) & (np.abs(Xp[:, 1]) < 0.5 * b.extent[1] + cs)
            if b.dim == 3:
                cand &= np.abs(Xp[:, 2]) < 0.5 * b.extent[2] + cs
            dels += [(b.k, int(i)) for i in idx[cand & (Xp[:, 0] > ha)]]
        elif b.bc in BIDIR:
            mine = lab == b.label
            inj += [(b.k, int(i)) for i in idx[mine & (Xp[:, 0] > ha)]]
            dels += [(b.k, int(i)) for i in idx[mine & (Xp[:, 0] < -ha)]]
    inj.sort()
    dels.sort()
    return inj, dels
