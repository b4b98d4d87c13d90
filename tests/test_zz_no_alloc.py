"""The allocation-free cell-linked-list entry point agrees with the allocating one.

sphbuf_cell_list_build_noalloc serves callers that cannot allocate device memory (a program
whose GPU memory is already reserved by another allocator, or a latency-bound loop in which a
cudaMalloc/cudaFree, which can synchronise the device, is not acceptable).  Its scratch is a
fixed array inside the library, shared by every call and keeping the previous call's
contents.  Two different inputs in a row check that each call starts from cleared scratch.
The entry point is called through the C ABI (ctypes), like sphbuf_cell_list_build.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20
MAX_CELLS = (1 << 20) - 1


def _call(fn, cell, ids, label, n, ncell, start, order):
    return fn(ctypes.c_void_p(cell.data_ptr()), ctypes.c_void_p(ids.data_ptr()),
              None if label is None else ctypes.c_void_p(label.data_ptr()), n, ncell,
              ctypes.c_void_p(start.data_ptr()), ctypes.c_void_p(order.data_ptr()), None)


def test_noalloc_matches_allocating_cell_list_on_two_calls_in_a_row():
    import torch

    from paper_2406_16786_gb300 import _ffi

    lib = _ffi.load()
    for rep, (n, ncell) in enumerate([(700_001, 1_000_003), (123_457, 40_961)]):
        rng = np.random.default_rng(90 + rep)
        cell = torch.from_numpy(rng.integers(0, ncell, n).astype(np.int32)).cuda()
        ids = torch.from_numpy(rng.permutation(n).astype(np.int32) * 5 + 3).cuda()
        label = torch.from_numpy(np.where(rng.random(n) < 0.02, 255, 0).astype(np.uint8)).cuda()
        outs = []
        for fn in (lib.sphbuf_cell_list_build, lib.sphbuf_cell_list_build_noalloc):
            start = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
            order = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            assert _call(fn, cell, ids, label, n, ncell, start, order) == 0
            outs.append((start.cpu().numpy(), order.cpu().numpy()))
        (s_ref, o_ref), (s_na, o_na) = outs
        assert np.array_equal(s_na, s_ref)
        assert np.array_equal(o_na, o_ref)
        kept = int(s_ref[-1])
        assert kept == int((label.cpu().numpy() != 255).sum())


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    import torch

    from paper_2406_16786_gb300 import _ffi

    lib = _ffi.load()
    small = torch.zeros(8, dtype=torch.int32, device="cuda")
    # size checks come before any device work, so the small arrays are never read
    assert _call(lib.sphbuf_cell_list_build_noalloc, small, small, None, MAX_N + 1, 10, small, small) == 2
    assert _call(lib.sphbuf_cell_list_build_noalloc, small, small, None, 4, MAX_CELLS + 1, small, small) == 2


def test_noalloc_bad_cell_index_then_valid_call():
    """A call with a cell index outside [0, ncell) returns SPHBUF_ERR_INVALID_ARG; the error
    flag lives in the shared scratch, so the next valid call must start with it cleared and
    give the allocating entry point's result."""
    import torch

    from paper_2406_16786_gb300 import _ffi

    lib = _ffi.load()
    n, ncell = 5000, 977
    rng = np.random.default_rng(17)
    bad = rng.integers(0, ncell, n).astype(np.int32)
    bad[1234] = ncell + 3
    ids = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    start = torch.zeros(ncell + 1, dtype=torch.int32, device="cuda")
    order = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert _call(lib.sphbuf_cell_list_build_noalloc, torch.from_numpy(bad).cuda(), ids, None, n, ncell,
                 start, order) == 1
    good = torch.from_numpy(rng.integers(0, ncell, n).astype(np.int32)).cuda()
    outs = []
    for fn in (lib.sphbuf_cell_list_build, lib.sphbuf_cell_list_build_noalloc):
        s = torch.full((ncell + 1,), -7, dtype=torch.int32, device="cuda")
        o = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        assert _call(fn, good, ids, None, n, ncell, s, o) == 0
        outs.append((s.cpu().numpy(), o.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_noalloc_dense_cell_bound():
    """1024 particles in one cell are sorted; 1025 are rejected (the in-cell rank compares
    every pair of the cell, so the stand-alone entry points bound a cell's occupancy)."""
    import torch

    from paper_2406_16786_gb300 import _ffi

    lib = _ffi.load()
    for m, want in ((1024, 0), (1025, 1)):
        n, ncell = m + 10, 4
        cell = np.zeros(n, dtype=np.int32)
        cell[m:] = 3
        ids_np = np.random.default_rng(m).permutation(n).astype(np.int32)
        ids = torch.from_numpy(ids_np).cuda()
        s = torch.zeros(ncell + 1, dtype=torch.int32, device="cuda")
        o = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        assert _call(lib.sphbuf_cell_list_build_noalloc, torch.from_numpy(cell).cuda(), ids, None, n, ncell, s,
                     o) == want
        if want == 0:
            assert np.array_equal(o.cpu().numpy(), np.lexsort((ids_np, cell)))
