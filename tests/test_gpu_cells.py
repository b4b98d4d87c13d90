"""Stand-alone counting-sort cell-linked list (device arrays) vs a plain sort by (cell, id)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,ncell", [(0, 7), (1, 1), (1000, 17), (300001, 4096 * 3 + 5), (2_000_000, 1_000_003)])
def test_cell_list_matches_lexsort(n, ncell):
    import torch

    from paper_2406_16786_gb300.domain import cell_list_build

    rng = np.random.default_rng(n + ncell)
    cell = rng.integers(0, ncell, n).astype(np.int32)
    ids = rng.permutation(np.arange(n, dtype=np.uint32) * 3 + 1).astype(np.uint32)
    label = np.where(rng.random(n) < 0.03, 255, 0).astype(np.uint8)
    dc = torch.from_numpy(cell).cuda()
    di = torch.from_numpy(ids.view(np.int32)).cuda()
    dl = torch.from_numpy(label).cuda()
    start = torch.zeros(ncell + 1, dtype=torch.int32, device="cuda")
    order = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
    cell_list_build(dc.data_ptr(), di.data_ptr(), dl.data_ptr(), n, ncell, start.data_ptr(), order.data_ptr())
    keep = np.nonzero(label != 255)[0]
    want = keep[np.lexsort((ids[keep], cell[keep]))]
    got = order.cpu().numpy()[: keep.size]
    assert np.array_equal(got, want)
    counts = np.bincount(cell[keep], minlength=ncell)
    assert np.array_equal(start.cpu().numpy().astype(np.int64), np.concatenate([[0], np.cumsum(counts)]))


def test_cell_index_out_of_range_is_rejected():
    import torch

    from paper_2406_16786_gb300.domain import SphbufError, cell_list_build

    cell = torch.tensor([0, 5, 99, 2], dtype=torch.int32, device="cuda")
    ids = torch.arange(4, dtype=torch.int32, device="cuda")
    start = torch.zeros(11, dtype=torch.int32, device="cuda")
    order = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(SphbufError) as e:
        cell_list_build(cell.data_ptr(), ids.data_ptr(), None, 4, 10, start.data_ptr(), order.data_ptr())
    assert e.value.status == 1
