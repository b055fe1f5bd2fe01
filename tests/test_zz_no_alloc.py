"""hcao_cell_sort_noalloc: the stable cell sort for callers that cannot
allocate device memory (their own pool owns the device, or a cudaMalloc's
possible device-wide synchronisation is not acceptable to them).  Its scratch
is a fixed device array in the library; it must give the same permutation and
cell offsets as hcao_cell_sort, call after call, and refuse inputs larger than
that array.
"""
import numpy as np
import pytest

from paper_2606_31548_b300 import hcao

pytestmark = pytest.mark.gpu


def _sort_both(ctx, keys, n_cells):
    import torch
    n = keys.shape[0]
    dk = torch.from_numpy(keys.view(np.int32)).cuda()
    out = []
    for use_noalloc in (False, True):
        perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
        off = torch.full((n_cells + 1,), -1, dtype=torch.int32, device="cuda")
        if use_noalloc:
            hcao.cell_sort_noalloc(dk, n, n_cells, perm, off, torch.cuda.current_stream().cuda_stream)
        else:
            ctx.cell_sort(dk, n, n_cells, perm, off)
            ctx.sync()
        torch.cuda.synchronize()
        out.append((perm.cpu().numpy()[:n].view(np.uint32), off.cpu().numpy().view(np.uint32)))
    return out


def test_noalloc_sort_matches_the_allocating_sort_twice():
    ctx = hcao.Context()
    rng = np.random.default_rng(2024)
    # two calls in a row with different inputs: the shared scratch keeps the
    # first call's contents, which must not leak into the second result
    for n, n_cells in ((300_001, 5000), (hcao.NOALLOC_SORT_MAX_KEYS, 70_000)):
        keys = rng.integers(0, n_cells, size=n).astype(np.uint32)
        (p_ref, o_ref), (p_na, o_na) = _sort_both(ctx, keys, n_cells)
        assert np.array_equal(p_na, p_ref)
        assert np.array_equal(o_na, o_ref)
        assert np.array_equal(p_ref, np.argsort(keys, kind="stable").astype(np.uint32))


def test_noalloc_sort_rejects_more_keys_than_its_scratch():
    import torch
    n = hcao.NOALLOC_SORT_MAX_KEYS + 1
    dk = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.zeros(n, dtype=torch.int32, device="cuda")
    off = torch.zeros(2, dtype=torch.int32, device="cuda")
    with pytest.raises(hcao.HcaoError) as e:
        hcao.cell_sort_noalloc(dk, n, 1, perm, off)
    assert e.value.code == -1  # HCAO_EINVAL
