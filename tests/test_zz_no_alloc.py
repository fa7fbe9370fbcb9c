"""The allocation-free cell sort against the context's reference setup, through the C-ABI.

tlsph_cell_sort_noalloc serves callers that cannot call cudaMalloc: it keeps its scratch
in a fixed device array inside the library.  Its permutation must equal the one
tlsph_build_ref_neighbours computes (an integer result: compared exactly), on two calls
in a row, since every call reuses the same scratch.  This file runs last so that a
failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W

pytestmark = pytest.mark.gpu


def _cases():
    block = W.block_3d(nx=20, ny=18, nz=12, jitter=0.01, seed=7)
    ragged = W.block_3d(nx=37, ny=11, nz=9, jitter=0.3, seed=5)
    plate = W.notched_plate(nx=125, ny=50)
    batch = W.batched(nspec=12, n_min=200, n_max=3000, seed=3)
    return [block, ragged, plate, batch]


@pytest.mark.parametrize("k", range(4))
def test_noalloc_sort_equals_reference_setup(k):
    import torch

    case = _cases()[k]
    assert case.n <= tlsph.NOALLOC_MAX_PARTICLES
    ref = tlsph.from_case(case).permutation()
    dev = torch.device("cuda", 0)
    X0 = torch.from_numpy(np.ascontiguousarray(case.X0)).to(dev)
    spec = None if case.specimen_id is None else torch.from_numpy(case.specimen_id.astype(np.int32)).to(dev)
    for _ in range(2):  # two calls in a row share the scratch
        perm = torch.full((case.n,), -1, dtype=torch.int32, device=dev)
        st = tlsph.cell_sort_noalloc(X0, perm, case.h, 2.0, spec)
        torch.cuda.synchronize()
        assert st == tlsph.OK
        assert np.array_equal(perm.cpu().numpy().astype(np.int64), ref)


def test_noalloc_rejects_oversize_and_bad_arguments():
    import torch

    dev = torch.device("cuda", 0)
    n = tlsph.NOALLOC_MAX_PARTICLES + 1
    X0 = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    perm = torch.zeros(n, dtype=torch.int32, device=dev)
    assert tlsph.cell_sort_noalloc(X0, perm, 1e-3) == tlsph.ERR_ARG
    assert tlsph.cell_sort_noalloc(X0[:10], perm[:10], -1.0) == tlsph.ERR_ARG
