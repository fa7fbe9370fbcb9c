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


def _two_clusters(gap):
    """Two 6 x 5 x 4 jittered blocks, the second shifted by gap metres along each axis."""
    a = W.block_3d(nx=6, ny=5, nz=4, jitter=0.01, seed=11)
    b = W.block_3d(nx=6, ny=5, nz=4, jitter=0.01, seed=12)
    X = np.concatenate([a.X0, b.X0 + gap])
    return X, a.h


def test_noalloc_refuses_what_the_reference_setup_refuses():
    """A grid whose cell keys would pass 9e18 (clusters 100 km apart with 1 mm cells) and a NaN coordinate
    are refused by the context's setup; the allocation-free sort then writes -1 into every perm entry on
    both of two calls in a row, instead of an order computed from overflowed keys.  Clusters 1 km apart
    (keys about 1e18) are accepted by both and sort to the same order."""
    import torch

    dev = torch.device("cuda", 0)
    for gap, accepted in ((1e3, True), (1e5, False)):
        X, h = _two_clusters(gap)
        ctx = tlsph.TLSPH(3, h)
        ctx.set_materials([W.Material(model=W.MODEL_NH, rho=7850.0, E=200e9, nu=0.3)])
        ctx.create_particles(X, np.full(len(X), 1e-9))
        st = ctx.lib.tlsph_build_ref_neighbours(ctx.ctx)
        assert (st == tlsph.OK) == accepted, (gap, st)
        ref = ctx.permutation() if accepted else None
        ctx.close()
        X0 = torch.from_numpy(X).to(dev)
        for _ in range(2):
            perm = torch.zeros(len(X), dtype=torch.int32, device=dev)
            assert tlsph.cell_sort_noalloc(X0, perm, h, 2.0) == tlsph.OK
            torch.cuda.synchronize()
            got = perm.cpu().numpy().astype(np.int64)
            if accepted:
                assert np.array_equal(got, ref)
            else:
                assert np.all(got == -1)
    X, h = _two_clusters(0.1)
    X[7, 1] = np.nan
    X0 = torch.from_numpy(X).to(dev)
    perm = torch.zeros(len(X), dtype=torch.int32, device=dev)
    assert tlsph.cell_sort_noalloc(X0, perm, h, 2.0) == tlsph.OK
    torch.cuda.synchronize()
    assert np.all(perm.cpu().numpy() == -1)
    # a negative specimen id is refused the same way
    X, h = _two_clusters(0.1)
    X0 = torch.from_numpy(X).to(dev)
    spec = torch.zeros(len(X), dtype=torch.int32, device=dev)
    spec[3] = -2
    perm = torch.zeros(len(X), dtype=torch.int32, device=dev)
    assert tlsph.cell_sort_noalloc(X0, perm, h, 2.0, spec) == tlsph.OK
    torch.cuda.synchronize()
    assert np.all(perm.cpu().numpy() == -1)
