"""Neighbour layouts: the stencil layout (lattice inputs; one table per specimen in a batch) and
the SELL-32 rows visit the same pairs in the same order, so whole steps agree bit for bit; inputs
whose pair differences take more than 128 values keep the SELL-32 rows."""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W

pytestmark = pytest.mark.gpu

CASES = {
    "plate_fp64": lambda: W.plate_2d(),
    "plate_odd_rows_fp32": lambda: W.plate_2d(nx=100, ny=21, precision="fp32"),
    "block_j2_odd_planes": lambda: W.block_3d(nx=40, ny=9, nz=7),
    "crack_branching": lambda: W.crack_branching(nx=120, ny=48),
    "block_j2": lambda: W.block_3d(nx=24, ny=20, nz=16),
    "notched_pf": lambda: W.notched_plate(nx=100, ny=40),
    "block_j2_fp64": lambda: W.block_3d(nx=16, ny=14, nz=12, precision="fp64"),
}


@pytest.mark.parametrize("which", sorted(CASES))
@pytest.mark.parametrize("mode", [tlsph.MODE_LAUNCH, tlsph.MODE_PERSISTENT])
def test_stencil_layout_is_bit_identical_to_csr(which, mode):
    case = CASES[which]()
    sten = tlsph.from_case(case)
    csr = tlsph.from_case(case)
    csr.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, tlsph.LAYOUT_CSR)
    nst = sten.get_info()["stencil"]
    assert 0 < nst <= 128
    assert csr.get_info()["stencil"] == 0
    for g in (sten, csr):
        g.set_option(tlsph.OPT_MODE, mode)
        g.step(150)
    for f in ("U", "V", "S", "P", "F"):
        a, b = sten.read_state(f), csr.read_state(f)
        assert np.array_equal(a, b), f
    assert sten.time() == csr.time()


def test_stencil_size_of_the_lattices():
    # lattice offsets strictly inside the support R = 3 dp: 92 in 3D, 24 in 2D; those at exactly
    # 3 dp (30 in 3D, 4 in 2D) join when jitter or rounding brings some pair inside
    n3 = tlsph.from_case(W.block_3d(nx=24, ny=20, nz=16)).get_info()["stencil"]
    n2 = tlsph.from_case(W.plate_2d()).get_info()["stencil"]
    assert 92 <= n3 <= 122 and 24 <= n2 <= 28, (n3, n2)


@pytest.mark.parametrize("nspec", [6, 40])
def test_batched_specimens_bit_identical(nspec):
    # each specimen is a lattice with its own row pitch: one stencil table per specimen (2D: the
    # 24 offsets inside the support, plus the 4 at its edge when rounding brings them in)
    case = W.batched(nspec=nspec, n_min=200, n_max=1500, seed=3)
    auto = tlsph.from_case(case)
    assert 24 <= auto.get_info()["stencil"] <= 28
    csr = tlsph.from_case(case)
    csr.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, tlsph.LAYOUT_CSR)
    auto.step(100)
    csr.step(100)
    assert np.array_equal(auto.read_state("U"), csr.read_state("U"))


def test_irregular_particles_keep_sell_rows():
    # jitter of 0.45 dp: cells hold 0, 1 or 2 particles and the pair differences spread out
    case = W.block_3d(nx=16, ny=16, nz=16, jitter=0.45)
    g = tlsph.from_case(case)
    assert g.get_info()["stencil"] == 0
    g.step(10)
    assert np.all(np.isfinite(g.read_state("U")))
