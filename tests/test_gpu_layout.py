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


def pf_block(nx=16, ny=12, nz=10):
    """3D jittered block of a brittle SVK solid with the phase field, pressed at 1 m/s after a ramp."""
    case = W.block_3d(nx=nx, ny=ny, nz=nz, jitter=0.01, seed=5, v_press=1.0)
    case.materials = [W.Material(model=W.MODEL_SVK, rho=2450.0, E=32e9, nu=0.2, beta1=0.2, fracture=1, Gc=30.0,
                                 eps0=2.0 * case.dp, s_lim=0.1)]
    case.bcs[1].ramp = 300 * 0.3 * case.h / W.REF_WAVE_SPEED
    return case


# (case, nx, ny)
LATTICE_CASES = {
    "block_j2": (lambda: W.block_3d(nx=24, ny=20, nz=16), 24, 20),
    # odd y and z counts: the two rows of a thread straddle a z plane, and the last thread has one row
    "block_j2_odd_planes": (lambda: W.block_3d(nx=40, ny=9, nz=7), 40, 9),
    # without jitter no pair lies at exactly 3 dp: the table holds 92 of the ball's 122 entries
    "block_j2_no_jitter": (lambda: W.block_3d(nx=20, ny=18, nz=10, jitter=0.0), 20, 18),
    "svk_phase_field_block": (pf_block, 16, 12),
}


@pytest.mark.parametrize("which", sorted(LATTICE_CASES))
@pytest.mark.parametrize("rows", [(1, 2), (2, 1), (1, 1), (2, 2), (1, 4), (2, 4)])
@pytest.mark.parametrize("fuse", [1, 0])
def test_lattice_layout_is_bit_identical_to_stencil_and_csr(which, rows, fuse):
    # the lattice kernels walk the ball at compile time, rows per thread 1 or 2, with the stress in the
    # gradient kernel or in its own pass: same pairs, same order, same arithmetic as the table walks
    make, nx, ny = LATTICE_CASES[which]
    case = make()
    lat, sten, csr = tlsph.from_case(case), tlsph.from_case(case), tlsph.from_case(case)
    sten.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, tlsph.LAYOUT_STENCIL)
    csr.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, tlsph.LAYOUT_CSR)
    lat.set_option(tlsph.OPT_LATTICE_ROWS_GRADIENT, rows[0])
    lat.set_option(tlsph.OPT_LATTICE_ROWS_FORCE, rows[1])
    lat.set_option(tlsph.OPT_FUSE_STRESS, fuse)
    info = lat.get_info()
    assert info["lattice_nx"] == nx and info["lattice_nxny"] == nx * ny, info
    assert sten.get_info()["lattice_nx"] == 0 and sten.get_info()["stencil"] > 0
    assert csr.get_info()["lattice_nx"] == 0 and csr.get_info()["stencil"] == 0
    for g in (lat, sten, csr):
        g.step(120)
    for f in ("U", "V", "S", "P", "F", "EPSP"):
        a, b, c = lat.read_state(f), sten.read_state(f), csr.read_state(f)
        assert np.array_equal(a, b), f
        assert np.array_equal(a, c), f
    assert lat.time() == sten.time() == csr.time()
    assert lat.get_info()["kernel_launches"] < sten.get_info()["kernel_launches"] or not fuse


@pytest.mark.parametrize("which", sorted(LATTICE_CASES))
@pytest.mark.parametrize("patch", [32, 64, 128])
@pytest.mark.parametrize("rows", [(1, 2), (2, 4), (1, 1)])
def test_lattice_patches_are_bit_identical_to_whole_lines(which, patch, rows):
    # blocks that take patches of x (none of these lattices has an x line a multiple of 32 long but the
    # 128-wide patch of the 24 and 40 wide ones: the last patch of each band has idle threads) give the
    # same step as blocks that take whole lines
    make, _, _ = LATTICE_CASES[which]
    case = make()
    ref, pat = tlsph.from_case(case), tlsph.from_case(case)
    for g in (ref, pat):
        g.set_option(tlsph.OPT_LATTICE_ROWS_GRADIENT, rows[0])
        g.set_option(tlsph.OPT_LATTICE_ROWS_FORCE, rows[1])
    pat.set_option(tlsph.OPT_LATTICE_PATCH, patch)
    assert pat.get_info()["lattice_nx"] > 0
    for g in (ref, pat):
        g.step(60)
    for f in ("U", "V", "S", "P", "F", "EPSP"):
        assert np.array_equal(ref.read_state(f), pat.read_state(f)), f
    assert ref.time() == pat.time()
    with pytest.raises(tlsph.TLSPHError):
        pat.set_option(tlsph.OPT_LATTICE_PATCH, 48)


@pytest.mark.parametrize("which", sorted(LATTICE_CASES))
@pytest.mark.parametrize("zc", [1, 3, 5, 64])
def test_force_pass_streaming_along_z_is_bit_identical(which, zc):
    # columns of zc planes per thread (one plane; chunks that do not divide the plane count; one chunk
    # for the whole lattice): each row still adds its entries in ascending difference
    make, _, _ = LATTICE_CASES[which]
    case = make()
    ref, zs = tlsph.from_case(case), tlsph.from_case(case)
    zs.set_option(tlsph.OPT_LATTICE_ZSTREAM, zc)
    for g in (ref, zs):
        g.step(60)
    for f in ("U", "V", "S", "P", "F", "EPSP"):
        assert np.array_equal(ref.read_state(f), zs.read_state(f)), f
    assert ref.time() == zs.time()
    # the energy sums meet in FP64 atomics across blocks, whose order varies from run to run
    e_ref, e_zs = ref.energies(), zs.energies()
    assert all(np.isclose(e_ref[k], e_zs[k], rtol=1e-12, atol=0) for k in e_ref), (e_ref, e_zs)
    with pytest.raises(tlsph.TLSPHError):
        zs.set_option(tlsph.OPT_LATTICE_ZSTREAM, -1)


def test_force_pass_streaming_along_z_in_graphs_and_with_kernel_timing():
    case = W.block_3d(nx=24, ny=20, nz=16)
    ref, zs = tlsph.from_case(case), tlsph.from_case(case)
    zs.set_option(tlsph.OPT_LATTICE_ZSTREAM, 4)
    zs.set_option(tlsph.OPT_MODE, tlsph.MODE_GRAPH)
    ref.step(30)
    zs.step(30)
    zs.set_option(tlsph.OPT_KERNEL_TIMING, 1)
    ref.step(10)
    zs.step(10)
    assert zs.kernel_times()["pass2_launches"] > 0
    assert np.array_equal(ref.read_state("U"), zs.read_state("U"))


def test_lattice_layout_only_where_it_applies():
    # FP64, 2D, several specimens and a jitter that reaches the next lattice shell keep the table walks
    assert tlsph.from_case(W.block_3d(nx=16, ny=14, nz=12, precision="fp64")).get_info()["lattice_nx"] == 0
    assert tlsph.from_case(W.plate_2d(nx=100, ny=21, precision="fp32")).get_info()["lattice_nx"] == 0
    wide = tlsph.from_case(W.block_3d(nx=16, ny=16, nz=12, jitter=0.08))
    assert wide.get_info()["stencil"] > 122 or wide.get_info()["stencil"] == 0
    assert wide.get_info()["lattice_nx"] == 0
