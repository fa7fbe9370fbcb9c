"""Edge cases of the boundary on a device: empty and invalid inputs return statuses, a zero-step
call changes nothing, the smallest lattices and the smallest batches still match the oracle, and
the surrogate and network calls reject what they cannot serve."""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle

pytestmark = pytest.mark.gpu


def fresh(case, precision=tlsph.FP64):
    t = tlsph.TLSPH(case.dim, case.h, precision)
    t.set_materials(case.materials)
    return t


def test_empty_and_invalid_particle_sets():
    case = W.plate_2d(nx=6, ny=4)
    t = fresh(case)
    with pytest.raises(tlsph.TLSPHError) as e:
        t.create_particles(np.zeros((0, 2)), np.zeros(0))
    assert e.value.status == tlsph.ERR_ARG
    with pytest.raises(tlsph.TLSPHError) as e:
        t.create_particles(case.X0, case.vol, material_id=np.full(case.n, 5, np.int32))
    assert e.value.status == tlsph.ERR_ARG
    with pytest.raises(tlsph.TLSPHError) as e:
        t.create_particles(case.X0, case.vol, material_id=np.full(case.n, -1, np.int32))
    assert e.value.status == tlsph.ERR_ARG


def test_zero_steps_change_nothing():
    case = W.block_3d(nx=9, ny=8, nz=7)
    g = tlsph.from_case(case)
    g.step(7)
    U, info = g.read_state("U"), g.get_info()
    g.step(0)
    assert np.array_equal(g.read_state("U"), U) and g.get_info()["steps"] == info["steps"]


@pytest.mark.parametrize("shape", [(4, 4), (7, 3)])
def test_smallest_lattices_match_oracle(shape):
    """Lattices of a few particles, every one of them at the boundary (FP64, 200 steps)."""
    case = W.plate_2d(nx=shape[0], ny=shape[1], ramp_steps=20)
    g = tlsph.from_case(case, precision=tlsph.FP64)
    o = make_oracle(case)
    rp_g, col_g = g.neighbours()
    rp_o, col_o = o.neighbours()
    assert np.array_equal(rp_g, rp_o) and np.array_equal(col_g, col_o)
    g.step(200)
    o.step(200)
    u_g, u_o = g.read_state("U"), o.read("U")
    assert np.linalg.norm(u_g - u_o) <= 1e-5 * np.linalg.norm(u_o)


def test_batch_of_tiny_specimens_matches_oracle():
    """Specimens much smaller than a warp: every warp spans several specimens and stencil tables."""
    case = W.batched(nspec=24, n_min=24, n_max=60, seed=9)
    g = tlsph.from_case(case)
    o = make_oracle(case)
    assert g.get_info()["stencil"] > 0
    g.step(150)
    o.step(150)
    u_g, u_o = g.read_state("U"), o.read("U")
    assert np.linalg.norm(u_g - u_o) <= 1e-4 * np.linalg.norm(u_o)


def test_surrogate_rejects_what_it_cannot_serve():
    net = tlsph.MLP(batch=256)
    fp64 = tlsph.from_case(W.block_3d(nx=8, ny=8, nz=6, precision="fp64"))
    with pytest.raises(tlsph.TLSPHError) as e:
        fp64.set_surrogate(net)
    assert e.value.status == tlsph.ERR_ARG
    fp32 = tlsph.from_case(W.block_3d(nx=8, ny=8, nz=6))
    with pytest.raises(tlsph.TLSPHError) as e:
        fp32.set_surrogate(net, 7)
    assert e.value.status == tlsph.ERR_ARG
    with pytest.raises(tlsph.TLSPHError) as e:
        net.set_tensor_path(3)
    assert e.value.status == tlsph.ERR_ARG
