"""Algorithm 2 (leapfrog time integration) on the device against the FP64 oracle, and its
bookkeeping: exact free fall, parity on the plate, the J2 block and the notched phase-field plate,
bit-identical launch and graph modes and neighbour layouts, checkpoints that carry the half-step
acceleration, and the refusal of the persistent mode."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def leap(case):
    case.integrator = tlsph.INTEGRATOR_LEAPFROG
    return case


def test_free_fall_is_exact():
    case = leap(W.plate_2d(nx=6, ny=5, beta1=0.0))
    case.bcs = []
    case.dt_mode, case.fixed_dt = O.DT_FIXED, 1e-4
    case.gravity = (0.0, -9.81, 0.0)
    g = tlsph.from_case(case, precision=tlsph.FP64)
    g.step(250)
    t = 250 * 1e-4
    assert np.allclose(g.read_state("U")[:, 1], -9.81 * 0.5 * t * t, rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-5), (tlsph.FP32_U64, 1e-4)])
def test_plate_1000_steps(precision, tol):
    case = leap(W.plate_2d())
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    o.step(1000)
    g.step(1000)
    assert rel_l2(g.read_state("U"), o.read("U")) <= tol
    assert rel_l2(g.read_state("V"), o.read("V")) <= tol
    assert rel_l2(g.read_state("ACC"), o.read("ACC")) <= 10 * tol
    to, _ = o.time()
    tg, _ = g.time()
    assert abs(tg - to) <= 1e-12 * to


@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-8), (tlsph.FP32_U64, 1e-4)])
def test_j2_block_1000_steps(precision, tol):
    case = leap(W.block_3d(nx=16, ny=16, nz=8))
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    o.step(1000)
    g.step(1000)
    assert rel_l2(g.read_state("U"), o.read("U")) <= tol
    ep_o, ep_g = o.read("EPSP"), g.read_state("EPSP")
    assert ep_o.max() > 1e-3
    assert np.abs(ep_g - ep_o).max() <= 10 * tol * ep_o.max() + 1e-7


@pytest.mark.parametrize("precision", [tlsph.FP64, tlsph.FP32_U64])
def test_notched_plate_phase_field(precision):
    case = leap(W.notched_plate(nx=125, ny=50))
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    o.step(600)
    g.step(600)
    tol = 1e-5 if precision == tlsph.FP64 else 1e-4
    assert rel_l2(g.read_state("U"), o.read("U")) <= tol
    s_o, s_g = o.read("S"), g.read_state("S")
    assert s_o.min() < 0.999
    assert np.abs(s_g - s_o).max() <= 1e-3


def test_modes_and_layouts_bit_identical():
    case = leap(W.block_3d(nx=14, ny=12, nz=9))
    ref = None
    for mode, layout in [(tlsph.MODE_LAUNCH, tlsph.LAYOUT_AUTO), (tlsph.MODE_GRAPH, tlsph.LAYOUT_AUTO),
                         (tlsph.MODE_LAUNCH, tlsph.LAYOUT_CSR)]:
        g = tlsph.from_case(case)
        g.set_option(tlsph.OPT_MODE, mode)
        g.set_option(tlsph.OPT_NEIGHBOUR_LAYOUT, layout)
        g.step(51)
        g.step(24)
        out = (g.read_state("U"), g.read_state("V"), g.time())
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]) and out[2] == ref[2]
    g = tlsph.from_case(case)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_PERSISTENT)
    with pytest.raises(tlsph.TLSPHError) as e:
        g.step(1)
    assert e.value.status == tlsph.ERR_ARG


def test_checkpoint_carries_the_half_step_acceleration():
    case = leap(W.notched_plate(nx=60, ny=24))
    a = tlsph.from_case(case)
    a.step(100)
    blob = a.read_state("STATE").copy()
    a.step(100)
    b = tlsph.from_case(case)
    b.write_state("STATE", blob)
    b.step(100)
    assert np.array_equal(b.read_state("U"), a.read_state("U"))
    assert np.array_equal(b.read_state("S"), a.read_state("S"))
