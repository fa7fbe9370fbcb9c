"""St. Venant-Kirchhoff with the spectral strain split (Sec. 2.3.1) on the sm_103a path against the
FP64 oracle, through the C-ABI.

Tolerances: stress of a static random strain field element by element (FP64 1e-10, FP32 1e-5 of the
largest entry); dynamic runs as for the neo-Hookean cases, relative L2 displacement <= 1e-5 (FP64) /
1e-4 (FP32) and damage within 1e-3.
"""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def svk_block(nx=12, ny=10, nz=8, precision="fp64"):
    """3D jittered block of a brittle SVK solid whose top face is pressed at 1 m/s after a ramp (lateral
    expansion gives strains of both signs); damage grows through the whole block within 200 steps."""
    case = W.block_3d(nx=nx, ny=ny, nz=nz, jitter=0.05, seed=5, precision=precision, v_press=1.0)
    case.materials = [W.Material(model=W.MODEL_SVK, rho=2450.0, E=32e9, nu=0.2, beta1=0.2, fracture=1, Gc=30.0,
                                 eps0=2.0 * case.dp, s_lim=0.1)]
    case.bcs[1].ramp = 300 * 0.3 * case.h / W.REF_WAVE_SPEED
    return case


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-10), (tlsph.FP32_U64, 1e-5)])
def test_static_random_strain_stress(dim, precision, tol):
    """Random displacement and phase fields: P of every particle, element by element."""
    case = svk_block() if dim == 3 else W.notched_plate(nx=60, ny=24, model="svk")
    rng = np.random.default_rng(21 + dim)
    u = rng.normal(scale=1.5e-3 * case.dp, size=case.X0.shape)
    s = rng.uniform(0.0, 1.0, size=case.n)
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    for obj in (o, g):
        (obj.write if obj is o else obj.write_state)("U", u)
        (obj.write if obj is o else obj.write_state)("S", s)
    Po, Pg = o.read("P"), g.read_state("P")
    assert (s <= case.materials[0].s_lim).any() and (s > 0.9).any()
    assert np.abs(Pg - Po).max() <= tol * np.abs(Po).max()


@pytest.mark.parametrize("precision", [tlsph.FP64, tlsph.FP32_U64])
def test_notched_svk_plate(precision):
    """SVK notched plate (125 x 50), 600 steps: u <= 1e-4 (1e-5 FP64), damage within 1e-3, H close."""
    case = W.notched_plate(nx=125, ny=50, model="svk")
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    o.step(600)
    g.step(600)
    tol = 1e-5 if precision == tlsph.FP64 else 1e-4
    assert rel_l2(g.read_state("U"), o.read("U")) <= tol
    s_o, s_g = o.read("S"), g.read_state("S")
    assert s_o.min() < 0.999  # damage develops at the notch tip
    assert np.abs(s_g - s_o).max() <= 1e-3
    assert rel_l2(g.read_state("H"), o.read("H")) <= 1e-3


@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-8), (tlsph.FP32_U64, 1e-4)])
def test_svk_block_3d(precision, tol):
    """3D SVK block, 150 steps (partial damage everywhere): displacement, stress, history and damage."""
    case = svk_block()
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    o.step(150)
    g.step(150)
    s_o = o.read("S")
    assert 0.5 < s_o.min() < 0.95
    assert np.abs(g.read_state("S") - s_o).max() <= max(10 * tol, 1e-6)
    assert rel_l2(g.read_state("U"), o.read("U")) <= tol
    assert rel_l2(g.read_state("P"), o.read("P")) <= 10 * tol
    H_o = o.read("H")
    assert H_o.max() > 0.0
    assert rel_l2(g.read_state("H"), H_o) <= 10 * tol
    info = g.get_info()
    assert info["nonfinite"] == 0


def test_svk_modes_bit_identical():
    """Launch-per-kernel, graph and persistent modes give bit-identical SVK runs."""
    case = W.notched_plate(nx=60, ny=24, model="svk")
    out = []
    for mode in (tlsph.MODE_LAUNCH, tlsph.MODE_GRAPH, tlsph.MODE_PERSISTENT):
        g = tlsph.from_case(case)
        g.set_option(tlsph.OPT_MODE, mode)
        g.step(200)
        out.append((g.read_state("U"), g.read_state("S")))
    for u, s in out[1:]:
        assert np.array_equal(u, out[0][0]) and np.array_equal(s, out[0][1])
