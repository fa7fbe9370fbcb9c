"""Parity of the sm_103a CUDA path with the FP64 CPU oracle, through the C-ABI.

Tolerances: neighbour lists and the cell-sorted permutation bit-exact; relative L2
displacement after 1000 steps <= 1e-5 on the FP64 path and <= 1e-4 on the FP32
path; damage <= 1e-3 (max abs).  Inputs are the seeded lattices of
paper_2602_15149_b300.workloads at sizes the oracle finishes in seconds; the
full-size block is checked on properties that hold at any size.
"""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu(case, precision=None, **kw):
    return tlsph.from_case(case, precision=precision, **kw)


# ---------------------------------------------------------------- reference setup
@pytest.mark.parametrize("which", ["plate", "block", "notched", "block_ragged"])
def test_neighbours_and_permutation_bit_exact(which):
    case = {"plate": lambda: W.plate_2d(),
            "block": lambda: W.block_3d(nx=20, ny=18, nz=12, jitter=0.01, seed=7),
            "notched": lambda: W.notched_plate(nx=125, ny=50),
            "block_ragged": lambda: W.block_3d(nx=13, ny=7, nz=5, jitter=0.2, seed=3)}[which]()
    o = make_oracle(case)
    g = gpu(case)
    rp_o, col_o = o.neighbours()
    rp_g, col_g = g.neighbours()
    assert np.array_equal(rp_o, rp_g)
    assert np.array_equal(col_o, col_g)
    assert np.array_equal(o.perm(), g.permutation())


def test_patch_test_on_gpu():
    rng = np.random.default_rng(0)
    for prec, tol in [(tlsph.FP64, 1e-12), (tlsph.FP32_U64, 2e-6)]:
        case = W.block_3d(nx=9, ny=8, nz=7, jitter=0.05, seed=4)
        g = gpu(case, precision=prec)
        A = rng.normal(scale=1e-3, size=(3, 3))
        g.write_state("U", case.X0 @ A.T)
        F = g.read_state("F")
        assert np.abs(F - (np.eye(3) + A)).max() < tol


# ---------------------------------------------------------------- full runs vs the oracle
def compare_run(case, steps, precision, chunks=1):
    o = make_oracle(case)
    g = gpu(case, precision=precision)
    per = steps // chunks
    for _ in range(chunks):
        o.step(per)
        g.step(per)
    out = {}
    for f in ["U", "V"]:
        out[f] = rel_l2(g.read_state(f), o.read(f))
    return o, g, out


def test_plate_fp64_1000_steps():
    """2D Neo-Hookean plate, 100 x 20, FP64: rel-L2(u) <= 1e-5 after 1000 steps."""
    case = W.plate_2d()
    o, g, err = compare_run(case, 1000, tlsph.FP64)
    assert err["U"] <= 1e-5, err
    assert err["V"] <= 1e-5, err
    to, dto = o.time()
    tg, dtg = g.time()
    assert abs(tg - to) <= 1e-12 * to and dtg == dto


def test_plate_fp32_1000_steps():
    case = W.plate_2d(precision="fp32")
    o, g, err = compare_run(case, 1000, tlsph.FP32_U64)
    assert err["U"] <= 1e-4, err


@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-8), (tlsph.FP32_U64, 1e-4)])
def test_j2_block_1000_steps(precision, tol):
    """3D J2 block (16 x 16 x 8, jittered), pressed at 5 m/s: u within tol, plastic strain close."""
    case = W.block_3d(nx=16, ny=16, nz=8)
    o, g, err = compare_run(case, 1000, precision)
    assert err["U"] <= tol, err
    ep_o, ep_g = o.read("EPSP"), g.read_state("EPSP")
    assert ep_o.max() > 1e-3  # the block yields
    assert np.abs(ep_g - ep_o).max() <= 10 * tol * max(ep_o.max(), 1e-30) + 1e-7
    info = g.get_info()
    assert info["noconverge"] == 0 and info["nonfinite"] == 0


@pytest.mark.parametrize("precision", [tlsph.FP64, tlsph.FP32_U64])
def test_notched_plate_phase_field(precision):
    """Phase-field plate with edge notch (125 x 50), 600 steps (damage initiated at the tip):
    u <= 1e-4 (1e-5 FP64) and s within 1e-3."""
    case = W.notched_plate(nx=125, ny=50)
    o, g, err = compare_run(case, 600, precision)
    tol = 1e-5 if precision == tlsph.FP64 else 1e-4
    assert err["U"] <= tol, err
    s_o, s_g = o.read("S"), g.read_state("S")
    assert s_o.min() < 0.999  # damage develops
    assert np.abs(s_g - s_o).max() <= 1e-3
    H_o, H_g = o.read("H"), g.read_state("H")
    assert rel_l2(H_g, H_o) <= 1e-3
    # fracture energy (the regularised crack functional) and the work of the tractions
    eo, eg = o.energies(), g.energies()
    etol = 1e-6 if precision == tlsph.FP64 else 2e-3
    for k in ("FE", "Wext", "KE", "SE"):
        assert abs(eg[k] - eo[k]) <= etol * abs(eo[k]), (k, eg[k], eo[k])
    assert eo["FE"] > 0 and eo["Wext"] > 0


def test_stress_and_energies_match():
    case = W.block_3d(nx=12, ny=10, nz=8)
    o = make_oracle(case)
    g = gpu(case, precision=tlsph.FP64)
    o.step(300)
    g.step(300)
    assert rel_l2(g.read_state("P"), o.read("P")) <= 1e-8
    assert rel_l2(g.read_state("F"), o.read("F")) <= 1e-10
    eo, eg = o.energies(), g.energies()
    for k in ["KE", "SE", "PW", "Wext"]:  # Wext: the reactions of the pressing and the fixed face
        assert abs(eg[k] - eo[k]) <= 1e-8 * max(abs(eo[k]), 1e-30), (k, eg[k], eo[k])
    assert eo["Wext"] > 0


def test_cpinv_matches_oracle_plastic_state():
    case = W.block_3d(nx=12, ny=10, nz=8)
    o = make_oracle(case)
    g = gpu(case, precision=tlsph.FP64)
    o.step(500)
    g.step(500)
    assert np.abs(g.read_state("CPINV") - o.read("CPINV")).max() <= 1e-9


# ---------------------------------------------------------------- invariants on the GPU
def test_momentum_conservation_gpu():
    case = W.block_3d(nx=10, ny=9, nz=8, jitter=0.05, seed=4, beta1=0.0)
    case.bcs = []
    g = gpu(case, precision=tlsph.FP64)
    g.set_option(tlsph.OPT_RECORD_ACC, 1)
    g.write_state("U", np.random.default_rng(0).normal(scale=2e-7, size=case.X0.shape))
    g.step(1)
    a = g.read_state("ACC")
    m = case.materials[0].rho * case.vol
    tot = (m[:, None] * a).sum(axis=0)
    assert np.abs(tot).max() < 1e-10 * (m[:, None] * np.abs(a)).sum()


def test_checkpoint_round_trip_bit_identical():
    case = W.notched_plate(nx=60, ny=24)
    a = gpu(case)
    a.step(100)
    blob = a.read_state("STATE").copy()
    a.step(100)
    u1 = a.read_state("U")
    b = gpu(case)
    b.write_state("STATE", blob)
    b.step(100)
    assert np.array_equal(b.read_state("U"), u1)
    assert np.array_equal(b.read_state("S"), a.read_state("S"))


def test_determinism_run_twice():
    case = W.block_3d(nx=14, ny=12, nz=9)
    u = []
    for _ in range(2):
        g = gpu(case)
        g.step(200)
        u.append(g.read_state("U"))
    assert np.array_equal(u[0], u[1])


def test_adaptive_dt_tracks_oracle():
    case = W.plate_2d(precision="fp64")
    case.dt_mode = W.DT_ADAPTIVE
    o = make_oracle(case)
    g = gpu(case)
    o.step(200)
    g.step(200)
    to, dto = o.time()
    tg, dtg = g.time()
    assert abs(tg - to) <= 1e-7 * to and abs(dtg - dto) <= 1e-7 * dto


# ---------------------------------------------------------------- error handling
def test_errors_are_statuses():
    case = W.plate_2d(nx=10, ny=5)
    t = tlsph.TLSPH(2, case.h, tlsph.FP64)
    t.set_materials(case.materials)
    t.create_particles(case.X0, case.vol)
    with pytest.raises(tlsph.TLSPHError) as e:
        t.step(1)
    assert e.value.status == tlsph.ERR_STATE
    # an isolated particle has a singular correction matrix
    X = np.vstack([case.X0, [[1.0, 1.0]]])
    t.create_particles(X, np.full(X.shape[0], case.dp ** 2))
    with pytest.raises(tlsph.TLSPHError) as e:
        t.build_ref_neighbours()
    assert e.value.status == tlsph.ERR_SINGULAR_L
    with pytest.raises(tlsph.TLSPHError) as e:
        t.create_particles(np.array([[np.nan, 0.0]]), np.array([1.0]))
    assert e.value.status == tlsph.ERR_ARG


@pytest.mark.parametrize("integrator", [1, 2])
def test_external_work_of_a_constant_traction_on_the_gpu(integrator):
    """A clamped bar pulled by a constant traction: the GPU's Wext equals sum f . u of its own displacement
    (the work of a constant force along the path is its value times the displacement) and the oracle's
    Wext, under both integrators."""
    case = W.plate_2d(nx=40, ny=6, beta1=0.0, beta2=0.0)
    X = case.X0
    left = np.isclose(X[:, 0], X[:, 0].min()).astype(np.uint8)
    right = np.isclose(X[:, 0], X[:, 0].max())
    case.bcs = [W.BC(left, W.BC_VEL, 0b11, (0.0, 0.0, 0.0)),
                W.BC(right.astype(np.uint8), W.BC_TRACTION, 0b01, (2e8, 0.0, 0.0), area=case.dp)]
    case.integrator = integrator
    o = make_oracle(case)
    g = gpu(case, precision=tlsph.FP64)
    o.step(400)
    g.step(400)
    w = g.energies()["Wext"]
    ref = np.sum(2e8 * case.dp * g.read_state("U")[right, 0])
    assert abs(w - ref) <= 1e-12 * abs(ref)
    assert abs(w - o.energies()["Wext"]) <= 1e-9 * abs(ref)
