"""Oracle pins for the energy outputs (Sec. 3.5 energy tracking) and for the reading of the
phase-field update (eq. phasefieldddot, Algorithm 1), each against something other than the oracle:

* the fracture energy FE of a uniform phase field is its closed form (no gradient term);
* FE of the steady 1D profile s = 1 - exp(-|x| / (2 eps0)) tends to Gc per unit crack length as
  dp / eps0 -> 0 (Sec. 2.2: the regularised crack functional of that profile integrates to Gc),
  at first order in dp / eps0;
* the external work of constant forces (a traction, gravity) is sum f . u, and with it the
  scheme's conserved energy (the staggered energy of Algorithm 1 minus the external work)
  stays constant;
* Algorithm 1's printed explicit update of sdot diverges at the notch tip of the notched plate
  once the history functional grows there, while the reading taken (local terms at the new
  time level) stays bounded; the two agree as dt -> 0 (their difference halves with dt).
"""
import math

import numpy as np
import pytest

from paper_2602_15149_b300 import workloads as W
from tests.oracle_cases import make_oracle


# ---------------------------------------------------------------- fracture energy
def _strip(k, dp=1e-3, ny=10, half_width_eps=12):
    """A phase-field strip 2 x 12 eps0 wide (eps0 = k dp), no loads, no notch."""
    eps0 = k * dp
    nx = int(round(2 * half_width_eps * eps0 / dp))
    case = W.notched_plate(nx=nx, ny=ny, width=nx * dp, height=ny * dp, notch_len=0.0, traction=0.0)
    case.bcs = []
    case.notches = []
    case.materials[0].eps0 = eps0
    return case, eps0


def test_fracture_energy_of_a_uniform_field_is_the_closed_form():
    """FE = sum_i V_i Gc (1 - s)^2 / (4 eps0) when s is uniform (the corrected gradient of a constant is
    zero, so the gradient term adds nothing)."""
    case, eps0 = _strip(3)
    o = make_oracle(case)
    Gc = case.materials[0].Gc
    for s0 in (1.0, 0.7, 0.25, 0.0):
        o.write("S", np.full(case.n, s0))
        fe = o.energies()["FE"]
        ref = np.sum(case.vol) * Gc * (1.0 - s0) ** 2 / (4.0 * eps0)
        assert abs(fe - ref) <= 1e-12 * max(ref, 1e-30), (s0, fe, ref)


def test_fracture_energy_of_the_steady_profile_tends_to_gc():
    """The steady 1D profile s = 1 - exp(-|x| / (2 eps0)) across a crack line of length L has
    integral of (1 - s)^2 / (4 eps0) + eps0 s'^2 equal to 1 per unit length (each term 1/2), so
    FE -> Gc L.  The discrete FE (corrected SPH gradient, kink at the crack line) approaches it at
    first order in dp / eps0: the deficit halves when eps0 / dp doubles."""
    deficits = []
    for k in (2, 4, 8, 16):
        case, eps0 = _strip(k)
        o = make_oracle(case)
        x = case.X0[:, 0] - 0.5 * (case.X0[:, 0].min() + case.X0[:, 0].max())
        o.write("S", 1.0 - np.exp(-np.abs(x) / (2.0 * eps0)))
        L = case.X0[:, 1].max() - case.X0[:, 1].min() + case.dp
        deficits.append(1.0 - o.energies()["FE"] / (case.materials[0].Gc * L))
    assert all(d > 0 for d in deficits)
    for a, b in zip(deficits, deficits[1:]):
        assert 1.7 <= a / b <= 2.3, deficits
    assert deficits[-1] < 0.04, deficits


# ---------------------------------------------------------------- external work
def _bar(kind, integrator=1):
    """A 40 x 6 plane-strain bar without viscosity, clamped at x = 0 and loaded by a constant traction on
    its far end, by gravity, or pulled there at a constant velocity."""
    case = W.plate_2d(nx=40, ny=6, beta1=0.0, beta2=0.0)
    X = case.X0
    left = np.isclose(X[:, 0], X[:, 0].min()).astype(np.uint8)
    right = np.isclose(X[:, 0], X[:, 0].max()).astype(np.uint8)
    clamp = W.BC(left, W.BC_VEL, 0b11, (0.0, 0.0, 0.0))
    if kind == "traction":
        case.bcs = [clamp, W.BC(right, W.BC_TRACTION, 0b01, (2e8, 0.0, 0.0), area=case.dp)]
    elif kind == "gravity":
        case.bcs = [clamp]
        case.gravity = (0.0, -9.81e5, 0.0)
    else:
        case.bcs = [clamp, W.BC(right, W.BC_VEL, 0b01, (0.5, 0.0, 0.0))]
    case.integrator = integrator
    return case


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("kind", ["traction", "gravity"])
def test_external_work_of_constant_forces_is_force_times_displacement(kind, integrator):
    case = _bar(kind, integrator)
    o = make_oracle(case)
    m = case.materials[0].rho * case.vol
    right = np.isclose(case.X0[:, 0], case.X0[:, 0].max())
    for _ in range(8):
        o.step(60)
        U = o.read("U")
        ref = np.sum(2e8 * case.dp * U[right, 0]) if kind == "traction" else np.sum(m * -9.81e5 * U[:, 1])
        w = o.energies()["Wext"]
        assert abs(ref) > 0 and abs(w - ref) <= 1e-12 * abs(ref), (w, ref)


def _staggered_minus_work(o, case):
    """1/2 m v_{n-1/2} . v_{n+1/2} + SE(u_n) - Wext(u_n), Algorithm 1's conserved energy under a constant
    external force (the work is then the potential -f . u).  Advances the oracle by one step."""
    m = case.materials[0].rho * case.vol
    e = o.energies()
    v0 = o.read("V")
    o.step(1)
    v1 = o.read("V")
    return 0.5 * np.sum(m[:, None] * v0 * v1) + e["SE"] - e["Wext"], abs(e["Wext"])


@pytest.mark.parametrize("kind,tol", [("traction", 5e-6), ("gravity", 5e-7), ("velocity", 3e-3)])
def test_energy_balance_with_external_work(kind, tol):
    """KE + SE - Wext (staggered) of a loaded bar without viscosity stays constant: to roundoff-level
    drift for constant forces, within a bounded drift when a velocity condition pulls (its reaction is
    the external force)."""
    case = _bar(kind)
    o = make_oracle(case)
    E0, _ = _staggered_minus_work(o, case)
    worst, wmax = 0.0, 0.0
    for _ in range(20):
        o.step(49)
        E, w = _staggered_minus_work(o, case)
        worst, wmax = max(worst, abs(E - E0)), max(wmax, w)
    assert wmax > 1.0
    assert worst <= tol * wmax, (worst / wmax)


# ---------------------------------------------------------------- phase-field update (reading R20)
def test_printed_explicit_update_diverges_at_the_notch_tip():
    """On the notched plate (125 x 50, +-1 MPa) the printed update sdot_{n+1} = sdot_n + dt sddot_n grows
    without bound once the history functional at the notch tip is large (dt gamma > 2 for the damping
    gamma = (c / eps0) sqrt(4 eps0 H / Gc + 1)); the reading taken stays bounded on the same run."""
    case = W.notched_plate(nx=125, ny=50)
    o_impl, o_expl = make_oracle(case), make_oracle(case, pf_explicit=True)
    o_impl.step(400)
    o_expl.step(400)
    sd_i, sd_e = np.abs(o_impl.read("SDOT")), np.abs(o_expl.read("SDOT"))
    assert sd_i.max() < 1e6
    assert sd_e.max() > 1e20
    k = int(np.argmax(sd_e))
    tip = np.array([0.05, 0.02])
    assert np.linalg.norm(case.X0[k] - tip) <= 4 * case.dp, case.X0[k]


def test_phase_field_readings_agree_as_dt_shrinks():
    """Before the explicit form breaks down (150 steps of the CFL step, damage down to s = 0.58 at the
    tip), the reading and the printed form differ at first order in dt: the largest difference of s
    halves each time dt halves (to the same simulated time)."""
    base = make_oracle(W.notched_plate(nx=125, ny=50))
    base.step(1)
    dt0 = base.time()[1]
    diffs = []
    for f in (1, 2, 4):
        res = []
        for explicit in (False, True):
            case = W.notched_plate(nx=125, ny=50)
            case.dt_mode, case.fixed_dt = W.DT_FIXED, dt0 / f
            o = make_oracle(case, pf_explicit=explicit)
            o.step(150 * f)
            res.append(o.read("S"))
        assert res[0].min() < 0.7  # damage is under way
        diffs.append(np.abs(res[0] - res[1]).max())
    for a, b in zip(diffs, diffs[1:]):
        assert 1.8 <= a / b <= 2.2, diffs
