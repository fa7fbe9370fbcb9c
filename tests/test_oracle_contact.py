"""Pins of the oracle's contact between bodies (reading of Sec. 3.3 <contcoeff>, <restcoef>: a linear
spring-dashpot normal force between particles of different bodies closer than the particle spacing).

The force law is checked against the damped oscillator it defines: a head-on pair leaves with e times its
approach speed after half a damped period, pi / (w_n sqrt(1 - zeta^2)).  The step is checked on plates
that collide: momentum is conserved exactly, energy (kinetic + strain + contact) is conserved without
damping and lost with it, and the collision of two identical plates is mirror-symmetric."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleMaterial, contact_force
from paper_2602_15149_b300 import workloads as W
from tests.oracle_cases import make_oracle

STEEL = OracleMaterial(model=2, rho=7870.0, E=200e9, nu=0.29)
SOFT = OracleMaterial(model=2, rho=1000.0, E=1e6, nu=0.4)


def test_pair_force_is_antisymmetric_normal_and_short_ranged():
    rng = np.random.default_rng(0)
    for _ in range(50):
        xi, xj = rng.uniform(0, 1e-2, 2), rng.uniform(0, 1e-2, 2)
        vi, vj = rng.normal(size=2), rng.normal(size=2)
        Fij = contact_force(2, 1e-2, 5.0, xi, xj, vi, vj, 0.5, 0.7, STEEL, SOFT, 0.9, 0.6)
        Fji = contact_force(2, 1e-2, 5.0, xj, xi, vj, vi, 0.7, 0.5, SOFT, STEEL, 0.6, 0.9)
        assert np.allclose(Fij, -Fji, rtol=1e-14, atol=0)
        d = xi - xj
        if np.linalg.norm(d) >= 1e-2:
            assert not Fij.any()
        else:
            assert abs(Fij[0] * d[1] - Fij[1] * d[0]) <= 1e-12 * np.linalg.norm(Fij) * np.linalg.norm(d)


@pytest.mark.parametrize("e", [1.0, 0.95, 0.5])
def test_head_on_pair_restitution_and_duration(e):
    """Integrate the pair's relative motion with the oracle's force (dt 1/2000 of the contact time)."""
    dc, kc, m1, m2, v0 = 1e-2, 5.0, 0.8, 0.4, 3.0
    ms = m1 * m2 / (m1 + m2)
    k = kc / (2 * (1 - STEEL.nu ** 2) / STEEL.E)
    le = math.log(e)
    zeta = -le / math.sqrt(math.pi ** 2 + le ** 2)
    tc = math.pi / (math.sqrt(k / ms) * math.sqrt(1 - zeta ** 2))
    dt = tc / 2000
    x1, x2 = np.array([0.0, 0.0]), np.array([dc, 0.0])  # just touching
    v1, v2 = np.array([v0, 0.0]), np.array([0.0, 0.0])
    t, in_contact, t_in = 0.0, False, None
    for _ in range(10000):
        F = contact_force(2, dc, kc, x1, x2, v1, v2, m1, m2, STEEL, STEEL, e, e)
        v1 = v1 + dt * F / m1
        v2 = v2 - dt * F / m2
        x1, x2 = x1 + dt * v1, x2 + dt * v2
        t += dt
        touching = np.linalg.norm(x2 - x1) < dc
        if touching and not in_contact:
            in_contact, t_in = True, t - dt
        if in_contact and not touching:
            break
    assert abs((v2[0] - v1[0]) / v0 - e) < 2e-3
    assert abs((t - t_in) - tc) < 5e-3 * tc
    assert abs(m1 * v1[0] + m2 * v2[0] - m1 * v0) < 1e-12 * m1 * v0


def _plates(e, v=1.0, n=8, model="nh", beta1=None):
    """Two touching 8 x 8 plates (closest rows one spacing apart, the contact distance) closing at 2 v.  The
    contact spring's w dt is about 0.15 at C_CFL = 0.05."""
    case = W.flyer_plate(n=n, dx=1e-3, gap=0.0, v=v, restitution=e, model=model, precision="fp64")
    case.cfl = 0.05
    if beta1 is not None:
        case.materials[0].beta1 = beta1
    return case


def test_momentum_conserved_through_the_collision():
    case = _plates(0.8, v=2.0)
    o = make_oracle(case)
    m = case.materials[0].rho * case.vol
    p0 = (m[:, None] * o.read("V")).sum(axis=0)
    touched = False
    for _ in range(30):
        o.step(20)
        p = (m[:, None] * o.read("V")).sum(axis=0)
        assert np.abs(p - p0).max() <= 1e-12 * (m * 2.0).sum()
        touched |= o.contact_energy() > 0
    assert touched


def _total_energy(o, case):
    e = o.energies()
    return e["KE"] + e["SE"] + o.contact_energy()


def test_energy_without_and_with_damping():
    """Without viscosity: e = 1 keeps kinetic + strain + contact energy within 2% through impact and rebound
    (the symplectic Euler energy, sampled with v at half steps, oscillates by about 1%); e = 0.3 loses
    about a tenth of it for good."""
    out = {}
    for e in (1.0, 0.3):
        case = _plates(e, beta1=0.0)
        o = make_oracle(case)
        E0 = _total_energy(o, case)
        hist, contact = [], []
        for _ in range(100):
            o.step(10)
            hist.append(_total_energy(o, case))
            contact.append(o.contact_energy())
        assert max(contact) > 0 and contact[-1] == 0.0  # they met and separated
        out[e] = (E0, np.array(hist))
    E0, h = out[1.0]
    assert np.abs(h - E0).max() < 0.02 * E0
    E0, h = out[0.3]
    assert h[-1] < 0.95 * E0 and np.abs(h[-30:] - h[-1]).max() < 0.01 * E0


def test_symmetric_collision():
    case = _plates(0.9, v=2.0)
    o = make_oracle(case)
    o.step(300)
    u = o.read("U")
    m = case.n // 2
    lo, hi = u[:m], u[m:]
    # the upper plate is the lower one mirrored about the mid-plane: u_y flips sign, rows reverse
    n = int(round(math.sqrt(m)))
    lo = lo.reshape(n, n, 2)
    hi = hi.reshape(n, n, 2)[::-1]
    assert np.abs(hi[..., 0] - lo[..., 0]).max() <= 1e-9 * np.abs(u).max()
    assert np.abs(hi[..., 1] + lo[..., 1]).max() <= 1e-9 * np.abs(u).max()
