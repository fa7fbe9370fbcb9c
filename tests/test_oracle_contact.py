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


# ---------------------------------------------------------------- friction (<kfric>)
def _split(F, d):
    n = d / np.linalg.norm(d)
    fn = F @ n
    return fn, F - fn * n


@pytest.mark.parametrize("mu", [0.1, 0.6])
def test_friction_is_tangential_bounded_dissipative_and_reciprocal(mu):
    """Coulomb's law in every contact: the friction changes only the tangential part of the pair force, its
    size never exceeds mu times the compressive normal force, it opposes the sliding velocity, there is none
    while the pair pulls apart under tension, and j feels the opposite force."""
    rng = np.random.default_rng(7)
    seen_sliding = seen_tension = 0
    for _ in range(400):
        xi, xj = rng.uniform(0, 1e-2, 2), rng.uniform(0, 1e-2, 2)
        vi, vj = rng.normal(size=2) * rng.choice([1e-4, 1.0, 30.0]), rng.normal(size=2)
        d = xi - xj
        if np.linalg.norm(d) >= 1e-2:
            continue
        F0 = contact_force(2, 1e-2, 5.0, xi, xj, vi, vj, 0.5, 0.7, STEEL, SOFT, 0.9, 0.6)
        F = contact_force(2, 1e-2, 5.0, xi, xj, vi, vj, 0.5, 0.7, STEEL, SOFT, 0.9, 0.6, mu=mu)
        Fji = contact_force(2, 1e-2, 5.0, xj, xi, vj, vi, 0.7, 0.5, SOFT, STEEL, 0.6, 0.9, mu=mu)
        assert np.allclose(F, -Fji, rtol=1e-13, atol=1e-300)
        fn0, ft0 = _split(F0, d)
        fn, ft = _split(F, d)
        scale = abs(fn0) + np.linalg.norm(F)
        assert abs(fn - fn0) <= 1e-12 * scale and np.linalg.norm(ft0) <= 1e-12 * scale
        vt = (vi - vj) - ((vi - vj) @ d) * d / (d @ d)
        if fn0 <= 0:
            seen_tension += 1
            assert np.linalg.norm(ft) <= 1e-12 * scale
            continue
        assert np.linalg.norm(ft) <= mu * fn0 * (1 + 1e-12)
        assert ft @ vt <= 0
        assert abs(ft[0] * vt[1] - ft[1] * vt[0]) <= 1e-9 * np.linalg.norm(ft) * np.linalg.norm(vt)
        seen_sliding += np.linalg.norm(ft) >= mu * fn0 * (1 - 1e-12)
    assert seen_sliding > 20 and seen_tension >= 3


def test_friction_is_coulomb_when_sliding_and_vanishes_at_rest():
    """A pair pressed together (no normal motion) and sliding fast feels exactly mu f_n; as the sliding speed
    goes to zero the friction goes to zero in proportion to it (no jump for an explicit step to chatter on).
    The crossover speed is mu delta w / 2 (about 0.07 m/s for this soft pair at 1% overlap)."""
    dc, kc, mu = 1e-2, 5.0, 0.4
    xi, xj = np.array([0.0, 0.0]), np.array([0.99 * dc, 0.0])
    fn = -contact_force(2, dc, kc, xi, xj, np.zeros(2), np.zeros(2), 0.5, 0.5, SOFT, SOFT, 1.0, 1.0)[0]
    assert fn > 0
    for vt in (5.0, 50.0):
        F = contact_force(2, dc, kc, xi, xj, np.array([0.0, vt]), np.zeros(2), 0.5, 0.5, SOFT, SOFT, 1.0, 1.0, mu)
        assert abs(F[1] + mu * fn) <= 1e-12 * mu * fn
        assert abs(-F[0] - fn) <= 1e-12 * fn
    r = [contact_force(2, dc, kc, xi, xj, np.array([0.0, v]), np.zeros(2), 0.5, 0.5, SOFT, SOFT, 1.0, 1.0, mu)[1] / v
         for v in (1e-9, 1e-8, 1e-7)]
    assert r[0] < 0 and abs(r[1] / r[0] - 1) < 1e-9 and abs(r[2] / r[0] - 1) < 1e-9


def test_sliding_pair_stops_as_coulomb_predicts():
    """A particle pressed onto another by a constant load and sliding at v0 decelerates at mu f_n / m*
    (Coulomb) and never slides back: it stops after about m* v0 / (mu f_n).  Soft pair at 1% overlap, whose
    crossover speed (0.05 m/s) is 1% of v0, with w dt = 0.025 as the solver's Courant number gives."""
    dc, kc, mu, m1, m2, v0 = 1e-2, 5.0, 0.3, 0.8, 0.4, 5.0
    ms = m1 * m2 / (m1 + m2)
    x1, x2 = np.array([0.0, 0.0]), np.array([0.99 * dc, 0.0])
    fn = -contact_force(2, dc, kc, x1, x2, np.zeros(2), np.zeros(2), m1, m2, SOFT, SOFT, 1.0, 1.0)[0]
    k = fn / (0.01 * dc)
    t_stop = ms * v0 / (mu * fn)
    dt = 0.025 / math.sqrt(k / ms)
    v1, v2 = np.array([0.0, v0]), np.zeros(2)
    t, t_end, vrel = 0.0, None, []
    for _ in range(int(1.2 * t_stop / dt)):
        F = contact_force(2, dc, kc, x1, x2, v1, v2, m1, m2, SOFT, SOFT, 1.0, 1.0, mu)
        F[0] = 0.0  # the normal load is held (the pair stays pressed at the same overlap)
        v1 = v1 + dt * F / m1
        v2 = v2 - dt * F / m2
        t += dt
        vrel.append(v1[1] - v2[1])
        if t_end is None and vrel[-1] <= 1e-3 * v0:
            t_end = t
    assert t_end is not None and abs(t_end - t_stop) < 0.03 * t_stop
    assert min(vrel) >= -1e-9 * v0 and abs(vrel[-1]) < 1e-6 * v0


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


def test_friction_stops_the_sliding_at_most_in_one_step():
    """With a step long for the contact spring (omega dt = 2, where the viscous regularisation alone would
    reverse the sliding), friction is capped at m* |v_t| / dt: one explicit step brings the pair's relative
    tangential velocity to zero and not past it.  With a short step (omega dt = 0.1) the cap is inactive."""
    dc, kc, mu = 1e-2, 5.0, 0.5
    m1 = m2 = 0.5
    xi, xj = np.array([0.0, 0.0]), np.array([0.009, 0.0])  # pressed: r < dc
    fn = -contact_force(2, dc, kc, xi, xj, np.zeros(2), np.zeros(2), m1, m2, SOFT, SOFT, 1.0, 1.0)[0]
    assert fn > 0
    kn = kc / (2 * (1 - SOFT.nu ** 2) / SOFT.E)
    ms = m1 * m2 / (m1 + m2)
    omega = math.sqrt(kn / ms)
    vt = 0.5 * mu * fn / (2 * math.sqrt(kn * ms))  # slow enough that the viscous bound is below Coulomb
    vi = np.array([0.0, vt])
    for wdt, capped in ((2.0, True), (0.1, False)):
        dt = wdt / omega
        F = contact_force(2, dc, kc, xi, xj, vi, np.zeros(2), m1, m2, SOFT, SOFT, 1.0, 1.0, mu, dt)
        Fu = contact_force(2, dc, kc, xi, xj, vi, np.zeros(2), m1, m2, SOFT, SOFT, 1.0, 1.0, mu)
        ft = -F[1]
        if capped:
            assert abs(ft - ms * vt / dt) <= 1e-12 * ft
            assert vt - ft / ms * dt >= -1e-15  # relative tangential velocity after the step (pair's own frame)
            assert ft < -Fu[1]
        else:
            assert ft == -Fu[1]
