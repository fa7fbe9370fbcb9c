"""Pins of the phase-field bound (<restrictphi> of Sec. 3.3; Sec. 4 keeps the particles near the loads of the
four-point bend intact with s >= 0.9999): the particles a bound covers keep s_{n+1} >= its value.

A bound of 0 changes nothing (s is never negative), a bound of 1 on every particle leaves the notched plate
undamaged and moving like the same plate without a phase field, a bound around the notch tip keeps the tip
intact while the rest of the plate evolves as before, and a bound given by an expression that skips outside
a region acts exactly like the same constant bound on that region."""
import copy

import numpy as np
import pytest

from paper_2602_15149_b300 import workloads as W
from tests.oracle_cases import make_oracle

BOUND = W.BC_PHASE_BOUND


def _plate(**kw):
    case = W.notched_plate(nx=60, ny=24, precision="fp64", traction=4e6, **kw)
    return case


def _with(case, bcs=(), exbcs=()):
    c = copy.copy(case)
    c.bcs = list(case.bcs) + list(bcs)
    c.expr_bcs = list(getattr(case, "expr_bcs", []) or []) + list(exbcs)
    return c


def _run(case, steps, every=50):
    o = make_oracle(case)
    snaps = []
    for _ in range(steps // every):
        o.step(every)
        snaps.append((o.read("S").copy(), o.read("U").copy()))
    return o, snaps


def test_zero_bound_changes_nothing():
    case = _plate()
    all_ = np.ones(case.n, np.uint8)
    _, a = _run(case, 200)
    _, b = _run(_with(case, [W.BC(all_, BOUND, 1, (0.0, 0.0, 0.0))]), 200)
    for (sa, ua), (sb, ub) in zip(a, b):
        assert np.array_equal(sa, sb) and np.array_equal(ua, ub)


@pytest.mark.parametrize("integrator", [1, 2])
def test_full_bound_keeps_the_plate_intact(integrator):
    """s = 1 everywhere: no damage, and the displacement is that of the plate without a phase field.  Under
    Algorithm 2 this needs the bound at the half level as well: the forces and the degradation of a step are
    taken at s_{n+1/2}, which a negative sdot would otherwise pull below 1."""
    case = _plate()
    case.integrator = integrator
    assert case.materials[0].fracture
    bounded = _with(case, [W.BC(np.ones(case.n, np.uint8), BOUND, 1, (1.0, 0.0, 0.0))])
    intact = copy.copy(case)
    intact.materials = [copy.copy(m) for m in case.materials]
    for m in intact.materials:
        m.fracture = False
    _, a = _run(bounded, 300)
    _, b = _run(intact, 300)
    for (sa, ua), (_, ub) in zip(a, b):
        assert np.all(sa == 1.0)
        assert np.abs(ua - ub).max() <= 1e-9 * np.abs(ub).max()


def test_bound_at_the_notch_tip_holds_and_is_needed():
    case = _plate()
    X = case.X0
    tip = np.array([0.05, 0.02])  # the notch runs from x = 0 to 0.05 at mid-height
    near = (np.linalg.norm(X - tip, axis=1) < 4 * case.dp).astype(np.uint8)
    _, free = _run(case, 600, every=100)
    _, held = _run(_with(case, [W.BC(near, BOUND, 1, (0.9999, 0.0, 0.0))]), 600, every=100)
    assert free[-1][0][near == 1].min() < 0.99  # without the bound the tip damages
    for s, _ in held:
        assert s[near == 1].min() >= 0.9999


def test_expression_bound_equals_the_constant_bound_on_its_region():
    case = _plate()
    region = (case.X0[:, 0] > 0.04) & (case.X0[:, 0] < 0.07)
    const = _with(case, [W.BC(region.astype(np.uint8), BOUND, 1, (0.9999, 0.0, 0.0))])
    expr = _with(case, exbcs=[W.ExprBC(np.ones(case.n, np.uint8), BOUND, 1,
                                       [("if(x0 > 0.04 and x0 < 0.07, 0.9999, skip)", ""), None, None])])
    _, a = _run(const, 300)
    _, b = _run(expr, 300)
    for (sa, ua), (sb, ub) in zip(a, b):
        assert np.array_equal(sa, sb) and np.array_equal(ua, ub)


def test_expression_bound_is_kept_in_the_unit_interval():
    """An expression bound of 1.5 acts as the bound 1 (s stays a fraction), and one of -0.5 as no bound."""
    case = _plate()
    all_ = np.ones(case.n, np.uint8)
    one = _with(case, [W.BC(all_, BOUND, 1, (1.0, 0.0, 0.0))])
    big = _with(case, exbcs=[W.ExprBC(all_, BOUND, 1, [("1.5", ""), None, None])])
    neg = _with(case, exbcs=[W.ExprBC(all_, BOUND, 1, [("-0.5", ""), None, None])])
    _, a = _run(one, 200)
    _, b = _run(big, 200)
    _, c = _run(case, 200)
    _, d = _run(neg, 200)
    for (sa, ua), (sb, ub) in zip(a, b):
        assert np.array_equal(sa, sb) and np.array_equal(ua, ub) and sb.max() <= 1.0
    for (sc, uc), (sd, ud) in zip(c, d):
        assert np.array_equal(sc, sd) and np.array_equal(uc, ud)


def test_bad_phase_bounds_are_refused():
    o = make_oracle(_plate())
    all_ = np.ones(o.n, np.uint8)
    for value, comp in ((1.5, 1), (-0.1, 1), (float("nan"), 1), (0.5, 2), (0.5, 0)):
        with pytest.raises(RuntimeError):
            o.add_bc(all_, BOUND, comp, (value, 0.0, 0.0))
