"""The phase-field bound (<restrictphi> of Sec. 3.3) on the sm_103a path against the FP64 oracle: a constant
bound around the notch tip and the same bound given by an expression that skips outside its region, on the
notched plate under the traction that damages the tip without the bound.  u within 1e-5 (FP64) / 1e-4
(FP32) of the oracle (relative L2), s within 1e-3, and the covered particles keep s >= 0.9999 in both."""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle
from tests.test_oracle_phase_bound import _plate, _with

pytestmark = pytest.mark.gpu


def _cases():
    case = _plate()
    tip = np.array([0.05, 0.02])
    near = np.linalg.norm(case.X0 - tip, axis=1) < 4 * case.dp
    const = _with(case, [W.BC(near.astype(np.uint8), W.BC_PHASE_BOUND, 1, (0.9999, 0.0, 0.0))])
    expr = _with(case, exbcs=[W.ExprBC(np.ones(case.n, np.uint8), W.BC_PHASE_BOUND, 1,
                                       [("if((x0 - 0.05)^2 + (y0 - 0.02)^2 < (4*dx)^2, 0.9999, skip)", ""),
                                        None, None])])
    return near, {"constant": const, "expression": expr}


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("which", ["constant", "expression"])
@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-5), (tlsph.FP32_U64, 1e-4)])
def test_phase_bound_matches_oracle(which, precision, tol, integrator):
    near, cases = _cases()
    case = cases[which]
    case.integrator = integrator
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    for _ in range(3):
        o.step(200)
        g.step(200)
        u_o, u_g = o.read("U"), g.read_state("U")
        assert np.linalg.norm(u_g - u_o) <= tol * np.linalg.norm(u_o)
        s_o, s_g = o.read("S"), g.read_state("S")
        assert np.abs(s_g - s_o).max() <= 1e-3
        assert s_g[near].min() >= np.float32(0.9999) and s_o[near].min() >= 0.9999


def test_phase_bound_is_refused_for_a_bad_kind():
    case = _plate()
    g = tlsph.from_case(case, build=False)
    with pytest.raises(tlsph.TLSPHError):
        g.add_bc(np.ones(case.n, np.uint8), 5, 1, (1.0, 0.0, 0.0))


def test_full_bound_under_algorithm_2_keeps_the_plate_intact_on_the_gpu():
    """Bound 1 on every particle under Algorithm 2: the half level is bounded as well, so the plate moves as
    the same plate without a phase field (FP64, 1e-9)."""
    import copy

    case = _plate()
    case.integrator = 2
    bounded = _with(case, [W.BC(np.ones(case.n, np.uint8), W.BC_PHASE_BOUND, 1, (1.0, 0.0, 0.0))])
    intact = copy.copy(case)
    intact.materials = [copy.copy(m) for m in case.materials]
    for m in intact.materials:
        m.fracture = False
    a = tlsph.from_case(bounded, precision=tlsph.FP64)
    b = tlsph.from_case(intact, precision=tlsph.FP64)
    a.step(300)
    b.step(300)
    assert np.all(a.read_state("S") == 1.0)
    ua, ub = a.read_state("U"), b.read_state("U")
    assert np.abs(ua - ub).max() <= 1e-9 * np.abs(ub).max()


def test_bad_phase_bounds_are_refused_by_the_library():
    case = _plate()
    g = tlsph.from_case(case, build=False)
    all_ = np.ones(case.n, np.uint8)
    for value, comp in ((1.5, 1), (-0.1, 1), (float("nan"), 1), (0.5, 2)):
        with pytest.raises(tlsph.TLSPHError) as e:
            g.add_bc(all_, W.BC_PHASE_BOUND, comp, (value, 0.0, 0.0))
        assert e.value.status == tlsph.ERR_ARG
