"""User-defined expressions (Sec. 3.3) on the sm_103a path against the oracle's evaluator, through the
C-ABI: the device bytecode interpreter, boundary conditions given by expressions in both integrators and
all execution modes, and initial fields.

Tolerances: trees of correctly rounded operations (+ - * /, sqrt, abs, comparisons, logic, if) bit-exact;
the transcendental functions within 4 ulp of numpy; runs with expression conditions bit-identical to the
same conditions written as constants, and within 1e-8 (FP64, max norm relative to the largest value) of the
oracle, whose neighbour sums run in another order (a condition applied at the wrong time level would be off
by about w dt ~ 1e-2 here).
"""
import copy

import numpy as np
import pytest

from oracle.expr import VARIABLES, Expression
from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle
from tests.test_oracle_expr import CANTILEVER_EXPR, CANTILEVER_LOCALS, _paper

pytestmark = pytest.mark.gpu

EXACT_F1 = ["sqrt", "abs"]
_PREC_OPS = ["or", "and", "<", ">", "<=", ">=", "==", "!=", "+", "-", "*", "/"]


def _gen_exact(rng, depth):
    """Random trees of correctly rounded operations only."""
    r = rng.random()
    if depth == 0 or r < 0.2:
        if rng.random() < 0.5:
            return ("num", float(np.round(rng.uniform(-3, 3), 3)))
        return ("var", VARIABLES[rng.integers(len(VARIABLES))])
    r = rng.random()
    if r < 0.6:
        return (_PREC_OPS[rng.integers(len(_PREC_OPS))], _gen_exact(rng, depth - 1), _gen_exact(rng, depth - 1))
    if r < 0.7:
        return ("neg", _gen_exact(rng, depth - 1))
    if r < 0.8:
        return ("call", EXACT_F1[rng.integers(2)], _gen_exact(rng, depth - 1))
    return ("if", _gen_exact(rng, depth - 1), _gen_exact(rng, depth - 1), _gen_exact(rng, depth - 1))


@pytest.fixture(scope="module")
def ctx():
    return tlsph.from_case(W.plate_2d(nx=10, ny=4), precision=tlsph.FP64)


def _vars(rng, n):
    V = rng.uniform(-2, 2, size=(n, 12))
    V[::5] = np.round(V[::5])      # exact integers and zeros exercise ties in comparisons
    V[1::7] = 0.0
    return V


def test_exact_trees_bit_identical(ctx):
    rng = np.random.default_rng(11)
    n = 257  # two blocks and a ragged tail
    for _ in range(300):
        src = _paper(_gen_exact(rng, 5))
        V = _vars(rng, n)
        ref, rskip = Expression(src).evaluate(**{k: V[:, q] for q, k in enumerate(VARIABLES)})
        val, skip = ctx.expr_eval(ctx.expr_compile(src), V)
        assert np.array_equal(skip, rskip)
        same = (val == ref) | (np.isnan(val) & np.isnan(ref))
        assert same.all(), (src, val[~same][:3], ref[~same][:3])


@pytest.mark.parametrize("fn", ["sin", "cos", "tan", "cot", "sinh", "cosh", "tanh", "coth", "log", "ln", "pow"])
def test_functions_within_ulps(ctx, fn):
    rng = np.random.default_rng(12)
    V = np.zeros((1000, 12))
    V[:, 0] = rng.uniform(0.01, 5.0, 1000) * rng.choice([-1, 1], 1000) if fn not in ("log", "ln", "pow") \
        else rng.uniform(1e-3, 50.0, 1000)
    V[:, 1] = rng.uniform(-3, 3, 1000)
    src = "pow(x0, y0)" if fn == "pow" else f"{fn}(x0)"
    ref, _ = Expression(src).evaluate(x0=V[:, 0], y0=V[:, 1])
    val, skip = ctx.expr_eval(ctx.expr_compile(src), V)
    assert not skip.any()
    ulp = np.spacing(np.abs(ref))
    assert np.all(np.abs(val - ref) <= 4 * ulp), src


def test_skip_and_locals_on_device(ctx):
    x0 = np.array([-1.0, 0.0, 1.0])
    V = np.zeros((3, 12))
    V[:, 0] = x0
    for src, loc in [("if(x0 < 0, 0, skip)", ""), ("1 + skip", ""), ("if(skip, 1, 2)", ""), ("if(1, 3, skip)", ""),
                     ("a", "a = skip"), ("1", "a = skip"), ("a*b", "a = 2; b = a + x0"), (CANTILEVER_EXPR, CANTILEVER_LOCALS)]:
        ref, rskip = Expression(src, loc).evaluate(x0=x0)
        val, skip = ctx.expr_eval(ctx.expr_compile(src, loc), V)
        assert np.array_equal(skip, rskip), src
        assert np.allclose(val[~skip], ref[~rskip], rtol=1e-14, atol=0), src


def test_compile_errors_are_reported(ctx):
    for src in ["1+", "foo(1)", "if(1,2)"]:
        with pytest.raises(tlsph.TLSPHError):
            ctx.expr_compile(src)


# ---- boundary conditions ---------------------------------------------------------------------------------
def _plate(integrator=1):
    case = W.plate_2d(nx=30, ny=8, beta1=0.2)
    case.bcs[1].ramp = 0.0
    case.integrator = integrator
    return case


def _without(case, drop):
    c = copy.copy(case)  # keeps attributes beyond the dataclass fields (batched specimen loads)
    c.bcs = [b for k, b in enumerate(case.bcs) if k not in drop]
    return c


def _gpu_with(case, exbcs, drop=(), precision=tlsph.FP64, mode=None):
    """exbcs: (mask, kind, comp_mask, [(expr, locals) or None per component], area)."""
    c = _without(case, drop)
    g = tlsph.from_case(c, precision=precision, build=False)
    for mask, kind, cm, exprs, area in exbcs:
        ids = [-1 if e is None else g.expr_compile(*e) for e in exprs]
        g.add_bc_expr(mask, kind, cm, ids, area=area)
    g.build_ref_neighbours()
    if mode is not None:
        g.set_option(tlsph.OPT_MODE, mode)
    return g


def _oracle_with(case, exbcs, drop=()):
    o = make_oracle(_without(case, drop))
    for mask, kind, cm, exprs, area in exbcs:
        o.add_bc_expr(mask, kind, cm, [None if e is None else Expression(e[0], e[1]) for e in exprs], area=area)
    return o


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("mode", [tlsph.MODE_LAUNCH, tlsph.MODE_GRAPH])
def test_constant_expressions_equal_constant_conditions(integrator, mode):
    case = _plate(integrator)
    ref = tlsph.from_case(case, precision=tlsph.FP64)
    ref.step(150)
    left, right = case.bcs[0].mask, case.bcs[1].mask
    ex = [(left, 0, 0b11, [("0", ""), ("0", "")], 0.0), (right, 0, 0b01, [(repr(case.bcs[1].value[0]), "")], 0.0)]
    g = _gpu_with(case, ex, drop=(0, 1), mode=mode)
    g.step(150)
    assert np.array_equal(g.read_state("U"), ref.read_state("U"))
    clamp = ("if(x0 < dx, 0, skip)", "")
    g = _gpu_with(case, [(np.ones(case.n, np.uint8), 0, 0b11, [clamp, clamp], 0.0)], drop=(0,), mode=mode)
    g.step(150)
    assert np.array_equal(g.read_state("U"), ref.read_state("U"))


@pytest.mark.parametrize("integrator", [1, 2])
def test_time_dependent_velocity_matches_oracle(integrator):
    case = _plate(integrator)
    ex = [(case.bcs[1].mask, 0, 0b01, [("A*sin(w*t) + 0.1*ux/dx", "A = 0.3; w = 2e5")], 0.0)]
    g = _gpu_with(case, ex, drop=(1,))
    o = _oracle_with(case, ex, drop=(1,))
    g.step(200)
    o.step(200)
    u_o = o.read("U")
    assert np.abs(g.read_state("U") - u_o).max() <= 1e-8 * np.abs(u_o).max()
    assert np.abs(g.read_state("V") - o.read("V")).max() <= 1e-8 * np.abs(o.read("V")).max()


def test_traction_expression_matches_oracle():
    case = W.notched_plate(nx=60, ny=24, precision="fp64")
    top, bot = case.bcs
    ex = [(top.mask, top.kind, 0b10, [None, ("if(t < 2e-6, 1e6*t/2e-6, 1e6)*(1 + 0.5*x0/0.1)", "")], top.area),
          (bot.mask, bot.kind, 0b10, [None, ("-1e6", "")], bot.area)]
    g = _gpu_with(case, ex, drop=(0, 1))
    o = _oracle_with(case, ex, drop=(0, 1))
    g.step(300)
    o.step(300)
    u_o = o.read("U")
    assert np.abs(g.read_state("U") - u_o).max() <= 1e-8 * np.abs(u_o).max()
    assert np.abs(g.read_state("S") - o.read("S")).max() <= 1e-6  # damaged to s ~ 0.03, which amplifies rounding


def test_persistent_mode_refuses_expression_conditions():
    case = _plate()
    g = _gpu_with(case, [(case.bcs[1].mask, 0, 0b01, [("1.0", "")], 0.0)], drop=(1,), mode=tlsph.MODE_PERSISTENT)
    with pytest.raises(tlsph.TLSPHError):
        g.step(4)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_LAUNCH)
    g.step(4)


@pytest.mark.parametrize("precision", [tlsph.FP64, tlsph.FP32_U64])
def test_initial_velocity_from_expression(precision):
    X, _ = W.lattice((44, 4), 5e-3, origin=(-0.02, 0.0))
    n = X.shape[0]
    case = W.Case("beam", 2, 5e-3, 7.5e-3, 0.3, W.DT_CFL_STATIC, 0.0,
                  [W.Material(model=W.MODEL_SVK, rho=1000.0, E=2e6, nu=0.4, beta1=0.0)], X, np.full(n, 25e-6),
                  np.zeros_like(X), np.zeros(n, np.int32), None)
    g = tlsph.from_case(case, precision=precision)
    e = g.expr_compile(CANTILEVER_EXPR, CANTILEVER_LOCALS)
    g.apply_expr("V", [-1, e])
    want, _ = Expression(CANTILEVER_EXPR, CANTILEVER_LOCALS).evaluate(x0=X[:, 0], t=0.0)
    v = g.read_state("V")
    tol = 1e-15 if precision == tlsph.FP64 else 1e-7
    assert np.allclose(v[:, 1], want, rtol=tol, atol=tol * 0.57) and np.all(v[:, 0] == 0.0)
    g.apply_expr("U", [g.expr_compile("1e-4*x0"), -1])
    assert np.allclose(g.read_state("U")[:, 0], 1e-4 * X[:, 0], rtol=1e-15, atol=0)


@pytest.mark.parametrize("integrator", [1, 2])
def test_expression_conditions_3d_match_oracle(integrator):
    """A 3D NH block: the bottom face held by an expression over every particle, the top face pulled with a
    time- and position-dependent velocity in z and x."""
    case = W.block_3d(nx=7, ny=6, nz=5, jitter=0.05, seed=4, precision="fp64", beta1=0.2)
    case.materials = [W.Material(model=W.MODEL_NH, rho=7850.0, E=200e9, nu=0.3, beta1=0.2)]
    case.integrator = integrator
    top = case.bcs[1].mask
    dz = case.dp
    ex = [(np.ones(case.n, np.uint8), 0, 0b111, [("if(z0 < dx, 0, skip)", "")] * 3, 0.0),
          (top, 0, 0b101, [("0.2*sin(w*t)*y0/0.006", "w = 3e5"), None, ("-2*min1", "w = 3e5; min1 = 1 - cos(w*t)")],
           0.0)]
    g = _gpu_with(case, ex, drop=(0, 1))
    o = _oracle_with(case, ex, drop=(0, 1))
    g.step(200)
    o.step(200)
    u_o = o.read("U")
    assert np.abs(g.read_state("U") - u_o).max() <= 1e-8 * np.abs(u_o).max()
    assert np.abs(u_o[case.X0[:, 2] < dz]).max() == 0.0


def test_expression_conditions_with_specimen_clocks():
    """Batched specimens keep their own clocks (and step sizes): an expression condition on every particle
    sees its own specimen's t and dt, in the library as in the oracle."""
    case = W.batched(nspec=6, n_min=40, n_max=300, seed=4, precision="fp64")
    ex = [(np.ones(case.n, np.uint8), 0, 0b10, [None, ("if(x0 < 2.5*dx, 1e3*t + 0.01*dt/1e-7, skip)", "")], 0.0)]
    g = _gpu_with(case, ex)
    o = _oracle_with(case, ex)
    g.step(150)
    o.step(150)
    u_o = o.read("U")
    assert np.abs(g.read_state("U") - u_o).max() <= 1e-8 * np.abs(u_o).max()
    ts = [g.time(s) for s in range(6)]
    assert len({round(t[1], 18) for t in ts}) > 1  # the specimens do run on different steps
