"""Pins of the oracle's expression evaluator (Sec. 3.3, user-defined expressions) against facts that do
not come from it: textbook values, Python's own parser on random expressions, the paper's skip
examples and the cantilever mode shape the paper builds with an expression."""
import math

import numpy as np
import pytest

from oracle.expr import VARIABLES, Expression, ExprError, particle_variables
from paper_2602_15149_b300 import workloads as W


def ev(src, locals_="", **v):
    val, skip = Expression(src, locals_).evaluate(**v)
    return val, skip


@pytest.mark.parametrize("src,want", [
    ("1+2*3", 7.0), ("(1+2)*3", 9.0), ("10/4/5", 0.5), ("10-4-3", 3.0), ("2^3^2", 512.0), ("-2^2", -4.0),
    ("2^-1", 0.5), ("-3*-2", 6.0), ("2*-3^2", -18.0), ("1.5e2+.5", 150.5), ("log(1000)", 3.0), ("ln(1)", 0.0),
    ("pow(2,10)", 1024.0), ("sqrt(16)", 4.0), ("abs(-3)", 3.0), ("cot(1)", 1 / math.tan(1)),
    ("coth(2)", 1 / math.tanh(2)), ("1<2 and 3<2", 0.0), ("1<2 or 3<2", 1.0), ("1 or 0 and 0", 1.0),
    ("(1 or 0) and 0", 0.0), ("2==2", 1.0), ("2!=2", 0.0), ("1<=1", 1.0), ("1>=2", 0.0), ("3>2>0", 1.0),
    ("1+1<3 and 2*2==4", 1.0), ("if(0,1,2)", 2.0), ("if(-0.5,1,2)", 1.0), ("if(1<2,if(0,5,6),7)", 6.0),
])
def test_textbook_values(src, want):
    val, skip = ev(src)
    assert not skip.any()
    assert val[0] == pytest.approx(want, rel=1e-15, abs=1e-15)


def test_variables_and_locals():
    X0 = np.array([[0.1, 0.2], [0.3, -0.4]])
    u = np.array([[1e-3, 0.0], [0.0, 2e-3]])
    v = particle_variables(X0, u, 0.5, 1e-6, 1e-3)
    val, _ = ev("x0 + 10*y0 + 100*x + 1000*uy + t + dt/dx", **v)
    ref = X0[:, 0] + 10 * X0[:, 1] + 100 * (X0[:, 0] + u[:, 0]) + 1000 * u[:, 1] + 0.5 + 1e-3
    assert np.allclose(val, ref, rtol=1e-15)
    val, _ = ev("a*b", "a = 2; b = a + x0", **v)
    assert np.allclose(val, 2 * (2 + X0[:, 0]))
    assert ev("z + uz + z0", **v)[0].tolist() == [0.0, 0.0]


def test_skip_semantics():
    x0 = np.array([-1.0, 0.0, 1.0])
    # a clamp: zero left of the wall, nothing elsewhere
    val, skip = ev("if(x0 < 0, 0, skip)", x0=x0)
    assert skip.tolist() == [False, True, True] and val[0] == 0.0
    val, skip = ev("if(x0 <= 0, 0, if(t <= 0, 5, skip))", x0=x0, t=0.0)
    assert skip.tolist() == [False, False, False] and val.tolist() == [0.0, 0.0, 5.0]
    val, skip = ev("if(x0 <= 0, 0, if(t <= 0, 5, skip))", x0=x0, t=1.0)
    assert skip.tolist() == [False, False, True]
    assert ev("1 + skip")[1].all() and ev("if(skip, 1, 2)")[1].all() and ev("sin(Skip)")[1].all()
    assert not ev("if(1, 3, skip)")[1].any()  # the branch not taken does nothing
    assert ev("a", "a = skip")[1].all() and not ev("1", "a = skip")[1].any()


@pytest.mark.parametrize("src", ["1+", "(1+2", "foo(1)", "sin(1,2)", "pow(1)", "x0 y0", "1 $ 2", "q + 1",
                                 "if(1,2)", "and"])
def test_errors(src):
    with pytest.raises(ExprError):
        Expression(src)


def test_bad_locals():
    for loc in ("sin = 1", "x0 = 2", "a b = 1", "a"):
        with pytest.raises(ExprError):
            Expression("1", loc)


# ---- random expressions against Python's own parser -------------------------------------------------
_PREC = {"or": 1, "and": 2, "<": 3, ">": 3, "<=": 3, ">=": 3, "==": 3, "!=": 3, "+": 4, "-": 4, "*": 5, "/": 5,
         "^": 6}
_F1 = ["sin", "cos", "tan", "sinh", "cosh", "tanh", "cot", "coth", "sqrt", "abs", "log", "ln"]


def _gen(rng, depth):
    r = rng.random()
    if depth == 0 or r < 0.2:
        if rng.random() < 0.5:
            return ("num", float(np.round(rng.uniform(-3, 3), 3)))
        return ("var", VARIABLES[rng.integers(len(VARIABLES))])
    r = rng.random()
    if r < 0.55:
        op = list(_PREC)[rng.integers(len(_PREC))]
        return (op, _gen(rng, depth - 1), _gen(rng, depth - 1))
    if r < 0.65:
        return ("neg", _gen(rng, depth - 1))
    if r < 0.8:
        return ("call", _F1[rng.integers(len(_F1))], _gen(rng, depth - 1))
    if r < 0.87:
        return ("call", "pow", _gen(rng, depth - 1), _gen(rng, depth - 1))
    return ("if", _gen(rng, depth - 1), _gen(rng, depth - 1), _gen(rng, depth - 1))


def _paper(node, ctx=0, right=False):
    """The paper's syntax with only the parentheses the precedence table needs."""
    op = node[0]
    if op == "num":
        s = repr(node[1])
        return f"({s})" if node[1] < 0 else s
    if op == "var":
        return node[1]
    if op == "neg":
        s = "-" + _paper(node[1], 5.5)
        return f"({s})" if ctx > 5.5 or ctx == 5.5 and right else s
    if op == "call":
        return node[1] + "(" + ",".join(_paper(a) for a in node[2:]) + ")"
    if op == "if":
        return "if(" + ",".join(_paper(a) for a in node[1:]) + ")"
    p = _PREC[op]
    if op == "^":  # right-associative: parenthesise a left operand of equal precedence
        s = _paper(node[1], p + 0.1) + "^" + _paper(node[2], p, True)
    else:
        s = _paper(node[1], p) + f" {op} " + _paper(node[2], p + 0.1)
    return f"({s})" if p < ctx else s


def _py(node):
    """Fully parenthesised Python with the same meaning (floats, NaN on domain errors)."""
    op = node[0]
    if op == "num":
        return repr(node[1])
    if op == "var":
        return f"V[{node[1]!r}]"
    if op == "neg":
        return f"(-{_py(node[1])})"
    if op == "call":
        return f"F[{node[1]!r}](" + ",".join(_py(a) for a in node[2:]) + ")"
    if op == "if":
        return f"({_py(node[2])} if ({_py(node[1])}) != 0.0 else {_py(node[3])})"
    a, b = _py(node[1]), _py(node[2])
    if op == "^":
        return f"F['pow']({a},{b})"
    if op == "/":
        return f"F['div']({a},{b})"
    if op == "and":
        return f"float(({a}) != 0.0 and ({b}) != 0.0)"
    if op == "or":
        return f"float(({a}) != 0.0 or ({b}) != 0.0)"
    if op in ("<", ">", "<=", ">=", "==", "!="):
        return f"float(({a}) {op} ({b}))"
    return f"F['fin']({a} {op} {b})"


class _Domain(Exception):
    pass


def _safe(f):
    """Python's math routine, with any domain error or non-finite intermediate ending the case (IEEE and
    Python disagree there, and the comparison is about parsing)."""
    def g(*a):
        try:
            r = f(*a)
        except (ValueError, ZeroDivisionError, OverflowError):
            raise _Domain
        if isinstance(r, complex) or not math.isfinite(r):
            raise _Domain
        return float(r)
    return g


def _pyfuncs():
    import math as m
    F = {"sin": m.sin, "cos": m.cos, "tan": m.tan, "sinh": m.sinh, "cosh": m.cosh, "tanh": m.tanh,
         "cot": lambda a: 1.0 / m.tan(a), "coth": lambda a: 1.0 / m.tanh(a), "sqrt": m.sqrt, "abs": abs,
         "log": m.log10, "ln": m.log, "pow": m.pow, "div": lambda a, b: a / b, "fin": lambda a: a}
    return {k: _safe(f) for k, f in F.items()}


def test_random_expressions_against_python():
    """2000 random trees: the oracle parses the minimally parenthesised text into the same values Python
    gives for the fully parenthesised one (trees whose evaluation leaves the finite reals are dropped)."""
    rng = np.random.default_rng(7)
    F = _pyfuncs()
    checked = 0
    for _ in range(2000):
        tree = _gen(rng, 4)
        V = {k: float(np.round(rng.uniform(-2, 2), 3)) for k in VARIABLES}
        try:
            ref = eval(_py(tree), {"F": F, "V": V})
        except (_Domain, OverflowError):
            continue
        if not math.isfinite(ref):
            continue
        val, skip = Expression(_paper(tree)).evaluate(**V)
        assert not skip.any()
        assert val[0] == pytest.approx(ref, rel=1e-12, abs=1e-12), (_paper(tree), val[0], ref)
        checked += 1
    assert checked > 1000


# ---- the cantilever's initial velocity (eq. freeoscivel) is the first bending mode ---------------------
CANTILEVER_LOCALS = W.CANTILEVER_MODE_LOCALS
CANTILEVER_EXPR = W.CANTILEVER_MODE


def test_cantilever_expression_is_the_first_mode():
    """v(x0) = 0.01 cs f(x0)/f(L0) (eq. freeoscivel written as an expression): 0 and slope 0 at the clamp,
    0.57 m/s at the tip, and (k_w L0 = 1.875 being the first root of 1 + cos cosh = 0 to four digits) nearly
    zero curvature at the free end."""
    e = Expression(CANTILEVER_EXPR, CANTILEVER_LOCALS)
    L0, h = 0.2, 1e-4

    def v(x):
        val, skip = e.evaluate(x0=np.asarray(x, float), t=0.0)
        assert not skip.any()
        return val

    assert v([L0])[0] == pytest.approx(0.57, rel=1e-14)
    assert v([-0.01, 0.0]).tolist() == [0.0, 0.0]
    small = v([1e-4])[0]
    assert 0 < small < 1e-5  # f ~ x^2 near the clamp: value and slope vanish
    d2 = (v([L0 - 2 * h])[0] - 2 * v([L0 - h])[0] + v([L0])[0]) / h ** 2
    d2_mid = (v([0.1 - h])[0] - 2 * v([0.1])[0] + v([0.1 + h])[0]) / h ** 2
    assert abs(d2) < 0.02 * abs(d2_mid)


# ---- expressions as boundary conditions in the oracle's step ------------------------------------------
from tests.oracle_cases import make_oracle  # noqa: E402


def _plate(integrator=1, pull_ramp=False):
    case = W.plate_2d(nx=30, ny=8, beta1=0.2)
    if not pull_ramp:
        case.bcs[1].ramp = 0.0
    case.integrator = integrator
    return case


def _run(case, steps, exbcs=(), drop=()):
    bcs = [b for k, b in enumerate(case.bcs) if k not in drop]
    c = W.Case(**{**case.__dict__, "bcs": bcs})
    o = make_oracle(c)
    for mask, kind, cm, exprs in exbcs:
        o.add_bc_expr(mask, kind, cm, exprs)
    o.step(steps)
    return o


def test_constant_expressions_equal_constant_conditions():
    """The clamp and the pull written as expressions give bit-identical runs (Algorithms 1 and 2)."""
    for integ in (1, 2):
        case = _plate(integ)
        ref = _run(case, 150).read("U")
        left, right = case.bcs[0].mask, case.bcs[1].mask
        zero = Expression("0")
        pull = Expression(repr(case.bcs[1].value[0]))
        got = _run(case, 150, [(left, 0, 0b11, [zero, zero]), (right, 0, 0b01, [pull])], drop=(0, 1)).read("U")
        assert np.array_equal(got, ref)
        # the clamp as one expression over every particle, skipping all but the left column
        clamp = Expression("if(x0 < dx, 0, skip)")
        everyone = np.ones(case.n, np.uint8)
        got = _run(case, 150, [(everyone, 0, 0b11, [clamp, clamp])], drop=(0,)).read("U")
        assert np.array_equal(got, ref)


def test_skipped_condition_does_nothing():
    case = _plate()
    ref = _run(case, 100).read("U")
    got = _run(case, 100, [(np.ones(case.n, np.uint8), 0, 0b11, [Expression("skip"), Expression("Skip")])]).read("U")
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("integrator", [1, 2])
def test_time_dependent_velocity_integrates_exactly(integrator):
    """v_x = A sin(w t) on the right edge.  Algorithm 1 prescribes v_{n+1} at t_{n+1}, so u_N = sum_k dt v(t_k),
    k = 1..N; Algorithm 2 adds dt/2 (v_n + v_{n+1}) with v_0 = 0 (the trapezoid rule)."""
    case = _plate(integrator)
    A, w, N = 0.3, 2e5, 120
    o = _run(case, N, [(case.bcs[1].mask, 0, 0b01, [Expression(f"{A}*sin({w}*t)")])], drop=(1,))
    _, dt = o.time()
    tk = dt * np.arange(N + 1)
    v = A * np.sin(w * tk)
    want = dt * v[1:].sum() if integrator == 1 else 0.5 * dt * (v[:-1] + v[1:]).sum()
    ux = o.read("U")[case.bcs[1].mask.astype(bool), 0]
    assert np.allclose(ux, want, rtol=1e-12, atol=0)
    assert abs(want) > 1e-9


def test_traction_expression_equals_constant_traction():
    case = W.notched_plate(nx=40, ny=16, steps=100)
    ref = _run(case, 100).read("U")
    top, bot = case.bcs[0], case.bcs[1]
    o = make_oracle(W.Case(**{**case.__dict__, "bcs": []}))
    o.add_bc_expr(top.mask, top.kind, top.comp_mask, [None, Expression(repr(top.value[1]))], area=top.area)
    o.add_bc_expr(bot.mask, bot.kind, bot.comp_mask, [None, Expression(repr(bot.value[1]))], area=bot.area)
    o.step(100)
    assert np.array_equal(o.read("U"), ref)


def test_initial_velocity_from_the_cantilever_expression():
    """apply_expr sets v at t = 0 from the paper's expression; the clamped part (x0 <= 0) gets 0."""
    X, _ = W.lattice((44, 4), 5e-3, origin=(-0.02, 0.0))
    case = W.Case("beam", 2, 5e-3, 7.5e-3, 0.3, W.DT_CFL_STATIC, 0.0, [W.Material(model=W.MODEL_SVK)], X,
                  np.full(X.shape[0], 25e-6), np.zeros_like(X), np.zeros(X.shape[0], np.int32), None)
    o = make_oracle(case)
    e = Expression(CANTILEVER_EXPR, CANTILEVER_LOCALS)
    o.apply_expr("V", [None, e])
    v = o.read("V")
    want, _ = e.evaluate(x0=X[:, 0], t=0.0)
    assert np.array_equal(v[:, 1], want) and np.all(v[:, 0] == 0.0)
    assert np.all(v[X[:, 0] <= 0.0, 1] == 0.0) and v[:, 1].max() > 0.5
