"""Oracle: user-defined expressions (Sec. 3.3, user-defined expressions; the tables of built-in
variables, functions and operators with precedence).

TEST INFRASTRUCTURE.  Only tests/, the smoke check and the benchmark's CPU legs use this module.  It is
a plain recursive-descent parser that evaluates directly on numpy arrays (one value per particle),
written from the paper's description and independent of the library's bytecode compiler.

Language (as the paper lists it):

* variables x0 y0 z0 (initial position), x y z (current position), ux uy uz (displacement),
  t (time), dt (time step), dx (particle spacing);
* numbers, parentheses, + - * / and ^ (exponentiation, right-associative);
* comparisons < > <= >= == != and the logical operators ``and``, ``or`` (1 for true, 0 for false; a
  value is true when it is not 0);
* functions sin cos tan cot sinh cosh tanh coth sqrt abs, log (base 10), ln (natural), pow(x, y) and
  the conditional if(c, a, b);
* the keyword ``skip`` / ``Skip``: a branch that does nothing;
* locals ``name = expression; ...`` evaluated in order before the expression.

Precedence, lowest first: or (1), and (2), comparisons (3), + - (4), * / (5), ^ (6); all left-associative
except ^.  Readings where the paper is silent:

* unary minus binds looser than ^ and tighter than * and / (so -2^2 = -4 and 2^-1 = 0.5);
* skip is a property of a value: an operation on a skipped operand gives a skipped result, if() with a
  skipped condition is skipped, and only the branch if() takes is evaluated, so a skip in the other
  branch has no effect.  A skipped result leaves the quantity the expression sets untouched;
* arithmetic is IEEE double (division by zero gives inf or nan, pow of a negative base with a
  non-integer exponent gives nan).
"""
from __future__ import annotations

import re

import numpy as np

VARIABLES = ("x0", "y0", "z0", "x", "y", "z", "ux", "uy", "uz", "t", "dt", "dx")

_FUNCS1 = {
    "sin": np.sin, "cos": np.cos, "tan": np.tan,
    "cot": lambda a: 1.0 / np.tan(a),
    "sinh": np.sinh, "cosh": np.cosh, "tanh": np.tanh,
    "coth": lambda a: 1.0 / np.tanh(a),
    "sqrt": np.sqrt, "abs": np.abs,
    "log": np.log10, "ln": np.log,
}
_FUNCS2 = {"pow": np.power}
_KEYWORDS = {"and", "or", "if", "skip", "Skip"}

_TOKEN = re.compile(r"\s*(?:(?P<num>(?:\d+\.?\d*|\.\d+)(?:[eE][+-]?\d+)?)|(?P<id>[A-Za-z_][A-Za-z_0-9]*)"
                    r"|(?P<op><=|>=|==|!=|[-+*/^<>(),]))")


class ExprError(ValueError):
    pass


def _tokens(src):
    pos, out = 0, []
    src = src.rstrip()
    while pos < len(src):
        m = _TOKEN.match(src, pos)
        if not m or m.end() == pos:
            raise ExprError(f"unexpected character at {pos}: {src[pos:pos + 10]!r}")
        kind = m.lastgroup
        out.append((kind, m.group(kind), m.start(kind)))
        pos = m.end()
    out.append(("end", None, len(src)))
    return out


class _Parser:
    """Recursive descent over the precedence table; builds a tree of tuples."""

    def __init__(self, src, names):
        self.toks = _tokens(src)
        self.k = 0
        self.names = names  # locals defined so far

    def peek(self):
        return self.toks[self.k]

    def take(self, kind=None, value=None):
        tok = self.toks[self.k]
        if (kind and tok[0] != kind) or (value is not None and tok[1] != value):
            raise ExprError(f"expected {value or kind} at {tok[2]}, found {tok[1]!r}")
        self.k += 1
        return tok

    def parse(self):
        node = self.or_expr()
        if self.peek()[0] != "end":
            raise ExprError(f"unexpected {self.peek()[1]!r} at {self.peek()[2]}")
        return node

    def or_expr(self):
        node = self.and_expr()
        while self.peek()[:2] == ("id", "or"):
            self.take()
            node = ("or", node, self.and_expr())
        return node

    def and_expr(self):
        node = self.cmp_expr()
        while self.peek()[:2] == ("id", "and"):
            self.take()
            node = ("and", node, self.cmp_expr())
        return node

    def cmp_expr(self):
        node = self.add_expr()
        while self.peek()[0] == "op" and self.peek()[1] in ("<", ">", "<=", ">=", "==", "!="):
            op = self.take()[1]
            node = (op, node, self.add_expr())
        return node

    def add_expr(self):
        node = self.mul_expr()
        while self.peek()[0] == "op" and self.peek()[1] in ("+", "-"):
            op = self.take()[1]
            node = (op, node, self.mul_expr())
        return node

    def mul_expr(self):
        node = self.unary()
        while self.peek()[0] == "op" and self.peek()[1] in ("*", "/"):
            op = self.take()[1]
            node = (op, node, self.unary())
        return node

    def unary(self):
        if self.peek()[0] == "op" and self.peek()[1] in ("-", "+"):
            op = self.take()[1]
            inner = self.unary()
            return ("neg", inner) if op == "-" else inner
        return self.power()

    def power(self):
        base = self.primary()
        if self.peek()[0] == "op" and self.peek()[1] == "^":
            self.take()
            return ("^", base, self.unary())  # right-associative; the exponent may carry a sign
        return base

    def primary(self):
        kind, val, pos = self.peek()
        if kind == "num":
            self.take()
            return ("num", float(val))
        if kind == "op" and val == "(":
            self.take()
            node = self.or_expr()
            self.take("op", ")")
            return node
        if kind == "id":
            self.take()
            if val in ("skip", "Skip"):
                return ("skip",)
            if val == "if":
                self.take("op", "(")
                c = self.or_expr()
                self.take("op", ",")
                a = self.or_expr()
                self.take("op", ",")
                b = self.or_expr()
                self.take("op", ")")
                return ("if", c, a, b)
            if val in _FUNCS1 or val in _FUNCS2:
                self.take("op", "(")
                args = [self.or_expr()]
                while self.peek()[:2] == ("op", ","):
                    self.take()
                    args.append(self.or_expr())
                self.take("op", ")")
                want = 1 if val in _FUNCS1 else 2
                if len(args) != want:
                    raise ExprError(f"{val} takes {want} argument(s), got {len(args)} at {pos}")
                return ("call", val, *args)
            if val in self.names:
                return ("local", val)
            if val in VARIABLES:
                return ("var", val)
            raise ExprError(f"unknown name {val!r} at {pos}")
        raise ExprError(f"unexpected {val!r} at {pos}")


def _eval(node, env, n):
    """(value array, skip mask) of a tree node; env maps names to (value, skip)."""
    op = node[0]
    if op == "num":
        return np.full(n, node[1]), np.zeros(n, bool)
    if op == "skip":
        return np.zeros(n), np.ones(n, bool)
    if op in ("var", "local"):
        return env[node[1]]
    if op == "neg":
        v, s = _eval(node[1], env, n)
        return -v, s
    if op == "call":
        args = [_eval(a, env, n) for a in node[2:]]
        f = _FUNCS1.get(node[1]) or _FUNCS2[node[1]]
        sk = np.zeros(n, bool)
        for _, s in args:
            sk = sk | s
        return f(*[v for v, _ in args]), sk
    if op == "if":
        c, cs = _eval(node[1], env, n)
        take = c != 0.0
        v = np.zeros(n)
        s = cs.copy()
        if take.any():  # only the particles that take a branch evaluate it (the result is the same)
            av, ask = _eval(node[2], env, n)
            v = np.where(take, av, v)
            s = s | (take & ask)
        if (~take).any():
            bv, bsk = _eval(node[3], env, n)
            v = np.where(take, v, bv)
            s = s | (~take & bsk)
        return v, s
    a, sa = _eval(node[1], env, n)
    b, sb = _eval(node[2], env, n)
    s = sa | sb
    if op == "+":
        return a + b, s
    if op == "-":
        return a - b, s
    if op == "*":
        return a * b, s
    if op == "/":
        return a / b, s
    if op == "^":
        return np.power(a, b), s
    if op == "<":
        return (a < b).astype(float), s
    if op == ">":
        return (a > b).astype(float), s
    if op == "<=":
        return (a <= b).astype(float), s
    if op == ">=":
        return (a >= b).astype(float), s
    if op == "==":
        return (a == b).astype(float), s
    if op == "!=":
        return (a != b).astype(float), s
    if op == "and":
        return ((a != 0.0) & (b != 0.0)).astype(float), s
    if op == "or":
        return ((a != 0.0) | (b != 0.0)).astype(float), s
    raise ExprError(f"bad node {op}")


class Expression:
    """A parsed expression with its locals."""

    def __init__(self, expr: str, locals_: str = ""):
        self.locals = []
        names = set()
        for part in [p for p in locals_.split(";") if p.strip()]:
            if "=" not in part:
                raise ExprError(f"local without '=': {part!r}")
            name, rhs = part.split("=", 1)
            name = name.strip()
            if not re.fullmatch(r"[A-Za-z_][A-Za-z_0-9]*", name) or name in _KEYWORDS or name in _FUNCS1 \
                    or name in _FUNCS2 or name in VARIABLES:
                raise ExprError(f"bad local name {name!r}")
            self.locals.append((name, _Parser(rhs, set(names)).parse()))
            names.add(name)
        self.tree = _Parser(expr, names).parse()

    def evaluate(self, **vars_):
        """Evaluate over arrays of the built-in variables (each scalar or shape (n,); missing ones are 0).
        Returns (values, skip) as arrays of shape (n,)."""
        n = max([np.size(v) for v in vars_.values()] + [1])
        env = {}
        for name in VARIABLES:
            v = np.broadcast_to(np.asarray(vars_.get(name, 0.0), dtype=np.float64), (n,)).copy()
            env[name] = (v, np.zeros(n, bool))
        with np.errstate(all="ignore"):
            for name, tree in self.locals:
                env[name] = _eval(tree, env, n)
            return _eval(self.tree, env, n)


def particle_variables(X0, u, t, dt, dx):
    """The built-in variables of every particle: X0 and u of shape (n, dim); t, dt per particle or scalar."""
    d = X0.shape[1]
    out = {"t": t, "dt": dt, "dx": dx}
    for k, c in enumerate("xyz"):
        x0 = X0[:, k] if k < d else np.zeros(X0.shape[0])
        uk = u[:, k] if k < d else np.zeros(X0.shape[0])
        out[c + "0"] = x0
        out["u" + c] = uk
        out[c] = x0 + uk
    return out
