"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/tlsph.h declares.

No compute calls are made here (no GPU needed): only argument validation that
returns before any device work.
"""
import ctypes
import os
import re

import pytest

from paper_2602_15149_b300 import build, tlsph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tlsph_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return tlsph.load_library()


def test_every_declared_symbol_is_exported(lib):
    decl = declared_functions()
    assert len(decl) >= 20
    missing = [n for n in decl if not hasattr(lib, n)]
    assert not missing
    assert sorted(tlsph.EXPORTS) == decl


def test_argument_errors_without_device_work(lib):
    ctx = ctypes.c_void_p()
    bad = tlsph.Params(4, 1, 1, 1e-3, 2.0, 0.3, 2, 0.0, (ctypes.c_double * 3)(0, 0, 0), None, 0)
    assert lib.tlsph_create(ctypes.byref(bad), ctypes.byref(ctx)) == tlsph.ERR_ARG
    neg_h = tlsph.Params(3, 1, 1, -1.0, 2.0, 0.3, 2, 0.0, (ctypes.c_double * 3)(0, 0, 0), None, 0)
    assert lib.tlsph_create(ctypes.byref(neg_h), ctypes.byref(ctx)) == tlsph.ERR_ARG
    assert lib.tlsph_create(None, ctypes.byref(ctx)) == tlsph.ERR_ARG
    assert lib.tlsph_step(None, 1) == tlsph.ERR_ARG
    assert lib.tlsph_nnz(None) == -1
    assert lib.tlsph_field_bytes(None, 0) == -1
    lib.tlsph_destroy(None)


def test_library_targets_sm103a():
    cmd = build.nvcc_command()
    assert "arch=compute_103a,code=sm_103a" in " ".join(cmd)
    assert os.path.exists(build.LIB)


def test_expr_check_accepts_what_the_oracle_parses():
    """The library's expression compiler (no GPU needed) accepts and rejects the same texts as the oracle's
    parser: the paper's examples, error cases, and random expressions of the full grammar."""
    import numpy as np
    from oracle.expr import Expression, ExprError
    from paper_2602_15149_b300 import tlsph
    from tests.test_oracle_expr import CANTILEVER_EXPR, CANTILEVER_LOCALS, _gen, _paper
    cases = [(CANTILEVER_EXPR, CANTILEVER_LOCALS), ("if(x0 < 0, 0, skip)", ""), ("a*b", "a = 2; b = a + x0"),
             ("2^-1", ""), ("-2^2", ""), ("1 or 0 and 0", ""), ("1+", ""), ("(1+2", ""), ("foo(1)", ""),
             ("sin(1,2)", ""), ("pow(1)", ""), ("x0 y0", ""), ("1 $ 2", ""), ("q + 1", ""), ("if(1,2)", ""),
             ("and", ""), ("1", "sin = 1"), ("1", "x0 = 2"), ("1", "a b = 1"), ("1", "a"), ("", ""), ("1e", ""),
             ("1.5.3", ""), (".5e-3*dx", "")]
    rng = np.random.default_rng(3)
    cases += [(_paper(_gen(rng, 5)), "") for _ in range(300)]
    for src, loc in cases:
        try:
            Expression(src, loc)
            want_ok = True
        except ExprError:
            want_ok = False
        msg = tlsph.expr_check(src, loc)
        assert (msg is None) == want_ok, (src, loc, msg)
        if msg is not None:
            assert msg
