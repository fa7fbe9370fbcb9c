"""Batched form: many independent specimens in one launch, execution modes, autotuner.

* a small batch of uneven 2D specimens (NH and J2) against the FP64 oracle;
* a specimen run alone and inside a batch gives bit-identical fields (specimens never
  interact and each keeps its own clock);
* kernel launches, a replayed CUDA graph and the persistent cooperative launch give
  bit-identical results;
* the autotuner leaves no trace in the state;
* the persistent launch's grid barrier gives up after its time limit and reports
  TLSPH_ERR_TIMEOUT, leaving the context usable (the barrier waits for a block that is
  never launched: nothing faults or hangs).
"""
import copy

import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def small_batch(nspec=8, seed=11):
    return W.batched(nspec=nspec, n_min=200, n_max=1500, seed=seed)


def specimen_alone(case, s):
    """The particles, material and boundary conditions of specimen s of a batch, as their own case."""
    sel = case.specimen_id == s
    idx = np.nonzero(sel)[0]
    sub = copy.copy(case)
    sub.X0 = case.X0[idx].copy()
    sub.vol = case.vol[idx].copy()
    sub.v0 = case.v0[idx].copy()
    sub.material_id = np.zeros(len(idx), np.int32)
    sub.materials = [case.materials[int(case.material_id[idx[0]])]]
    sub.specimen_id = None
    sub.bcs = [W.BC(b.mask[idx], b.kind, b.comp_mask, b.value, b.t_start, b.t_end, b.ramp, b.area)
               for b in case.bcs]
    sub.specimen_loads = [W.BC(case.specimen_loads[s].mask[idx], case.specimen_loads[s].kind,
                               case.specimen_loads[s].comp_mask, case.specimen_loads[s].value,
                               ramp=case.specimen_loads[s].ramp)]
    return sub, idx


def test_batch_matches_oracle():
    case = small_batch()
    o = make_oracle(case)
    g = tlsph.from_case(case)
    o.step(500)
    g.step(500)
    assert rel_l2(g.read_state("U"), o.read("U")) <= 1e-4
    assert rel_l2(g.read_state("V"), o.read("V")) <= 1e-4
    for s in range(8):  # every specimen has its own clock
        to, dto = o.time(s)
        tg, dtg = g.time(s)
        assert dtg == dto and abs(tg - to) <= 1e-12 * to
    assert len({round(g.time(s)[1], 20) for s in range(8)}) > 1  # the step sizes differ


def test_specimen_alone_equals_in_batch():
    case = small_batch(6, seed=4)
    g = tlsph.from_case(case)
    g.step(200)
    U = g.read_state("U")
    for s in (0, 3, 5):
        sub, idx = specimen_alone(case, s)
        a = tlsph.from_case(sub)
        a.step(200)
        assert np.array_equal(a.read_state("U"), U[idx])
        assert a.time() == g.time(s)


@pytest.mark.parametrize("which", ["block", "batch", "notched"])
def test_execution_modes_bit_identical(which):
    case = {"block": lambda: W.block_3d(nx=14, ny=12, nz=9),
            "batch": lambda: small_batch(5, seed=2),
            "notched": lambda: W.notched_plate(nx=60, ny=24)}[which]()
    ref = None
    for mode, block in [(tlsph.MODE_LAUNCH, 128), (tlsph.MODE_LAUNCH, 64), (tlsph.MODE_GRAPH, 128),
                        (tlsph.MODE_PERSISTENT, 128), (tlsph.MODE_PERSISTENT, 256)]:
        g = tlsph.from_case(case)
        g.set_option(tlsph.OPT_MODE, mode)
        g.set_option(tlsph.OPT_BLOCK, block)
        g.step(51)
        g.step(24)
        out = (g.read_state("U"), g.read_state("V"), g.read_state("S"), g.time())
        if ref is None:
            ref = out
        else:
            assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
            assert np.array_equal(out[2], ref[2]) and out[3] == ref[3]


def test_autotune_leaves_no_trace():
    case = small_batch(6, seed=8)
    a = tlsph.from_case(case)
    a.step(50)
    ref = a.read_state("U")
    b = tlsph.from_case(case)
    b.step(20)
    best, allt = b.autotune(trial_steps=5)
    assert best["ms_per_step"] > 0 and len(allt) == 6
    assert all(np.isfinite(t["ms_per_step"]) for t in allt)
    assert b.get_info()["steps"] == 20
    b.step(30)
    assert np.array_equal(b.read_state("U"), ref)


def test_persistent_barrier_timeout_is_a_status():
    case = W.block_3d(nx=10, ny=10, nz=8)
    g = tlsph.from_case(case)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_PERSISTENT)
    g.set_option(tlsph.OPT_BARRIER_TEST, 1)
    st = g.step(3, check=False)
    assert st == tlsph.ERR_TIMEOUT
    g.set_option(tlsph.OPT_BARRIER_TEST, 0)
    assert g.step(5, check=False) == tlsph.OK
    assert np.all(np.isfinite(g.read_state("U")))
