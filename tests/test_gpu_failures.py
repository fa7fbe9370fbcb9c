"""Failure detection without faulting a GPU: faults are made on the host (bad inputs, an allocation cap,
a non-finite state written into the context) and each must come back as a status with a message, with
the context still usable afterwards.  The bounded grid-barrier wait of the persistent mode is covered in
tests/test_gpu_batched.py."""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W

pytestmark = pytest.mark.gpu


def _ctx(case, precision=tlsph.FP64):
    t = tlsph.TLSPH(case.dim, case.h, precision, dx=case.dp)
    t.set_materials(case.materials)
    return t


def test_coincident_particles_are_refused_then_fixed():
    case = W.plate_2d(nx=12, ny=5)
    X = case.X0.copy()
    X[7] = X[6]
    t = _ctx(case)
    t.create_particles(X, case.vol)
    with pytest.raises(tlsph.TLSPHError) as e:
        t.build_ref_neighbours()
    assert e.value.status == tlsph.ERR_ARG and "reference position" in str(e.value)
    t.create_particles(case.X0, case.vol)
    t.build_ref_neighbours()
    t.step(10)


def test_bad_materials_and_notches():
    case = W.notched_plate(nx=20, ny=8)
    t = tlsph.TLSPH(case.dim, case.h, tlsph.FP64)
    m = case.materials[0]
    for kw in ({"nu": 0.5}, {"E": -1.0}, {"rho": 0.0}):
        bad = W.Material(**{**m.__dict__, **kw})
        with pytest.raises(tlsph.TLSPHError) as e:
            t.set_materials([bad])
        assert e.value.status == tlsph.ERR_ARG
    t.set_materials(case.materials)
    t.create_particles(case.X0, case.vol)
    q = np.array(case.notches[0], dtype=float).reshape(12)
    q[4] = np.inf
    with pytest.raises(tlsph.TLSPHError) as e:
        t.add_notch(q)
    assert e.value.status == tlsph.ERR_ARG


def test_allocation_failure_is_a_status():
    """A 1 MiB cap makes the setup's allocations fail with TLSPH_ERR_OOM; lifting it, the same context
    builds and steps, bit-identically to a fresh one."""
    case = W.block_3d(nx=12, ny=10, nz=8)
    g = tlsph.from_case(case, build=False)
    g.set_option(tlsph.OPT_MEMORY_LIMIT, 1)
    with pytest.raises(tlsph.TLSPHError) as e:
        g.build_ref_neighbours()
    assert e.value.status == tlsph.ERR_OOM
    with pytest.raises(tlsph.TLSPHError) as e:
        g.step(1)
    assert e.value.status == tlsph.ERR_STATE
    g.set_option(tlsph.OPT_MEMORY_LIMIT, 0)
    g.build_ref_neighbours()
    g.step(50)
    ref = tlsph.from_case(case)
    ref.step(50)
    assert np.array_equal(g.read_state("U"), ref.read_state("U"))
    with pytest.raises(tlsph.TLSPHError):
        g.set_option(tlsph.OPT_MEMORY_LIMIT, -1)


def test_non_finite_state_is_reported_and_recoverable():
    """A NaN written into the displacement makes the next step report TLSPH_ERR_NONFINITE; writing a clean
    checkpoint back, the context steps on and matches a run that never saw the NaN."""
    case = W.plate_2d(nx=20, ny=6)
    g = tlsph.from_case(case, precision=tlsph.FP64)
    g.step(20)
    blob = g.read_state("STATE").copy()
    u = g.read_state("U")
    u[3, 0] = np.nan
    g.write_state("U", u)
    st = g.step(5, check=False)
    assert st == tlsph.ERR_NONFINITE
    g.write_state("STATE", blob)
    assert g.step(30, check=False) == tlsph.OK
    ref = tlsph.from_case(case, precision=tlsph.FP64)
    ref.step(50)
    assert np.array_equal(g.read_state("U"), ref.read_state("U"))
