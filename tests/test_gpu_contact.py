"""Contact between bodies (reading of Sec. 3.3 <contcoeff>, <restcoef>) on the sm_103a path against the
FP64 oracle, through the C-ABI, and the paper's flyer-plate impact (Sec. 4) at its published size.

Parity: two touching 8 x 8 plates colliding (FP64 within 1e-8 of the largest displacement, FP32 within
1e-4), both integrators, and the same plates sliding past each other with friction (<kfric>); momentum
conserved to rounding; launch and graph modes bit-identical.
Flyer plate: what the paper states about its run (the figures carry no numbers) -- plasticity starts at
the contact interface, the impact is symmetric about the mid-plane, and the plates spread laterally.
"""
import numpy as np
import pytest

from paper_2602_15149_b300 import tlsph, workloads as W
from tests.oracle_cases import make_oracle
from tests.test_oracle_contact import _plates

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-8), (tlsph.FP32_U64, 1e-4)])
def test_colliding_plates_match_oracle(integrator, precision, tol):
    case = _plates(0.8, v=2.0)
    case.integrator = integrator
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    for _ in range(3):  # approach, impact, rebound
        o.step(100)
        g.step(100)
        u_o = o.read("U")
        assert np.abs(g.read_state("U") - u_o).max() <= tol * np.abs(u_o).max()
        v_o = o.read("V")
        assert np.abs(g.read_state("V") - v_o).max() <= tol * np.abs(v_o).max()


def _sliding_plates(kfric, v_shear=1.0):
    """The touching 8 x 8 plates of the parity test, closing at 2 x 2 m/s and sliding past each other at
    2 x v_shear along the contact plane, with friction coefficient kfric on both bodies."""
    case = W.flyer_plate(n=8, dx=1e-3, gap=0.0, v=2.0, restitution=0.8, model="nh", precision="fp64",
                         kfric=kfric, v_shear=v_shear)
    case.cfl = 0.05
    return case


@pytest.mark.parametrize("integrator", [1, 2])
@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-8), (tlsph.FP32_U64, 1e-4)])
def test_sliding_plates_with_friction_match_oracle(precision, tol, integrator):
    # friction acts at the level of the forces: t_n under Algorithm 1, the half level under Algorithm 2
    case = _sliding_plates(0.3)
    case.integrator = integrator
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    for _ in range(3):
        o.step(100)
        g.step(100)
        for f in ("U", "V"):
            a = o.read(f)
            assert np.abs(g.read_state(f) - a).max() <= tol * np.abs(a).max(), f


def test_friction_slows_the_sliding_and_keeps_momentum():
    """With friction the plates' relative sliding speed drops during the contact (without it, it does not
    change beyond what the impact's elastic waves carry), and the total momentum is kept to rounding."""
    out = {}
    for mu in (0.0, 0.5):
        case = _sliding_plates(mu)
        m = case.materials[0].rho * case.vol
        g = tlsph.from_case(case, precision=tlsph.FP64)
        p0 = (m[:, None] * g.read_state("V")).sum(axis=0)
        g.step(300)
        v = g.read_state("V")
        p = (m[:, None] * v).sum(axis=0)
        assert np.abs(p - p0).max() <= 1e-12 * (m * 3.0).sum()
        lo = case.specimen_id == 0
        out[mu] = v[lo, 0].mean() - v[~lo, 0].mean()
    assert out[0.5] < 0.8 * out[0.0], out


@pytest.mark.parametrize("kfric", [0.0, 0.4])
def test_momentum_and_modes(kfric):
    # launch and graph modes share the contact launches: bit-identical with and without friction
    case = _plates(0.8, v=2.0) if kfric == 0.0 else _sliding_plates(kfric)
    m = case.materials[0].rho * case.vol
    out = []
    for mode in (tlsph.MODE_LAUNCH, tlsph.MODE_GRAPH):
        g = tlsph.from_case(case, precision=tlsph.FP64)
        g.set_option(tlsph.OPT_MODE, mode)
        p0 = (m[:, None] * g.read_state("V")).sum(axis=0)
        for _ in range(3):
            g.step(100)
            p = (m[:, None] * g.read_state("V")).sum(axis=0)
            assert np.abs(p - p0).max() <= 1e-12 * (m * 3.0).sum()
        out.append((g.read_state("U"), g.read_state("V")))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    g = tlsph.from_case(case, precision=tlsph.FP64)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_PERSISTENT)
    with pytest.raises(tlsph.TLSPHError):
        g.step(2)


def test_friction_arguments_are_checked():
    case = _sliding_plates(None)
    g = tlsph.from_case(case, precision=tlsph.FP64, build=False)
    g2 = tlsph.TLSPH(case.dim, case.h, tlsph.FP64, dx=case.dp)
    g2.set_materials(case.materials)
    g2.create_particles(case.X0, case.vol, specimen_id=case.specimen_id)
    with pytest.raises(tlsph.TLSPHError) as e:  # no contact yet
        g2._ck(g2.lib.tlsph_set_contact_friction(g2.ctx, 2, tlsph._d(np.array([0.1, 0.1]))), "friction")
    assert e.value.status == tlsph.ERR_STATE
    for bad in ([0.1], [0.1, -0.2], [0.1, np.inf], [np.nan, 0.0]):
        with pytest.raises(tlsph.TLSPHError) as e:
            g.set_contact(case.contact["contcoeff"], case.contact["restitution"], bad)
        assert e.value.status == tlsph.ERR_ARG
    g.set_contact(case.contact["contcoeff"], case.contact["restitution"], [0.0, 0.0])  # zero = none
    g.build_ref_neighbours()
    ref = tlsph.from_case(case, precision=tlsph.FP64)
    g.step(50)
    ref.step(50)
    assert np.array_equal(g.read_state("U"), ref.read_state("U"))


def test_contact_needs_a_shared_clock():
    case = _plates(0.8)
    case.dt_mode = W.DT_ADAPTIVE
    with pytest.raises(tlsph.TLSPHError):
        tlsph.from_case(case, precision=tlsph.FP64)


def test_flyer_plate_as_published():
    """Two 100 x 100 J2 plates at +-200 m/s (FP32), run to 300 us: impact at about 125 us (0.05 m closed at
    400 m/s), plastic strain first at the contact rows, a symmetric state, lateral spreading at the
    interface, momentum still zero."""
    case = W.flyer_plate()
    g = tlsph.from_case(case)
    g.set_option(tlsph.OPT_MODE, tlsph.MODE_GRAPH)
    n = 100
    m = n * n
    X = case.X0
    t, first_plastic, ep = 0.0, None, None
    while t < 300e-6:
        g.step(200)
        t, _ = g.time()
        ep = g.read_state("EPSP")
        if first_plastic is None and ep.max() > 0.0:
            first_plastic = (t, np.nonzero(ep > 0.5 * ep.max())[0])
    assert first_plastic is not None and 110e-6 < first_plastic[0] < 160e-6
    rows = np.rint(X[first_plastic[1], 1] / case.dp - 0.5).astype(int)
    assert np.all((rows >= n - 3) & (rows < n + 3 + 5))  # the rows at the interface (the gap is 5 rows)
    u = g.read_state("U")
    lo, hi = u[:m].reshape(n, n, 2), u[m:].reshape(n, n, 2)[::-1]
    scale = np.abs(u).max()
    assert np.abs(hi[..., 0] - lo[..., 0]).max() <= 1e-3 * scale
    assert np.abs(hi[..., 1] + lo[..., 1]).max() <= 1e-3 * scale
    # the interface rows widen (barrelling): the outer columns move outwards
    assert u[:m].reshape(n, n, 2)[n - 1, n - 1, 0] > 0 and u[:m].reshape(n, n, 2)[n - 1, 0, 0] < 0
    v = g.read_state("V")
    rho = case.materials[0].rho
    p = (rho * case.vol[:, None] * v).sum(axis=0)
    assert np.abs(p).max() <= 1e-4 * rho * case.vol.sum() * 200.0
    assert g.get_info()["nonfinite"] == 0


@pytest.mark.parametrize("precision,tol", [(tlsph.FP64, 1e-8), (tlsph.FP32_U64, 1e-4)])
def test_colliding_blocks_3d_match_oracle(precision, tol):
    """Two 5 x 4 x 5 NH blocks stacked along y, touching, closing at 4 m/s (the 3D contact stiffness carries
    the spacing: k = contcoeff E* dc)."""
    n = (5, 4, 5)
    lo, _ = W.lattice(n, 1e-3)
    hi, _ = W.lattice(n, 1e-3, origin=(0.0, n[1] * 1e-3, 0.0))
    X = np.vstack([lo, hi])
    m = lo.shape[0]
    v0 = np.zeros_like(X)
    v0[:m, 1], v0[m:, 1] = 2.0, -2.0
    spec = np.repeat(np.array([0, 1], np.int32), m)
    mat = W.Material(model=W.MODEL_NH, rho=7870.0, E=200e9, nu=0.29, beta1=0.05)
    case = W.Case("blocks_3d_contact", 3, 1e-3, 1.5e-3, 0.05, W.DT_CFL_STATIC, 0.0, [mat], X, np.full(2 * m, 1e-9),
                  v0, np.zeros(2 * m, np.int32), spec, [], [], 300, "fp64")
    case.contact = {"contcoeff": 5.0, "restitution": [0.9, 0.7]}
    o = make_oracle(case)
    g = tlsph.from_case(case, precision=precision)
    for _ in range(3):
        o.step(100)
        g.step(100)
        u_o = o.read("U")
        assert np.abs(g.read_state("U") - u_o).max() <= tol * np.abs(u_o).max()
    assert o.contact_energy() >= 0.0
