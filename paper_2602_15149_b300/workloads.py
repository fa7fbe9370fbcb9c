"""Seeded synthetic inputs for the TLSPH step (arXiv 2602.15149).

This module only lays out particles, materials, boundary conditions and
notches.  It holds none of the method's arithmetic; both the CUDA library and
the CPU oracle receive the same arrays from here.

Recipes (the paper's own workloads use CAD geometry that is not available, so
these lattices stand in for them at the same scale):

* ``plate_2d``      -- 2D plane-strain elastic plate, square lattice
  X = ((i + 1/2) dp, (j + 1/2) dp), no jitter; neo-Hookean (or St. Venant-
  Kirchhoff); left edge clamped,
  right edge pulled in x at ``v_pull`` with a linear ramp over ``ramp_steps``
  steps (100 x 20 particles, dp = 1 mm is the full case).
* ``block_3d``      -- 3D block, lattice jittered by U(-jitter dp, +jitter dp)
  per axis from ``numpy.random.default_rng(seed)``; J2 plasticity; bottom face
  fixed, top face pressed down at ``v_press`` (128 x 128 x 64 is the full case).
* ``notched_plate`` -- 2D plate 0.1 x 0.04 m with an edge notch of length
  0.05 m at mid-height, phase-field fracture of a neo-Hookean (or St. Venant-
  Kirchhoff) solid, +-1 MPa traction on the top and bottom rows (500 x 200
  particles is the full case).
* ``crack_branching`` -- the paper's dynamic crack-branching benchmark (Sec. 4,
  crack branching): the notched plate in plane strain at dx = 0.0625 mm
  (1600 x 640 = 1,024,000 particles), St. Venant-Kirchhoff, eps0 = 2 dx,
  s_l = 0.05, C_CFL = 0.2, beta1 = 0.2, constant 1 MPa traction, run to 80-120 us.
* ``cantilever_beam`` -- the paper's freely oscillating cantilever (Sec. 4,
  free oscillation of a cantilever beam): a 0.2 x 0.02 m plane-strain SVK beam
  (mu = 0.715 MPa, kappa = 3.25 MPa, rho = 1000) whose columns with x0 <= 0
  (1.5 mm) are held by expression conditions, started with the first-mode
  velocity profile of eq. freeoscivel through an expression initial field.
* ``flyer_plate``   -- the paper's flyer-plate impact (Sec. 4): two 1 x 1 m
  plane-strain J2 steel plates 0.05 m apart (100 x 100 particles each at
  dx = 0.01 m) closing at +-200 m/s, contact between the two bodies
  (contcoeff 5, restitution 0.95), Courant number 0.01.
* ``taylor_bar``    -- the paper's 3D Taylor impact (Sec. 4): a copper-like J2
  cylinder (L0 = 32.4 mm, R0 = 3.2 mm; the lattice cells whose centres lie in
  the cylinder) moving at -227 m/s onto a rigid wall at z = 0, the wall and
  the start given by expressions, Courant number 0.02.
* ``batched``       -- many independent 2D specimens of log-uniform size with
  random materials and loading (512 specimens is the full case).

Ramp lengths are given in steps of 0.3 h / REF_WAVE_SPEED, a fixed reference
speed (the elastic wave speed of the steel of ``plate_2d``, 5,856 m/s), so that
this module computes nothing of the method; for the steel cases this is the
solvers' own ``cfl_static`` step.
"""
from __future__ import annotations

import copy
import math
from dataclasses import dataclass, field

import numpy as np

REF_WAVE_SPEED = 5856.0  # m/s, sets ramp durations (see the module docstring)

MODEL_SVK, MODEL_NH, MODEL_J2 = 1, 2, 3
_MODELS = {"svk": MODEL_SVK, "nh": MODEL_NH}
BC_VEL, BC_TRACTION, BC_ACCEL, BC_POINTFORCE, BC_PHASE_BOUND = 0, 1, 2, 3, 4
DT_FIXED, DT_ADAPTIVE, DT_CFL_STATIC = 0, 1, 2


@dataclass
class Material:
    model: int = MODEL_NH
    rho: float = 7850.0
    E: float = 200e9
    nu: float = 0.3
    sigma_y0: float = 0.0
    H_hard: float = 0.0
    beta1: float = 0.2
    beta2: float = 0.0
    fracture: int = 0
    Gc: float = 0.0
    eps0: float = 0.0
    s_lim: float = 0.1


@dataclass
class BC:
    mask: np.ndarray            # uint8 per particle
    kind: int                   # BC_*
    comp_mask: int              # bit k -> component k
    value: tuple                # 3 values
    t_start: float = 0.0
    t_end: float = -1.0         # < 0: no end
    ramp: float = 0.0           # linear ramp time, 0 = step
    area: float = 0.0           # traction: area per particle


@dataclass
class ExprBC:
    """A boundary condition whose components are user-defined expressions: (text, locals) or None each."""
    mask: np.ndarray
    kind: int
    comp_mask: int
    exprs: list
    t_start: float = 0.0
    t_end: float = -1.0
    area: float = 0.0


@dataclass
class Case:
    name: str
    dim: int
    dp: float
    h: float
    cfl: float
    dt_mode: int
    fixed_dt: float
    materials: list
    X0: np.ndarray              # (n, dim) float64
    vol: np.ndarray             # (n,) float64
    v0: np.ndarray              # (n, dim) float64
    material_id: np.ndarray     # (n,) int32
    specimen_id: np.ndarray | None
    bcs: list = field(default_factory=list)
    notches: list = field(default_factory=list)
    steps: int = 1000
    precision: str = "fp32"     # "fp64" or "fp32" (fp32 fields, fp64 displacement)
    gravity: tuple = (0.0, 0.0, 0.0)
    integrator: int = 1         # 1: Algorithm 1 (symplectic Euler), 2: Algorithm 2 (leapfrog)
    expr_bcs: list = field(default_factory=list)  # ExprBC
    expr_ics: list = field(default_factory=list)  # (field "U" or "V", [(text, locals) or None per component])
    contact: dict | None = None  # {"contcoeff": kc, "restitution": [e per specimen], optional "kfric": [mu per
    #                              specimen]}: bodies = specimens

    @property
    def n(self) -> int:
        return int(self.X0.shape[0])


def lattice(shape, dp, jitter=0.0, seed=0, origin=None):
    """Particles at ((i + 1/2) dp, ...) with id = i + nx (j + ny k); optional uniform jitter."""
    dim = len(shape)
    idx = np.indices(shape[::-1]).reshape(dim, -1)[::-1].T.astype(np.float64)  # x fastest
    X = (idx + 0.5) * dp
    if origin is not None:
        X = X + np.asarray(origin, dtype=np.float64)
    if jitter:
        rng = np.random.default_rng(seed)
        X = X + rng.uniform(-jitter * dp, jitter * dp, size=X.shape)
    return np.ascontiguousarray(X), idx.astype(np.int64)


def plate_2d(nx=100, ny=20, dp=1e-3, v_pull=1.0, ramp_steps=100, steps=1000, precision="fp64",
             beta1=1.0, beta2=0.0, model="nh"):
    """2D plane-strain hyperelastic plate (``model`` "nh" or "svk"), left edge clamped, right edge
    pulled (ramped)."""
    X, idx = lattice((nx, ny), dp)
    n = X.shape[0]
    mat = Material(model=_MODELS[model], rho=7850.0, E=200e9, nu=0.3, beta1=beta1, beta2=beta2)
    h = 1.5 * dp
    dt = 0.3 * h / REF_WAVE_SPEED
    left = (idx[:, 0] == 0).astype(np.uint8)
    right = (idx[:, 0] == nx - 1).astype(np.uint8)
    bcs = [BC(left, BC_VEL, 0b11, (0.0, 0.0, 0.0)),
           BC(right, BC_VEL, 0b01, (v_pull, 0.0, 0.0), ramp=ramp_steps * dt)]
    return Case("plate_2d_" + model, 2, dp, h, 0.3, DT_CFL_STATIC, 0.0, [mat], X, np.full(n, dp * dp),
                np.zeros((n, 2)), np.zeros(n, np.int32), None, bcs, [], steps, precision)


def block_3d(nx=128, ny=128, nz=64, dp=1e-3, jitter=0.01, seed=2602, v_press=5.0, steps=2000,
             precision="fp32", sigma_y0=250e6, H_hard=1e9, beta1=0.2):
    """3D J2 block: bottom face fixed, top face pressed down at v_press."""
    X, idx = lattice((nx, ny, nz), dp, jitter=jitter, seed=seed)
    n = X.shape[0]
    mat = Material(model=MODEL_J2, rho=7850.0, E=200e9, nu=0.3, sigma_y0=sigma_y0, H_hard=H_hard, beta1=beta1)
    bottom = (idx[:, 2] == 0).astype(np.uint8)
    top = (idx[:, 2] == nz - 1).astype(np.uint8)
    bcs = [BC(bottom, BC_VEL, 0b111, (0.0, 0.0, 0.0)),
           BC(top, BC_VEL, 0b100, (0.0, 0.0, -v_press))]
    return Case("block_3d_j2", 3, dp, 1.5 * dp, 0.3, DT_CFL_STATIC, 0.0, [mat], X, np.full(n, dp ** 3),
                np.zeros((n, 3)), np.zeros(n, np.int32), None, bcs, [], steps, precision)


def notched_plate(nx=500, ny=200, width=0.1, height=0.04, notch_len=0.05, traction=1e6, steps=4000,
                  precision="fp32", s_lim=0.1, beta1=0.2, model="nh"):
    """2D phase-field plate with an edge notch at mid-height, pulled by +-traction on top/bottom rows
    (``model`` "nh" or "svk" for the degraded hyperelastic law)."""
    dp = width / nx
    assert abs(dp * ny - height) < 1e-12 * height
    X, idx = lattice((nx, ny), dp)
    n = X.shape[0]
    mat = Material(model=_MODELS[model], rho=2450.0, E=32e9, nu=0.2, beta1=beta1, fracture=1, Gc=3.0,
                   eps0=2.0 * dp, s_lim=s_lim)
    top = (idx[:, 1] == ny - 1).astype(np.uint8)
    bot = (idx[:, 1] == 0).astype(np.uint8)
    area = dp * 1.0  # unit thickness
    bcs = [BC(top, BC_TRACTION, 0b10, (0.0, traction, 0.0), area=area),
           BC(bot, BC_TRACTION, 0b10, (0.0, -traction, 0.0), area=area)]
    y0 = 0.5 * height
    notch = [(0.0, y0, 0.0), (notch_len, y0, 0.0), (notch_len, y0, 1.0), (0.0, y0, 1.0)]
    return Case("notched_plate_pf" if model == "nh" else "notched_plate_pf_" + model, 2, dp, 1.5 * dp, 0.3, DT_CFL_STATIC, 0.0, [mat], X, np.full(n, dp * dp),
                np.zeros((n, 2)), np.zeros(n, np.int32), None, bcs, [np.array(notch, dtype=np.float64)], steps,
                precision)


def crack_branching(nx=1600, ny=640, t_end=80e-6, precision="fp32"):
    """The paper's crack-branching case: the 100 x 40 mm notched plate with the degraded SVK law,
    its soft-particle limit (0.05) and Courant number (0.2).  ``steps`` is only a size hint (t_end
    over 0.2 h / REF_WAVE_SPEED); runs of this case stop on the simulated time instead."""
    case = notched_plate(nx=nx, ny=ny, traction=1e6, precision=precision, s_lim=0.05, beta1=0.2, model="svk")
    case.name = "crack_branching_svk"
    case.cfl = 0.2
    case.steps = int(math.ceil(t_end / (0.2 * case.h / REF_WAVE_SPEED)))
    return case


# The first bending mode as an initial velocity (eq. freeoscivel): v(X1) = 0.01 c_s f(X1) / f(L0) with
# f(x) = [cos kL + cosh kL][cosh kx - cos kx] + [sin kL - sinh kL][sinh kx - sin kx], k L0 = 1.875, and the
# clamp at X1 <= 0.  Written as the expression language's (text, locals); c_s = 57 m/s as the paper states.
CANTILEVER_MODE_LOCALS = ("L = 0.2; k = 1.875 / L; A = 0.01 * 57.0; c1 = cos(k*L) + cosh(k*L); "
                          "s1 = sin(k*L) - sinh(k*L); fL = c1*(cosh(k*L) - cos(k*L)) + s1*(sinh(k*L) - sin(k*L))")
CANTILEVER_MODE = "if(x0 <= 0, 0, A * (c1*(cosh(k*x0) - cos(k*x0)) + s1*(sinh(k*x0) - sin(k*x0))) / fL)"
CANTILEVER_CLAMP = "if(x0 <= 0, 0, skip)"


def cantilever_beam(dx=0.5e-3, L0=0.2, H0=0.02, clamp=1.5e-3, steps=20000, precision="fp64"):
    """The paper's 2D cantilever (x along the beam, y transverse): lattice from x = -clamp to L0, the columns
    with x0 <= 0 held at zero velocity by expression conditions, the first-mode transverse velocity as an
    expression initial field.  SVK with mu = 0.715 MPa, kappa = 3.25 MPa (E = 9 kappa mu / (3 kappa + mu),
    nu = (3 kappa - 2 mu) / (2 (3 kappa + mu)) written out below), rho = 1000, artificial viscosity
    (0.015, 0.01), Courant number 0.2."""
    nx, ny = int(round((L0 + clamp) / dx)), int(round(H0 / dx))
    X, _ = lattice((nx, ny), dx, origin=(-clamp, 0.0))
    n = X.shape[0]
    mat = Material(model=MODEL_SVK, rho=1000.0, E=1998447.2049689442, nu=0.39751552795031053, beta1=0.015,
                   beta2=0.01)
    case = Case("cantilever_beam_svk", 2, dx, 1.5 * dx, 0.2, DT_CFL_STATIC, 0.0, [mat], X, np.full(n, dx * dx),
                np.zeros((n, 2)), np.zeros(n, np.int32), None, [], [], steps, precision)
    mode = (CANTILEVER_MODE, CANTILEVER_MODE_LOCALS)
    clampx = (CANTILEVER_CLAMP, "")
    case.expr_bcs = [ExprBC(np.ones(n, np.uint8), BC_VEL, 0b11, [clampx, clampx])]
    case.expr_ics = [("V", [None, mode])]
    return case


def flyer_plate(n=100, dx=0.01, gap=0.05, v=200.0, steps=20000, precision="fp32", contcoeff=5.0, restitution=0.95,
                model="j2", kfric=None, v_shear=0.0):
    """Two identical square plates (specimens 0 and 1 = the two bodies) moving towards each other along y;
    the lower one at +v, the upper one at -v.  J2 steel as the paper's case (rho 7870, E 200 GPa, nu 0.29,
    sigma_y0 400 MPa, H 100 MPa, artificial viscosity 0.05), or "nh" for the same elastic constants.
    kfric: friction coefficient of both bodies (None = the paper's default, none); v_shear: the plates also
    slide past each other along x at +-v_shear."""
    lo, _ = lattice((n, n), dx)
    hi, _ = lattice((n, n), dx, origin=(0.0, n * dx + gap))
    X = np.vstack([lo, hi])
    m = n * n
    spec = np.concatenate([np.zeros(m, np.int32), np.ones(m, np.int32)])
    v0 = np.zeros((2 * m, 2))
    v0[:m, 1] = v
    v0[m:, 1] = -v
    v0[:m, 0] = v_shear  # optional sliding of the lower plate along the contact plane
    v0[m:, 0] = -v_shear
    mat = Material(model=MODEL_J2 if model == "j2" else MODEL_NH, rho=7870.0, E=200e9, nu=0.29,
                   sigma_y0=400e6 if model == "j2" else 0.0, H_hard=100e6 if model == "j2" else 0.0, beta1=0.05)
    case = Case("flyer_plate_" + model, 2, dx, 1.5 * dx, 0.01, DT_CFL_STATIC, 0.0, [mat], X, np.full(2 * m, dx * dx), v0,
                np.zeros(2 * m, np.int32), spec, [], [], steps, precision)
    case.contact = {"contcoeff": contcoeff, "restitution": [restitution, restitution]}
    if kfric is not None:  # <kfric> per body (the paper's case leaves it at 0)
        case.contact["kfric"] = [kfric, kfric]
    return case


def taylor_bar(dx=0.4e-3, L0=32.4e-3, R0=3.2e-3, v=227.0, steps=40000, precision="fp32"):
    """The paper's Taylor bar: lattice cells of the box [-R0, R0]^2 x [0, L0] whose centres lie within R0 of the
    axis.  A particle whose current z is below 3/4 dx (the layer on the wall) has no axial velocity; every other
    particle starts at -v along z.  J2 with rho 8930, E 117 GPa, nu 0.35, sigma_y0 400 MPa, H 100 MPa,
    artificial viscosity 0.05."""
    nxy, nz = int(math.ceil(2 * R0 / dx)), int(round(L0 / dx))
    X, _ = lattice((nxy, nxy, nz), dx, origin=(-nxy * dx / 2, -nxy * dx / 2, 0.0))
    X = np.ascontiguousarray(X[X[:, 0] ** 2 + X[:, 1] ** 2 <= R0 ** 2])
    n = X.shape[0]
    mat = Material(model=MODEL_J2, rho=8930.0, E=117e9, nu=0.35, sigma_y0=400e6, H_hard=100e6, beta1=0.05)
    case = Case("taylor_bar_j2", 3, dx, 1.5 * dx, 0.02, DT_CFL_STATIC, 0.0, [mat], X, np.full(n, dx ** 3),
                np.zeros((n, 3)), np.zeros(n, np.int32), None, [], [], steps, precision)
    wall = ("if(z < 0.75*dx, 0, skip)", "")
    case.expr_bcs = [ExprBC(np.ones(n, np.uint8), BC_VEL, 0b100, [None, None, wall])]
    case.expr_ics = [("V", [None, None, ("if(z < 0.75*dx, 0, -v0)", f"v0 = {v!r}")])]
    return case


def batched(nspec=512, n_min=500, n_max=50000, dp=1e-3, seed=0, steps=1000, precision="fp32"):
    """Independent 2D specimens laid side by side (each its own specimen id).

    Per specimen s (seeded by ``seed + s``): N_s = round(exp(U(ln n_min, ln n_max))), aspect U(1, 4),
    E log-U(1, 200) GPa, nu U(0.2, 0.45), Neo-Hookean or J2 with p = 1/2 (sigma_y0 U(100, 500) MPa,
    H = 1 GPa), rho = 7850, one clamped edge and a different loaded edge (velocity log-U(0.1, 5) m/s
    along the edge normal, ramped over 100 steps).  Specimens are ordered by size.
    """
    specs = []
    for s in range(nspec):
        rng = np.random.default_rng(seed + s)
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        aspect = rng.uniform(1.0, 4.0)
        ny = max(3, int(round(math.sqrt(N / aspect))))
        nx = max(3, int(round(N / ny)))
        E = math.exp(rng.uniform(math.log(1e9), math.log(200e9)))
        nu = rng.uniform(0.2, 0.45)
        j2 = rng.uniform() < 0.5
        sy = rng.uniform(100e6, 500e6)
        sides = rng.permutation(4)[:2]
        rate = math.exp(rng.uniform(math.log(0.1), math.log(5.0)))
        specs.append((nx * ny, nx, ny, E, nu, j2, sy, int(sides[0]), int(sides[1]), rate))
    specs.sort(key=lambda t: t[0])
    Xs, mids, sids, bc_clamp, bc_load, mats, loads = [], [], [], [], [], [], []
    x_off = 0.0
    for s, (N, nx, ny, E, nu, j2, sy, clamp, load, rate) in enumerate(specs):
        X, idx = lattice((nx, ny), dp, origin=(x_off, 0.0))
        x_off += (nx + 4) * dp  # specimens never touch (gap > support radius)
        m = Material(model=MODEL_J2 if j2 else MODEL_NH, rho=7850.0, E=E, nu=nu, sigma_y0=sy if j2 else 0.0,
                     H_hard=1e9 if j2 else 0.0, beta1=0.2)
        mats.append(m)
        edges = [idx[:, 0] == 0, idx[:, 0] == nx - 1, idx[:, 1] == 0, idx[:, 1] == ny - 1]
        normals = [(-1.0, 0.0), (1.0, 0.0), (0.0, -1.0), (0.0, 1.0)]
        Xs.append(X)
        mids.append(np.full(X.shape[0], s, np.int32))
        sids.append(np.full(X.shape[0], s, np.int32))
        bc_clamp.append(edges[clamp])
        bc_load.append(edges[load])
        loads.append((load, rate, normals[load], REF_WAVE_SPEED))
    X0 = np.concatenate(Xs)
    n = X0.shape[0]
    clamp_mask = np.concatenate(bc_clamp).astype(np.uint8)
    bcs = [BC(clamp_mask, BC_VEL, 0b11, (0.0, 0.0, 0.0))]
    # one loaded-edge BC per specimen (its own edge, direction and rate), ramped over 100
    # reference steps
    case = Case("batched_2d", 2, dp, 1.5 * dp, 0.3, DT_CFL_STATIC, 0.0, mats, X0, np.full(n, dp * dp),
                np.zeros((n, 2)), np.concatenate(mids), np.concatenate(sids), bcs, [], steps, precision)
    case.specimen_loads = []
    off = 0
    for s, X in enumerate(Xs):
        load, rate, nrm, c = loads[s]
        mask = np.zeros(n, np.uint8)
        mask[off:off + X.shape[0]] = bc_load[s]
        dt = 0.3 * case.h / c
        case.specimen_loads.append(BC(mask, BC_VEL, 0b01 if nrm[0] != 0.0 else 0b10,
                                      (rate * nrm[0], rate * nrm[1], 0.0), ramp=100 * dt))
        off += X.shape[0]
    return case


def subset(case: Case, specimens) -> Case:
    """The given specimens of a batched case as a case of their own (specimens renumbered
    0 .. k-1 in the given order's sorted order; materials, boundary conditions and loads kept).
    A rank of a multi-GPU run takes its share of the specimens this way."""
    keep = np.sort(np.asarray(list(specimens), dtype=np.int64))
    sel = np.isin(case.specimen_id, keep)
    idx = np.nonzero(sel)[0]
    renum = np.full(int(case.specimen_id.max()) + 1, -1, np.int64)
    renum[keep] = np.arange(keep.size)
    sub = copy.copy(case)
    sub.X0 = case.X0[idx].copy()
    sub.vol = case.vol[idx].copy()
    sub.v0 = case.v0[idx].copy()
    sub.material_id = case.material_id[idx].copy()
    sub.specimen_id = renum[case.specimen_id[idx]].astype(np.int32)
    sub.bcs = [BC(b.mask[idx], b.kind, b.comp_mask, b.value, b.t_start, b.t_end, b.ramp, b.area) for b in case.bcs]
    loads = getattr(case, "specimen_loads", [])
    sub.specimen_loads = [BC(loads[s].mask[idx], loads[s].kind, loads[s].comp_mask, loads[s].value,
                             ramp=loads[s].ramp) for s in keep] if loads else []
    return sub

