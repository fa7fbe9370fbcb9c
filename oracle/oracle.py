"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

Mirrors the operations of the C-ABI library (create_particles /
build_ref_neighbours / step / read_state) so that one test harness drives
both; it does not import the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tlsph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_tlsph.so")

MODEL_SVK, MODEL_NH, MODEL_J2 = 1, 2, 3
BC_VEL, BC_TRACTION, BC_ACCEL, BC_POINTFORCE = 0, 1, 2, 3
DT_FIXED, DT_ADAPTIVE, DT_CFL_STATIC = 0, 1, 2
FIELDS = {"U": 0, "V": 1, "X": 2, "S": 3, "SDOT": 4, "H": 5, "EPSP": 6, "P": 7, "F": 8, "FP": 9,
          "L": 10, "ACC": 11, "CPINV": 12, "SDD": 13, "LAP": 14}


class _Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("h", C.c_double), ("support", C.c_double), ("cfl", C.c_double),
                ("dt_mode", C.c_int), ("fixed_dt", C.c_double), ("gravity", C.c_double * 3),
                ("visc_literal", C.c_int), ("lap_uncorrected", C.c_int), ("integrator", C.c_int),
                ("pf_explicit", C.c_int)]


class _Material(C.Structure):
    _fields_ = [("model", C.c_int), ("rho", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("sigma_y0", C.c_double), ("H_hard", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("fracture", C.c_int), ("Gc", C.c_double), ("eps0", C.c_double),
                ("s_lim", C.c_double)]


@dataclass
class OracleMaterial:
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

    def c_struct(self) -> _Material:
        return _Material(self.model, self.rho, self.E, self.nu, self.sigma_y0, self.H_hard, self.beta1,
                         self.beta2, self.fracture, self.Gc, self.eps0, self.s_lim)


def build_oracle(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/liboracle_tlsph.so`` (FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def load_oracle():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build_oracle())
    P, D, I64, I32, U8 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32), \
        C.POINTER(C.c_uint8)
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.POINTER(_Params)]
    lib.orc_destroy.argtypes = [P]
    lib.orc_set_materials.argtypes = [P, C.c_int, C.POINTER(_Material)]
    lib.orc_create_particles.argtypes = [P, C.c_int64, D, D, D, I32, I32]
    lib.orc_add_bc.argtypes = [P, U8, C.c_int, C.c_int, D, C.c_double, C.c_double, C.c_double, C.c_double]
    lib.orc_add_notch.argtypes = [P, D]
    lib.orc_build_neighbours.argtypes = [P, C.c_int]
    lib.orc_nnz.restype = C.c_int64
    lib.orc_nnz.argtypes = [P]
    lib.orc_neighbours.argtypes = [P, I64, I32, C.c_int64]
    lib.orc_perm.argtypes = [P, I64]
    lib.orc_step.argtypes = [P, C.c_int64]
    lib.orc_read.argtypes = [P, C.c_int, D]
    lib.orc_write.argtypes = [P, C.c_int, D]
    lib.orc_energies.argtypes = [P, D]
    lib.orc_noconv.restype = C.c_int64
    lib.orc_noconv.argtypes = [P]
    lib.orc_time.argtypes = [P, C.c_int, D, D]
    lib.orc_expm.argtypes = [D, D]
    lib.orc_wendland.argtypes = [C.c_int, C.c_double, C.c_double, D, D]
    lib.orc_sound_speed.restype = C.c_double
    lib.orc_sound_speed.argtypes = [C.POINTER(_Material)]
    lib.orc_nh_stress.argtypes = [D, C.c_double, C.POINTER(_Material), D, D, D]
    lib.orc_svk_stress.argtypes = [D, C.c_double, C.POINTER(_Material), D, D, D]
    lib.orc_sym_eig3.argtypes = [D, D, D]
    lib.orc_sym_eig3.restype = None
    lib.orc_j2_update.argtypes = [D, D, C.c_double, C.POINTER(_Material), D, D, D, D, C.POINTER(C.c_int)]
    lib.orc_set_bc_values.argtypes = [C.c_void_p, C.c_int, C.c_int, D, C.POINTER(C.c_uint8)]
    lib.orc_set_contact.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_int, D]
    lib.orc_contact_energy.argtypes = [C.c_void_p]
    lib.orc_contact_energy.restype = C.c_double
    lib.orc_contact_force.argtypes = [C.c_int, C.c_double, C.c_double, D, D, D, D, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, D]
    lib.orc_set_contact_friction.argtypes = [C.c_void_p, C.c_int, D]
    lib.orc_prepare_step.argtypes = [C.c_void_p]
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


class Oracle:
    """One FP64 CPU simulation (the oracle)."""

    def __init__(self, dim: int, h: float, cfl: float = 0.3, dt_mode: int = DT_CFL_STATIC,
                 fixed_dt: float = 0.0, gravity=(0.0, 0.0, 0.0), support: float = 2.0,
                 visc_literal: bool = False, lap_uncorrected: bool = False, integrator: int = 1,
                 dx: float | None = None, pf_explicit: bool = False):
        self.lib = load_oracle()
        p = _Params(dim, h, support, cfl, dt_mode, fixed_dt, (C.c_double * 3)(*gravity), int(visc_literal),
                    int(lap_uncorrected), int(integrator), int(pf_explicit))
        self.ctx = self.lib.orc_create(C.byref(p))
        if not self.ctx:
            raise ValueError("invalid oracle parameters")
        self.dim = dim
        self.n = 0
        self.dx = h / 1.5 if dx is None else dx  # the expression variable dx (particle spacing)
        self.integrator = integrator
        self._exbcs = []
        self._nbc = 0

    def __del__(self):
        if getattr(self, "ctx", None):
            self.lib.orc_destroy(self.ctx)
            self.ctx = None

    def set_materials(self, mats):
        arr = (_Material * len(mats))(*[m.c_struct() for m in mats])
        _check(self.lib.orc_set_materials(self.ctx, len(mats), arr), "set_materials")

    def create_particles(self, X0, vol, v0=None, material_id=None, specimen_id=None):
        X0 = np.ascontiguousarray(X0, dtype=np.float64)
        n = X0.shape[0]
        vol = np.ascontiguousarray(vol, dtype=np.float64)
        v0p = None if v0 is None else _dp(np.ascontiguousarray(v0, dtype=np.float64))
        self._keep = [X0, vol]
        if v0 is not None:
            self._keep.append(np.ascontiguousarray(v0, dtype=np.float64))
            v0p = _dp(self._keep[-1])
        mid = np.zeros(n, np.int32) if material_id is None else np.ascontiguousarray(material_id, np.int32)
        sid = None if specimen_id is None else np.ascontiguousarray(specimen_id, np.int32)
        _check(self.lib.orc_create_particles(self.ctx, n, _dp(X0), _dp(vol), v0p,
                                             mid.ctypes.data_as(C.POINTER(C.c_int32)),
                                             None if sid is None else sid.ctypes.data_as(C.POINTER(C.c_int32))),
               "create_particles")
        self.n = n
        self._X0 = X0.copy()
        self._spec = np.zeros(n, np.int64) if sid is None else sid.astype(np.int64)

    def add_bc(self, mask, kind, comp_mask, value, t_start=0.0, t_end=-1.0, ramp=0.0, area=0.0):
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        val = np.zeros(3)
        val[:len(value)] = value
        _check(self.lib.orc_add_bc(self.ctx, m.ctypes.data_as(C.POINTER(C.c_uint8)), kind, comp_mask, _dp(val),
                                   t_start, t_end, ramp, area), "add_bc")
        self._nbc += 1
        return self._nbc - 1

    def add_bc_expr(self, mask, kind, comp_mask, exprs, t_start=0.0, t_end=-1.0, area=0.0):
        """A condition whose component k takes the value of exprs[k] (an oracle.expr.Expression) per particle
        and per step; skipped values leave the component alone.  Velocity values are evaluated at the time
        the step prescribes them (t_{n+1}; Algorithm 2 also t_{n+1/2} for the predictor), force values at
        the time of the forces, all with the displacement at the start of the step."""
        b = self.add_bc(mask, kind, comp_mask, (0.0, 0.0, 0.0), t_start, t_end, 0.0, area)
        self._exbcs.append((b, kind, comp_mask, list(exprs) + [None] * (3 - len(exprs))))
        return b

    def set_contact(self, contcoeff, restitution, dc=None):
        """Contact between bodies (the specimens), reading of Sec. 3.3 <contcoeff>/<restcoef>: a linear
        spring-dashpot normal force between particles of different specimens closer than dc (default the
        particle spacing dx); the specimens then share one clock."""
        r = np.ascontiguousarray(restitution, dtype=np.float64)
        _check(self.lib.orc_set_contact(self.ctx, contcoeff, self.dx if dc is None else dc, r.size, _dp(r)),
               "set_contact")

    def set_contact_friction(self, kfric):
        """Friction coefficient <kfric> per body (Coulomb friction, regularised near rest; reading of Sec. 3.3)."""
        f = np.ascontiguousarray(kfric, dtype=np.float64)
        _check(self.lib.orc_set_contact_friction(self.ctx, f.size, _dp(f)), "set_contact_friction")

    def contact_energy(self):
        return float(self.lib.orc_contact_energy(self.ctx))

    def variables(self, t_offset=0.0):
        """The built-in expression variables of every particle at t_n + t_offset * dt (state at t_n)."""
        from oracle.expr import particle_variables
        nspec = int(self._spec.max()) + 1 if self.n else 1
        ts = np.array([self.time(s) for s in range(nspec)])
        t, dt = ts[self._spec, 0], ts[self._spec, 1]
        return particle_variables(self._X0, self.read("U"), t + t_offset * dt, dt, self.dx)

    def apply_expr(self, field: str, exprs, t_offset=0.0):
        """Set the components of a state field ("U" or "V") to expressions evaluated now (t = the current time,
        dt = the coming step; None or a skipped value leaves a component as it is)."""
        _check(self.lib.orc_prepare_step(self.ctx), "prepare_step")
        vars_ = self.variables(t_offset)
        cur = self.read(field).copy()
        for k, e in enumerate(list(exprs)[:self.dim]):
            if e is None:
                continue
            val, skip = e.evaluate(**vars_)
            cur[~skip, k] = val[~skip]
        self.write(field, cur)

    def _set_expr_values(self):
        _check(self.lib.orc_prepare_step(self.ctx), "prepare_step")
        leap = self.integrator == 2
        for b, kind, cm, exprs in self._exbcs:
            if kind == 0:
                phases = [(0, 1.0)] + ([(1, 0.5)] if leap else [])
            elif kind == 4:  # phase-field bound: the new level s_{n+1} (Algorithm 2: also s_{n+1/2})
                phases = [(0, 1.0)] + ([(1, 0.5)] if leap else [])
            else:
                phases = [(0, 0.5 if leap else 0.0)]
            for phase, off in phases:
                vars_ = self.variables(off)
                val = np.zeros((self.n, 3))
                skip = np.ones((self.n, 3), np.uint8)
                for k in range(3):
                    if (cm >> k) & 1 and exprs[k] is not None:
                        v, sk = exprs[k].evaluate(**vars_)
                        val[:, k] = v
                        skip[:, k] = sk
                _check(self.lib.orc_set_bc_values(self.ctx, b, phase, _dp(val), skip.ctypes.data_as(
                    C.POINTER(C.c_uint8))), "set_bc_values")

    def add_notch(self, quad):
        q = np.ascontiguousarray(quad, dtype=np.float64).reshape(12)
        _check(self.lib.orc_add_notch(self.ctx, _dp(q)), "add_notch")

    def build_ref_neighbours(self, method: int | None = None):
        if method is None:
            method = 0 if self.n <= 20000 else 1
        _check(self.lib.orc_build_neighbours(self.ctx, method), "build_neighbours")

    def neighbours(self):
        nnz = self.lib.orc_nnz(self.ctx)
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        _check(self.lib.orc_neighbours(self.ctx, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                       col.ctypes.data_as(C.POINTER(C.c_int32)), nnz), "neighbours")
        return rp, col[:nnz]

    def perm(self):
        p = np.zeros(self.n, np.int64)
        _check(self.lib.orc_perm(self.ctx, p.ctypes.data_as(C.POINTER(C.c_int64))), "perm")
        return p

    def step(self, nsteps: int = 1):
        if not self._exbcs:
            _check(self.lib.orc_step(self.ctx, nsteps), "step")
            return
        for _ in range(nsteps):  # expressions are evaluated before every step
            self._set_expr_values()
            _check(self.lib.orc_step(self.ctx, 1), "step")

    def read(self, field: str):
        per = {"U": self.dim, "V": self.dim, "X": self.dim, "ACC": self.dim, "P": 9, "F": 9, "FP": 9, "L": 9,
               "CPINV": 9}.get(field, 1)
        out = np.zeros(self.n * per)
        _check(self.lib.orc_read(self.ctx, FIELDS[field], _dp(out)), "read " + field)
        if per == 9:
            return out.reshape(self.n, 3, 3)
        return out.reshape(self.n, per) if per > 1 else out

    def write(self, field: str, values):
        a = np.ascontiguousarray(values, dtype=np.float64).ravel()
        _check(self.lib.orc_write(self.ctx, FIELDS[field], _dp(a)), "write " + field)

    def energies(self):
        out = np.zeros(6)
        _check(self.lib.orc_energies(self.ctx, _dp(out)), "energies")
        return {"KE": out[0], "SE": out[1], "FE": out[2], "PW": out[3], "Wext": out[4], "t": out[5],
                "dt": self.time()[1]}

    def time(self, spec: int = 0):
        t, dt = C.c_double(), C.c_double()
        _check(self.lib.orc_time(self.ctx, spec, C.byref(t), C.byref(dt)), "time")
        return t.value, dt.value

    def noconv(self) -> int:
        return int(self.lib.orc_noconv(self.ctx))


# ---- pointwise routines (for pin tests) -------------------------------------------------
def expm(A):
    lib = load_oracle()
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    out = np.zeros(9)
    lib.orc_expm(_dp(A), _dp(out))
    return out.reshape(3, 3)


def wendland(dim, h, r):
    lib = load_oracle()
    W, dW = C.c_double(), C.c_double()
    lib.orc_wendland(dim, h, r, C.byref(W), C.byref(dW))
    return W.value, dW.value


def sound_speed(mat: OracleMaterial) -> float:
    m = mat.c_struct()
    return load_oracle().orc_sound_speed(C.byref(m))


def nh_stress(F, s, mat: OracleMaterial):
    lib = load_oracle()
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    S = np.zeros(9)
    pp, pm = C.c_double(), C.c_double()
    m = mat.c_struct()
    st = lib.orc_nh_stress(_dp(F), s, C.byref(m), _dp(S), C.byref(pp), C.byref(pm))
    if st != 0:
        raise ValueError("nh_stress: invalid F")
    return S.reshape(3, 3), pp.value, pm.value


def svk_stress(F, s, mat: OracleMaterial):
    """St. Venant-Kirchhoff stress with the spectral split: (S, psi_plus, psi_minus)."""
    lib = load_oracle()
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    S = np.zeros(9)
    pp, pm = C.c_double(), C.c_double()
    m = mat.c_struct()
    st = lib.orc_svk_stress(_dp(F), s, C.byref(m), _dp(S), C.byref(pp), C.byref(pm))
    if st != 0:
        raise ValueError("svk_stress: invalid F")
    return S.reshape(3, 3), pp.value, pm.value


def contact_force(dim, dc, contcoeff, xi, xj, vi, vj, mi, mj, mat_i: OracleMaterial, mat_j: OracleMaterial,
                  e_i, e_j, mu=0.0, dt=0.0):
    """Contact force on particle i from particle j (zero out of contact); mu = the pair's friction coefficient,
    dt = the step the force acts over (> 0 caps friction so that it at most stops the sliding in one step)."""
    lib = load_oracle()
    a = [np.zeros(3) for _ in range(4)]
    for dst, src in zip(a, (xi, xj, vi, vj)):
        dst[:len(src)] = src
    F = np.zeros(3)
    ci = (1 - mat_i.nu ** 2) / mat_i.E
    cj = (1 - mat_j.nu ** 2) / mat_j.E
    lib.orc_contact_force(dim, dc, contcoeff, *[_dp(x) for x in a], mi, mj, ci, cj, e_i, e_j, mu, dt, _dp(F))
    return F[:dim]


def sym_eig3(A):
    """Jacobi eigen-decomposition of a symmetric 3x3 matrix: (eigenvalues, Q with the eigenvectors as columns)."""
    lib = load_oracle()
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    w, Q = np.zeros(3), np.zeros(9)
    lib.orc_sym_eig3(_dp(A), _dp(w), _dp(Q))
    return w, Q.reshape(3, 3)


def j2_update(F, Fp, ep, mat: OracleMaterial):
    lib = load_oracle()
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(9)
    Fp = np.ascontiguousarray(Fp, dtype=np.float64).reshape(9)
    Fpo, S = np.zeros(9), np.zeros(9)
    epo, dg = C.c_double(), C.c_double()
    it = C.c_int()
    m = mat.c_struct()
    st = lib.orc_j2_update(_dp(F), _dp(Fp), ep, C.byref(m), _dp(Fpo), C.byref(epo), _dp(S), C.byref(dg),
                           C.byref(it))
    return {"Fp": Fpo.reshape(3, 3), "ep": epo.value, "S": S.reshape(3, 3), "dgamma": dg.value,
            "iters": it.value, "status": st}
