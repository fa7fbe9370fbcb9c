"""Thin ctypes binding of the C-ABI in ``include/tlsph.h`` (argument marshalling only).

Every computation runs in ``_lib/libtlsph.so`` (sm_103a CUDA).  There is no
fallback: if the library is missing this module raises on load.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# the library to load; TLSPH_LIBRARY selects another build, e.g. _lib/libtlsph_debug.so (bounds-checked kernels)
LIB_PATH = os.environ.get("TLSPH_LIBRARY") or os.path.join(HERE, "_lib", "libtlsph.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_SINGULAR_L, ERR_NONFINITE, ERR_NOCONVERGE, ERR_TIMEOUT, ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, FP32_U64 = 0, 1
DT_FIXED, DT_ADAPTIVE, DT_CFL_STATIC = 0, 1, 2
MODEL_SVK, MODEL_NH, MODEL_J2 = 1, 2, 3
BC_VEL, BC_TRACTION, BC_ACCEL, BC_POINTFORCE, BC_PHASE_BOUND = 0, 1, 2, 3, 4
FIELD = {"U": 0, "V": 1, "X": 2, "S": 3, "SDOT": 4, "H": 5, "EPSP": 6, "P": 7, "F": 8, "ACC": 11, "CPINV": 12,
         "STATE": 100}
OPT_KERNEL_TIMING, OPT_RECORD_ACC, OPT_MODE, OPT_BLOCK, OPT_BARRIER_TEST, OPT_NEIGHBOUR_LAYOUT = 1, 2, 3, 4, 5, 6
OPT_MEMORY_LIMIT = 7
OPT_LATTICE_ROWS_GRADIENT, OPT_LATTICE_ROWS_FORCE, OPT_FUSE_STRESS, OPT_LATTICE_PATCH = 8, 9, 10, 11
OPT_LATTICE_ZSTREAM = 12
LAYOUT_AUTO, LAYOUT_CSR, LAYOUT_STENCIL = 0, 1, 2
MODE_LAUNCH, MODE_GRAPH, MODE_PERSISTENT = 0, 1, 2
INTEGRATOR_EULER, INTEGRATOR_LEAPFROG = 1, 2
MODE_NAMES = {MODE_LAUNCH: "launch", MODE_GRAPH: "graph", MODE_PERSISTENT: "persistent"}

# every entry point declared in include/tlsph.h
EXPORTS = ["tlsph_create", "tlsph_destroy", "tlsph_last_error", "tlsph_set_materials", "tlsph_create_particles",
           "tlsph_add_bc", "tlsph_add_notch", "tlsph_build_ref_neighbours", "tlsph_step", "tlsph_step_async",
           "tlsph_sync", "tlsph_read_state", "tlsph_write_state", "tlsph_field_bytes", "tlsph_energies", "tlsph_time",
           "tlsph_neighbours", "tlsph_permutation", "tlsph_nnz", "tlsph_get_info", "tlsph_set_option",
           "tlsph_kernel_times", "tlsph_cell_sort_noalloc", "tlsph_autotune", "tlsph_mlp_create",
           "tlsph_mlp_destroy", "tlsph_mlp_last_error", "tlsph_mlp_set_params", "tlsph_mlp_get_params",
           "tlsph_mlp_set_normalization", "tlsph_mlp_get_normalization", "tlsph_mlp_fit_normalization",
           "tlsph_mlp_train_step", "tlsph_mlp_gradients", "tlsph_mlp_forward", "tlsph_set_surrogate",
           "tlsph_surrogate_counts", "tlsph_j2_samples",
           "tlsph_mlp_set_tensor_path", "tlsph_expr_check", "tlsph_expr_compile", "tlsph_add_bc_expr",
           "tlsph_apply_expr", "tlsph_expr_eval", "tlsph_set_contact", "tlsph_set_contact_friction", "tlsph_mlp_save",
           "tlsph_mlp_load", "tlsph_load_surrogate"]
MLP_NUM_PARAMS = 37264
SURROGATE_ALL, SURROGATE_PLASTIC = 0, 1
TENSOR_MMA_SYNC, TENSOR_TCGEN05 = 0, 1
NOALLOC_MAX_PARTICLES = 131072


class Params(C.Structure):
    _fields_ = [("dim", C.c_int), ("precision", C.c_int), ("integrator", C.c_int), ("h", C.c_double),
                ("support", C.c_double), ("cfl", C.c_double), ("dt_mode", C.c_int), ("fixed_dt", C.c_double),
                ("gravity", C.c_double * 3), ("cuda_stream", C.c_void_p), ("device", C.c_int), ("dx", C.c_double)]


class Material(C.Structure):
    _fields_ = [("model", C.c_int), ("rho", C.c_double), ("E", C.c_double), ("nu", C.c_double),
                ("sigma_y0", C.c_double), ("H_hard", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("fracture", C.c_int), ("Gc", C.c_double), ("eps0", C.c_double), ("s_lim", C.c_double)]


class Info(C.Structure):
    _fields_ = [("steps", C.c_int64), ("kernel_launches", C.c_int64), ("noconverge", C.c_int64),
                ("nonfinite", C.c_int64), ("nnz", C.c_int64), ("max_row", C.c_int64), ("bytes_per_step", C.c_double),
                ("stencil", C.c_int64), ("lattice_nx", C.c_int64), ("lattice_nxny", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("mode", C.c_int), ("block", C.c_int), ("ms_per_step", C.c_double)]


class TLSPHError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tlsph status {status}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtlsph.so and declare the C signatures (raises if the library is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2602_15149_b300.build.build_library()")
    lib = C.CDLL(path)
    P, D, I64, I32, U8, V = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32), \
        C.POINTER(C.c_uint8), C.c_void_p
    sig = {
        "tlsph_create": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_void_p)]),
        "tlsph_destroy": (None, [P]),
        "tlsph_last_error": (C.c_char_p, [P]),
        "tlsph_set_materials": (C.c_int, [P, C.c_int, C.POINTER(Material)]),
        "tlsph_create_particles": (C.c_int, [P, C.c_int64, D, D, D, I32, I32]),
        "tlsph_add_bc": (C.c_int, [P, U8, C.c_int, C.c_int, D, C.c_double, C.c_double, C.c_double, C.c_double]),
        "tlsph_add_notch": (C.c_int, [P, D]),
        "tlsph_expr_check": (C.c_int, [C.c_char_p, C.c_char_p, C.c_char_p, C.c_size_t]),
        "tlsph_expr_compile": (C.c_int, [P, C.c_char_p, C.c_char_p, C.POINTER(C.c_int)]),
        "tlsph_add_bc_expr": (C.c_int, [P, U8, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_double, C.c_double,
                                        C.c_double]),
        "tlsph_apply_expr": (C.c_int, [P, C.c_int, C.POINTER(C.c_int)]),
        "tlsph_expr_eval": (C.c_int, [P, C.c_int, C.c_int64, D, D, U8]),
        "tlsph_set_contact": (C.c_int, [P, C.c_double, C.c_int, D]),
        "tlsph_set_contact_friction": (C.c_int, [P, C.c_int, D]),
        "tlsph_mlp_save": (C.c_int, [P, C.c_char_p]),
        "tlsph_mlp_load": (C.c_int, [P, C.c_char_p]),
        "tlsph_load_surrogate": (C.c_int, [P, C.c_char_p, C.c_int]),
        "tlsph_build_ref_neighbours": (C.c_int, [P]),
        "tlsph_step": (C.c_int, [P, C.c_int64]),
        "tlsph_step_async": (C.c_int, [P, C.c_int64]),
        "tlsph_sync": (C.c_int, [P]),
        "tlsph_read_state": (C.c_int, [P, C.c_int, V, C.c_size_t, C.c_int]),
        "tlsph_write_state": (C.c_int, [P, C.c_int, V, C.c_size_t, C.c_int]),
        "tlsph_field_bytes": (C.c_int64, [P, C.c_int]),
        "tlsph_energies": (C.c_int, [P, D]),
        "tlsph_time": (C.c_int, [P, C.c_int, D, D]),
        "tlsph_neighbours": (C.c_int, [P, I64, I32, C.c_int64]),
        "tlsph_permutation": (C.c_int, [P, I64]),
        "tlsph_nnz": (C.c_int64, [P]),
        "tlsph_get_info": (C.c_int, [P, C.POINTER(Info)]),
        "tlsph_set_option": (C.c_int, [P, C.c_int, C.c_int]),
        "tlsph_kernel_times": (C.c_int, [P, D, I64]),
        "tlsph_cell_sort_noalloc": (C.c_int, [C.c_int, V, C.c_int64, C.c_int, C.c_double, C.c_double, V, V, V]),
        "tlsph_autotune": (C.c_int, [P, C.c_int, C.POINTER(Tuning), C.POINTER(Tuning)]),
        "tlsph_mlp_create": (C.c_int, [C.c_int, V, C.c_int, C.POINTER(C.c_void_p)]),
        "tlsph_mlp_destroy": (None, [P]),
        "tlsph_mlp_last_error": (C.c_char_p, [P]),
        "tlsph_mlp_set_params": (C.c_int, [P, V]),
        "tlsph_mlp_get_params": (C.c_int, [P, V]),
        "tlsph_mlp_set_normalization": (C.c_int, [P, V]),
        "tlsph_mlp_get_normalization": (C.c_int, [P, V]),
        "tlsph_mlp_fit_normalization": (C.c_int, [P, C.c_int64, V, V, C.c_float]),
        "tlsph_mlp_train_step": (C.c_int, [P, V, V, C.c_float, C.POINTER(C.c_float)]),
        "tlsph_mlp_gradients": (C.c_int, [P, V, V, V, C.POINTER(C.c_float)]),
        "tlsph_mlp_forward": (C.c_int, [P, C.c_int64, V, V, V]),
        "tlsph_set_surrogate": (C.c_int, [P, P, C.c_int]),
        "tlsph_surrogate_counts": (C.c_int, [P, I64]),
        "tlsph_j2_samples": (C.c_int, [P, C.c_int, C.c_int, C.c_uint, V, V, V, C.c_int64, I64]),
        "tlsph_mlp_set_tensor_path": (C.c_int, [P, C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class TLSPH:
    """One TLSPH context on a CUDA device (methods carry the C-ABI names without the prefix)."""

    def __init__(self, dim, h, precision=FP32_U64, cfl=0.3, dt_mode=DT_CFL_STATIC, fixed_dt=0.0,
                 gravity=(0.0, 0.0, 0.0), support=2.0, device=0, stream=None, integrator=INTEGRATOR_EULER, dx=0.0):
        self.lib = load_library()
        p = Params(dim, precision, integrator, h, support, cfl, dt_mode, fixed_dt, (C.c_double * 3)(*gravity),
                   stream, device, dx)
        ctx = C.c_void_p()
        st = self.lib.tlsph_create(C.byref(p), C.byref(ctx))
        if st != OK:
            raise TLSPHError(st, "tlsph_create failed (no CUDA device or bad parameters)")
        self.ctx = ctx
        self.dim = dim
        self.precision = precision
        self.n = 0

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tlsph_destroy(self.ctx)
            self.ctx = None

    __del__ = close

    def _ck(self, st, what=""):
        if st != OK:
            raise TLSPHError(st, f"{what}: {self.last_error()}")
        return st

    def last_error(self) -> str:
        return self.lib.tlsph_last_error(self.ctx).decode()

    def set_materials(self, mats):
        arr = (Material * len(mats))(*[Material(m.model, m.rho, m.E, m.nu, m.sigma_y0, m.H_hard, m.beta1, m.beta2,
                                                m.fracture, m.Gc, m.eps0, m.s_lim) for m in mats])
        self._ck(self.lib.tlsph_set_materials(self.ctx, len(mats), arr), "set_materials")

    def create_particles(self, X0, vol, v0=None, material_id=None, specimen_id=None):
        X0 = np.ascontiguousarray(X0, np.float64)
        n = X0.shape[0]
        vol = np.ascontiguousarray(vol, np.float64)
        mid = np.zeros(n, np.int32) if material_id is None else np.ascontiguousarray(material_id, np.int32)
        v0a = None if v0 is None else np.ascontiguousarray(v0, np.float64)
        sid = None if specimen_id is None else np.ascontiguousarray(specimen_id, np.int32)
        I32 = C.POINTER(C.c_int32)
        self._ck(self.lib.tlsph_create_particles(self.ctx, n, _d(X0), _d(vol), None if v0a is None else _d(v0a),
                                                 mid.ctypes.data_as(I32),
                                                 None if sid is None else sid.ctypes.data_as(I32)),
                 "create_particles")
        self.n = n

    def add_bc(self, mask, kind, comp_mask, value, t_start=0.0, t_end=-1.0, ramp=0.0, area=0.0):
        m = np.ascontiguousarray(mask, np.uint8)
        val = np.zeros(3)
        val[:len(value)] = value
        self._ck(self.lib.tlsph_add_bc(self.ctx, m.ctypes.data_as(C.POINTER(C.c_uint8)), kind, comp_mask, _d(val),
                                       t_start, t_end, ramp, area), "add_bc")

    def add_notch(self, quad):
        q = np.ascontiguousarray(quad, np.float64).reshape(12)
        self._ck(self.lib.tlsph_add_notch(self.ctx, _d(q)), "add_notch")

    def set_contact(self, contcoeff, restitution, kfric=None):
        """Contact between the bodies (specimens): potential multiplier, one restitution per body and,
        optionally, one friction coefficient per body."""
        r = np.ascontiguousarray(restitution, np.float64)
        self._ck(self.lib.tlsph_set_contact(self.ctx, contcoeff, r.size, _d(r)), "set_contact")
        if kfric is not None:
            f = np.ascontiguousarray(kfric, np.float64)
            self._ck(self.lib.tlsph_set_contact_friction(self.ctx, f.size, _d(f)), "set_contact_friction")

    def expr_compile(self, expr, locals_=""):
        """Compile a user-defined expression; returns its id."""
        i = C.c_int()
        self._ck(self.lib.tlsph_expr_compile(self.ctx, locals_.encode(), expr.encode(), C.byref(i)), "expr_compile")
        return i.value

    def add_bc_expr(self, mask, kind, comp_mask, expr_ids, t_start=0.0, t_end=-1.0, area=0.0):
        """A boundary condition whose components take the values of compiled expressions (ids, -1 for none)."""
        m = np.ascontiguousarray(mask, np.uint8)
        ids = (C.c_int * 3)(*(list(expr_ids) + [-1] * (3 - len(expr_ids))))
        self._ck(self.lib.tlsph_add_bc_expr(self.ctx, m.ctypes.data_as(C.POINTER(C.c_uint8)), kind, comp_mask, ids,
                                            t_start, t_end, area), "add_bc_expr")

    def apply_expr(self, field, expr_ids):
        """Set the components of field "U" or "V" from compiled expressions evaluated now (ids, -1 for none)."""
        ids = (C.c_int * 3)(*(list(expr_ids) + [-1] * (3 - len(expr_ids))))
        self._ck(self.lib.tlsph_apply_expr(self.ctx, FIELD[field], ids), "apply_expr")

    def expr_eval(self, expr_id, variables):
        """Evaluate a compiled expression on the device for rows of the 12 built-in variables (n x 12, order
        x0 y0 z0 x y z ux uy uz t dt dx); returns (values, skip)."""
        v = np.ascontiguousarray(variables, np.float64).reshape(-1, 12)
        out = np.zeros(v.shape[0])
        skip = np.zeros(v.shape[0], np.uint8)
        self._ck(self.lib.tlsph_expr_eval(self.ctx, expr_id, v.shape[0], _d(v), _d(out),
                                          skip.ctypes.data_as(C.POINTER(C.c_uint8))), "expr_eval")
        return out, skip.astype(bool)

    def build_ref_neighbours(self):
        self._ck(self.lib.tlsph_build_ref_neighbours(self.ctx), "build_ref_neighbours")

    def step(self, nsteps=1, check=True):
        st = self.lib.tlsph_step(self.ctx, nsteps)
        if check:
            self._ck(st, "step")
        return st

    def step_async(self, nsteps=1):
        self._ck(self.lib.tlsph_step_async(self.ctx, nsteps), "step_async")

    def sync(self, check=True):
        st = self.lib.tlsph_sync(self.ctx)
        if check:
            self._ck(st, "sync")
        return st

    def field_bytes(self, field: str) -> int:
        return int(self.lib.tlsph_field_bytes(self.ctx, FIELD[field]))

    def read_state(self, field: str, out=None):
        """Read a field in the caller's order into a new numpy array, or into ``out``
        (a numpy array, or a torch CUDA tensor of float64 for a device-side read)."""
        nb = self.field_bytes(field)
        if field == "STATE":
            buf = np.zeros(nb, np.uint8) if out is None else out
            self._ck(self.lib.tlsph_read_state(self.ctx, FIELD[field], buf.ctypes.data, nb, 0), "read_state")
            return buf
        if out is not None and hasattr(out, "data_ptr"):
            self._ck(self.lib.tlsph_read_state(self.ctx, FIELD[field], out.data_ptr(), nb, 1), "read_state")
            return out
        a = np.zeros(nb // 8) if out is None else out
        self._ck(self.lib.tlsph_read_state(self.ctx, FIELD[field], a.ctypes.data, nb, 0), "read_state " + field)
        per = nb // 8 // self.n
        if per == 9:
            return a.reshape(self.n, 3, 3)
        return a.reshape(self.n, per) if per > 1 else a

    def write_state(self, field: str, values):
        nb = self.field_bytes(field)
        if hasattr(values, "data_ptr"):
            self._ck(self.lib.tlsph_write_state(self.ctx, FIELD[field], values.data_ptr(), nb, 1), "write_state")
            return
        a = np.ascontiguousarray(values, np.uint8 if field == "STATE" else np.float64)
        self._ck(self.lib.tlsph_write_state(self.ctx, FIELD[field], a.ctypes.data, nb, 0), "write_state " + field)

    def energies(self):
        out = np.zeros(6)
        self._ck(self.lib.tlsph_energies(self.ctx, _d(out)), "energies")
        return {"KE": out[0], "SE": out[1], "FE": out[2], "PW": out[3], "Wext": out[4], "t": out[5],
                "dt": self.time()[1]}

    def time(self, specimen=0):
        t, dt = C.c_double(), C.c_double()
        self._ck(self.lib.tlsph_time(self.ctx, specimen, C.byref(t), C.byref(dt)), "time")
        return t.value, dt.value

    def nnz(self) -> int:
        return int(self.lib.tlsph_nnz(self.ctx))

    def neighbours(self):
        nnz = self.nnz()
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        self._ck(self.lib.tlsph_neighbours(self.ctx, rp.ctypes.data_as(C.POINTER(C.c_int64)),
                                           col.ctypes.data_as(C.POINTER(C.c_int32)), nnz), "neighbours")
        return rp, col[:nnz]

    def permutation(self):
        p = np.zeros(self.n, np.int64)
        self._ck(self.lib.tlsph_permutation(self.ctx, p.ctypes.data_as(C.POINTER(C.c_int64))), "permutation")
        return p

    def get_info(self) -> dict:
        info = Info()
        self._ck(self.lib.tlsph_get_info(self.ctx, C.byref(info)), "get_info")
        return {k: getattr(info, k) for k, _ in Info._fields_}

    def set_option(self, option: int, value: int):
        self._ck(self.lib.tlsph_set_option(self.ctx, option, value), "set_option")

    def autotune(self, trial_steps=10):
        """Time every execution mode / block size on the live problem and keep the fastest
        (the state is restored); returns (best, all) as dicts."""
        best = Tuning()
        allt = (Tuning * 6)()
        self._ck(self.lib.tlsph_autotune(self.ctx, trial_steps, C.byref(best), allt), "autotune")
        conv = lambda t: {"mode": MODE_NAMES[t.mode], "block": t.block, "ms_per_step": t.ms_per_step}
        return conv(best), [conv(t) for t in allt]

    def set_surrogate(self, mlp, scope=None):
        """Attach a network (None detaches); scope SURROGATE_ALL (default) or SURROGATE_PLASTIC."""
        scope = SURROGATE_ALL if scope is None else scope
        self._ck(self.lib.tlsph_set_surrogate(self.ctx, None if mlp is None else mlp.h, scope), "set_surrogate")

    def load_surrogate(self, path, scope=None):
        """Attach the network stored in a file written by MLP.save."""
        scope = SURROGATE_ALL if scope is None else scope
        self._ck(self.lib.tlsph_load_surrogate(self.ctx, os.fsencode(path), scope), "load_surrogate")

    def surrogate_counts(self):
        """(network, outside the envelope, elastic trial kept exact), cumulative."""
        c = np.zeros(3, np.int64)
        self._ck(self.lib.tlsph_surrogate_counts(self.ctx, c.ctypes.data_as(C.POINTER(C.c_int64))), "surrogate_counts")
        return int(c[0]), int(c[1]), int(c[2])

    def j2_samples(self, x, y, stride_elastic=1, stride_plastic=1, salt=0, pnorm=None):
        """Return-map samples of the current state into torch CUDA float32 tensors x, y (cap x 16)
        and optionally pnorm (cap, |P|_F of each row); returns the number of rows written."""
        cnt = np.zeros(1, np.int64)
        self._ck(self.lib.tlsph_j2_samples(self.ctx, stride_elastic, stride_plastic, salt, x.data_ptr(), y.data_ptr(),
                                           None if pnorm is None else pnorm.data_ptr(), int(x.shape[0]),
                                           cnt.ctypes.data_as(C.POINTER(C.c_int64))), "j2_samples")
        return int(cnt[0])

    def kernel_times(self):
        ms = np.zeros(3)
        cnt = np.zeros(3, np.int64)
        self._ck(self.lib.tlsph_kernel_times(self.ctx, _d(ms), cnt.ctypes.data_as(C.POINTER(C.c_int64))),
                 "kernel_times")
        return {"pass2_ms": ms[0], "pass2_launches": int(cnt[0]), "gradient_ms": ms[1],
                "gradient_launches": int(cnt[1]), "stress_ms": ms[2], "stress_launches": int(cnt[2])}


class MLP:
    """The surrogate network on a CUDA device (tlsph_mlp_*); data arguments are torch CUDA tensors."""

    def __init__(self, batch=4096, device=0, stream=None):
        self.lib = load_library()
        h = C.c_void_p()
        st = self.lib.tlsph_mlp_create(device, stream, batch, C.byref(h))
        if st != OK:
            raise TLSPHError(st, "tlsph_mlp_create failed")
        self.h = h
        self.batch = batch

    def close(self):
        if getattr(self, "h", None):
            self.lib.tlsph_mlp_destroy(self.h)
            self.h = None

    __del__ = close

    def _ck(self, st, what):
        if st != OK:
            raise TLSPHError(st, f"{what}: {self.lib.tlsph_mlp_last_error(self.h).decode()}")

    def set_params(self, p):
        a = np.ascontiguousarray(p, np.float32)
        assert a.size == MLP_NUM_PARAMS
        self._ck(self.lib.tlsph_mlp_set_params(self.h, a.ctypes.data), "set_params")

    def get_params(self):
        a = np.zeros(MLP_NUM_PARAMS, np.float32)
        self._ck(self.lib.tlsph_mlp_get_params(self.h, a.ctypes.data), "get_params")
        return a

    def save(self, path):
        """Write the parameters and normalisation to a network file."""
        self._ck(self.lib.tlsph_mlp_save(self.h, os.fsencode(path)), "save")

    def load(self, path):
        """Replace the parameters and normalisation from a network file."""
        self._ck(self.lib.tlsph_mlp_load(self.h, os.fsencode(path)), "load")

    def set_tensor_path(self, path):
        """TENSOR_TCGEN05 (default) or TENSOR_MMA_SYNC for the inference kernels and the training GEMMs."""
        self._ck(self.lib.tlsph_mlp_set_tensor_path(self.h, int(path)), "set_tensor_path")

    def set_normalization(self, norm):
        a = np.ascontiguousarray(norm, np.float32).reshape(96)
        self._ck(self.lib.tlsph_mlp_set_normalization(self.h, a.ctypes.data), "set_normalization")

    def get_normalization(self):
        a = np.zeros(96, np.float32)
        self._ck(self.lib.tlsph_mlp_get_normalization(self.h, a.ctypes.data), "get_normalization")
        return a

    def fit_normalization(self, x, y, margin=0.02):
        self._ck(self.lib.tlsph_mlp_fit_normalization(self.h, int(x.shape[0]), x.data_ptr(), y.data_ptr(),
                                                      float(margin)), "fit_normalization")

    def train_step(self, x, y, lr):
        loss = C.c_float()
        self._ck(self.lib.tlsph_mlp_train_step(self.h, x.data_ptr(), y.data_ptr(), float(lr), C.byref(loss)),
                 "train_step")
        return loss.value

    def gradients(self, x, y):
        g = np.zeros(MLP_NUM_PARAMS, np.float32)
        loss = C.c_float()
        self._ck(self.lib.tlsph_mlp_gradients(self.h, x.data_ptr(), y.data_ptr(), g.ctypes.data, C.byref(loss)),
                 "gradients")
        return loss.value, g

    def forward(self, x, y, outside=None):
        self._ck(self.lib.tlsph_mlp_forward(self.h, int(x.shape[0]), x.data_ptr(), y.data_ptr(),
                                            None if outside is None else outside.data_ptr()), "forward")


def pack_params(params):
    """[(W0, b0), ..., (W3, b3)] -> the packed float32 layout of the C-ABI."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def unpack_params(p, sizes=(16, 128, 128, 128, 16)):
    out, off = [], 0
    for n_in, n_out in zip(sizes[:-1], sizes[1:]):
        W = p[off:off + n_in * n_out].reshape(n_out, n_in)
        off += n_in * n_out
        b = p[off:off + n_out]
        off += n_out
        out.append((W, b))
    return out


def cell_sort_noalloc(X0, perm, h, support=2.0, specimen_id=None, device=0, stream=None) -> int:
    """tlsph_cell_sort_noalloc on caller-owned device buffers (torch CUDA tensors): X0 (n, dim)
    float64, perm (n,) int32 out, specimen_id (n,) int32 or None.  Returns the status; the
    library allocates nothing."""
    lib = load_library()
    n, dim = int(X0.shape[0]), int(X0.shape[1])
    return lib.tlsph_cell_sort_noalloc(device, stream, n, dim, h, support, X0.data_ptr(),
                                       None if specimen_id is None else specimen_id.data_ptr(), perm.data_ptr())


def expr_check(expr, locals_=""):
    """Check an expression without a context or a GPU: None when it compiles, else the error message."""
    lib = load_library()
    buf = C.create_string_buffer(512)
    st = lib.tlsph_expr_check(locals_.encode(), expr.encode(), buf, 512)
    return None if st == OK else buf.value.decode()


def from_case(case, precision=None, device=0, build=True, stream=None) -> TLSPH:
    """Create a context from a :class:`workloads.Case` (marshalling only)."""
    prec = precision if precision is not None else (FP64 if case.precision == "fp64" else FP32_U64)
    t = TLSPH(case.dim, case.h, prec, case.cfl, case.dt_mode, case.fixed_dt, case.gravity, device=device,
              stream=stream, integrator=getattr(case, "integrator", INTEGRATOR_EULER), dx=case.dp)
    t.set_materials(case.materials)
    t.create_particles(case.X0, case.vol, case.v0, case.material_id, case.specimen_id)
    for b in list(case.bcs) + list(getattr(case, "specimen_loads", [])):
        t.add_bc(b.mask, b.kind, b.comp_mask, b.value, b.t_start, b.t_end, b.ramp, b.area)
    for q in case.notches:
        t.add_notch(q)
    if getattr(case, "contact", None):
        t.set_contact(case.contact["contcoeff"], case.contact["restitution"], case.contact.get("kfric"))
    for b in getattr(case, "expr_bcs", []):
        ids = [-1 if e is None else t.expr_compile(e[0], e[1]) for e in b.exprs]
        t.add_bc_expr(b.mask, b.kind, b.comp_mask, ids, b.t_start, b.t_end, b.area)
    if build:
        t.build_ref_neighbours()
        for fld, exprs in getattr(case, "expr_ics", []):
            t.apply_expr(fld, [-1 if e is None else t.expr_compile(e[0], e[1]) for e in exprs])
    elif getattr(case, "expr_ics", []):
        raise ValueError("initial fields given by expressions need build=True")
    return t
