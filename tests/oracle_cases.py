"""Drive the FP64 oracle from a workload Case (test helper; imports only oracle/ and workloads)."""
import numpy as np

from oracle.expr import Expression
from oracle.oracle import Oracle, OracleMaterial
from paper_2602_15149_b300 import workloads as W


def oracle_material(m: W.Material) -> OracleMaterial:
    return OracleMaterial(m.model, m.rho, m.E, m.nu, m.sigma_y0, m.H_hard, m.beta1, m.beta2, m.fracture, m.Gc,
                          m.eps0, m.s_lim)


def make_oracle(case: W.Case, build=True, method=None, **kw) -> Oracle:
    kw.setdefault("integrator", getattr(case, "integrator", 1))
    kw.setdefault("dx", case.dp)
    o = Oracle(case.dim, case.h, cfl=case.cfl, dt_mode=case.dt_mode, fixed_dt=case.fixed_dt,
               gravity=case.gravity, **kw)
    o.set_materials([oracle_material(m) for m in case.materials])
    o.create_particles(case.X0, case.vol, case.v0, case.material_id, case.specimen_id)
    for b in list(case.bcs) + list(getattr(case, "specimen_loads", [])):
        o.add_bc(b.mask, b.kind, b.comp_mask, b.value, b.t_start, b.t_end, b.ramp, b.area)
    for q in case.notches:
        o.add_notch(q)
    if getattr(case, "contact", None):
        o.set_contact(case.contact["contcoeff"], case.contact["restitution"])
        if case.contact.get("kfric") is not None:
            o.set_contact_friction(case.contact["kfric"])
    for b in getattr(case, "expr_bcs", []):
        o.add_bc_expr(b.mask, b.kind, b.comp_mask, [None if e is None else Expression(e[0], e[1]) for e in b.exprs],
                      b.t_start, b.t_end, b.area)
    if build:
        o.build_ref_neighbours(method)
        for fld, exprs in getattr(case, "expr_ics", []):
            o.apply_expr(fld, [None if e is None else Expression(e[0], e[1]) for e in exprs])
    return o
