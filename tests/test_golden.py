"""The synthetic workloads reuse the paper's printed defaults and case values (tests/golden/paper_values.json)."""
import json
import os

from paper_2602_15149_b300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def v(k):
    return GOLD[k]["value"]


def test_defaults_follow_paper():
    m = W.Material()
    assert m.s_lim == v("soft_particle_limit_s_l")
    assert m.beta1 == v("artificial_viscosity_default_factor1")
    assert m.beta2 == v("artificial_viscosity_default_factor2")


def test_notched_plate_uses_crack_branching_material():
    c = W.notched_plate(nx=50, ny=20)
    m = c.materials[0]
    assert (m.E, m.nu, m.rho, m.Gc) == (v("crack_branching_E_Pa"), v("crack_branching_nu"), v("crack_branching_rho"),
                                        v("crack_branching_Gc"))
    assert c.bcs[0].value[1] == v("crack_branching_traction_Pa")
    assert c.notches[0][1][0] == v("crack_branching_notch_tip_x_m")


def test_crack_branching_case_is_the_published_one():
    ref = GOLD["crack_branching"]
    c = W.crack_branching()
    m = c.materials[0]
    assert c.n == 1600 * 640 and abs(c.dp - ref["dx_m"]) < 1e-15
    assert abs(m.eps0 - ref["eps0_m"]) < 1e-15 and m.s_lim == ref["s_lim"] and c.cfl == ref["cfl"]
    assert m.beta1 == ref["beta1"] and m.model == W.MODEL_SVK and m.fracture == 1
    assert (m.E, m.nu, m.rho, m.Gc) == (v("crack_branching_E_Pa"), v("crack_branching_nu"), v("crack_branching_rho"),
                                        v("crack_branching_Gc"))
