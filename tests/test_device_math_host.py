"""The library's constitutive device code, compiled for the host, against the FP64 oracle.

tests/native/constitutive_host.cu includes csrc/constitutive.cuh unchanged and is built
with nvcc as host code, so the GPU's SVK (spectral split), NH and J2 (C_p^-1 form) arithmetic is checked on
the CPU in both FP64 and FP32, without a GPU.
"""
import ctypes as C
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_pins import (STEEL_J2, STEEL_NH, SVK, _F_of_E, _plastic_state, _trial_F, lame,
                                     rand_rotation)

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "constitutive_host.cu")
LIB = os.path.join(HERE, "native", "_build", "libconstitutive_host.so")


@pytest.fixture(scope="module")
def hc():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    deps = [SRC] + [os.path.join(HERE, "..", "paper_2602_15149_b300", "csrc", f)
                    for f in ("constitutive.cuh", "tensor3.cuh")]
    if not os.path.exists(LIB) or any(os.path.getmtime(d) > os.path.getmtime(LIB) for d in deps):
        subprocess.check_call(["nvcc", "-std=c++17", "-O2", "-Xcompiler", "-fPIC", "-shared", "-o", LIB, SRC])
    lib = C.CDLL(LIB)
    D = C.POINTER(C.c_double)
    for f in (lib.hc_j2_d, lib.hc_j2_f):
        f.argtypes = [D, D, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, D, D, D, D]
    for f in (lib.hc_nh_d, lib.hc_nh_f):
        f.argtypes = [D, C.c_double, C.c_double, C.c_double, D, D, D]
    lib.hc_svk.argtypes = [C.c_int, C.c_int, D, C.c_double, C.c_double, C.c_double, D, D, D]
    return lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _j2(fn, F, Fp0, ep0):
    Fpi = np.linalg.inv(Fp0)
    K = Fpi @ Fpi.T - np.eye(3)
    K6 = np.array([K[0, 0], K[1, 1], K[2, 2], K[0, 1], K[0, 2], K[1, 2]])
    G = np.ascontiguousarray(F - np.eye(3)).ravel()
    K6o, S = np.zeros(6), np.zeros(9)
    epo, dg = C.c_double(), C.c_double()
    st = fn(_p(G), _p(K6), ep0, STEEL_J2.E, STEEL_J2.nu, STEEL_J2.sigma_y0, STEEL_J2.H_hard, _p(K6o), C.byref(epo),
            _p(S), C.byref(dg))
    Ko = np.array([[K6o[0], K6o[3], K6o[4]], [K6o[3], K6o[1], K6o[5]], [K6o[4], K6o[5], K6o[2]]]) + np.eye(3)
    return st, S.reshape(3, 3), epo.value, Ko


@pytest.mark.parametrize("prec,tol", [("d", 1e-9), ("f", 2e-3)])
def test_j2_cpinv_form_matches_fp_oracle(hc, prec, tol):
    """Stress, plastic strain and C_p^-1 of the device return map equal the oracle's F_p return map."""
    fn = hc.hc_j2_d if prec == "d" else hc.hc_j2_f
    rng = np.random.default_rng(0)
    nplastic = 0
    for k in range(200):
        Fp0, ep0 = _plastic_state(rng) if k % 2 else (np.eye(3), 0.0)
        F = _trial_F(rng, rng.uniform(0.0005, 0.0025), rng.uniform(-2e-3, 2e-3))
        ro = O.j2_update(F, Fp0, ep0, STEEL_J2)
        st, S, ep, Cpi = _j2(fn, F, Fp0, ep0)
        assert st == 0
        scale = np.abs(ro["S"]).max()
        assert np.abs(S - ro["S"]).max() <= tol * scale
        assert abs(ep - ro["ep"]) <= tol * max(ro["ep"], 1e-3)
        Fpi = np.linalg.inv(ro["Fp"])
        assert np.abs(Cpi - Fpi @ Fpi.T).max() <= tol
        nplastic += ro["dgamma"] > 0
    assert nplastic > 50


@pytest.mark.parametrize("prec", ["d", "f"])
def test_j2_barely_yielding_states_converge(hc, prec):
    """Trial states just above the yield surface (f / sigma_y from 1e-8 to 1e-3), where the residual is at
    the level of rounding: the bracket search must not mistake a rounding rise of r for its minimum."""
    fn = hc.hc_j2_d if prec == "d" else hc.hc_j2_f
    rng = np.random.default_rng(7)
    lam, mu = lame(STEEL_J2.E, STEEL_J2.nu)
    # the deviatoric strain at which a trial state reaches the yield surface from F_p = I, about
    e_y = STEEL_J2.sigma_y0 / (math.sqrt(6.0) * mu)
    for k in range(400):
        over = 10.0 ** rng.uniform(-8, -3)
        F = _trial_F(rng, e_y * (1.0 + over), rng.uniform(-1e-3, 1e-3))
        st, S, ep, Cpi = _j2(fn, F, np.eye(3), 0.0)
        assert st == 0, (k, over)
        assert np.all(np.isfinite(S))


@pytest.mark.parametrize("prec,tol", [("d", 1e-9), ("f", 2e-3)])
def test_j2_far_outside_the_yield_surface_matches_oracle(hc, prec, tol):
    """Trial stresses of 2 to 6 sigma_y (one random strain increment of 0.3%), where doubling the bracket
    steps over the negative interval of the V-shaped residual: the device code's search converges to the
    oracle's root (both bracket the first root, tests/test_oracle_pins.py pins it independently)."""
    fn = hc.hc_j2_d if prec == "d" else hc.hc_j2_f
    rng = np.random.default_rng(1)
    far = 0
    for _ in range(20):
        F = np.eye(3) + rng.normal(scale=3e-3, size=(3, 3))
        ro = O.j2_update(F, np.eye(3), 0.0, STEEL_J2)
        st, S, ep, Cpi = _j2(fn, F, np.eye(3), 0.0)
        assert st == 0 and ro["status"] == 0
        assert np.abs(S - ro["S"]).max() <= tol * np.abs(ro["S"]).max()
        assert abs(ep - ro["ep"]) <= tol * max(ro["ep"], 1e-3)
        far += ro["dgamma"] > 2.5e-3
    assert far >= 5


@pytest.mark.parametrize("prec,tol", [("d", 1e-11), ("f", 1e-5)])
def test_nh_matches_oracle(hc, prec, tol):
    fn = hc.hc_nh_d if prec == "d" else hc.hc_nh_f
    rng = np.random.default_rng(2)
    for scale in [1e-5, 1e-3, 5e-2]:
        for _ in range(20):
            F = np.eye(3) + rng.normal(scale=scale, size=(3, 3))
            s = rng.uniform(0.2, 1.0)
            So, ppo, pmo = O.nh_stress(F, s, STEEL_NH)
            S, pp, pm = np.zeros(9), C.c_double(), C.c_double()
            fn(_p(np.ascontiguousarray(F - np.eye(3)).ravel()), s, STEEL_NH.E, STEEL_NH.nu, _p(S), C.byref(pp),
               C.byref(pm))
            # (the oracle's literal I - tr C / 3 C^-1 cancels to ~1e-15 E in FP64 near F = I)
            assert np.abs(S.reshape(3, 3) - So).max() <= tol * np.abs(So).max() + 1e-15 * STEEL_NH.E
            # the tensile energy drives damage: relative accuracy even at tiny strain (the oracle's
            # literal mu/2 (J^-2/3 tr C - 3) itself cancels to ~1e-15 E in FP64)
            floor = 1e-15 * STEEL_NH.E
            assert abs(pp.value - ppo) <= 50 * tol * abs(ppo) + floor
            assert abs(pm.value - pmo) <= 50 * tol * abs(pmo) + floor


# ---------------------------------------------------------------- St. Venant-Kirchhoff split
def _svk(hc, prec, dim, F, s):
    G = np.ascontiguousarray(F - np.eye(3)).ravel()
    S = np.zeros(9)
    pp, pm = C.c_double(), C.c_double()
    hc.hc_svk(prec, dim, _p(G), s, SVK.E, SVK.nu, _p(S), C.byref(pp), C.byref(pm))
    return S.reshape(3, 3), pp.value, pm.value


def _svk_strains(rng, dim):
    """Strains whose spectra the split finds hardest: repeated, near-equal straddling zero, isotropic,
    single-signed, and generic, in random frames (in-plane frames in 2D)."""
    spectra = [(1e-3, -2e-4, -2e-4), (-1e-3, 2e-4, 2e-4), (1e-3, 1e-9, -1e-9), (1e-3, -1e-9, -1e-9),
               (3e-4, 3e-4, 3e-4), (-3e-4, -3e-4, -3e-4), (1e-3, 5e-4, 2e-4), (-1e-3, -5e-4, -2e-4),
               (1e-3, 0.0, 0.0), (2e-3, -1e-3, 3e-7), (1e-3, 1e-3 * (1 + 1e-7), -4e-4), (0.0, 0.0, 0.0)]
    spectra += [tuple(rng.normal(scale=1e-3, size=3)) for _ in range(40)]
    out = []
    for lam in spectra:
        if dim == 2:
            R = np.eye(3)
            th = rng.uniform(0, np.pi)
            R[:2, :2] = [[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]]
            E = R @ np.diag([lam[0], lam[1], 0.0]) @ R.T
        else:
            R = rand_rotation(rng)
            E = R @ np.diag(lam) @ R.T
        out.append(E)
    return out


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec,tol", [(64, 2e-12), (32, 2e-6)])
def test_svk_split_matches_oracle(hc, dim, prec, tol):
    """Stress and both energies of the device split against the oracle's Jacobi split, for degraded and
    intact particles, relative to the stress scale of the strain (FP32 is bounded by the rounding of E
    itself, about eps |E|)."""
    rng = np.random.default_rng(11 + dim)
    lam, mu = lame(SVK.E, SVK.nu)
    for E in _svk_strains(rng, dim):
        F = _F_of_E(E)
        for s in (1.0, 0.4, 0.0):
            So, ppo, pmo = O.svk_stress(F, s, SVK)
            Sd, ppd, pmd = _svk(hc, prec, dim, F, s)
            scale = max((lam + 2 * mu) * np.abs(E).max(), 1.0)
            assert np.abs(Sd - So).max() <= tol * scale, (E, s, Sd, So)
            escale = max((lam + 2 * mu) * np.abs(E).max() ** 2, 1e-30)
            assert abs(ppd - ppo) <= tol * escale and abs(pmd - pmo) <= tol * escale
