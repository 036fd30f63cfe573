"""Pins of the oracle's explicit Cahn-Hilliard variant (Eq. ExpCH, reading R15).

  * closed form: with no solid, a uniform x1 velocity and C = eps cos(k x1) (uniform in x2),
    every term of the discrete update is a known multiple of cos(k x1), sin(k x1) and
    cos(3 k x1) (the cubic of psi' gives the third harmonic), at levels n and n-1 with
    different amplitudes and velocities, so the AB2 weights and the level of each term are
    checked;
  * the update conserves sum C before the ghost fill (divergence form, no flux through the
    walls, mirror rows) on a sinusoidal-wall case with ghosts;
  * consistency: the explicit and the (separately pinned) semi-implicit steps are two
    discretisations in time of the same equation, so from a smooth state with a first-order
    consistent history their one-step increments differ by O(dt^2): the relative
    difference shrinks in proportion to dt.
"""
import dataclasses
import math

import numpy as np

from oracle import ib_pf2d as O
from workloads import cases as W


def _scheme(case, s):
    return dataclasses.replace(case, params=dataclasses.replace(case.params, ch_scheme=s))


def _free_case(nx, ny, Cn, Pe, dt):
    h = 2.0 / nx
    d1, d2 = math.sqrt(2.0) * h, 0.5 * math.sqrt(2.0) * h
    p = W.Params(Cn=Cn, Pe=Pe, dt=dt, d1=d1, d2=d2, ch_scheme=1)
    return W.Case2D(f"free_{nx}x{ny}", nx, ny, 2.0, ny * h, W.GEOM_NONE, (0.0,) * 4, (1.0, 0.5),
                    0.0, p, 1)


def test_single_mode_closed_form():
    nx, ny, m = 64, 8, 3
    Cn, Pe, dt = 0.05, 40.0, 1.0e-3
    case = _free_case(nx, ny, Cn, Pe, dt)
    geo = O.build_geometry(case)
    h = case.h
    k = 2.0 * math.pi * m / case.lx
    x = (np.arange(nx) + 0.5) * h
    lam = lambda q: (2.0 * math.cos(q * k * h) - 2.0) / (h * h)   # discrete lap of cos(q k x)

    def F(eps, U):
        # -div(U C_f) with C_f the face means: -U (C_{i+1} - C_{i-1}) / (2h)
        adv = U * eps * math.sin(k * h) / h * np.sin(k * x)
        # phi = (3/4 eps^3 - eps - Cn^2 lam1 eps) cos(kx) + eps^3/4 cos(3kx)
        a1 = 0.75 * eps ** 3 - eps - Cn * Cn * lam(1) * eps
        a3 = 0.25 * eps ** 3
        diff = (lam(1) * a1 * np.cos(k * x) + lam(3) * a3 * np.cos(3.0 * k * x)) / Pe
        return adv + diff

    eps_n, eps_o, U_n, U_o = 0.6, 0.45, 0.7, -0.3
    row = lambda a: np.tile(a, (ny, 1))
    st = {"C": row(eps_n * np.cos(k * x)), "C_old": row(eps_o * np.cos(k * x)),
          "u": np.full((ny, nx), U_n), "u_old": np.full((ny, nx), U_o),
          "v": np.zeros((ny + 1, nx)), "v_old": np.zeros((ny + 1, nx))}
    got = O.ch_explicit(case, geo, st)
    want = row(eps_n * np.cos(k * x) + dt * (1.5 * F(eps_n, U_n) - 0.5 * F(eps_o, U_o)))
    assert np.abs(got - want).max() <= 1e-13, np.abs(got - want).max()


def test_explicit_update_conserves_sum_before_fill():
    case = _scheme(W.sinusoid_wall_512x256(theta_deg=90.0, l_s=0.0, nx=64, ny=32), 1)
    geo = O.build_geometry(case)
    assert len(geo.gcell) > 0
    st = W.random_state(case, seed=5)
    C_pre = O.ch_explicit(case, geo, st)
    assert abs(C_pre.sum() - st["C"].sum()) <= 1e-13 * np.abs(st["C"]).sum()
    # and the full step takes it: mass before the fill equals the input mass
    _, info = O.step(case, geo, st)
    assert abs(info["mass_pre"] - st["C"].sum()) <= 1e-13 * np.abs(st["C"]).sum()


def test_explicit_and_semi_implicit_agree_to_second_order():
    nx, ny = 64, 32
    ratios = []
    for dt in (4.0e-5, 5.0e-6):
        base = _free_case(nx, ny, Cn=0.06, Pe=20.0, dt=dt)
        base = dataclasses.replace(base, drop_c=(1.0, 0.5), drop_r=0.3)
        geo = O.build_geometry(base)
        st = W.initial_state(base)
        # a first-order consistent history: C^{n-1} = C^n - dt F(C^n) with u = 0
        F0 = O.laplacian(O.chemical_potential(base, geo, st["C"]), base.h) / base.params.Pe
        st = dict(st)
        st["C_old"] = st["C"] - dt * F0
        d = {}
        for s in (0, 1):
            c = _scheme(base, s)
            _, info = O.step(c, geo, st)
            d[s] = info["C_pre"] - st["C"]
        ratios.append(np.abs(d[1] - d[0]).max() / np.abs(d[0]).max())
    # dt shrinks 8x: the relative difference should shrink ~8x (first order in dt)
    r = ratios[1] / ratios[0]
    assert ratios[0] < 0.05 and 1.0 / 16.0 < r < 1.0 / 4.0, ratios
