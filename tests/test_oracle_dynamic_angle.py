"""Pins of the dynamic contact angle (mu_f > 0) of the oracle: Eq. WallBCS_recast with the
readings R4 and R18, and the slip condition with the wetting bracket (Eq. UpdateVtan).

* mu_f -> 0: the per-step update converges to the static root of reading R4 (which is
  pinned against Eq. WallBCS by test_oracle_pins);
* mu_f -> infinity: C_I only moves with the wall-tangential advection, exactly by
  -dt v_t dC/dx_t;
* a uniform tangential velocity over a field linear along the wall gives v_t dC/dx_t in
  closed form;
* the ghost velocity with the bracket satisfies the discrete stress balance of Eq.
  SlipVelocityTangen (re-derived here, not the oracle's closed form);
* droplets with finite friction relax to the same static angle (the bracket vanishes at
  rest), more slowly the larger mu_f.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

from oracle import ib_pf2d as O
from workloads import cases

import wetting


def _inputs(n=64, seed=2):
    rng = np.random.default_rng(seed)
    case = cases.flat_wall_case()
    return (case, rng.uniform(-0.95, 0.95, n), rng.uniform(1.2, 3.0, n),
            rng.uniform(0.2, 1.0, n) * case.h)


@pytest.mark.parametrize("theta", [30.0, 60.0, 120.0, 150.0])
def test_small_friction_converges_to_the_static_root(theta):
    case, CM, gam, dn = _inputs()
    case = cases.with_params(case, theta_deg=theta, mu_f=1e-9)
    _, CI_static, _ = O.contact_angle_ghost(case, CM, gam, dn)
    CG, CI, B = O.dynamic_contact_ghost(case, CM, gam, dn, np.zeros_like(CM), np.zeros_like(CM))
    assert np.abs(CI - CI_static).max() < 1e-6
    assert np.abs(B).max() < 1e-5
    # and from any start, with the wetting residual of Eq. WallBCS at the new level vanishing
    # as mu_f Cn (C_I^{n+1} - C_I^n)/dt
    case2 = cases.with_params(case, mu_f=0.5)
    CI0 = np.random.default_rng(1).uniform(-0.9, 0.9, len(CM))
    CG, CI, B = O.dynamic_contact_ghost(case2, CM, gam, dn, CI0, np.zeros_like(CM))
    p = case2.params
    assert np.allclose(B, p.mu_f * p.Cn * (CI - CI0) / p.dt, rtol=1e-9, atol=1e-12)


def test_infinite_friction_only_advects():
    case, CM, gam, dn = _inputs()
    case = cases.with_params(case, theta_deg=50.0, mu_f=1e300)
    rng = np.random.default_rng(3)
    CI0 = rng.uniform(-0.9, 0.9, len(CM))
    adv = rng.standard_normal(len(CM))
    CG, CI, B = O.dynamic_contact_ghost(case, CM, gam, dn, CI0, adv)
    assert np.allclose(CI, CI0 - case.params.dt * adv, rtol=0, atol=1e-15)
    assert np.allclose(CI, (gam * CG + CM) / (gam + 1.0), atol=1e-13)     # Eq. UpdateC


def test_uniform_tangential_velocity_over_a_linear_field():
    # flat wall (n = (0, 1), t = (1, 0)): u = U everywhere, v = 0 and C = a + b x1 give
    # v_t = U and dC/dx_t = b at every intersect point away from the periodic seam
    case = cases.flat_wall_case(nx=64, ny=32)
    geo = O.build_geometry(case)
    h, nx, ny = case.h, case.nx, case.ny
    U, a, b = 0.37, 0.1, -0.8
    x = (np.arange(nx) + 0.5) * h
    C = np.tile(a + b * x, (ny, 1))
    u = np.full((ny, nx), U)
    v = np.zeros((ny + 1, nx))
    adv, gt = O.wall_advection(case, geo, u, v, C)
    i = geo.gcell % nx
    inner = (i > 2) & (i < nx - 3)
    assert np.allclose(gt[inner], b, rtol=0, atol=1e-12)
    assert np.allclose(adv[inner], U * b, rtol=0, atol=1e-12)


@pytest.mark.parametrize("l_s", [0.005, 0.02])
def test_slip_with_bracket_satisfies_the_stress_balance(l_s):
    # mu V_t,I / l_s = mu (V_tM - V_tG)/((gamma+1) dn) - (1/Ca) B dC/dx_t, with
    # V_t,I = (gamma V_tG + V_tM)/(gamma + 1) and the 2-point slope through G and M
    case, _, gam, dn = _inputs(seed=7)
    case = cases.with_params(case, l_s=l_s, mu_f=1.0)
    rng = np.random.default_rng(8)
    k = len(gam)
    ang = rng.uniform(0.0, 2.0 * math.pi, k)
    n = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    uM, vM = rng.standard_normal(k), rng.standard_normal(k)
    B, gt, mu_I = rng.standard_normal(k), rng.standard_normal(k), rng.uniform(0.1, 1.0, k)
    uG, vG = O.slip_ghost(case, uM, vM, n, gam, dn, B, gt, mu_I)
    t = np.stack([n[:, 1], -n[:, 0]], axis=1)
    VtG = uG * t[:, 0] + vG * t[:, 1]
    VtM = uM * t[:, 0] + vM * t[:, 1]
    VtI = (gam * VtG + VtM) / (gam + 1.0)
    lhs = mu_I * VtI / l_s
    rhs = mu_I * (VtM - VtG) / ((gam + 1.0) * dn) - B * gt / case.params.Ca
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-9 * np.abs(rhs).max())
    # normal component: Eq. NoPenetration
    VnG = uG * n[:, 0] + vG * n[:, 1]
    assert np.allclose(VnG, -(uM * n[:, 0] + vM * n[:, 1]) / gam, atol=1e-13)


def _relax_dynamic(spec):
    import dataclasses
    from oracle import ib_pf2d as O2
    from workloads import cases as W
    import wetting as wt
    th, mu_f, start = spec
    case = W.flat_wall_case(nx=64, ny=32, theta_deg=th, Cn=0.04, dt=4e-4)
    case = W.with_params(case, mu_f=mu_f)
    if start == "cap":
        r, _, _ = wt.cap_shape(math.pi * 0.09 / 2.0, th)
        case = dataclasses.replace(case, drop_c=(1.0, 0.1 - r * math.cos(math.radians(th))), drop_r=r)
    geo = O2.build_geometry(case)
    st = W.initial_state(case)
    out = []
    for k in range(1, 12501):
        st, info = O2.step(case, geo, st)
        if k % 2500 == 0:
            out.append((wt.flat_wall_cap(case, st["C"], 0.1)[0], float(np.abs(info["B"]).max()),
                        bool(np.isfinite(st["C"]).all() and np.isfinite(st["C_I"]).all())))
    return out


RUNS = [(60.0, 0.1, "cap"), (60.0, 0.1, "semi"), (60.0, 1.0, "semi"), (120.0, 0.1, "semi")]


@pytest.fixture(scope="module")
def runs():
    with mp.get_context("spawn").Pool(len(RUNS)) as pool:
        return dict(zip(RUNS, pool.map(_relax_dynamic, RUNS)))


@pytest.mark.parametrize("spec", RUNS)
def test_finite_friction_reaches_the_static_angle(runs, spec):
    hist = runs[spec]
    assert all(h[2] for h in hist)
    assert abs(hist[-1][0] - spec[0]) < 1.0, [round(h[0], 3) for h in hist]


def test_larger_friction_spreads_more_slowly(runs):
    # at t = 1 the droplet with mu_f = 1 is further from 60 deg than the one with 0.1
    a_fast = runs[(60.0, 0.1, "semi")][0][0]
    a_slow = runs[(60.0, 1.0, "semi")][0][0]
    assert a_slow - 60.0 > a_fast - 60.0 > 0.0, (a_fast, a_slow)
