"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: dense brute-force
solves, closed forms (tanh profile, Laplace law, circular-cap geometry, 3-point Lagrange
derivatives), invariants (mass of the semi-implicit CH solve, discrete divergence) and
hand-derived geometry (tests/golden).
"""
import json
import math
from dataclasses import replace
from pathlib import Path

import numpy as np
import pytest

from oracle import ib_pf2d as O
from workloads import cases

GOLDEN = Path(__file__).resolve().parent / "golden"


def _dense_operator(fn, ny, nx):
    """Matrix of the linear map fn on ny x nx fields, column by column (brute force)."""
    n = nx * ny
    A = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = fn(e.reshape(ny, nx)).reshape(-1)
    return A


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 8)])
def test_ch_solve_matches_dense_brute_force(nx, ny):
    # Appendix A.1: the combined operator L^2 - (S/Cn^2) L + 1.5 Pe/(Cn^2 dt) built from
    # the 5-point stencil and inverted densely must equal the transform solve.
    case = cases.with_params(cases.flat_wall_case(nx=nx, ny=ny), Cn=0.05, dt=1e-3)
    p = case.params
    L = _dense_operator(lambda a: O.laplacian(a, case.h), ny, nx)
    eta2 = p.Cn ** 2
    A = L @ L - (p.S / eta2) * L + 1.5 * p.Pe / (eta2 * p.dt) * np.eye(nx * ny)
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((ny, nx))
    ref = np.linalg.solve(A, Q.reshape(-1)).reshape(ny, nx)
    got = O.ch_solve(case, Q)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 8)])
def test_poisson_solve_matches_dense_brute_force(nx, ny):
    # Eq. PressurePoisson with zero-flux x2 walls: minimum-norm (zero-mean) solution
    case = cases.flat_wall_case(nx=nx, ny=ny)
    L = _dense_operator(lambda a: O.laplacian(a, case.h), ny, nx)
    rng = np.random.default_rng(2)
    rhs = rng.standard_normal((ny, nx))
    rhs -= rhs.mean()
    ref = np.linalg.lstsq(L, rhs.reshape(-1), rcond=None)[0].reshape(ny, nx)
    got = O.poisson_solve(case, rhs)
    assert abs(got.mean()) < 1e-12 * np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


def test_two_stage_helmholtz_equals_combined_symbol():
    # With S >= Cn^2 sqrt(6 Pe/dt) alpha_s is real and the paper's two Helmholtz solves
    # (Eq. Helmholtz1 then Eq. Helmholtz2) must reproduce the combined solve.
    base = cases.flat_wall_case(nx=32, ny=16)
    p = base.params
    s_min = p.Cn * math.sqrt(6.0 * p.Pe / p.dt)
    case = cases.with_params(base, S=1.5 * s_min)
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((16, 32)) * 1e6
    a = O.ch_solve(case, Q)
    b = O.ch_solve_two_stage(case, Q)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()
    with pytest.raises(ValueError):
        O.ch_solve_two_stage(cases.with_params(base, S=0.5 * s_min), Q)


def test_laplacian_second_order():
    # 5-point stencil against the analytic Laplacian of a field with zero normal
    # derivative at the x2 walls; error must fall ~4x per refinement.
    errs = []
    for nx in (32, 64, 128):
        ny = nx // 2
        h = 2.0 / nx
        x = (np.arange(nx) + 0.5) * h
        y = (np.arange(ny) + 0.5) * h
        X, Y = np.meshgrid(x, y)
        f = np.sin(np.pi * X) * np.cos(np.pi * Y)
        ex = -2.0 * np.pi ** 2 * f
        errs.append(np.abs(O.laplacian(f, h) - ex).max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_momentum_rhs_second_order():
    # Convective + viscous bracket of Eq. PredictionExp with uniform rho = mu = 1 (C = 1)
    # against -(u.grad)u + (1/Re) lap u for a divergence-free field that vanishes on the
    # walls: u = pi sin(2 pi x) sin(2 pi y), v = -2 pi cos(2 pi x) sin^2(pi y).
    errs = []
    for nx in (32, 64, 128):
        ny = nx // 2
        case = cases.flat_wall_case(nx=nx, ny=ny)
        h = case.h
        Re = case.params.Re
        xf = np.arange(nx) * h
        xc = (np.arange(nx) + 0.5) * h
        yc = (np.arange(ny) + 0.5) * h
        yf = np.arange(ny + 1) * h

        def uf(x, y):
            return np.pi * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)

        def vf(x, y):
            return -2 * np.pi * np.cos(2 * np.pi * x) * np.sin(np.pi * y) ** 2

        Xu, Yu = np.meshgrid(xf, yc)
        Xv, Yv = np.meshgrid(xc, yf)
        u = uf(Xu, Yu)
        v = vf(Xv, Yv)
        C = np.ones((ny, nx))
        Hu, Hv = O.momentum_rhs(case, C, u, v)
        # analytic at the x1-faces
        ux = 2 * np.pi ** 2 * np.cos(2 * np.pi * Xu) * np.sin(2 * np.pi * Yu)
        uy = 2 * np.pi ** 2 * np.sin(2 * np.pi * Xu) * np.cos(2 * np.pi * Yu)
        lap_u = -8 * np.pi ** 2 * uf(Xu, Yu)
        ex_u = -(uf(Xu, Yu) * ux + vf(Xu, Yu) * uy) + lap_u / Re
        vx = 4 * np.pi ** 2 * np.sin(2 * np.pi * Xv) * np.sin(np.pi * Yv) ** 2
        vy = -2 * np.pi ** 2 * np.cos(2 * np.pi * Xv) * np.sin(2 * np.pi * Yv)
        lap_v = (8 * np.pi ** 3 * np.cos(2 * np.pi * Xv) * np.sin(np.pi * Yv) ** 2
                 - 4 * np.pi ** 3 * np.cos(2 * np.pi * Xv) * np.cos(2 * np.pi * Yv))
        ex_v = -(uf(Xv, Yv) * vx + vf(Xv, Yv) * vy) + lap_v / Re
        inner = slice(2, ny - 2)
        errs.append(max(np.abs(Hu - ex_u)[inner].max(), np.abs(Hv - ex_v)[2:ny - 1].max()))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0, errs


def _random_case_state(nx=64, ny=32, seed=5):
    case = cases.sinusoid_wall_512x256(nx=nx, ny=ny, theta_deg=60.0, l_s=0.01)
    return case, cases.random_state(case, seed=seed)


def test_mass_of_ch_solve_invariant():
    # k = 0 mode: sum C_pre^{n+1} = sum(2 C^n - C^{n-1}/2) / 1.5, to round-off, because
    # the advective flux divergence and the Laplacian sum to zero (periodic x1, zero
    # flux at the walls).
    case, st = _random_case_state()
    geo = O.build_geometry(case)
    for _ in range(3):
        expect = float((2.0 * st["C"] - 0.5 * st["C_old"]).sum()) / 1.5
        st, info = O.step(case, geo, st)
        assert abs(info["mass_pre"] - expect) <= 1e-12 * np.abs(st["C"]).sum()


def test_tanh_profile_is_discrete_steady_state():
    # Eq. InitializingC: two flat interfaces across a periodic channel without walls; with
    # equal densities the profile is an equilibrium of the CH + NS system, so it must stay
    # put (to the O((h/Cn)^2) discretisation error) and the velocity must stay ~0.
    case = cases.with_params(cases.free_droplet_case(nx=128, ny=32, Cn=0.02), dt=1e-4)
    nx, ny, h = case.nx, case.ny, case.h
    x = (np.arange(nx) + 0.5) * h
    C0 = np.tanh((0.25 * case.lx - np.abs(x - 0.5 * case.lx)) / (math.sqrt(2) * case.params.Cn))
    st = cases.initial_state(case)
    st["C"] = np.tile(C0, (ny, 1))
    st["C_old"] = st["C"].copy()
    geo = O.build_geometry(case)
    assert len(geo.gcell) == 0
    phi0 = (C0 ** 3 - C0) - case.params.Cn ** 2 * O.laplacian(st["C"], h)[0]
    assert np.abs(phi0).max() < 0.05          # discrete chemical potential ~ 0
    for _ in range(50):
        st, info = O.step(case, geo, st)
    assert np.abs(st["C"] - C0[None, :]).max() < 5e-3
    assert np.abs(st["u"]).max() < 1e-8 and np.abs(st["v"]).max() < 1e-8


def test_geometry_flat_wall_matches_hand_derivation():
    g = json.loads((GOLDEN / "flat_wall_128x64_geometry.json").read_text())
    case = cases.flat_wall_128x64()
    geo = O.build_geometry(case)
    gj, gi = np.divmod(geo.gcell, case.nx)
    assert len(geo.gcell) == g["ghost_count"]
    assert sorted(set(gj.tolist())) == g["ghost_rows"]
    assert np.array_equal(geo.n, np.tile(g["normal"], (len(gi), 1)))
    assert np.allclose(geo.dn, g["dn"], rtol=1e-12, atol=0)
    assert np.allclose(geo.gamma, g["gamma"], rtol=1e-12, atol=0)
    for key, arr in (("alpha_c_rows", geo.alpha_c), ("alpha_u_rows", geo.alpha_u),
                     ("alpha_v_rows", geo.alpha_v)):
        for row, val in g[key].items():
            assert np.all(arr[int(row)] == val), (key, row)
    assert len(geo.fu) == g["face_u_count"] and len(geo.fv) == g["face_v_count"]
    ap1_rows = np.unique(geo.ap1 // case.nx)
    assert g["ip1_row"] in ap1_rows and set(ap1_rows) == {g["ip1_row"] - 1, g["ip1_row"], g["ip1_row"] + 1}
    ap2_rows = np.unique(geo.ap2 // case.nx)
    assert set(ap2_rows) == {g["ip2_row"] - 1, g["ip2_row"], g["ip2_row"] + 1}


def _ip_positions(case, geo, s):
    """IP_s = G + (dn + d1 + s d2) n (Sec. 4.1.2), from the ghost centres and the tables."""
    h, nx = case.h, case.nx
    gx = (geo.gcell % nx + 0.5) * h
    gy = (geo.gcell // nx + 0.5) * h
    d = geo.dn + case.params.d1 + s * case.params.d2
    return gx + d * geo.n[:, 0], gy + d * geo.n[:, 1]


def _linear_gather_error(case, geo, a=3.0, b=0.7, c=1.3):
    """max |gathered - exact| of f = a + b x + c y at IP1 and IP2, with the x1 coordinate of
    each averaging point unwrapped to the side of the periodic box nearest the IP."""
    h, nx = case.h, case.nx
    err = 0.0
    for s, ap, w in ((1, geo.ap1, geo.w1), (2, geo.ap2, geo.w2)):
        px, py = _ip_positions(case, geo, s)
        ax = (ap % nx + 0.5) * h
        ax = ax - case.lx * np.round((ax - px[:, None]) / case.lx)
        ay = (ap // nx + 0.5) * h
        got = (w * (a + b * ax + c * ay)).sum(axis=1)
        err = max(err, float(np.abs(got - (a + b * px + c * py)).max()))
    return err


def test_idw_weights_constants_and_symmetric_linear_fields():
    # Eq. weright averaged (plain inverse-distance weights, params.weights = 1): sum W = 1
    # (constants exact) and W >= 0 on a curved wall; on the flat wall the stencil is
    # symmetric in x1 about the IP, so fields linear in x1 are exact.
    case, _ = _random_case_state()
    case = cases.with_params(case, weights=1)
    geo = O.build_geometry(case)
    assert np.allclose(geo.w1.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(geo.w2.sum(axis=1), 1.0, atol=1e-14)
    assert (geo.w1 >= 0).all() and (geo.w2 >= 0).all()
    flat = cases.with_params(cases.flat_wall_case(nx=64, ny=32), weights=1)
    gf = O.build_geometry(flat)
    h = flat.h
    x = (np.arange(flat.nx) + 0.5) * h
    f = np.tile(3.0 + 0.7 * x, (flat.ny, 1)).reshape(-1)
    ip = O._gather(f, gf.ap1, gf.w1)
    gx = (gf.gcell % flat.nx + 0.5) * h
    interior = (gf.gcell % flat.nx > 0) & (gf.gcell % flat.nx < flat.nx - 1)
    assert np.allclose(ip[interior], (3.0 + 0.7 * gx)[interior], rtol=0, atol=1e-13)


def test_idw_weights_first_order_on_general_linear_fields():
    # The plain inverse-distance average is not exact for a general linear field on the
    # sinusoidal wall (asymmetric stencils): its error is first order, bounded by a fraction
    # of h |grad f| and about halved when h is halved.
    errs = []
    for nx in (256, 512):
        case = cases.with_params(cases.sinusoid_wall_512x256(nx=nx, ny=nx // 2), weights=1)
        e = _linear_gather_error(case, O.build_geometry(case))
        errs.append(e / (case.h * math.hypot(0.7, 1.3)))
    assert 0.05 < errs[0] < 0.5 and 0.05 < errs[1] < 0.5, errs
    assert abs(errs[0] / errs[1] - 1.0) < 0.25, errs     # error / h constant: first order


@pytest.mark.parametrize("nx", [64, 256])
def test_linear_exact_weights_reproduce_linear_fields(nx):
    # Reading R17 (default weights): W1/W2 reproduce constants and every linear field
    # exactly at IP1 and IP2, on the curved wall and the flat one.
    for case in (cases.sinusoid_wall_512x256(nx=nx, ny=nx // 2), cases.flat_wall_case(nx=nx, ny=nx // 2)):
        geo = O.build_geometry(case)
        assert np.allclose(geo.w1.sum(axis=1), 1.0, atol=1e-13)
        assert np.allclose(geo.w2.sum(axis=1), 1.0, atol=1e-13)
        assert _linear_gather_error(case, geo) < 1e-12
        assert _linear_gather_error(case, geo, a=-1.0, b=-5.0, c=2.5) < 1e-12


def _lagrange_slope_at_I(CG, CI, CM, dn, gamma):
    """d/dn at I of the parabola through (-dn, CG), (0, CI), (gamma dn, CM)."""
    coef = np.polyfit([-dn, 0.0, gamma * dn], [CG, CI, CM], 2)
    return coef[1]


@pytest.mark.parametrize("theta", [30.0, 60.0, 90.0, 120.0, 150.0])
def test_contact_angle_ghost_satisfies_wetting_condition(theta):
    # Static form of Eq. WallBCS at I, with the normal derivative taken from the 3-point
    # parabola through G, I, M (numpy.polyfit, independent of the oracle's algebra).
    case = cases.with_params(cases.flat_wall_case(), theta_deg=theta)
    p = case.params
    rng = np.random.default_rng(4)
    CM = rng.uniform(-1.0, 1.0, 64)
    gamma = rng.uniform(1.2, 3.0, 64)
    dn = rng.uniform(0.2, 1.0, 64) * case.h
    CG, CI, clamped = O.contact_angle_ghost(case, CM, gamma, dn)
    assert clamped == 0
    assert np.all(np.abs(CI) <= 1.0)
    # I lies on the straight line between G and M (Eq. interpolationAtWall)
    assert np.allclose(CI, (gamma * CG + CM) / (gamma + 1.0), atol=1e-13)
    ct = math.cos(math.radians(theta))
    for k in range(64):
        slope = _lagrange_slope_at_I(CG[k], CI[k], CM[k], dn[k], gamma[k])
        resid = O.KAPPA * p.Cn * slope + ct * 0.75 * (1.0 - CI[k] ** 2)
        assert abs(resid) < 1e-9
    if theta == 90.0:
        assert np.allclose(CG, CM, atol=1e-14)   # zero normal gradient
    # pure phases are fixed points; beyond them the wall energy is flat (g' = 0), so an
    # overshooting mirror value is simply continued (zero normal gradient)
    CG1, _, _ = O.contact_angle_ghost(case, np.array([1.0, -1.0, 1.07, -1.2]),
                                      np.array([1.5, 1.5, 1.5, 2.0]),
                                      np.array([0.5, 0.5, 0.5, 0.7]) * case.h)
    assert np.allclose(CG1, [1.0, -1.0, 1.07, -1.2], atol=1e-14)


def test_contact_angle_fill_reproduces_inclined_tanh_profile():
    # A planar interface meeting the flat wall at theta: C = tanh(s / (sqrt 2 Cn)) with s
    # the signed distance to the line; in the continuum it satisfies kappa Cn dC/dn =
    # -cos(theta) g'(C) exactly.  Fed the exact value at the mirror point, the ghost fill
    # must reproduce C at the ghost centres with an error that falls with h; fed the
    # inverse-distance average, the error stays small.  Liquid (C = +1) on the side the
    # angle is measured through, so theta < 90 deg tilts the liquid over the wall.
    th = math.radians(60.0)
    nrm = np.array([math.sin(th), math.cos(th)])      # points from liquid to gas

    def profile(case, X, Y):
        s = -((X - 1.0) * nrm[0] + (Y - 0.1) * nrm[1])
        return np.tanh(s / (math.sqrt(2) * case.params.Cn))

    errs_exact, errs_idw = [], []
    for nx in (128, 256, 512):
        case = cases.flat_wall_case(nx=nx, ny=nx // 2, theta_deg=60.0, Cn=0.04)
        h = case.h
        geo = O.build_geometry(case)
        x = (np.arange(case.nx) + 0.5) * h
        y = (np.arange(case.ny) + 0.5) * h
        X, Y = np.meshgrid(x, y)
        C = profile(case, X, Y)
        gx = X.reshape(-1)[geo.gcell]
        gy = Y.reshape(-1)[geo.gcell]
        near = np.abs(gx - 1.0) < 0.3
        exact = C.reshape(-1)[geo.gcell]
        sM = geo.dn + case.params.d1
        CM_exact = profile(case, gx + sM * geo.n[:, 0], gy + sM * geo.n[:, 1])
        CG, _, _ = O.contact_angle_ghost(case, CM_exact, geo.gamma, geo.dn)
        errs_exact.append(np.abs(CG - exact)[near].max())
        CM = O.mirror_value(C.reshape(-1), geo)
        CG, _, _ = O.contact_angle_ghost(case, CM, geo.gamma, geo.dn)
        errs_idw.append(np.abs(CG - exact)[near].max())
    assert errs_exact[0] / errs_exact[1] > 3.0 and errs_exact[1] / errs_exact[2] > 3.0, errs_exact
    assert max(errs_idw) < 0.03, errs_idw
    # the opposite sign of cos(theta) must not fit the same profile
    case120 = cases.with_params(case, theta_deg=120.0)
    CG, _, _ = O.contact_angle_ghost(case120, CM_exact, geo.gamma, geo.dn)
    assert np.abs(CG - exact)[near].max() > 100 * errs_exact[2]


def test_slip_ghost_special_cases():
    # Eqs. NoPenetration and UpdateVtan: the velocity at I, linearly interpolated between
    # G and M, has zero normal component; l_s = 0 gives V_G = -V_M / gamma; l_s -> inf
    # gives V_tG = V_tM; in general (V_tI / l_s) = (V_tM - V_tG) / ((gamma + 1) dn).
    rng = np.random.default_rng(6)
    n = 50
    ang = rng.uniform(0, 2 * np.pi, n)
    nrm = np.stack([np.cos(ang), np.sin(ang)], axis=1)
    gamma = rng.uniform(1.2, 3.0, n)
    dn = rng.uniform(0.002, 0.01, n)
    uM, vM = rng.standard_normal(n), rng.standard_normal(n)
    t = np.stack([nrm[:, 1], -nrm[:, 0]], axis=1)
    VnM = uM * nrm[:, 0] + vM * nrm[:, 1]
    VtM = uM * t[:, 0] + vM * t[:, 1]
    for ls in (0.0, 0.004, 0.03, 1e30):
        case = cases.with_params(cases.flat_wall_case(), l_s=ls)
        uG, vG = O.slip_ghost(case, uM, vM, nrm, gamma, dn)
        VnG = uG * nrm[:, 0] + vG * nrm[:, 1]
        VtG = uG * t[:, 0] + vG * t[:, 1]
        for k in range(n):   # value at I by linear interpolation along the normal line
            VnI = np.interp(0.0, [-dn[k], gamma[k] * dn[k]], [VnG[k], VnM[k]])
            assert abs(VnI) < 1e-12
        VtI = (gamma * VtG + VtM) / (gamma + 1.0)
        if ls == 0.0:
            assert np.allclose(uG, -uM / gamma, atol=1e-14) and np.allclose(vG, -vM / gamma, atol=1e-14)
        elif ls > 1e20:
            assert np.allclose(VtG, VtM, atol=1e-12)
        else:
            assert np.allclose(VtI / ls, (VtM - VtG) / ((gamma + 1.0) * dn), rtol=1e-10)


def test_properties_stay_within_the_phase_values():
    # reading R11: rho and mu are bounded by the pure-phase values for any C, so
    # rho >= rho0 = min(rho_l, rho_g) as the Dodd-Ferrante split requires
    case = cases.flat_wall_case(rho_ratio=10.0, mu_ratio=20.0)
    rho, mu, rho0 = O._props(case)
    c = np.linspace(-1.5, 1.5, 301)
    assert rho(c).min() >= rho0 - 1e-15 and rho(c).max() <= 1.0 + 1e-15
    assert mu(c).min() >= 1.0 / 20.0 - 1e-15 and mu(c).max() <= 1.0 + 1e-15
    assert rho(np.array([0.3]))[0] == pytest.approx(0.5 * (1.3 * 1.0 + 0.7 * 0.1))


@pytest.mark.parametrize("ratio", [1.0, 10.0])
def test_projection(ratio):
    # Eq. correction: with equal densities the corrected velocity is discretely
    # divergence free; with a density ratio the Dodd-Ferrante split leaves div u at the
    # level of the lagged P^ term, and the Poisson residual lap P - rhs is round-off
    # (checked with the stencil, independent of the transform solver).
    case = cases.flat_wall_case(nx=64, ny=32, theta_deg=70.0, rho_ratio=ratio, mu_ratio=ratio)
    geo = O.build_geometry(case)
    st = cases.random_state(case, seed=8)
    if ratio == 1.0:
        st["P"][:] = 0.0
        st["P_old"][:] = 0.0
    new, info = O.step(case, geo, st)
    res = O.laplacian(info["P"], case.h) - info["rhs_p"]
    assert np.abs(res).max() <= 1e-10 * np.abs(info["rhs_p"]).max()
    div = O.divergence(new["u"], new["v"], case.h)
    if ratio == 1.0:
        assert np.abs(div).max() < 1e-10
    assert np.isfinite(div).all()


def test_laplace_pressure_jump():
    # Free 2D droplet, equal densities: the pressure jump across the interface equals
    # sigma / R with sigma = 1/(Re Ca) (reading of the surface-tension prefactor); the
    # diffuse-interface error shrinks as the interface is resolved by more cells.
    errs = []
    for nx in (128, 256):
        case = cases.free_droplet_case(nx=nx, ny=nx // 2, R=0.3, Cn=0.02)
        geo = O.build_geometry(case)
        st = cases.initial_state(case)
        st, info = O.step(case, geo, st)
        P = info["P"]
        dp = P[case.ny // 2, case.nx // 2] - P[5, 5]
        expect = 1.0 / (case.params.Re * case.params.Ca * case.drop_r)
        errs.append(abs(dp - expect) / expect)
    assert errs[1] < 0.02 and errs[0] > 2.0 * errs[1], errs


def test_face_fix_on_flat_wall_in_closed_form():
    # Reading R10 on a 32 x 16 grid with the wall at x2 = 0.1 (h = 1/16): row 1 holds the
    # ghosts, row 0 solid cells, rows >= 2 fluid.  Listed faces, derived by hand: every
    # x1-face of row 1 (alpha_u = 0.4), and the x2-faces of rows 1 (alpha_v = 0) and 2
    # (alpha_v = 0.9).  With distinct ghost values per column the re-interpolated faces are
    # u(1, i) = (uG(i-1) + uG(i))/2 (periodic), v(1, i) = (0 + vG(i))/2 and
    # v(2, i) = (vG(i) + vcen(2, i))/2; no other face changes.
    case = cases.flat_wall_case(nx=32, ny=16)
    geo = O.build_geometry(case)
    nx, ny = 32, 16
    assert np.array_equal(geo.gcell, np.arange(nx) + nx)
    assert np.array_equal(np.sort(geo.fu), np.arange(nx) + nx)
    assert np.array_equal(np.sort(geo.fv), np.r_[np.arange(nx) + nx, np.arange(nx) + 2 * nx])
    rng = np.random.default_rng(5)
    uss = rng.standard_normal((ny, nx))
    vss = rng.standard_normal((ny + 1, nx))
    ucen = rng.standard_normal((ny, nx))
    vcen = rng.standard_normal((ny, nx))
    uG = rng.standard_normal(nx)
    vG = rng.standard_normal(nx)
    u2, v2 = O.face_fix(case, geo, uss, vss, ucen, vcen, uG, vG)
    i = np.arange(nx)
    assert np.array_equal(u2[1], 0.5 * (uG[(i - 1) % nx] + uG))
    assert np.array_equal(v2[1], 0.5 * (0.0 + vG))
    assert np.array_equal(v2[2], 0.5 * (vG + vcen[2]))
    keep_u = np.ones((ny, nx), bool)
    keep_u[1] = False
    keep_v = np.ones((ny + 1, nx), bool)
    keep_v[1:3] = False
    assert np.array_equal(u2[keep_u], uss[keep_u]) and np.array_equal(v2[keep_v], vss[keep_v])


def test_penalisation_zeroes_solid_faces_and_keeps_fluid_faces():
    # Eq. Penalization2, u** = alpha u*: on the flat wall of the 128 x 64 case the x1-faces of
    # rows 0..4 are wholly solid (alpha_u = 0, not re-interpolated) and those of rows >= 7
    # wholly fluid (alpha_u = 1): u** = 0 there and u** = u* respectively.
    case = cases.flat_wall_128x64()
    geo = O.build_geometry(case)
    st = cases.random_state(case, seed=21)
    _, info = O.step(case, geo, st)
    assert np.all(geo.alpha_u[:5] == 0.0) and np.all(geo.alpha_u[7:] == 1.0)
    assert np.all(info["u_ss"][:5] == 0.0)
    assert np.array_equal(info["u_ss"][7:], info["u_star"][7:])
    assert np.all(info["v_ss"][:5] == 0.0)
    assert np.array_equal(info["v_ss"][8:], info["v_star"][8:])


def test_mirror_value_of_linear_fields_is_the_value_at_M():
    # Eq. extrapolation with IP1 = M + d2 n, IP2 = M + 2 d2 n: 2 f(IP1) - f(IP2) = f(M) for a
    # linear f, and M = G + (1 + gamma) dn n (I = G + dn n, M = I + d1 n, gamma = d1/dn);
    # with the linear-exact weights (R17) every gather is exact, so the mirror value of a
    # linear field is its value at M -- on the sinusoidal wall, whose ghosts have normals in
    # every direction.  The phi fill (Sec. 4.2.2) copies that value: phi_G = phi_M.
    case = cases.sinusoid_wall_512x256(theta_deg=90.0, l_s=0.0)
    d1, d2 = cases._ghost_lengths(2.0 / 128)
    case = replace(case, nx=128, ny=64, params=replace(case.params, d1=d1, d2=d2))
    geo = O.build_geometry(case)
    nx, ny, h = case.nx, case.ny, case.h
    gi, gj = geo.gcell % nx, geo.gcell // nx
    G = np.stack([(gi + 0.5) * h, (gj + 0.5) * h], axis=1)
    M = G + ((1.0 + geo.gamma) * geo.dn)[:, None] * geo.n
    xc = (np.arange(nx) + 0.5) * h
    yc = (np.arange(ny) + 0.5) * h
    f = 0.3 + 0.0 * xc[None, :] - 1.7 * yc[:, None]           # linear in x2 (x1 is periodic)
    fM = O.mirror_value(f.reshape(-1), geo)
    assert np.abs(fM - (0.3 - 1.7 * M[:, 1])).max() < 1e-12
    rng = np.random.default_rng(4)
    C = np.tanh(rng.standard_normal((ny, nx)) * 0.1 + (yc[:, None] - 0.5) / 0.05)
    phi = O.chemical_potential(case, geo, C)
    assert np.array_equal(phi.reshape(-1)[geo.gcell], O.mirror_value(phi.reshape(-1).copy(), geo))
