"""Pins of the semi-implicit momentum predictor of the oracle (params.ns_scheme = 1;
Appendix A.2, Eq. predictionSemi; reading R19).

* the velocity Helmholtz solves against a dense brute-force matrix of (1 - a L), L the
  5-point Laplacian of each component with its own x2 boundary rows (no-slip ghost rows for
  u, v = 0 on the walls), applied column by column;
* a discrete eigenvector (Fourier in x1 times sin(pi m (j + 1/2)/ny) for u) is divided by
  1 - a lambda exactly;
* with equal densities and viscosities (no mass-flux term) one semi-implicit predictor step
  agrees with the explicit AB2 one to O(dt^2) (the implicit half-viscous correction);
* the mass-flux term vanishes for equal densities and converges at second order to
  (rho'/(rho Pe)) (grad phi . grad) u for smooth fields.
"""
import math

import numpy as np
import pytest

from oracle import ib_pf2d as O
from workloads import cases


def _dense(fn, shape):
    n = shape[0] * shape[1]
    A = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = fn(e.reshape(shape)).reshape(-1)
    return A


def _lap_u(u, h):
    upad = np.vstack([-u[:1], u, -u[-1:]])
    return ((np.roll(u, -1, 1) + np.roll(u, 1, 1)) + (upad[2:] + upad[:-2]) - 4.0 * u) / (h * h)


def _lap_v(vi, h):
    # interior faces j = 1..ny-1, v = 0 on the wall rows
    vpad = np.vstack([np.zeros((1, vi.shape[1])), vi, np.zeros((1, vi.shape[1]))])
    return ((np.roll(vi, -1, 1) + np.roll(vi, 1, 1)) + (vpad[2:] + vpad[:-2]) - 4.0 * vi) / (h * h)


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 8)])
def test_velocity_helmholtz_matches_dense_solve(nx, ny):
    case = cases.flat_wall_case(nx=nx, ny=ny)
    h, a = case.h, 0.37 * case.h ** 2
    rng = np.random.default_rng(nx + ny)
    ru = rng.standard_normal((ny, nx))
    rv = np.zeros((ny + 1, nx))
    rv[1:ny] = rng.standard_normal((ny - 1, nx))
    du, dv = O.velocity_helmholtz(case, ru, rv, a)
    Au = np.eye(nx * ny) - a * _dense(lambda f: _lap_u(f, h), (ny, nx))
    Av = np.eye(nx * (ny - 1)) - a * _dense(lambda f: _lap_v(f, h), (ny - 1, nx))
    assert np.allclose(du.reshape(-1), np.linalg.solve(Au, ru.reshape(-1)), rtol=0, atol=1e-12)
    assert np.allclose(dv[1:ny].reshape(-1), np.linalg.solve(Av, rv[1:ny].reshape(-1)), rtol=0, atol=1e-12)
    assert np.all(dv[0] == 0.0) and np.all(dv[ny] == 0.0)


def test_eigenvector_is_divided_exactly():
    case = cases.flat_wall_case(nx=32, ny=16)
    nx, ny, h = case.nx, case.ny, case.h
    k, m, a = 3, 5, 2.0 * h * h
    x = np.arange(nx)
    j = np.arange(ny)
    u = np.cos(2 * np.pi * k * x / nx)[None, :] * np.sin(np.pi * m * (j + 0.5) / ny)[:, None]
    lam = -(4 / h ** 2) * (np.sin(np.pi * k / nx) ** 2 + np.sin(np.pi * m / (2 * ny)) ** 2)
    assert np.allclose(_lap_u(u, h), lam * u, atol=1e-9 * abs(lam))
    du, _ = O.velocity_helmholtz(case, u, np.zeros((ny + 1, nx)), a)
    assert np.allclose(du, u / (1.0 - a * lam), rtol=0, atol=1e-13)


def _predictor_pair(dt):
    case = cases.free_droplet_case(nx=64, ny=32, rho_ratio=1.0, mu_ratio=1.0, dt=dt)
    geo = O.build_geometry(case)
    st = cases.random_state(case, seed=5)
    st["u_old"], st["v_old"] = st["u"].copy(), st["v"].copy()
    out = {}
    for scheme in (0, 1):
        c = cases.with_params(case, ns_scheme=scheme)
        s = dict(st)
        # consistent start: the history bracket of each scheme at the current level
        C1 = s["C"]
        Nu, Nv, Vu, Vv = O.momentum_terms(c, C1, s["u"], s["v"])
        s["Hu"], s["Hv"] = (Nu + Vu, Nv + Vv) if scheme == 0 else (Nu, Nv)
        _, info = O.step(c, geo, s)
        out[scheme] = (info["u_star"] - st["u"], info["v_star"] - st["v"])
    return out


def test_semi_implicit_predictor_agrees_to_second_order():
    diffs = []
    for dt in (2e-4, 1e-4):
        out = _predictor_pair(dt)
        diffs.append(max(np.abs(out[1][0] - out[0][0]).max(), np.abs(out[1][1] - out[0][1]).max()))
        inc = np.abs(out[0][0]).max()
        assert diffs[-1] < 0.05 * inc, (diffs[-1], inc)
    assert 3.2 < diffs[0] / diffs[1] < 4.8, diffs


def test_mass_flux_term_vanishes_for_equal_densities():
    case = cases.with_params(cases.flat_wall_case(nx=32, ny=16, rho_ratio=1.0), ns_scheme=1)
    st = cases.random_state(case, seed=2)
    phi = np.random.default_rng(3).standard_normal((16, 32))
    mfu, mfv = O.mass_flux_term(case, st["C"], phi, st["u"], st["v"])
    assert np.all(mfu == 0.0) and np.all(mfv == 0.0)


def test_mass_flux_term_second_order():
    # u = sin(2 pi x) cos(pi y) with u = 0 at neither wall is not compatible with the ghost
    # rows, so the field lives in the interior rows only: C = 1 (liquid, rho = 1), phi and u
    # smooth and periodic in x1, compared on rows away from the walls
    errs = []
    for n in (32, 64):
        case = cases.flat_wall_case(nx=2 * n, ny=n, rho_ratio=10.0)
        h, nx, ny = case.h, case.nx, case.ny
        xf = np.arange(nx) * h                      # x1-faces
        yc = (np.arange(ny) + 0.5) * h
        xc = (np.arange(nx) + 0.5) * h
        X, Y = np.meshgrid(xc, yc)
        Xf, Yf = np.meshgrid(xf, yc)
        phi = np.sin(np.pi * X) * np.cos(2 * np.pi * Y)
        u = np.cos(np.pi * Xf) * np.sin(2 * np.pi * Yf)
        v = np.zeros((ny + 1, nx))
        C1 = np.ones((ny, nx))
        mfu, _ = O.mass_flux_term(case, C1, phi, u, v)
        rp = 0.5 * (1.0 - 1.0 / 10.0)
        exact = (rp / case.params.Pe) * (
            (np.pi * np.cos(np.pi * Xf) * np.cos(2 * np.pi * Yf)) * (-np.pi * np.sin(np.pi * Xf) * np.sin(2 * np.pi * Yf))
            + (-2 * np.pi * np.sin(np.pi * Xf) * np.sin(2 * np.pi * Yf)) * (2 * np.pi * np.cos(np.pi * Xf) * np.cos(2 * np.pi * Yf)))
        rows = slice(2, ny - 2)
        errs.append(np.abs(mfu[rows] - exact[rows]).max() / np.abs(exact).max())
    assert errs[1] < 0.3 * errs[0] and errs[1] < 1e-2, errs
