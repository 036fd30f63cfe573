"""Pins of the 3D CPU oracle against what the paper and the mathematics fix.

* a 3D step with no solid and data invariant along y (or along x) is the 2D step of the
  remaining plane: the 2D oracle is pinned on its own (test_oracle_pins,
  test_oracle_explicit_pins), so this pins every stencil, both solves (or the explicit
  Cahn-Hilliard update), the momentum terms, the projection and the correction of the 3D
  oracle, including the index conventions of each axis;
* the eigen-solves against a dense brute-force matrix of the 7-point operator;
* the pre-fill mass invariant of the CH solve and a divergence-free velocity after the
  projection;
* geometry: flat-wall fractions exact, sphere fractions against the sphere's volume,
  intersect points on the sphere, normals radial to O(h), x <-> y symmetry of a centred
  sphere;
* the vector slip formula against the 2D one where the normal lies in a plane, and its
  closed-form cases (no penetration at I, no slip, free slip, the slip-length law) for
  normals in any direction;
* the re-interpolated face lists of a flat wall, derived by hand;
* the semi-implicit predictor (Appendix A.2): the step's reduction to the pinned 2D one,
  the velocity Helmholtz solves against dense operators, the mass-flux term zero for equal
  densities and second order on smooth fields.
"""
import math

import numpy as np
import pytest

from oracle import ib_pf2d as O2
from oracle import ib_pf3d as O3
from workloads import cases as W


def _free3d(nx, ny, nz, rho_ratio=10.0, mu_ratio=10.0):
    return W.flat_wall_case3d(nx=nx, ny=ny, nz=nz, geom_kind=W.GEOM_NONE, Cn=0.1,
                              rho_ratio=rho_ratio, mu_ratio=mu_ratio)


def _case2d_like(c3, n1, n2, l1):
    p = c3.params
    return W.Case2D("plane", n1, n2, l1, n2 * c3.h, W.GEOM_NONE, (0.0,) * 4, (0.0, 0.0), 0.0,
                    p, 1)


def _plane_state(rng, n1, n2):
    """A smooth random 2D state (C, u, v, H, P at two levels) on an n2 x n1 plane."""
    def smooth(shape, amp):
        a = rng.standard_normal(shape)
        for _ in range(3):
            a = 0.25 * (np.roll(a, 1, 1) + np.roll(a, -1, 1)) + 0.5 * a
            a[1:-1] = 0.25 * (a[:-2] + a[2:]) + 0.5 * a[1:-1]
        return amp * a / np.abs(a).max()
    st = {"C": 0.8 * smooth((n2, n1), 1.0), "C_old": 0.8 * smooth((n2, n1), 1.0)}
    for k in ("u", "u_old", "Hu"):
        st[k] = smooth((n2, n1), 0.1)
    for k in ("v", "v_old", "Hv"):
        a = smooth((n2 + 1, n1), 0.1)
        a[0] = a[-1] = 0.0
        st[k] = a
    st["P"] = smooth((n2, n1), 1.0)
    st["P_old"] = smooth((n2, n1), 1.0)
    return st


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("axis,scheme,ns", [("y", 0, 0), ("x", 0, 0), ("y", 1, 0), ("x", 1, 0),
                                            ("y", 0, 1), ("x", 0, 1)])
def test_step_reduces_to_2d_plane(axis, scheme, ns):
    import dataclasses
    rng = np.random.default_rng(17)
    n1, n2, nrep = 16, 8, 4
    if axis == "y":      # data varies in (x, z), constant along y
        c3 = _free3d(n1, nrep, n2)
    else:                # data varies in (y, z), constant along x
        c3 = _free3d(nrep, n1, n2)
        c3 = W.Case3D(c3.name, nrep, n1, n2, nrep * c3.h, n1 * c3.h, n2 * c3.h, c3.geom_kind,
                      c3.geom_p, c3.drop_c, c3.drop_r, c3.params, 1)
    c3 = dataclasses.replace(c3, params=dataclasses.replace(c3.params, ch_scheme=scheme, ns_scheme=ns))
    c2 = _case2d_like(c3, n1, n2, n1 * c3.h)
    s2 = _plane_state(rng, n1, n2)
    zero3 = np.zeros((n2, c3.ny, c3.nx))
    s3 = {}
    if axis == "y":
        ext = lambda a: np.repeat(a[:, None, :], nrep, axis=1)
        s3 = {"C": ext(s2["C"]), "C_old": ext(s2["C_old"]),
              "u": ext(s2["u"]), "u_old": ext(s2["u_old"]), "Hu": ext(s2["Hu"]),
              "v": zero3.copy(), "v_old": zero3.copy(), "Hv": zero3.copy(),
              "w": ext(s2["v"]), "w_old": ext(s2["v_old"]), "Hw": ext(s2["Hv"]),
              "P": ext(s2["P"]), "P_old": ext(s2["P_old"])}
    else:
        ext = lambda a: np.repeat(a[:, :, None], nrep, axis=2)
        s3 = {"C": ext(s2["C"]), "C_old": ext(s2["C_old"]),
              "v": ext(s2["u"]), "v_old": ext(s2["u_old"]), "Hv": ext(s2["Hu"]),
              "u": zero3.copy(), "u_old": zero3.copy(), "Hu": zero3.copy(),
              "w": ext(s2["v"]), "w_old": ext(s2["v_old"]), "Hw": ext(s2["Hv"]),
              "P": ext(s2["P"]), "P_old": ext(s2["P_old"])}
    g2 = O2.build_geometry(c2)
    g3 = O3.build_geometry3(c3)
    assert len(g3.gcell) == 0
    r2, _ = O2.step(c2, g2, s2)
    r3, _ = O3.step3(c3, g3, s3)
    tang = "u" if axis == "y" else "v"
    other = "v" if axis == "y" else "u"
    for rep in range(nrep):
        sl = (slice(None), rep, slice(None)) if axis == "y" else (slice(None), slice(None), rep)
        assert _rel(r3["C"][sl], r2["C"]) < 1e-12
        assert _rel(r3[tang][sl], r2["u"]) < 1e-12
        assert _rel(r3["H" + tang][sl], r2["Hu"]) < 1e-12
        assert _rel(r3["w"][sl], r2["v"]) < 1e-12
        assert _rel(r3["Hw"][sl], r2["Hv"]) < 1e-12
        p3 = r3["P"][sl] - r3["P"][sl].mean()
        p2 = r2["P"] - r2["P"].mean()
        assert _rel(p3, p2) < 1e-11
    assert np.abs(r3[other]).max() < 1e-14


def test_solves_against_dense_operator():
    nx, ny, nz, h = 4, 4, 4, 0.25
    n = nx * ny * nz
    L = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = 1.0
        L[:, col] = O3.laplacian3(e.reshape(nz, ny, nx), h).reshape(-1)
    case = _free3d(nx, ny, nz)
    case = W.Case3D(case.name, nx, ny, nz, nx * h, ny * h, nz * h, case.geom_kind, case.geom_p,
                    case.drop_c, case.drop_r, case.params, 1)
    rng = np.random.default_rng(3)
    Q = rng.standard_normal((nz, ny, nx))
    p = case.params
    eta2 = p.Cn ** 2
    A = L @ L - (p.S / eta2) * L + 1.5 * p.Pe / (eta2 * p.dt) * np.eye(n)
    c_dense = np.linalg.solve(A, Q.reshape(-1))
    assert _rel(O3.ch_solve3(case, Q).reshape(-1), c_dense) < 1e-12
    rhs = Q - Q.mean()
    P = O3.poisson_solve3(case, rhs)
    assert _rel(O3.laplacian3(P, h), rhs) < 1e-11
    assert abs(P.mean()) < 1e-12


def test_mass_invariant_and_divergence_free():
    case = W.small_sphere_case(16)
    geo = O3.build_geometry3(case)
    st = W.random_state3d(case, seed=5)
    st["C_old"] = st["C"].copy()          # equal levels: sum C_pre = sum C
    new, info = O3.step3(case, geo, st)
    assert abs(info["mass_pre"] - st["C"].sum()) <= 1e-11 * np.abs(st["C"]).sum()
    div = O3.divergence3(new["u"], new["v"], new["w"], case.h)
    vel = max(np.abs(new["u"]).max(), np.abs(new["v"]).max(), np.abs(new["w"]).max())
    assert np.abs(div).max() * case.h < 1e-10 * vel


def test_flat_wall_fractions_exact():
    case = W.flat_wall_case3d(nx=8, ny=8, nz=8, wall_z=0.55)   # h = 0.25: wall inside cell 2
    a = O3.volume_fractions3(case, (0.0, 0.0, 0.0), (8, 8, 8))
    assert np.all(a[:2] == 0.0) and np.all(a[3:] == 1.0)
    assert np.allclose(a[2], (0.75 - 0.55) / 0.25 + 0.0, atol=1.0 / O3.NSUB3)
    # subgrid planes z = 0.5 + (a + 1/2) / 64: plane 2 (0.5390625) is solid, plane 3
    # (0.5546875) is fluid, so 13 of the 16 planes count as fluid
    assert np.all(a[2] == 13.0 / 16.0)


def test_sphere_fractions_volume_and_symmetry():
    case = W.small_sphere_case(16)
    a = O3.volume_fractions3(case, (0.0, 0.0, 0.0), (16, 16, 16))
    solid_vol = ((1.0 - a).sum()) * case.h ** 3
    exact = 4.0 / 3.0 * math.pi * 0.25 ** 3
    assert abs(solid_vol - exact) < 2e-3 * exact
    assert np.array_equal(a, np.transpose(a, (0, 2, 1)))        # x <-> y
    assert np.array_equal(a, a[:, :, ::-1]) and np.array_equal(a, a[::-1])


def test_sphere_ghost_geometry():
    case = W.small_sphere_case(16)
    geo = O3.build_geometry3(case)
    h = case.h
    c = np.array([0.5, 0.5, 0.5])
    k, r = np.divmod(geo.gcell, 16 * 16)
    j, i = np.divmod(r, 16)
    G = np.stack([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h], axis=1)
    I = G + geo.dn[:, None] * geo.n
    assert np.abs(np.linalg.norm(I - c, axis=1) - 0.25).max() < 1e-12
    radial = (G - c) / np.linalg.norm(G - c, axis=1)[:, None]
    cosang = np.sum(radial * geo.n, axis=1)
    assert cosang.min() > math.cos(math.radians(15.0))
    assert np.all(np.abs(geo.w1.sum(axis=1) - 1.0) < 1e-13)
    assert np.all(geo.gamma > 0.0) and geo.n_fallback_ap == 0
    assert np.all(geo.cls.reshape(-1)[geo.ap1[geo.w1 != 0]] == O3.CELL_FLUID)


@pytest.mark.parametrize("weights", [0, 1])
def test_averaging_weights_on_linear_fields_3d(weights):
    # Default weights (reading R17): every linear field is reproduced exactly at IP1 and IP2
    # around the sphere.  Plain inverse-distance weights (Eq. weright averaged): constants
    # exact, linear fields with a first-order error below h |grad f|.
    import dataclasses
    case = W.small_sphere_case(16)
    case = dataclasses.replace(case, params=dataclasses.replace(case.params, weights=weights))
    geo = O3.build_geometry3(case)
    h, n = case.h, case.nx
    k, r = np.divmod(geo.gcell, n * n)
    j, i = np.divmod(r, n)
    G = np.stack([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h], axis=1)
    grad = np.array([0.7, -1.1, 1.9])
    worst = 0.0
    for s_, ap, w in ((1, geo.ap1, geo.w1), (2, geo.ap2, geo.w2)):
        ip = G + (geo.dn + case.params.d1 + s_ * case.params.d2)[:, None] * geo.n
        ak, ar = np.divmod(ap, n * n)
        aj, ai = np.divmod(ar, n)
        A = np.stack([(ai + 0.5) * h, (aj + 0.5) * h, (ak + 0.5) * h], axis=-1)
        # periodic x and y: each averaging point on the side of the box nearest its IP
        A[..., :2] -= case.lx * np.round((A[..., :2] - ip[:, None, :2]) / case.lx)
        f = 2.0 + A @ grad
        got = (w * f).sum(axis=1)
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-13)
        worst = max(worst, float(np.abs(got - (2.0 + ip @ grad)).max()))
    if weights == 0:
        assert worst < 1e-12, worst
    else:
        assert 1e-3 * h < worst < h * np.linalg.norm(grad), worst


def test_slip_vector_form_matches_2d():
    rng = np.random.default_rng(9)
    ng = 50
    th = rng.uniform(0, 2 * math.pi, ng)
    n2d = np.stack([np.cos(th), np.sin(th)], axis=1)
    uM, vM = rng.standard_normal(ng), rng.standard_normal(ng)
    gamma = rng.uniform(0.5, 3.0, ng)
    dn = rng.uniform(0.01, 0.02, ng)
    c2 = W.flat_wall_128x64()
    c2 = W.with_params(c2, l_s=0.01)
    u2, v2 = O2.slip_ghost(c2, uM, vM, n2d, gamma, dn)
    c3 = W.flat_wall_case3d(l_s=0.01)
    n3 = np.stack([n2d[:, 0], np.zeros(ng), n2d[:, 1]], axis=1)
    u3, v3, w3 = O3.slip_ghost3(c3, uM, np.zeros(ng), vM, n3, gamma, dn)
    assert np.abs(u3 - u2).max() < 1e-13 and np.abs(w3 - v2).max() < 1e-13
    assert np.abs(v3).max() == 0.0


def test_explicit_update_conserves_sum_before_fill_3d():
    import dataclasses
    case = W.small_sphere_case(16)
    case = dataclasses.replace(case, params=dataclasses.replace(case.params, ch_scheme=1))
    geo = O3.build_geometry3(case)
    assert len(geo.gcell) > 0
    st = W.random_state3d(case, seed=9)
    C_pre = O3.ch_explicit3(case, geo, st)
    assert abs(C_pre.sum() - st["C"].sum()) <= 1e-13 * np.abs(st["C"]).sum()


def test_face_lists_on_flat_wall_by_hand():
    # 16 x 8 x 16 cells of h = 1/8 with the wall at z = 0.3: plane k = 0 solid, plane 1
    # (centres at z = 0.1875) solid with fluid above, so every cell of it is a ghost; plane 2
    # fluid.  Listed faces (fluid fraction below 1, touching a ghost), derived by hand: all
    # x- and y-faces of plane 1 (alpha = 0), the z-faces of plane 1 (between plane 0 and the
    # ghosts, alpha_w = 0) and of plane 2 (between the ghosts and the fluid: of the 16 subgrid
    # levels (c + 1/2) h/16 above z = 0.1875, the two with c >= 14 lie above the wall, so
    # alpha_w = 2/16).
    case = W.flat_wall_case3d(nx=16, ny=8, nz=16, wall_z=0.3)
    geo = O3.build_geometry3(case)
    nxy = 16 * 8
    assert case.h == 0.125
    assert np.array_equal(geo.gcell, np.arange(nxy) + nxy)
    assert np.array_equal(np.sort(geo.fu), np.arange(nxy) + nxy)
    assert np.array_equal(np.sort(geo.fv), np.arange(nxy) + nxy)
    assert np.array_equal(np.sort(geo.fw), np.r_[np.arange(nxy) + nxy, np.arange(nxy) + 2 * nxy])
    assert np.all(geo.alpha_w[1] == 0.0) and np.all(geo.alpha_w[2] == 2.0 / 16.0)
    assert np.all(geo.n == np.array([0.0, 0.0, 1.0]))
    assert np.allclose(geo.dn, 0.3 - 0.1875, atol=1e-14)


def test_slip_ghost3_special_cases_for_any_normal():
    # Eqs. NoPenetration and UpdateVtan in vector form for normals in any direction: the
    # normal velocity interpolated linearly between G and M vanishes at I; l_s = 0 gives
    # u_G = -u_M / gamma; l_s -> inf keeps the tangential vector; in general
    # V_tI / l_s = (V_tM - V_tG) / ((gamma + 1) dn) with V_tI = (gamma V_tG + V_tM)/(gamma + 1).
    rng = np.random.default_rng(12)
    ng = 60
    n = rng.standard_normal((ng, 3))
    n /= np.linalg.norm(n, axis=1)[:, None]
    uM, vM, wM = rng.standard_normal((3, ng))
    gamma = rng.uniform(1.2, 3.0, ng)
    dn = rng.uniform(0.002, 0.01, ng)
    VM = np.stack([uM, vM, wM], axis=1)
    VnM = (VM * n).sum(axis=1)
    VtM = VM - VnM[:, None] * n
    for ls in (0.0, 0.004, 0.03, 1e30):
        case = W.flat_wall_case3d(l_s=ls)
        VG = np.stack(O3.slip_ghost3(case, uM, vM, wM, n, gamma, dn), axis=1)
        VnG = (VG * n).sum(axis=1)
        VtG = VG - VnG[:, None] * n
        assert np.abs((gamma * VnG + VnM) / (gamma + 1.0)).max() < 1e-12
        if ls == 0.0:
            assert np.allclose(VG, -VM / gamma[:, None], atol=1e-14)
        elif ls > 1e20:
            assert np.allclose(VtG, VtM, atol=1e-12)
        else:
            VtI = (gamma[:, None] * VtG + VtM) / (gamma[:, None] + 1.0)
            assert np.allclose(VtI / ls, (VtM - VtG) / ((gamma[:, None] + 1.0) * dn[:, None]), rtol=1e-10, atol=1e-10)


def test_velocity_helmholtz3_against_dense_operator():
    # (1 - a L) d = r by the transforms against a dense solve of the assembled 7-point
    # operators: x-faces (and y-faces) with no-slip ghost planes -u beyond the z walls,
    # z-faces on the interior planes with w = 0 on the walls; periodic x and y
    rng = np.random.default_rng(31)
    nx, ny, nz = 8, 4, 6
    c = W.flat_wall_case3d(nx=nx, ny=ny, nz=nz, geom_kind=W.GEOM_NONE)
    h, a = c.h, 0.37 * c.h ** 2

    def lap(nzz, ghost):
        n = nzz * ny * nx
        L = np.zeros((n, n))
        idx = lambda k, j, i: (k * ny + j % ny) * nx + i % nx
        for k in range(nzz):
            for j in range(ny):
                for i in range(nx):
                    r = idx(k, j, i)
                    L[r, r] -= 6.0
                    for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                        L[r, idx(k, j + dj, i + di)] += 1.0
                    for dk in (1, -1):
                        kk = k + dk
                        if 0 <= kk < nzz:
                            L[r, idx(kk, j, i)] += 1.0
                        elif ghost:
                            L[r, r] -= 1.0          # ghost plane -u
        return L / h ** 2

    ru = rng.standard_normal((nz, ny, nx))
    rv = rng.standard_normal((nz, ny, nx))
    rw = np.zeros((nz + 1, ny, nx))
    rw[1:nz] = rng.standard_normal((nz - 1, ny, nx))
    du, dv, dw = O3.velocity_helmholtz3(c, ru, rv, rw, a)
    Lt, Ln = lap(nz, True), lap(nz - 1, False)
    It, In = np.eye(Lt.shape[0]), np.eye(Ln.shape[0])
    assert _rel(du.ravel(), np.linalg.solve(It - a * Lt, ru.ravel())) < 1e-12
    assert _rel(dv.ravel(), np.linalg.solve(It - a * Lt, rv.ravel())) < 1e-12
    assert _rel(dw[1:nz].ravel(), np.linalg.solve(In - a * Ln, rw[1:nz].ravel())) < 1e-12
    assert np.all(dw[0] == 0.0) and np.all(dw[nz] == 0.0)


def test_mass_flux_term3_vanishes_for_equal_densities_and_is_second_order():
    # rho' = 0 for equal densities; otherwise the discrete (grad phi . grad) u of smooth
    # fields converges at second order in h (interior planes, away from the z walls)
    import dataclasses

    def fields(n):
        c = W.flat_wall_case3d(nx=n, ny=n, nz=n, geom_kind=W.GEOM_NONE)
        h = c.h
        x = (np.arange(n) + 0.5) * h
        xf = np.arange(n) * h
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        L = n * h
        k = 2.0 * np.pi / L
        phi = np.sin(k * X) * np.cos(k * Y) * np.cos(np.pi * Z / L)
        C = np.zeros_like(phi)
        Zu, Yu, Xu = np.meshgrid(x, x, xf, indexing="ij")
        u = np.cos(k * Xu) * np.sin(k * Yu) * np.sin(np.pi * Zu / L)
        v = np.zeros_like(u)
        w = np.zeros((n + 1, n, n))
        exact = (k * np.cos(k * Xu) * np.cos(k * Yu) * np.cos(np.pi * Zu / L)) * (-k * np.sin(k * Xu) * np.sin(k * Yu) * np.sin(np.pi * Zu / L)) \
            + (-k * np.sin(k * Xu) * np.sin(k * Yu) * np.cos(np.pi * Zu / L)) * (k * np.cos(k * Xu) * np.cos(k * Yu) * np.sin(np.pi * Zu / L)) \
            + (-(np.pi / L) * np.sin(k * Xu) * np.cos(k * Yu) * np.sin(np.pi * Zu / L)) * ((np.pi / L) * np.cos(k * Xu) * np.sin(k * Yu) * np.cos(np.pi * Zu / L))
        return c, C, phi, u, v, w, exact

    c, C, phi, u, v, w, _ = fields(16)
    c1 = dataclasses.replace(c, params=dataclasses.replace(c.params, rho_ratio=1.0))
    for m in O3.mass_flux_term3(c1, C, phi, u, v, w):
        assert np.all(m == 0.0)
    errs = []
    for n in (16, 32):
        c, C, phi, u, v, w, exact = fields(n)
        rho_f = 0.5 * (1.0 + 1.0 / c.params.rho_ratio)    # C = 0: the mean density
        scale = 0.5 * (1.0 - 1.0 / c.params.rho_ratio) / (rho_f * c.params.Pe)
        mfu, _, _ = O3.mass_flux_term3(c, C, phi, u, v, w)
        inner = slice(2, n - 2)
        errs.append(np.abs(mfu[inner] / scale - exact[inner]).max())
    assert errs[1] < errs[0] / 3.0, errs


def test_mirror_value3_of_linear_fields_is_the_value_at_M():
    # as in 2D: M = G + (1 + gamma) dn n and 2 f(IP1) - f(IP2) = f(M) for a linear f, with the
    # linear-exact weights every gather exact (the sphere's ghosts lie away from the periodic
    # edges, so a field linear in x, y and z is linear on every stencil); the phi fill copies it
    case = W.small_sphere_case(32)
    geo = O3.build_geometry3(case)
    nx, ny, h = case.nx, case.ny, case.h
    gi, gj, gk = geo.gcell % nx, (geo.gcell // nx) % ny, geo.gcell // (nx * ny)
    G = np.stack([(gi + 0.5) * h, (gj + 0.5) * h, (gk + 0.5) * h], axis=1)
    M = G + ((1.0 + geo.gamma) * geo.dn)[:, None] * geo.n
    x = (np.arange(nx) + 0.5) * h
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    f = 0.3 + 0.7 * X - 1.1 * Y + 1.9 * Z
    fM = O3.mirror_value3(f.reshape(-1), geo)
    assert np.abs(fM - (0.3 + 0.7 * M[:, 0] - 1.1 * M[:, 1] + 1.9 * M[:, 2])).max() < 1e-12
    st = W.random_state3d(case, seed=8)
    phi = O3.chemical_potential3(case, geo, st["C"])
    assert np.array_equal(phi.reshape(-1)[geo.gcell], O3.mirror_value3(phi.reshape(-1).copy(), geo))
