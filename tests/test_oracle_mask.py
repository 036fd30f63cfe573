"""Pins of the MASK geometry in the oracle (reading R20): a solid with no analytic form,
given by its volume fractions, with the solid where the cell-centre fractions interpolated
linearly between cell centres are below 1/2 (Sec. 4.1.1 and 4.1.2 then apply unchanged).

* the interpolation: exact at cell centres, the mean of two neighbours half-way between
  them, periodic in x (and y), continued beyond the first and last centre rows;
* a step in the fractions on a grid line is a flat wall on that line: the MASK geometry of a
  grid-aligned flat wall's fractions equals the flat wall's geometry (2D and 3D);
* on a curved wall the intersect points found by the march and bisection lie on the 1/2
  level of the interpolated fractions, and every ghost centre is solid with a fluid face
  neighbour.
"""
from dataclasses import replace

import numpy as np
import pytest

from oracle import ib_pf2d as O
from oracle import ib_pf3d as O3
from workloads import cases as W


def _mask2(case, geo):
    return replace(case, geom_kind=W.GEOM_MASK, alpha=(geo.alpha_c, geo.alpha_u, geo.alpha_v))


def test_mask_interpolation_by_hand():
    rng = np.random.Generator(np.random.PCG64(20))
    nx, ny = 5, 4
    A = rng.random((ny, nx))
    au, av = np.ones((ny, nx)), np.ones((ny + 1, nx))
    case = replace(W.flat_wall_case(nx=8, ny=4), nx=nx, ny=ny, lx=nx * 0.25, ly=ny * 0.25,
                   geom_kind=W.GEOM_MASK, alpha=(A, au, av))
    h = case.h
    assert h == 0.25
    xc, yc = (np.arange(nx) + 0.5) * h, (np.arange(ny) + 0.5) * h
    assert np.array_equal(O.mask_alpha(case, xc[None, :], yc[:, None]), A)
    # half-way between vertical and horizontal neighbours
    mid_y = O.mask_alpha(case, xc[None, :], (yc[:-1] + 0.5 * h)[:, None])
    assert np.allclose(mid_y, 0.5 * (A[:-1] + A[1:]), rtol=0, atol=1e-15)
    mid_x = O.mask_alpha(case, (xc[:-1] + 0.5 * h)[None, :], yc[:, None])
    assert np.allclose(mid_x, 0.5 * (A[:, :-1] + A[:, 1:]), rtol=0, atol=1e-15)
    # periodic in x: the point half-way between the last and the first centre
    wrap = O.mask_alpha(case, np.full(ny, nx * h), yc)
    assert np.allclose(wrap, 0.5 * (A[:, -1] + A[:, 0]), rtol=0, atol=1e-15)
    # below the first and above the last centre row: that row's values
    assert np.array_equal(O.mask_alpha(case, xc, np.full(nx, 0.1 * h)), A[0])
    assert np.array_equal(O.mask_alpha(case, xc, np.full(nx, ny * h - 0.1 * h)), A[-1])
    # a bilinear function is reproduced at any point inside the centre lattice
    Af = 0.3 + 0.1 * xc[None, :] + 0.2 * yc[:, None] + 0.05 * xc[None, :] * yc[:, None]
    case_f = replace(case, alpha=(Af, au, av))
    x, y = rng.uniform(xc[0], xc[-1], 50), rng.uniform(yc[0], yc[-1], 50)
    assert np.allclose(O.mask_alpha(case_f, x, y), 0.3 + 0.1 * x + 0.2 * y + 0.05 * x * y,
                       rtol=0, atol=1e-14)


def _same_tables(g, m, names_exact, names_close, tol=1e-12):
    for k in names_exact:
        assert np.array_equal(getattr(g, k), getattr(m, k)), k
    for k in names_close:
        a, b = getattr(g, k), getattr(m, k)
        assert a.shape == b.shape, k
        assert np.abs(a - b).max() <= tol, (k, np.abs(a - b).max())


def test_mask_of_grid_aligned_flat_wall_is_the_flat_wall():
    case = W.flat_wall_case(nx=64, ny=32, wall_y=0.25)      # the wall on the grid line j = 8
    geo = O.build_geometry(case)
    assert set(np.unique(geo.alpha_c)) == {0.0, 1.0}
    mgeo = O.build_geometry(_mask2(case, geo))
    _same_tables(geo, mgeo, ("cls", "gcell", "ap1", "ap2", "fu", "fv", "alpha_c", "alpha_u", "alpha_v"),
                 ("n", "dn", "gamma", "w1", "w2"))


def test_mask_intersect_points_on_the_half_level():
    case = W.sinusoid_wall_512x256(theta_deg=90.0, l_s=0.0)
    d1, d2 = W._ghost_lengths(2.0 / 128)
    case = replace(case, nx=128, ny=64, params=replace(case.params, d1=d1, d2=d2))
    geo = O.build_geometry(case)
    mcase = _mask2(case, geo)
    m = O.build_geometry(mcase)
    nx, h = case.nx, case.h
    gi, gj = m.gcell % nx, m.gcell // nx
    G = np.stack([(gi + 0.5) * h, (gj + 0.5) * h], axis=1)
    I = G + m.dn[:, None] * m.n
    assert len(m.gcell) > 0
    assert np.abs(O.mask_alpha(mcase, I[:, 0], I[:, 1]) - 0.5).max() <= 1e-9
    assert (O.mask_alpha(mcase, G[:, 0], G[:, 1]) < 0.5).all()
    ac = geo.alpha_c
    fluid = ac >= 0.5
    nb = np.roll(fluid, 1, 1) | np.roll(fluid, -1, 1)
    nb[1:] |= fluid[:-1]
    nb[:-1] |= fluid[1:]
    assert np.array_equal(np.nonzero((~fluid & nb).ravel())[0], m.gcell)
    assert np.allclose(m.w1.sum(axis=1), 1.0) and np.allclose(m.w2.sum(axis=1), 1.0)
    # the 1/2 level of the interpolated fractions lies within a cell of the analytic wall
    yw = 0.2 + 0.05 * np.sin(4.0 * np.pi * I[:, 0])
    assert np.abs(I[:, 1] - yw).max() <= h


def test_mask3_of_grid_aligned_flat_wall_is_the_flat_wall():
    case = W.flat_wall_case3d(nx=16, ny=8, nz=16, wall_z=0.625)   # z = 5 h
    geo = O3.build_geometry3(case)
    assert set(np.unique(geo.alpha_c)) == {0.0, 1.0}
    mcase = replace(case, geom_kind=W.GEOM_MASK, alpha=(geo.alpha_c, geo.alpha_u, geo.alpha_v, geo.alpha_w))
    m = O3.build_geometry3(mcase)
    _same_tables(geo, m, ("cls", "gcell", "ap1", "ap2", "fu", "fv", "fw", "alpha_c", "alpha_w"),
                 ("n", "dn", "gamma", "w1", "w2"))


def test_mask3_intersect_points_on_the_half_level():
    case = W.small_sphere_case(32)
    geo = O3.build_geometry3(case)
    mcase = replace(case, geom_kind=W.GEOM_MASK, alpha=(geo.alpha_c, geo.alpha_u, geo.alpha_v, geo.alpha_w))
    m = O3.build_geometry3(mcase)
    nx, ny, h = case.nx, case.ny, case.h
    gi, gj, gk = m.gcell % nx, (m.gcell // nx) % ny, m.gcell // (nx * ny)
    G = np.stack([(gi + 0.5) * h, (gj + 0.5) * h, (gk + 0.5) * h], axis=1)
    I = G + m.dn[:, None] * m.n
    assert len(m.gcell) > 0
    assert np.abs(O3.mask_alpha3(mcase, I[:, 0], I[:, 1], I[:, 2]) - 0.5).max() <= 1e-9
    assert (O3.mask_alpha3(mcase, G[:, 0], G[:, 1], G[:, 2]) < 0.5).all()
    assert np.allclose(m.w1.sum(axis=1), 1.0) and np.allclose(m.w2.sum(axis=1), 1.0)
