"""Plain FP64 CPU oracle of one time step of the hybrid IB / phase-field method, 3D.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module; the CUDA
library is an independent implementation and the two share no code.

The 3D step follows the same sections and equations as the 2D oracle (ib_pf2d), with the
third axis added: periodic in x and y, walls in z (the wall-normal axis), cell fields
(nz, ny, nx) with x fastest, u / v on x- / y-faces (nz, ny, nx), w on z-faces (nz+1, ny, nx)
with rows 0 and nz on the domain walls.  Readings R1-R11 of ib_pf2d hold unchanged; the
3D counterparts of the 2D-specific ones are:
  R5' Slip velocity in vector form: V_n = u.n, V_t = u - V_n n, u_G = V_nG n + V_tG
      (the 2D tangent t = (n2, -n1) is the special case).
  R6' Ghost = solid cell centre with a fluid centre among its 6 face neighbours; averaging
      points = the cell holding the IP plus its 6 face neighbours (solid centres and cells
      outside the z range dropped, weights renormalised).
  R7' d1 = sqrt(3) h, d2 = d1/2.
  R8' Edge viscosities (xy-, xz- and yz-edges) use the mean C of the four cells around the
      edge; convection in divergence form with products of face means at the edges.
  R12 Subgrid counting (Sec. 4.1.1) with NSUB3 = 16 points per direction (4096 per control
      volume) in 3D.  A control volume wholly outside every sphere (or wholly inside one)
      is counted without visiting its points: the count is the same.
  R13 Corner gradients of alpha (Eq. NormalVectors, 3D): at corner (i+1/2, j+1/2, k+1/2)
      each component is the difference of the two 2x2 faces of the 8 surrounding cells
      divided by 4h; the cell normal is the mean of its 8 corners.  Fallback neighbour
      order +z, -z, +x, -x, +y, -y.
  R14 Periodic images: the sphere test takes the nearest image in x and y
      (dx = x - cx, shifted by -L if dx > L/2 or +L if dx < -L/2).
  With params.ch_scheme = 1, a1 + a2 is the explicit AB2 update of Eq. ExpCH as in the 2D
  oracle (its reading R15), with the third axis.  With params.ns_scheme = 1, a5 is the
  semi-implicit predictor of Appendix A.2 (Eq. predictionSemi) as in the 2D oracle (its
  reading R19), with the third axis: DST-II along z for u and v, DST-I for w.
Library primitives used as steps: numpy elementwise arithmetic and scipy's FFT / DCT-II.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

from oracle.ib_pf2d import KAPPA, GAMMA0, MARCH_DIV, MARCH_MAX, BISECT, EPS0
from oracle.ib_pf2d import CELL_FLUID, CELL_GHOST, CELL_SOLID
from oracle.ib_pf2d import contact_angle_ghost, dynamic_contact_ghost, linear_exact_weights
from workloads.cases import GEOM_FLAT, GEOM_MASK, GEOM_NONE, GEOM_SPHERE, GEOM_SPHERES, Case3D

NSUB3 = 16     # subgrid points per direction in 3D (reading R12)
NAP3 = 7       # averaging points per interpolation point in 3D


# --------------------------------------------------------------------------- solids
def _spheres(case: Case3D):
    if case.geom_kind == GEOM_SPHERE:
        return np.array([case.geom_p[:4]], dtype=np.float64)
    if case.geom_kind == GEOM_SPHERES:
        return np.array(case.spheres, dtype=np.float64).reshape(-1, 4)
    return np.zeros((0, 4))


def _wrap(d, L):
    """Nearest periodic image of a coordinate difference (reading R14)."""
    d = np.where(d > 0.5 * L, d - L, d)
    return np.where(d < -0.5 * L, d + L, d)


def mask_alpha3(case: Case3D, x, y, z):
    """MASK walls (reading R20): alpha_c interpolated trilinearly at (x, y, z), centres at
    ((i + 1/2) h, (j + 1/2) h, (k + 1/2) h), periodic in x and y, the first and last centre
    planes continued beyond them."""
    A = np.asarray(case.alpha[0], dtype=np.float64)
    nz, ny, nx = A.shape
    h = case.h
    x, y, z = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(y, np.float64),
                                  np.asarray(z, np.float64))
    fx, fy, fz = x / h - 0.5, y / h - 0.5, z / h - 0.5
    fx0, fy0, fz0 = np.floor(fx), np.floor(fy), np.floor(fz)
    tx, ty, tz = fx - fx0, fy - fy0, fz - fz0
    i0 = fx0.astype(np.int64) % nx
    j0 = fy0.astype(np.int64) % ny
    i1, j1 = (i0 + 1) % nx, (j0 + 1) % ny
    k0 = np.clip(fz0.astype(np.int64), 0, nz - 1)
    k1 = np.clip(fz0.astype(np.int64) + 1, 0, nz - 1)

    def plane(k):
        a = (1.0 - tx) * A[k, j0, i0] + tx * A[k, j0, i1]
        b = (1.0 - tx) * A[k, j1, i0] + tx * A[k, j1, i1]
        return (1.0 - ty) * a + ty * b

    return (1.0 - tz) * plane(k0) + tz * plane(k1)


def solid3(case: Case3D, x, y, z, sph=None):
    """True where (x, y, z) lies inside the solid."""
    x, y, z = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(y, np.float64),
                                  np.asarray(z, np.float64))
    if case.geom_kind == GEOM_NONE:
        return np.zeros(x.shape, dtype=bool)
    if case.geom_kind == GEOM_MASK:
        return mask_alpha3(case, x, y, z) < 0.5
    if case.geom_kind == GEOM_FLAT:
        return z < case.geom_p[0]
    sph = _spheres(case) if sph is None else sph
    out = np.zeros(x.shape, dtype=bool)
    for cx, cy, cz, r in sph:
        dx = _wrap(x - cx, case.lx)
        dy = _wrap(y - cy, case.ly)
        dz = z - cz
        out |= ((dx * dx + dy * dy) + dz * dz) < r * r
    return out


def _candidates(case: Case3D, sph, x0, y0, z0, h):
    """Spheres whose periodic bounding box meets the box [x0, x0+h] x ... (any of them
    may contain a point of the box)."""
    if len(sph) == 0:
        return sph
    cx = _wrap(sph[:, 0] - (x0 + 0.5 * h), case.lx)
    cy = _wrap(sph[:, 1] - (y0 + 0.5 * h), case.ly)
    cz = sph[:, 2] - (z0 + 0.5 * h)
    lim = sph[:, 3] + 0.5 * h
    m = (np.abs(cx) <= lim) & (np.abs(cy) <= lim) & (np.abs(cz) <= lim)
    return sph[m]


def volume_fraction_cv(case: Case3D, x0: float, y0: float, z0: float, sph=None) -> float:
    """Fluid fraction of the h^3 control volume with lower corner (x0, y0, z0): the share of
    its NSUB3^3 subgrid points (x0 + (a+1/2) h/NSUB3, ...) outside the solid (Sec. 4.1.1)."""
    h = case.h
    if case.geom_kind == GEOM_NONE:
        return 1.0
    hs = h / NSUB3
    off = (np.arange(NSUB3, dtype=np.float64) + 0.5) * hs
    if case.geom_kind == GEOM_FLAT:
        zs = z0 + off
        n_fluid = np.count_nonzero(zs >= case.geom_p[0]) * NSUB3 * NSUB3
        return n_fluid / float(NSUB3 ** 3)
    sph = _spheres(case) if sph is None else sph
    cand = _candidates(case, sph, x0, y0, z0, h)
    # reading R12: a sphere whose nearest point of the volume is at or beyond its radius
    # holds no subpoint; one holding the 8 corners holds every subpoint (convexity)
    hh = 0.5 * h
    band = []
    for cx, cy, cz, r in cand:
        ax = abs(float(_wrap(np.float64(x0 + hh - cx), case.lx)))
        ay = abs(float(_wrap(np.float64(y0 + hh - cy), case.ly)))
        az = abs(z0 + hh - cz)
        nx_, ny_, nz_ = max(ax - hh, 0.0), max(ay - hh, 0.0), max(az - hh, 0.0)
        if (nx_ * nx_ + ny_ * ny_) + nz_ * nz_ >= r * r:
            continue
        fx, fy, fz = ax + hh, ay + hh, az + hh
        if (fx * fx + fy * fy) + fz * fz < r * r:
            return 0.0
        band.append((cx, cy, cz, r))
    if not band:
        return 1.0
    Z, Y, X = np.meshgrid(z0 + off, y0 + off, x0 + off, indexing="ij")
    n_fluid = np.count_nonzero(~solid3(case, X, Y, Z, np.array(band)))
    return n_fluid / float(NSUB3 ** 3)


def volume_fractions3(case: Case3D, shift: tuple, shape: tuple, sph=None) -> np.ndarray:
    """Fractions of every control volume of a staggered family: control volume (k, j, i)
    has its lower corner at ((i + sx) h, (j + sy) h, (k + sz) h)."""
    h = case.h
    sph = _spheres(case) if sph is None else sph
    nz, ny, nx = shape
    out = np.ones(shape)
    if case.geom_kind == GEOM_NONE:
        return out
    if case.geom_kind == GEOM_FLAT:
        for k in range(nz):
            out[k] = volume_fraction_cv(case, 0.0, 0.0, (k + shift[2]) * h)
        return out
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                out[k, j, i] = volume_fraction_cv(case, (i + shift[0]) * h, (j + shift[1]) * h,
                                                  (k + shift[2]) * h, sph)
    return out


@dataclass
class Geometry3D:
    alpha_c: np.ndarray    # (nz, ny, nx)
    alpha_u: np.ndarray    # (nz, ny, nx)   x-faces
    alpha_v: np.ndarray    # (nz, ny, nx)   y-faces
    alpha_w: np.ndarray    # (nz+1, ny, nx) z-faces
    cls: np.ndarray        # (nz, ny, nx)   CELL_FLUID / CELL_GHOST / CELL_SOLID
    gcell: np.ndarray      # (ng,) linear cell index (k*ny + j)*nx + i, ascending
    n: np.ndarray          # (ng, 3) unit normal, solid -> fluid
    dn: np.ndarray
    gamma: np.ndarray
    ap1: np.ndarray        # (ng, NAP3)
    w1: np.ndarray
    ap2: np.ndarray
    w2: np.ndarray
    fu: np.ndarray         # linear indices of fixed x-, y-, z-faces
    fv: np.ndarray
    fw: np.ndarray
    n_fallback_normal: int
    n_fallback_ap: int


def _alpha_at3(a, i, j, k):
    nz, ny, nx = a.shape
    k = min(max(k, 0), nz - 1)       # mirror planes at the z walls
    return a[k, j % ny, i % nx]


def _first_fluid_neighbour3(cls, i, j, k):
    nz, ny, nx = cls.shape
    for di, dj, dk in ((0, 0, 1), (0, 0, -1), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0)):
        kk = k + dk
        if 0 <= kk < nz and cls[kk, (j + dj) % ny, (i + di) % nx] == CELL_FLUID:
            return (i + di) % nx, (j + dj) % ny, kk, float(di), float(dj), float(dk)
    return None


def _normal3(case: Case3D, alpha_c, cls, i, j, k):
    """Reading R13 of Eqs. NormalVectors_part1/2 in 3D."""
    h = case.h

    def corner(ci, cj, ck):   # corner (ci+1/2, cj+1/2, ck+1/2)
        a = [[[_alpha_at3(alpha_c, ci + di, cj + dj, ck + dk) for di in (0, 1)]
              for dj in (0, 1)] for dk in (0, 1)]   # a[dk][dj][di]
        mx = ((a[0][0][1] + a[0][1][1]) + (a[1][0][1] + a[1][1][1])
              - ((a[0][0][0] + a[0][1][0]) + (a[1][0][0] + a[1][1][0]))) / (4.0 * h)
        my = ((a[0][1][0] + a[0][1][1]) + (a[1][1][0] + a[1][1][1])
              - ((a[0][0][0] + a[0][0][1]) + (a[1][0][0] + a[1][0][1]))) / (4.0 * h)
        mz = ((a[1][0][0] + a[1][0][1]) + (a[1][1][0] + a[1][1][1])
              - ((a[0][0][0] + a[0][0][1]) + (a[0][1][0] + a[0][1][1]))) / (4.0 * h)
        return mx, my, mz

    cs = [corner(i + di, j + dj, k + dk) for dk in (-1, 0) for dj in (-1, 0) for di in (-1, 0)]
    m = [0.0, 0.0, 0.0]
    for c in range(3):
        acc = 0.0
        for q in cs:
            acc += q[c]
        m[c] = acc / 8.0
    mag2 = (m[0] * m[0] + m[1] * m[1]) + m[2] * m[2]
    if math.sqrt(mag2) * h < 1.0e-12:
        nb = _first_fluid_neighbour3(cls, i, j, k)
        if nb is None:
            raise ValueError("ghost cell without fluid neighbour")
        return nb[3], nb[4], nb[5], True
    norm = math.sqrt(mag2 + EPS0)
    return m[0] / norm, m[1] / norm, m[2] / norm, False


def _normals3(case: Case3D, alpha_c, gi, gj, gk):
    """Mean of the 8 corner gradients of alpha (reading R13) for arrays of cells, in the
    order and grouping of _normal3."""
    h = case.h
    nz, ny, nx = alpha_c.shape

    def al(i, j, k):
        return alpha_c[np.clip(k, 0, nz - 1), j % ny, i % nx]

    acc = np.zeros((len(gi), 3))
    for dk in (-1, 0):
        for dj in (-1, 0):
            for di in (-1, 0):
                ci, cj, ck = gi + di, gj + dj, gk + dk
                a = [[[al(ci + ei, cj + ej, ck + ek) for ei in (0, 1)] for ej in (0, 1)]
                     for ek in (0, 1)]
                mx = ((a[0][0][1] + a[0][1][1]) + (a[1][0][1] + a[1][1][1])
                      - ((a[0][0][0] + a[0][1][0]) + (a[1][0][0] + a[1][1][0]))) / (4.0 * h)
                my = ((a[0][1][0] + a[0][1][1]) + (a[1][1][0] + a[1][1][1])
                      - ((a[0][0][0] + a[0][0][1]) + (a[1][0][0] + a[1][0][1]))) / (4.0 * h)
                mz = ((a[1][0][0] + a[1][0][1]) + (a[1][1][0] + a[1][1][1])
                      - ((a[0][0][0] + a[0][0][1]) + (a[0][1][0] + a[0][1][1]))) / (4.0 * h)
                acc[:, 0] = acc[:, 0] + mx
                acc[:, 1] = acc[:, 1] + my
                acc[:, 2] = acc[:, 2] + mz
    return acc / 8.0


def _averaging_points3(case: Case3D, cls, px, py, pz):
    """Reading R6': the cell holding (px, py, pz) and its 6 face neighbours, fluid centres
    only, inverse-squared-distance weights normalised (Eq. weright averaged)."""
    h = case.h
    nz, ny, nx = cls.shape
    i0, j0, k0 = math.floor(px / h), math.floor(py / h), math.floor(pz / h)
    idx, d2s, offs, rel = [], [], [], []
    for di, dj, dk in ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1),
                       (0, 0, -1)):
        ic, jc, kc = i0 + di, j0 + dj, k0 + dk
        if kc < 0 or kc >= nz:
            continue
        if cls[kc, jc % ny, ic % nx] != CELL_FLUID:
            continue
        dx = (ic + 0.5) * h - px
        dy = (jc + 0.5) * h - py
        dz = (kc + 0.5) * h - pz
        idx.append((kc * ny + jc % ny) * nx + ic % nx)
        d2s.append((dx * dx + dy * dy) + dz * dz)
        offs.append((di, dj, dk))
        rel.append((dx / h, dy / h, dz / h))
    if not idx:
        return None
    tiny = (1.0e-12 * h) * (1.0e-12 * h)
    for q, d2 in enumerate(d2s):
        if d2 < tiny:
            w = [0.0] * len(idx)
            w[q] = 1.0
            return idx, w
    wr = [1.0 / d2 for d2 in d2s]
    s = 0.0
    for x in wr:
        s += x
    w = [x / s for x in wr]
    if getattr(case.params, "weights", 0) == 0 and len(idx) >= 4 and spans_space(offs):
        w = linear_exact_weights(w, rel)
    return idx, w


def spans_space(offsets) -> bool:
    """True when the integer stencil offsets of the kept averaging points are not all in
    one plane (affinely independent in 3D); decided in integers."""
    o = [tuple(a - b for a, b in zip(p, offsets[0])) for p in offsets]
    n = len(o)
    for p in range(n):
        for q in range(p + 1, n):
            for r in range(q + 1, n):
                a, b, c = o[p], o[q], o[r]
                det = (a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0])
                       + a[2] * (b[0] * c[1] - b[1] * c[0]))
                if det != 0:
                    return True
    return False


def classify3(case: Case3D):
    """Cell classes: solid centres with a fluid face neighbour are ghosts (reading R6')."""
    h = case.h
    xc = (np.arange(case.nx) + 0.5) * h
    yc = (np.arange(case.ny) + 0.5) * h
    zc = (np.arange(case.nz) + 0.5) * h
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    sol = solid3(case, X, Y, Z)
    cls = np.where(sol, CELL_SOLID, CELL_FLUID).astype(np.int8)
    fl = ~sol
    nb = np.zeros_like(sol)
    for ax in (1, 2):
        nb |= np.roll(fl, 1, axis=ax) | np.roll(fl, -1, axis=ax)
    nb[1:] |= fl[:-1]
    nb[:-1] |= fl[1:]
    cls[sol & nb] = CELL_GHOST
    return cls


def build_geometry3(case: Case3D) -> Geometry3D:
    """All of Sec. 4.1 for one 3D case (small grids: every control volume is visited)."""
    nx, ny, nz, h = case.nx, case.ny, case.nz, case.h
    p = case.params
    sph = _spheres(case)
    if case.geom_kind == GEOM_MASK:   # the caller's fractions replace the count (R20)
        alpha_c, alpha_u, alpha_v, alpha_w = (
            np.asarray(a, dtype=np.float64).reshape(s) for a, s in
            zip(case.alpha, ((nz, ny, nx), (nz, ny, nx), (nz, ny, nx), (nz + 1, ny, nx))))
    else:
        alpha_c = volume_fractions3(case, (0.0, 0.0, 0.0), (nz, ny, nx), sph)
        alpha_u = volume_fractions3(case, (-0.5, 0.0, 0.0), (nz, ny, nx), sph)
        alpha_v = volume_fractions3(case, (0.0, -0.5, 0.0), (nz, ny, nx), sph)
        alpha_w = volume_fractions3(case, (0.0, 0.0, -0.5), (nz + 1, ny, nx), sph)
    cls = classify3(case)
    gk, gj, gi = np.nonzero(cls == CELL_GHOST)
    ng = len(gi)
    gcell = ((gk * ny + gj) * nx + gi).astype(np.int64)
    ap1 = np.zeros((ng, NAP3), dtype=np.int64)
    ap2 = np.zeros((ng, NAP3), dtype=np.int64)
    w1 = np.zeros((ng, NAP3))
    w2 = np.zeros((ng, NAP3))
    nfb_n = nfb_ap = 0
    # normals (reading R13), every ghost at once; the arithmetic of each ghost is the
    # scalar sequence of _normal3
    m = _normals3(case, alpha_c, gi, gj, gk)
    mag2 = (m[:, 0] * m[:, 0] + m[:, 1] * m[:, 1]) + m[:, 2] * m[:, 2]
    norm = np.sqrt(mag2 + EPS0)
    nrm = m / norm[:, None]
    for g in np.nonzero(np.sqrt(mag2) * h < 1.0e-12)[0]:
        nb = _first_fluid_neighbour3(cls, int(gi[g]), int(gj[g]), int(gk[g]))
        if nb is None:
            raise ValueError("ghost cell without fluid neighbour")
        nrm[g] = (nb[3], nb[4], nb[5])
        nfb_n += 1
    G = np.stack([(gi + 0.5) * h, (gj + 0.5) * h, (gk + 0.5) * h], axis=1)
    # intersect points: march h/100 along n to the first point outside, then bisect
    ds = h / MARCH_DIV
    qs = np.zeros(ng, dtype=np.int64)
    active = np.arange(ng)
    q = 1
    while len(active) and q <= MARCH_MAX:
        t = q * ds
        out = ~solid3(case, G[active, 0] + t * nrm[active, 0], G[active, 1] + t * nrm[active, 1],
                      G[active, 2] + t * nrm[active, 2], sph)
        qs[active[out]] = q
        active = active[~out]
        q += 1
    if len(active):
        raise ValueError(f"no intersect point found for {len(active)} ghost(s)")
    lo, hi = (qs - 1) * ds, qs * ds
    for _ in range(BISECT):
        mid = 0.5 * (lo + hi)
        ins = solid3(case, G[:, 0] + mid * nrm[:, 0], G[:, 1] + mid * nrm[:, 1],
                     G[:, 2] + mid * nrm[:, 2], sph)
        lo = np.where(ins, mid, lo)
        hi = np.where(ins, hi, mid)
    dn = hi
    gamma = p.d1 / hi
    for g in range(ng):
        i, j, k = int(gi[g]), int(gj[g]), int(gk[g])
        n1, n2, n3 = nrm[g]
        gx, gy, gz = G[g]
        s1 = (dn[g] + p.d1) + p.d2
        s2 = (dn[g] + p.d1) + 2.0 * p.d2
        for sdist, aps, ws in ((s1, ap1, w1), (s2, ap2, w2)):
            res = _averaging_points3(case, cls, gx + sdist * n1, gy + sdist * n2, gz + sdist * n3)
            if res is None:
                nb = _first_fluid_neighbour3(cls, i, j, k)
                res = ([(nb[2] * ny + nb[1]) * nx + nb[0]], [1.0])
                nfb_ap += 1
            idx, w = res
            for aa in range(NAP3):
                aps[g, aa] = idx[aa] if aa < len(idx) else idx[0]
                ws[g, aa] = w[aa] if aa < len(idx) else 0.0
    isg = cls == CELL_GHOST
    fu = np.flatnonzero(((alpha_u < 1.0) & (isg | np.roll(isg, 1, axis=2))).reshape(-1))
    fv = np.flatnonzero(((alpha_v < 1.0) & (isg | np.roll(isg, 1, axis=1))).reshape(-1))
    fw_mask = np.zeros((nz + 1, ny, nx), dtype=bool)
    fw_mask[1:nz] = (alpha_w[1:nz] < 1.0) & (isg[1:] | isg[:-1])
    fw = np.flatnonzero(fw_mask.reshape(-1))
    return Geometry3D(alpha_c, alpha_u, alpha_v, alpha_w, cls, gcell, nrm, dn, gamma, ap1, w1,
                      ap2, w2, fu.astype(np.int64), fv.astype(np.int64), fw.astype(np.int64),
                      nfb_n, nfb_ap)


# ------------------------------------------------------------------ discrete operators
def _xp(a):
    return np.roll(a, -1, axis=-1)


def _xm(a):
    return np.roll(a, 1, axis=-1)


def _yp(a):
    return np.roll(a, -1, axis=-2)


def _ym(a):
    return np.roll(a, 1, axis=-2)


def _zp_mirror(a):
    return np.concatenate([a[1:], a[-1:]], axis=0)


def _zm_mirror(a):
    return np.concatenate([a[:1], a[:-1]], axis=0)


def laplacian3(a: np.ndarray, h: float) -> np.ndarray:
    """7-point Laplacian; periodic x, y; zero-gradient z walls."""
    return ((((_xp(a) + _xm(a)) + (_yp(a) + _ym(a))) + (_zp_mirror(a) + _zm_mirror(a)))
            - 6.0 * a) / (h * h)


def eigenvalues3(nx: int, ny: int, nz: int, h: float) -> np.ndarray:
    """Eigenvalues of laplacian3 in the real-Fourier (x) x Fourier (y) x DCT-II (z) basis,
    shape (nz, ny, nx//2 + 1)."""
    lx = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(nx // 2 + 1) / nx) ** 2
    ly = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(ny) / ny) ** 2
    lz = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(nz) / (2.0 * nz)) ** 2
    return (lz[:, None, None] + ly[None, :, None]) + lx[None, None, :]


def _forward3(a):
    s = sfft.fft(sfft.rfft(a, axis=2), axis=1)
    return sfft.dct(s.real, type=2, axis=0) + 1j * sfft.dct(s.imag, type=2, axis=0)


def _inverse3(s, nx):
    t = sfft.idct(s.real, type=2, axis=0) + 1j * sfft.idct(s.imag, type=2, axis=0)
    return sfft.irfft(sfft.ifft(t, axis=1), n=nx, axis=2)


def ch_solve3(case: Case3D, Q: np.ndarray) -> np.ndarray:
    """Appendix A.1 with the combined symbol of reading R2, 3D eigenbasis."""
    p = case.params
    lam = eigenvalues3(case.nx, case.ny, case.nz, case.h)
    eta2 = p.Cn * p.Cn
    sig = lam * lam - (p.S / eta2) * lam + GAMMA0 * p.Pe / (eta2 * p.dt)
    return _inverse3(_forward3(Q) / sig, case.nx)


def poisson_solve3(case: Case3D, rhs: np.ndarray) -> np.ndarray:
    """laplacian3(P) = rhs with the mean mode set to zero (Eq. PressurePoisson)."""
    lam = eigenvalues3(case.nx, case.ny, case.nz, case.h)
    lam0 = lam.copy()
    lam0[0, 0, 0] = 1.0
    s = _forward3(rhs) / lam0
    s[0, 0, 0] = 0.0
    return _inverse3(s, case.nx)


def _props(case: Case3D):
    p = case.params
    rho_l, rho_g = 1.0, 1.0 / p.rho_ratio
    mu_l, mu_g = 1.0, 1.0 / p.mu_ratio

    def rho(c):     # reading R11
        c = np.clip(c, -1.0, 1.0)
        return 0.5 * ((1.0 + c) * rho_l + (1.0 - c) * rho_g)

    def mu(c):
        c = np.clip(c, -1.0, 1.0)
        return 0.5 * ((1.0 + c) * mu_l + (1.0 - c) * mu_g)

    return rho, mu, min(rho_l, rho_g)


def ch_rhs3(case: Case3D, geo: "Geometry3D", st: dict) -> np.ndarray:
    """a1 in 3D: Q = (Pe/Cn^2)(C_check/dt - div(u~ C~)) + lap[(psi'(C~) - S C~)/Cn^2]
    + lap[(phi~_wall - phi~)/Cn^2], the last term the wall's no-flux condition on the
    chemical potential of C~ (reading R16 of the 2D oracle)."""
    p = case.params
    h, nz = case.h, case.nz
    eta2 = p.Cn * p.Cn
    C, Co = st["C"], st["C_old"]
    Ct = 2.0 * C - Co
    Cc = 2.0 * C - 0.5 * Co
    ut = 2.0 * st["u"] - st["u_old"]
    vt = 2.0 * st["v"] - st["v_old"]
    wt = 2.0 * st["w"] - st["w_old"]
    Fx = ut * (0.5 * (_xm(Ct) + Ct))
    Fy = vt * (0.5 * (_ym(Ct) + Ct))
    Fz = np.zeros((nz + 1,) + C.shape[1:])
    Fz[1:nz] = wt[1:nz] * (0.5 * (Ct[:-1] + Ct[1:]))
    div = ((_xp(Fx) - Fx) / h + (_yp(Fy) - Fy) / h) + (Fz[1:] - Fz[:-1]) / h
    g = ((Ct * Ct * Ct - Ct) - p.S * Ct) / eta2
    phi_t = (Ct * Ct * Ct - Ct) - eta2 * laplacian3(Ct, h)
    phi_t_wall = chemical_potential3(case, geo, Ct)
    return ((p.Pe / eta2) * (Cc / p.dt - div) + laplacian3(g, h)
            + laplacian3((phi_t_wall - phi_t) / eta2, h))


def chemical_potential3(case: Case3D, geo: "Geometry3D", C: np.ndarray) -> np.ndarray:
    """a4 in 3D: phi = psi'(C) - Cn^2 lap(C) on every cell, then phi_G = phi_M."""
    eta = case.params.Cn
    phi = (C * C * C - C) - (eta * eta) * laplacian3(C, case.h)
    pf = phi.reshape(-1)
    pf[geo.gcell] = mirror_value3(pf.copy(), geo)
    return phi


def ch_flux_div3(case: Case3D, C, u, v, w) -> np.ndarray:
    """div(u C_f) with face means of C, no flux through the z walls."""
    h, nz = case.h, case.nz
    Fx = u * (0.5 * (_xm(C) + C))
    Fy = v * (0.5 * (_ym(C) + C))
    Fz = np.zeros((nz + 1,) + C.shape[1:])
    Fz[1:nz] = w[1:nz] * (0.5 * (C[:-1] + C[1:]))
    return ((_xp(Fx) - Fx) / h + (_yp(Fy) - Fy) / h) + (Fz[1:] - Fz[:-1]) / h


def ch_explicit3(case: Case3D, geo: "Geometry3D", st: dict) -> np.ndarray:
    """a1 + a2, explicit variant in 3D (Eq. ExpCH, reading R15 of the 2D oracle):
    C^n + dt (3/2 F^n - 1/2 F^{n-1}), F = -div(u C_f) + (1/Pe) lap(phi)."""
    p = case.params

    def F(C, u, v, w):
        return -ch_flux_div3(case, C, u, v, w) + laplacian3(chemical_potential3(case, geo, C), case.h) / p.Pe

    Fn = F(st["C"], st["u"], st["v"], st["w"])
    Fo = F(st["C_old"], st["u_old"], st["v_old"], st["w_old"])
    return st["C"] + p.dt * (1.5 * Fn - 0.5 * Fo)


def _gather(field_flat, ap, w):
    acc = np.zeros(ap.shape[0])
    for a in range(ap.shape[1]):
        acc = acc + w[:, a] * field_flat[ap[:, a]]
    return acc


def mirror_value3(field_flat, geo: Geometry3D):
    """Eq. extrapolation with the 7-point averages (reading R6')."""
    return 2.0 * _gather(field_flat, geo.ap1, geo.w1) - _gather(field_flat, geo.ap2, geo.w2)


def slip_ghost3(case: Case3D, uM, vM, wM, n, gamma, dn, B=None, gt=None, mu_I=None):
    """a6 core in 3D (reading R5'): Eq. NoPenetration for V_n = u.n, Eq. UpdateVtan for the
    tangential vector, Eq. UpdateVandW back to the axes.  Dynamic angle (reading R18 of the
    2D oracle): the tangential vector gains -(1/Ca) B gt l_s (gamma + 1) dn / (mu_I (l_s +
    gamma dn)), gt (ng x 3) the tangential gradient of C at I."""
    p = case.params
    n1, n2, n3 = n[:, 0], n[:, 1], n[:, 2]
    VnM = (uM * n1 + vM * n2) + wM * n3
    f = (p.l_s - dn) / (p.l_s + gamma * dn)
    VnG = -VnM / gamma
    uG = VnG * n1 + f * (uM - VnM * n1)
    vG = VnG * n2 + f * (vM - VnM * n2)
    wG = VnG * n3 + f * (wM - VnM * n3)
    if B is not None:
        c = (B / p.Ca) * (p.l_s * (gamma + 1.0) * dn) / (mu_I * (p.l_s + gamma * dn))
        uG, vG, wG = uG - c * gt[:, 0], vG - c * gt[:, 1], wG - c * gt[:, 2]
    return uG, vG, wG


def _momentum_brackets3(case: Case3D, C1, u, v, w):
    """The convective brackets div(u u) and the viscous brackets div(mu (grad u + grad u^T))
    of the three components (readings R8, R8'); the z-face ones on the interior planes."""
    h, nz = case.h, case.nz
    _, mu, _ = _props(case)
    Cz = np.concatenate([C1[:1], C1, C1[-1:]], axis=0)            # mirror planes
    uz = np.concatenate([-u[:1], u, -u[-1:]], axis=0)              # no-slip ghost planes
    vz = np.concatenate([-v[:1], v, -v[-1:]], axis=0)
    mu_c = mu(C1)
    # edge viscosities: xy-edges (k, j-1/2, i-1/2); xz-edges (k-1/2, j, i-1/2), k = 0..nz;
    # yz-edges (k-1/2, j-1/2, i), k = 0..nz
    mu_xy = mu(0.25 * (((_xm(_ym(C1)) + _ym(C1)) + _xm(C1)) + C1))
    mu_xz = mu(0.25 * (((_xm(Cz[:-1]) + Cz[:-1]) + _xm(Cz[1:])) + Cz[1:]))
    mu_yz = mu(0.25 * (((_ym(Cz[:-1]) + Cz[:-1]) + _ym(Cz[1:])) + Cz[1:]))
    tau_xx = 2.0 * mu_c * ((_xp(u) - u) / h)
    tau_yy = 2.0 * mu_c * ((_yp(v) - v) / h)
    tau_zz = 2.0 * mu_c * ((w[1:] - w[:-1]) / h)
    tau_xy = mu_xy * ((u - _ym(u)) / h + (v - _xm(v)) / h)
    tau_xz = mu_xz * ((uz[1:] - uz[:-1]) / h + (w - _xm(w)) / h)
    tau_yz = mu_yz * ((vz[1:] - vz[:-1]) / h + (w - _ym(w)) / h)
    visc_u = ((tau_xx - _xm(tau_xx)) / h + (_yp(tau_xy) - tau_xy) / h) + (tau_xz[1:] - tau_xz[:-1]) / h
    visc_v = ((_xp(tau_xy) - tau_xy) / h + (tau_yy - _ym(tau_yy)) / h) + (tau_yz[1:] - tau_yz[:-1]) / h
    visc_w = ((_xp(tau_xz) - tau_xz)[1:nz] / h + (_yp(tau_yz) - tau_yz)[1:nz] / h) \
        + (tau_zz[1:] - tau_zz[:-1]) / h
    uc = 0.5 * (u + _xp(u))
    vc = 0.5 * (v + _yp(v))
    wc = 0.5 * (w[:-1] + w[1:])
    uv = (0.5 * (u + _ym(u))) * (0.5 * (v + _xm(v)))                     # xy-edges
    uw = (0.5 * (uz[1:] + uz[:-1])) * (0.5 * (w + _xm(w)))                # xz-edges
    vw = (0.5 * (vz[1:] + vz[:-1])) * (0.5 * (w + _ym(w)))                # yz-edges
    conv_u = ((uc * uc - _xm(uc * uc)) / h + (_yp(uv) - uv) / h) + (uw[1:] - uw[:-1]) / h
    conv_v = ((_xp(uv) - uv) / h + (vc * vc - _ym(vc * vc)) / h) + (vw[1:] - vw[:-1]) / h
    conv_w = ((_xp(uw) - uw)[1:nz] / h + (_yp(vw) - vw)[1:nz] / h) + (wc[1:] * wc[1:] - wc[:-1] * wc[:-1]) / h
    return conv_u, conv_v, conv_w, visc_u, visc_v, visc_w


def momentum_rhs3(case: Case3D, C1, u, v, w):
    """H = -div(u u) + div(mu (grad u + grad u^T)) / (Re rho) on the x-, y- and z-faces
    (Eq. PredictionExp; readings R8, R8').  Hw rows 0 and nz are zero."""
    p = case.params
    nz = case.nz
    rho, _, _ = _props(case)
    conv_u, conv_v, conv_w, visc_u, visc_v, visc_w = _momentum_brackets3(case, C1, u, v, w)
    Hu = -conv_u + visc_u / (p.Re * rho(0.5 * (_xm(C1) + C1)))
    Hv = -conv_v + visc_v / (p.Re * rho(0.5 * (_ym(C1) + C1)))
    Hw = np.zeros_like(w)
    Hw[1:nz] = -conv_w + visc_w / (p.Re * rho(0.5 * (C1[:-1] + C1[1:])))
    return Hu, Hv, Hw


def momentum_terms3(case: Case3D, C1, u, v, w):
    """The two brackets of momentum_rhs3 separately (the semi-implicit predictor of
    Appendix A.2, reading R19 of the 2D oracle): N = -div(u u) and
    V = div(mu (grad u + grad u^T)) / (Re rho), per component; the z-face wall planes zero."""
    p = case.params
    nz = case.nz
    rho, _, _ = _props(case)
    conv_u, conv_v, conv_w, visc_u, visc_v, visc_w = _momentum_brackets3(case, C1, u, v, w)
    Nw = np.zeros_like(w)
    Vw = np.zeros_like(w)
    Nw[1:nz] = -conv_w
    Vw[1:nz] = visc_w / (p.Re * rho(0.5 * (C1[:-1] + C1[1:])))
    return (-conv_u, -conv_v, Nw, visc_u / (p.Re * rho(0.5 * (_xm(C1) + C1))),
            visc_v / (p.Re * rho(0.5 * (_ym(C1) + C1))), Vw)


def mass_flux_term3(case: Case3D, C1, phi, u, v, w):
    """(rho'/(rho_f Pe)) (grad phi . grad) u on the x-, y- and z-faces (the last term of Eq.
    predictionSemi, reading R19 of the 2D oracle, with the third axis): rho' = (rho_l -
    rho_g)/2; the chemical potential's gradient by the face difference across the face and
    the mean of the two cells' central differences along it (phi continued by mirror planes
    beyond the z walls); the velocity's by central differences of its own faces (no-slip
    ghost planes -u, -v at the z walls; w on the interior z-faces, zero on the walls)."""
    p = case.params
    h, nz = case.h, case.nz
    rho, _, _ = _props(case)
    rp = 0.5 * (1.0 - 1.0 / p.rho_ratio)
    phx = (_xp(phi) - _xm(phi)) / (2.0 * h)
    phy = (_yp(phi) - _ym(phi)) / (2.0 * h)
    phz = (_zp_mirror(phi) - _zm_mirror(phi)) / (2.0 * h)
    uz = np.concatenate([-u[:1], u, -u[-1:]], axis=0)
    vz = np.concatenate([-v[:1], v, -v[-1:]], axis=0)
    mfu = (rp / (rho(0.5 * (_xm(C1) + C1)) * p.Pe)) * (
        (((phi - _xm(phi)) / h) * ((_xp(u) - _xm(u)) / (2.0 * h))
         + (0.5 * (phy + _xm(phy))) * ((_yp(u) - _ym(u)) / (2.0 * h)))
        + (0.5 * (phz + _xm(phz))) * ((uz[2:] - uz[:-2]) / (2.0 * h)))
    mfv = (rp / (rho(0.5 * (_ym(C1) + C1)) * p.Pe)) * (
        ((0.5 * (phx + _ym(phx))) * ((_xp(v) - _xm(v)) / (2.0 * h))
         + ((phi - _ym(phi)) / h) * ((_yp(v) - _ym(v)) / (2.0 * h)))
        + (0.5 * (phz + _ym(phz))) * ((vz[2:] - vz[:-2]) / (2.0 * h)))
    mfw = np.zeros_like(w)
    wi = w[1:nz]
    mfw[1:nz] = (rp / (rho(0.5 * (C1[:-1] + C1[1:])) * p.Pe)) * (
        ((0.5 * (phx[1:] + phx[:-1])) * ((_xp(wi) - _xm(wi)) / (2.0 * h))
         + (0.5 * (phy[1:] + phy[:-1])) * ((_yp(wi) - _ym(wi)) / (2.0 * h)))
        + ((phi[1:] - phi[:-1]) / h) * ((w[2:] - w[:-2]) / (2.0 * h)))
    return mfu, mfv, mfw


def velocity_helmholtz3(case: Case3D, ru, rv, rw, a):
    """(1 - a L) d = r for the three velocity components (Appendix A.2, Eq. predictionSemi,
    the implicit half of nu0 lap u): real Fourier in x, complex Fourier in y, and along z the
    DST-II of the tangential components (no-slip ghost planes, modes m = 1..nz) and the DST-I
    of w on the interior z-faces (w = 0 on the walls, modes m = 1..nz-1); eigenvalues
    -(4/h^2)(sin^2(pi kx/nx) + sin^2(pi ky/ny) + sin^2(pi m/(2 nz)))."""
    nx, ny, nz, h = case.nx, case.ny, case.nz, case.h
    lx = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(nx // 2 + 1) / nx) ** 2
    ly = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(ny) / ny) ** 2
    lt = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(1, nz + 1) / (2.0 * nz)) ** 2
    ln = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(1, nz) / (2.0 * nz)) ** 2

    def solve(r, typ, lz):
        s = sfft.fft(sfft.rfft(r, axis=2), axis=1)
        t = sfft.dst(s.real, type=typ, axis=0) + 1j * sfft.dst(s.imag, type=typ, axis=0)
        t = t / (1.0 - a * ((lz[:, None, None] + ly[None, :, None]) + lx[None, None, :]))
        t = sfft.idst(t.real, type=typ, axis=0) + 1j * sfft.idst(t.imag, type=typ, axis=0)
        return sfft.irfft(sfft.ifft(t, axis=1), n=nx, axis=2)

    du = solve(ru, 2, lt)
    dv = solve(rv, 2, lt)
    dw = np.zeros((nz + 1, ny, nx))
    dw[1:nz] = solve(rw[1:nz], 1, ln)
    return du, dv, dw


def step3(case: Case3D, geo: Geometry3D, st: dict) -> tuple[dict, dict]:
    """One full 3D time step a1..a8.  Returns (new state, intermediates)."""
    p = case.params
    nx, ny, nz, h = case.nx, case.ny, case.nz, case.h
    eta = p.Cn
    rho, mu, rho0 = _props(case)
    info = {}

    # a1 + a2 (semi-implicit, or the explicit variant with params.ch_scheme = 1)
    if getattr(p, "ch_scheme", 0) == 1:
        C_pre = ch_explicit3(case, geo, st)
    else:
        Q = ch_rhs3(case, geo, st)
        C_pre = ch_solve3(case, Q)
        info["Q"] = Q
    info["C_pre"], info["mass_pre"] = C_pre, float(C_pre.sum())

    # a3
    C1 = C_pre.copy()
    f = C1.reshape(-1)
    C_M = mirror_value3(C_pre.reshape(-1), geo)
    B = gt = None
    if p.mu_f > 0.0:
        # dynamic angle (reading R18 of the 2D oracle), vector form: v_t (dC/dx_t) = V_t . grad C
        g = geo.gcell
        gam = geo.gamma
        Cn_flat = st["C"].reshape(-1)
        CI_n = st.get("C_I")
        CI_n = np.full(len(g), np.nan) if CI_n is None else CI_n
        CI_n = np.where(np.isfinite(CI_n), CI_n,
                        (gam * Cn_flat[g] + mirror_value3(Cn_flat, geo)) / (gam + 1.0))
        at_I = lambda fld: (gam * fld.reshape(-1)[g] + mirror_value3(fld.reshape(-1), geo)) / (gam + 1.0)
        UI = np.stack([at_I(0.5 * (st["u"] + _xp(st["u"]))), at_I(0.5 * (st["v"] + _yp(st["v"]))),
                       at_I(0.5 * (st["w"][:-1] + st["w"][1:]))], axis=1)
        GI = np.stack([at_I((_xp(C_pre) - _xm(C_pre)) / (2.0 * h)),
                       at_I((_yp(C_pre) - _ym(C_pre)) / (2.0 * h)),
                       at_I((_zp_mirror(C_pre) - _zm_mirror(C_pre)) / (2.0 * h))], axis=1)
        nn = geo.n
        Vt = UI - (UI * nn).sum(axis=1)[:, None] * nn
        gt = GI - (GI * nn).sum(axis=1)[:, None] * nn
        adv = (Vt * GI).sum(axis=1)
        C_G, C_I, B = dynamic_contact_ghost(case, C_M, gam, geo.dn, CI_n, adv)
        clamped = 0
    else:
        C_G, C_I, clamped = contact_angle_ghost(case, C_M, geo.gamma, geo.dn)
    f[geo.gcell] = C_G
    info["C"], info["C_I"], info["disc_clamped"], info["B"] = C1, C_I, clamped, B
    info["mass"] = float(C1.sum())

    # a4
    phi = chemical_potential3(case, geo, C1)
    info["phi"] = phi

    # a5: the AB2 predictor (Eq. PredictionExp) or, with params.ns_scheme = 1, the
    # semi-implicit predictor of Appendix A.2 (Eq. predictionSemi; the history holds N)
    u, v, w = st["u"], st["v"], st["w"]
    semi = getattr(p, "ns_scheme", 0) == 1
    if semi:
        Hu, Hv, Hw, Vu, Vv, Vw = momentum_terms3(case, C1, u, v, w)
    else:
        Hu, Hv, Hw = momentum_rhs3(case, C1, u, v, w)
    rho_u = rho(0.5 * (_xm(C1) + C1))
    rho_v = rho(0.5 * (_ym(C1) + C1))
    rho_w = rho(0.5 * (C1[:-1] + C1[1:]))
    k_st = KAPPA / (p.Re * p.Ca * eta)
    st_u = k_st * (0.5 * (phi + _xm(phi))) * ((C1 - _xm(C1)) / h) / rho_u
    st_v = k_st * (0.5 * (phi + _ym(phi))) * ((C1 - _ym(C1)) / h) / rho_v
    st_w = k_st * (0.5 * (phi[1:] + phi[:-1])) * ((C1[1:] - C1[:-1]) / h) / rho_w
    w_star = np.zeros_like(w)
    if semi:
        mfu, mfv, mfw = mass_flux_term3(case, C1, phi, u, v, w)
        Fu = (((1.5 * Hu - 0.5 * st["Hu"]) + st_u) + Vu) + mfu
        Fv = (((1.5 * Hv - 0.5 * st["Hv"]) + st_v) + Vv) + mfv
        Fw = np.zeros_like(w)
        Fw[1:nz] = (((1.5 * Hw[1:nz] - 0.5 * st["Hw"][1:nz]) + st_w) + Vw[1:nz]) + mfw[1:nz]
        nu0 = 0.5 * (1.0 + (1.0 / p.mu_ratio) / (1.0 / p.rho_ratio)) / p.Re
        du, dv, dw = velocity_helmholtz3(case, p.dt * Fu, p.dt * Fv, p.dt * Fw, 0.5 * p.dt * nu0)
        u_star = u + du
        v_star = v + dv
        w_star[1:nz] = w[1:nz] + dw[1:nz]
    else:
        u_star = u + p.dt * ((1.5 * Hu - 0.5 * st["Hu"]) + st_u)
        v_star = v + p.dt * ((1.5 * Hv - 0.5 * st["Hv"]) + st_v)
        w_star[1:nz] = w[1:nz] + p.dt * ((1.5 * Hw[1:nz] - 0.5 * st["Hw"][1:nz]) + st_w)
    uss = geo.alpha_u * u_star
    vss = geo.alpha_v * v_star
    wss = geo.alpha_w * w_star
    info["Hu"], info["Hv"], info["Hw"] = Hu, Hv, Hw

    # a6
    ucen = 0.5 * (uss + _xp(uss))
    vcen = 0.5 * (vss + _yp(vss))
    wcen = 0.5 * (wss[:-1] + wss[1:])
    uM = mirror_value3(ucen.reshape(-1), geo)
    vM = mirror_value3(vcen.reshape(-1), geo)
    wM = mirror_value3(wcen.reshape(-1), geo)
    mu_I = mu(C_I) if B is not None else None
    uG, vG, wG = slip_ghost3(case, uM, vM, wM, geo.n, geo.gamma, geo.dn, B, gt, mu_I)
    solid_flat = (geo.cls == CELL_SOLID).reshape(-1)
    cells = []
    for cen, g in ((ucen, uG), (vcen, vG), (wcen, wG)):
        c = cen.copy().reshape(-1)
        c[solid_flat] = 0.0
        c[geo.gcell] = g
        cells.append(c)
    uss_f, vss_f, wss_f = uss.copy(), vss.copy(), wss.copy()
    nxy = nx * ny
    k_, r_ = np.divmod(geo.fu, nxy)
    j_, i_ = np.divmod(r_, nx)
    uss_f.reshape(-1)[geo.fu] = 0.5 * (cells[0][(k_ * ny + j_) * nx + (i_ - 1) % nx] + cells[0][geo.fu])
    k_, r_ = np.divmod(geo.fv, nxy)
    j_, i_ = np.divmod(r_, nx)
    vss_f.reshape(-1)[geo.fv] = 0.5 * (cells[1][(k_ * ny + (j_ - 1) % ny) * nx + i_] + cells[1][geo.fv])
    k_, r_ = np.divmod(geo.fw, nxy)
    wss_f.reshape(-1)[geo.fw] = 0.5 * (cells[2][(k_ - 1) * nxy + r_] + cells[2][k_ * nxy + r_])
    info["uG"], info["vG"], info["wG"] = uG, vG, wG
    info["u_ss"], info["v_ss"], info["w_ss"] = uss_f, vss_f, wss_f

    # a7
    Ph = 2.0 * st["P"] - st["P_old"]
    gx = (1.0 - rho0 / rho_u) * ((Ph - _xm(Ph)) / h)
    gy = (1.0 - rho0 / rho_v) * ((Ph - _ym(Ph)) / h)
    gz = np.zeros_like(w)
    gz[1:nz] = (1.0 - rho0 / rho_w) * ((Ph[1:] - Ph[:-1]) / h)
    div_g = ((_xp(gx) - gx) / h + (_yp(gy) - gy) / h) + (gz[1:] - gz[:-1]) / h
    div_u = ((_xp(uss_f) - uss_f) / h + (_yp(vss_f) - vss_f) / h) + (wss_f[1:] - wss_f[:-1]) / h
    rhs = div_g + (rho0 / p.dt) * div_u
    P1 = poisson_solve3(case, rhs)
    info["rhs_p"], info["P"] = rhs, P1

    # a8
    u1 = uss_f - p.dt * ((1.0 / rho0) * ((P1 - _xm(P1)) / h)
                         + (1.0 / rho_u - 1.0 / rho0) * ((Ph - _xm(Ph)) / h))
    v1 = vss_f - p.dt * ((1.0 / rho0) * ((P1 - _ym(P1)) / h)
                         + (1.0 / rho_v - 1.0 / rho0) * ((Ph - _ym(Ph)) / h))
    w1 = np.zeros_like(w)
    w1[1:nz] = wss_f[1:nz] - p.dt * ((1.0 / rho0) * ((P1[1:] - P1[:-1]) / h)
                                     + (1.0 / rho_w - 1.0 / rho0) * ((Ph[1:] - Ph[:-1]) / h))
    new = {"C": C1, "C_old": st["C"].copy(), "u": u1, "u_old": u.copy(), "v": v1,
           "v_old": v.copy(), "w": w1, "w_old": w.copy(), "Hu": Hu, "Hv": Hv, "Hw": Hw,
           "P": P1, "P_old": st["P"].copy()}
    if p.mu_f > 0.0:
        new["C_I"] = C_I.copy()
    return new, info


def divergence3(u, v, w, h):
    return ((_xp(u) - u) / h + (_yp(v) - v) / h) + (w[1:] - w[:-1]) / h
