"""Plain FP64 CPU oracle of one time step of the hybrid IB / phase-field method, 2D.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module; the CUDA
library is an independent implementation and the two share no code.

What it computes (Shahmardi, Rosti, Tammisola & Brandt, arXiv 2104.00350):
  * geometry precompute, Sec. 4.1: volume fractions by subgrid counting (Sec. 4.1.1),
    normals from corner gradients of alpha (Eqs. NormalVectors_part1/2), ghost /
    intersect / mirror / interpolation points (Sec. 4.1.2), inverse-distance weights
    W1/W2 (Eq. weright averaged);
  * per step, in the order of the block diagram of Sec. 4.2 / Appendix A:
      a1  RHS of the semi-implicit Cahn-Hilliard split (Eq. Helmholtz1, Appendix A.1)
      a2  the two Helmholtz solves (Eqs. Helmholtz1, Helmholtz2) in one eigenbasis
          (or, with params.ch_scheme = 1, a1+a2 as the explicit AB2 update of Eq. ExpCH)
      a3  contact-angle ghost fill of C (Eqs. interpolationAtWall, ProjectingToNT, UpdateC,
          static form of Eq. WallBCS)
      a4  chemical potential (Eq. Chemical-Potential) and its zero-gradient ghost fill
      a5  AB2 momentum predictor (Eq. PredictionExp) + volume penalisation (Eq. Penalization2)
      a6  ghost-cell slip / no-penetration fill (Eqs. NoPenetration, UpdateVtan, UpdateVandW)
      a7  Dodd-Ferrante pressure Poisson (Eq. PressurePoisson)
      a8  velocity correction (Eq. correction)
Library primitives used as steps: numpy elementwise arithmetic and scipy's FFT / DCT-II.

Readings of the paper where it is silent, garbled or inconsistent (all shared, by
restatement, with the CUDA path):
  R1  Nondimensional CH: dC/dt + div(uC) = (1/Pe) lap(phi), phi = psi'(C) - Cn^2 lap(C),
      psi'(C) = C^3 - C; surface tension force (kappa/(Re Ca Cn)) phi grad C with
      kappa = 3/(2 sqrt 2), so the interfacial tension is 1/(Re Ca).
  R2  The two Helmholtz solves are done back to back in one eigenbasis: the combined
      symbol (L - alpha_s - S/Cn^2)(L + alpha_s) = L^2 - (S/Cn^2) L + 1.5 Pe/(Cn^2 dt)
      is used, which is legal for any S >= 0 (the appendix's alpha_s is real only for
      S >= Cn^2 sqrt(6 Pe/dt)).  Appendix A.1 writes psi where psi' is meant.
  R3  gamma = d1/dn (the formula of Eq. interpolationAtWall, not its wording); the
      one-sided normal derivative is the 3-point Lagrange one through G, I, M, whose
      denominator is gamma(gamma+1)dn (Eq. ProjectingToNT prints gamma(gamma-1)dn).
  R4  Static angle (mu_f = 0, where Eq. WallBCS_recast divides by zero): C_I solves
      kappa Cn dC/dn + cos(theta) g'(C_I) = 0 with G, I, M tied by Eq. UpdateC, so the
      3-point derivative is the slope (C_M - C_I)/(gamma dn) -- the same reduction the
      paper makes for the slip velocity in Eq. UpdateVtan.  (Holding G at the estimate
      2C^n_G - C^{n-1}_G instead makes the ghost update an unstable recursion: at
      theta = 90 deg it multiplies ghost errors by about 5 per step.)  g' is taken as zero
      outside [-1, 1] (g constant beyond the pure phases), so C_I = C_M when |C_M| >= 1 and
      otherwise the quadratic's root inside [-1, 1] is taken (without this cut-off the
      quadratic has no real root once C_M overshoots 1 at a dewetting wall and the ghost
      value feeds the overshoot).  The wetting bracket of the slip condition is then zero,
      so the slip formula has no B term.
  R5  Tangent t = (n2, -n1); back transform x1 = Vn n1 + Vt n2, x2 = Vn n2 - Vt n1.
  R6  Ghost = solid cell centre with a fluid centre among its 4 face neighbours; averaging
      points = the cell holding the IP plus its 4 face neighbours, solid centres and
      out-of-domain cells excluded, weights renormalised.
  R7  d1 = sqrt(2) h, d2 = d1/2, IP1 = M + d2 n, IP2 = M + 2 d2 n.
  R8  Second-order FD on the staggered grid: arithmetic face/edge means, divergence-form
      convection, periodic in x1, mirror (Neumann) rows for C, phi, P and no-slip ghost
      rows for u in x2, v = 0 on the x2 walls.
  R9  AB2 on H = -conv + visc/(Re rho) with the n-1 term taken at the n-1 state; the
      surface tension term is single-level at n+1.
  R10 Face fix after the velocity ghost fill: faces with alpha_f < 1 touching a ghost cell
      take the mean of the two cell-centred values (ghost value; 0 for a solid non-ghost
      cell; pre-fix centred u** for a fluid cell).
  R11 rho(C) and mu(C) are evaluated with C clamped to [-1, 1]: the Dodd-Ferrante split of
      Eq. PressurePoisson rests on rho >= rho0 = min(rho_l, rho_g), which an unclamped
      linear law breaks wherever C overshoots -1 (observed inside the solid, where it ended
      runs after ~1e4 steps).
  R16 No flux through the immersed wall in the semi-implicit CH step.  The wall condition
      d(phi)/dn = 0 (Eq. AllBCs, second line; imposed by phi_G = phi_M, Sec. 4.2.2) enters
      the explicit part of the Appendix A.1 split: its right-hand side holds lap(phi~)/Cn^2
      with phi~ = psi'(C~) - Cn^2 lap(C~) ghost-filled, and only the stabilisation of the
      increment C^{n+1} - C~ stays implicit across the wall.  Appendix A.1 solves on the
      whole box with Neumann conditions at the box walls only; without this term C
      diffuses through the ghost layer into and out of the solid and a droplet settled 7 deg
      off the prescribed angle (52.9 deg for 60).
  R17 Averaging weights (Eq. weright averaged): the normalised 1/h_i^2 weights w_i are made
      linear-exact by moving least squares with a linear basis and the same weight
      function: xb = sum w_i d_i, S = sum w_i (d_i - xb)(d_i - xb)^T, W_i = w_i (1 + (d_i - xb)
      . S^{-1}(-xb)) (d_i: offset from the IP in cells), when the kept averaging points are
      not all on one line (else the plain weights).  Plain Shepard weights reproduce
      constants only; their first-order error moved the settled angle by 2-3 deg at
      Cn/h = 1.28.  params.weights = 1 selects the plain weights of the paper.
  R18 Dynamic contact angle (mu_f > 0): Eq. WallBCS_recast, nondimensional as
      dC_I/dt = -v_t (dC/dx_t)_I + (1/(mu_f Cn)) [kappa Cn dC/dn + cos(theta) g'(C_I)]
      (the paper's mu_f eps over sigma eps, with eps -> Cn and sigma -> 1), integrated by one
      backward-Euler step per time step for a per-ghost state C_I (the normal derivative,
      R4's slope (C_M - C_I)/(gamma dn), and g'(C_I) at the new level, solved as R4's
      quadratic with modified coefficients; an explicit g' is unstable for small mu_f), the
      advection explicit; v_t and dC/dx_t at I
      are gamma-weighted means of the ghost's and the mirror point's values (Eq.
      interpolationAtWall) of the level-n cell-centred velocity and of central differences
      of C^{n+1} before the fill.  An unset C_I (NaN) starts as (gamma C^n_G + C^n_M)/(gamma+1).
      The bracket B = kappa Cn dC/dn + cos(theta) g'(C_I) at the new level enters the slip
      condition (Eq. UpdateVtan) as -(1/Ca) B (dC/dx_t)_I l_s (gamma+1) dn / (mu_I (l_s +
      gamma dn)), mu_I = mu(C_I): the stress balance of Eq. SlipVelocity multiplied by Re,
      with the surface-tension scale 1/(Re Ca) of R1 (the paper's Eq. UpdateVtan drops kappa
      and eps).  mu_f -> 0 recovers R4's static root; mu_f -> infinity freezes C_I but for
      advection along the wall.
  R19 Semi-implicit momentum predictor (params.ns_scheme = 1; Appendix A.2, Eq.
      predictionSemi): u* = u^n + d with (1 - (dt nu0/2) L) d = dt [3/2 N^n - 1/2 N^{n-1} + ST
      + V^n + MF], N = -div(u u) (the history field holds N only), V^n = div(mu^{n+1}(grad u^n +
      grad u^n^T))/(Re rho^{n+1}) at level n, ST the surface tension of R9, nu0 =
      (mu_l/rho_l + mu_g/rho_g)/(2 Re), L the 5-point Laplacian of each component with its
      own x2 boundary rows (no-slip ghost rows for u: DST-II; v = 0 on the walls: DST-I),
      solved on the whole box like the CH split.  MF = (rho'/(rho_f Pe)) (grad phi . grad) u,
      rho' = (rho_l - rho_g)/2: the mass-flux consistency term, derived from the momentum
      equation with the diffusive mass flux rho' J, J = -(1/Pe) grad phi (the paper prints
      (rho_1 - rho_2)/2 M (grad phi . grad) u without the 1/rho); the discrete form is in
      mass_flux_term.
  R15 Explicit CH (Eq. ExpCH) in the form of R1 and R8: the update is
      C^{n+1} = C^n + dt (3/2 F^n - 1/2 F^{n-1}),  F = -div(u C_f) + (1/Pe) lap(phi),
      the convective term in divergence form (the paper writes u . grad C; equal for a
      divergence-free u) and the mobility term with the paper's 3/(2 sqrt 2) M absorbed into
      1/Pe.  F^{n-1} is evaluated from the level n-1 fields (C^{n-1}, u^{n-1}, v^{n-1}, and
      phi^{n-1} = phi(C^{n-1}) with its zero-gradient ghost fill), so the first step of a
      run started with C^{n-1} = C^n, u^{n-1} = u^n is a forward Euler step.  As in the
      semi-implicit variant every cell is updated (also inside the solid) before the a3
      ghost fill.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.fft as sfft

from workloads.cases import GEOM_FLAT, GEOM_MASK, GEOM_NONE, GEOM_SINUSOID, Case2D

KAPPA = 3.0 / (2.0 * math.sqrt(2.0))   # the 3/(2 sqrt 2) factor of Eq. Cahn-Hilliard
GAMMA0 = 1.5                           # BDF2 weight of Appendix A.1: (3/2 C^{n+1} - C_check)/dt
NSUB = 100                             # subgrid points per direction (Sec. 4.1.1)
MARCH_DIV = 100                        # march step h/100 along the normal (Sec. 4.1.2)
MARCH_MAX = 1000                       # give up after 10 h
BISECT = 60                            # bisection refinements of the intersect point
EPS0 = 1.0e-30                         # epsilon_0 of Eq. NormalVectors_part2
NAP = 5                                # averaging points per interpolation point in 2D

CELL_FLUID, CELL_GHOST, CELL_SOLID = 0, 1, 2


# --------------------------------------------------------------------------- walls
def wall_height(case: Case2D, x):
    """x2-position of the wall above abscissa x, or None when there is no solid."""
    p = case.geom_p
    if case.geom_kind == GEOM_FLAT:
        return np.full(np.shape(x), p[0])
    if case.geom_kind == GEOM_SINUSOID:
        w = (2.0 * math.pi) * p[2]
        return p[0] + p[1] * np.sin(w * np.asarray(x, dtype=np.float64))
    if case.geom_kind == GEOM_NONE:
        return None
    raise ValueError("unknown wall kind")


def mask_alpha(case: Case2D, x, y):
    """MASK walls (reading R20): the cell-centre fractions alpha_c interpolated bilinearly at
    (x, y), centres at ((i + 1/2) h, (j + 1/2) h), periodic in x1, the first and last centre
    rows continued beyond them."""
    A = np.asarray(case.alpha[0], dtype=np.float64)
    ny, nx = A.shape
    h = case.h
    x, y = np.broadcast_arrays(np.asarray(x, np.float64), np.asarray(y, np.float64))
    fx = x / h - 0.5
    fy = y / h - 0.5
    fx0 = np.floor(fx)
    fy0 = np.floor(fy)
    tx = fx - fx0
    ty = fy - fy0
    i0 = fx0.astype(np.int64) % nx
    i1 = (i0 + 1) % nx
    j0 = np.clip(fy0.astype(np.int64), 0, ny - 1)
    j1 = np.clip(fy0.astype(np.int64) + 1, 0, ny - 1)
    a = (1.0 - tx) * A[j0, i0] + tx * A[j0, i1]
    b = (1.0 - tx) * A[j1, i0] + tx * A[j1, i1]
    return (1.0 - ty) * a + ty * b


def solid(case: Case2D, x, y):
    """True where (x, y) lies inside the solid."""
    if case.geom_kind == GEOM_MASK:
        return mask_alpha(case, x, y) < 0.5
    yw = wall_height(case, x)
    if yw is None:
        return np.zeros(np.broadcast(np.asarray(x), np.asarray(y)).shape, dtype=bool)
    return np.asarray(y) < yw


# --------------------------------------------------------------- volume fractions
def volume_fractions(case: Case2D, x0: np.ndarray, y0: np.ndarray) -> np.ndarray:
    """Fluid fraction of the h x h control volumes with lower-left corners (x0[i], y0[j]):
    the share of the NSUB x NSUB subgrid points (x0 + (a+1/2) h/NSUB, y0 + (b+1/2) h/NSUB)
    that lie outside the solid (Sec. 4.1.1).  Control volumes that lie entirely above the
    highest or below the lowest wall height met by their subpoint columns are counted
    without visiting every subpoint (the count is the same)."""
    h = case.h
    hs = h / NSUB
    off = (np.arange(NSUB, dtype=np.float64) + 0.5) * hs
    out = np.empty((len(y0), len(x0)))
    for i, xl in enumerate(x0):
        xs = xl + off
        yw = wall_height(case, xs)
        if yw is None:
            out[:, i] = 1.0
            continue
        ys = y0[:, None] + off[None, :]
        all_fluid = ys[:, 0] >= yw.max()
        all_solid = ys[:, -1] < yw.min()
        out[all_fluid, i] = 1.0
        out[all_solid, i] = 0.0
        for j in np.nonzero(~(all_fluid | all_solid))[0]:
            n_fluid = np.count_nonzero(~solid(case, xs[:, None], ys[j][None, :]))
            out[j, i] = n_fluid / float(NSUB * NSUB)
    return out


@dataclass
class Geometry2D:
    """Precomputed tables (the paper's 'permanent arrays', Sec. 4.1.2)."""
    alpha_c: np.ndarray     # (ny, nx)   cell-centred control volumes
    alpha_u: np.ndarray     # (ny, nx)   x1-face control volumes
    alpha_v: np.ndarray     # (ny+1, nx) x2-face control volumes
    cls: np.ndarray         # (ny, nx)   CELL_FLUID / CELL_GHOST / CELL_SOLID
    gcell: np.ndarray       # (ng,) linear cell index j*nx + i, ascending
    n: np.ndarray           # (ng, 2) unit normal, solid -> fluid
    dn: np.ndarray          # (ng,) ghost-to-intersect distance
    gamma: np.ndarray       # (ng,) d1 / dn
    ap1: np.ndarray         # (ng, NAP) averaging-point cell indices around IP1
    w1: np.ndarray          # (ng, NAP) normalised weights (W1)
    ap2: np.ndarray
    w2: np.ndarray
    fu: np.ndarray          # linear indices of fixed x1-faces
    fv: np.ndarray          # linear indices (j*nx+i, j in 1..ny-1) of fixed x2-faces
    n_fallback_normal: int
    n_fallback_ap: int


def _alpha_at(alpha_c, i, j):
    ny, nx = alpha_c.shape
    j = min(max(j, 0), ny - 1)       # mirror rows at the x2 domain walls
    return alpha_c[j, i % nx]


def _normal(case: Case2D, alpha_c, cls, i, j):
    """Eqs. NormalVectors_part1/2: alpha gradients at the four corners, averaged to the
    centre, normalised with epsilon_0.  Points from the solid into the fluid."""
    h = case.h
    ny, nx = alpha_c.shape

    def corner(ci, cj):   # corner (ci+1/2, cj+1/2)
        a00 = _alpha_at(alpha_c, ci, cj)
        a10 = _alpha_at(alpha_c, ci + 1, cj)
        a01 = _alpha_at(alpha_c, ci, cj + 1)
        a11 = _alpha_at(alpha_c, ci + 1, cj + 1)
        mx = (a10 + a11 - a00 - a01) / (2.0 * h)
        my = (a01 + a11 - a00 - a10) / (2.0 * h)
        return mx, my

    c1 = corner(i, j)
    c2 = corner(i - 1, j)
    c3 = corner(i, j - 1)
    c4 = corner(i - 1, j - 1)
    mx = (((c1[0] + c2[0]) + c3[0]) + c4[0]) / 4.0
    my = (((c1[1] + c2[1]) + c3[1]) + c4[1]) / 4.0
    norm = math.sqrt(mx * mx + my * my + EPS0)
    if math.sqrt(mx * mx + my * my) * h < 1.0e-12:
        nb = _first_fluid_neighbour(cls, i, j)
        if nb is None:
            raise ValueError("ghost cell without fluid neighbour")
        return nb[2], nb[3], True
    return mx / norm, my / norm, False


def _first_fluid_neighbour(cls, i, j):
    """Face neighbour in the fixed order +x2, -x2, +x1, -x1 whose centre is fluid:
    (i, j, e1, e2) with (e1, e2) the unit vector towards it."""
    ny, nx = cls.shape
    for di, dj in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        jj = j + dj
        if 0 <= jj < ny and cls[jj, (i + di) % nx] == CELL_FLUID:
            return (i + di) % nx, jj, float(di), float(dj)
    return None


def spans_plane(offsets) -> bool:
    """True when the integer stencil offsets (di, dj) of the kept averaging points are not
    all on one line (affinely independent in 2D); decided in integers."""
    o = [(a - offsets[0][0], b - offsets[0][1]) for a, b in offsets]
    return any(o[p][0] * o[q][1] - o[p][1] * o[q][0] != 0
               for p in range(len(o)) for q in range(p + 1, len(o)))


def linear_exact_weights(w, d):
    """Reading R17: moving-least-squares weights with a linear basis and the weight function
    w of Eq. weright averaged (normalised, sum 1), for points at offsets d (k x D, in cells)
    from the interpolation point.  With xb = sum w_i d_i and S = sum w_i (d_i - xb)(d_i - xb)^T
    the weights are W_i = w_i (1 + (d_i - xb) . S^{-1} (0 - xb)); sum W_i = 1 and
    sum W_i d_i = 0, i.e. constants and linear fields are reproduced exactly.  Shepard's
    weights of the paper are the same construction with a constant basis (W = w)."""
    w = np.asarray(w, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    xb = w @ d
    e = d - xb
    S = (e * w[:, None]).T @ e
    v = np.linalg.solve(S, -xb)
    return list(w * (1.0 + e @ v))


def _averaging_points(case: Case2D, cls, px, py):
    """Cell holding (px, py) plus its 4 face neighbours; solid centres and cells outside
    the x2 range dropped; inverse-squared-distance weights, normalised (Eq. weright
    averaged); a coincident point takes the whole weight.  With params.weights = 0 the
    weights are made linear-exact (reading R17) when the kept points span the plane."""
    h = case.h
    ny, nx = cls.shape
    i0 = math.floor(px / h)
    j0 = math.floor(py / h)
    idx, d2s, offs, rel = [], [], [], []
    for di, dj in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
        ic, jc = i0 + di, j0 + dj
        if jc < 0 or jc >= ny:
            continue
        if cls[jc, ic % nx] != CELL_FLUID:
            continue
        cx = (ic + 0.5) * h
        cy = (jc + 0.5) * h
        dx = cx - px
        dy = cy - py
        idx.append(jc * nx + (ic % nx))
        d2s.append(dx * dx + dy * dy)
        offs.append((di, dj))
        rel.append((dx / h, dy / h))
    if not idx:
        return None
    tiny = (1.0e-12 * h) * (1.0e-12 * h)
    for k, d2 in enumerate(d2s):
        if d2 < tiny:
            w = [0.0] * len(idx)
            w[k] = 1.0
            return idx, w
    wr = [1.0 / d2 for d2 in d2s]
    q = 0.0
    for x in wr:
        q += x
    w = [x / q for x in wr]
    if getattr(case.params, "weights", 0) == 0 and len(idx) >= 3 and spans_plane(offs):
        w = linear_exact_weights(w, rel)
    return idx, w


def build_geometry(case: Case2D) -> Geometry2D:
    """All of Sec. 4.1 for one 2D case."""
    nx, ny, h = case.nx, case.ny, case.h
    p = case.params
    ii = np.arange(nx, dtype=np.float64)
    jj = np.arange(ny, dtype=np.float64)
    if case.geom_kind == GEOM_MASK:   # the caller's fractions replace the count (R20)
        alpha_c, alpha_u, alpha_v = (np.asarray(a, dtype=np.float64).reshape(s) for a, s in
                                     zip(case.alpha, ((ny, nx), (ny, nx), (ny + 1, nx))))
    else:
        alpha_c = volume_fractions(case, ii * h, jj * h)
        alpha_u = volume_fractions(case, (ii - 0.5) * h, jj * h)
        alpha_v = volume_fractions(case, ii * h, (np.arange(ny + 1, dtype=np.float64) - 0.5) * h)

    xc = (ii + 0.5) * h
    yc = (jj + 0.5) * h
    sol = solid(case, xc[None, :], yc[:, None])
    cls = np.where(sol, CELL_SOLID, CELL_FLUID).astype(np.int8)
    fl = ~sol
    nb_fluid = np.zeros_like(sol)
    nb_fluid |= np.roll(fl, 1, axis=1) | np.roll(fl, -1, axis=1)
    nb_fluid[1:] |= fl[:-1]
    nb_fluid[:-1] |= fl[1:]
    cls[sol & nb_fluid] = CELL_GHOST

    gj, gi = np.nonzero(cls == CELL_GHOST)          # row-major order = ascending j*nx+i
    ng = len(gi)
    gcell = (gj * nx + gi).astype(np.int64)
    nrm = np.zeros((ng, 2))
    dn = np.zeros(ng)
    gamma = np.zeros(ng)
    ap1 = np.zeros((ng, NAP), dtype=np.int64)
    ap2 = np.zeros((ng, NAP), dtype=np.int64)
    w1 = np.zeros((ng, NAP))
    w2 = np.zeros((ng, NAP))
    nfb_n = nfb_ap = 0
    ds = h / MARCH_DIV
    for g in range(ng):
        i, j = int(gi[g]), int(gj[g])
        n1, n2, fb = _normal(case, alpha_c, cls, i, j)
        nfb_n += int(fb)
        nrm[g] = (n1, n2)
        gx = (i + 0.5) * h
        gy = (j + 0.5) * h
        # intersect point: march along n until the first point outside the solid,
        # then bisect between the last inside and the first outside point
        k = 1
        while k <= MARCH_MAX:
            t = k * ds
            if not solid(case, gx + t * n1, gy + t * n2):
                break
            k += 1
        if k > MARCH_MAX:
            raise ValueError(f"no intersect point found for ghost ({i},{j})")
        lo, hi = (k - 1) * ds, k * ds
        for _ in range(BISECT):
            mid = 0.5 * (lo + hi)
            if solid(case, gx + mid * n1, gy + mid * n2):
                lo = mid
            else:
                hi = mid
        dn[g] = hi
        gamma[g] = p.d1 / hi
        s1 = (hi + p.d1) + p.d2
        s2 = (hi + p.d1) + 2.0 * p.d2
        for s, aps, ws in ((s1, ap1, w1), (s2, ap2, w2)):
            res = _averaging_points(case, cls, gx + s * n1, gy + s * n2)
            if res is None:
                nb = _first_fluid_neighbour(cls, i, j)
                res = ([nb[1] * nx + nb[0]], [1.0])
                nfb_ap += 1
            idx, w = res
            for a in range(NAP):
                aps[g, a] = idx[a] if a < len(idx) else idx[0]
                ws[g, a] = w[a] if a < len(idx) else 0.0

    isg = cls == CELL_GHOST
    fu_mask = (alpha_u < 1.0) & (isg | np.roll(isg, 1, axis=1))
    fv_mask = np.zeros((ny + 1, nx), dtype=bool)
    fv_mask[1:ny] = (alpha_v[1:ny] < 1.0) & (isg[1:] | isg[:-1])
    fu = np.flatnonzero(fu_mask.reshape(-1)).astype(np.int64)
    fv = np.flatnonzero(fv_mask.reshape(-1)).astype(np.int64)
    return Geometry2D(alpha_c, alpha_u, alpha_v, cls, gcell, nrm, dn, gamma, ap1, w1, ap2, w2,
                      fu, fv, nfb_n, nfb_ap)


# ------------------------------------------------------------------ discrete operators
def _xp(a):   # a[:, i+1] (periodic x1)
    return np.roll(a, -1, axis=1)


def _xm(a):   # a[:, i-1]
    return np.roll(a, 1, axis=1)


def _yp_mirror(a):   # a[j+1] with the mirror row a[ny] = a[ny-1]
    return np.vstack([a[1:], a[-1:]])


def _ym_mirror(a):   # a[j-1] with the mirror row a[-1] = a[0]
    return np.vstack([a[:1], a[:-1]])


def laplacian(a: np.ndarray, h: float) -> np.ndarray:
    """5-point Laplacian of a cell-centred field; periodic x1, zero-gradient x2 walls."""
    return (((_xp(a) + _xm(a)) + (_yp_mirror(a) + _ym_mirror(a))) - 4.0 * a) / (h * h)


def eigenvalues(nx: int, ny: int, h: float):
    """Eigenvalues of `laplacian` in the real-Fourier (x1) x DCT-II (x2) basis."""
    kx = np.arange(nx // 2 + 1, dtype=np.float64)
    my = np.arange(ny, dtype=np.float64)
    lx = -(4.0 / (h * h)) * np.sin(np.pi * kx / nx) ** 2
    ly = -(4.0 / (h * h)) * np.sin(np.pi * my / (2.0 * ny)) ** 2
    return ly[:, None] + lx[None, :]


def _forward(a):
    s = sfft.rfft(a, axis=1)
    return sfft.dct(s.real, type=2, axis=0) + 1j * sfft.dct(s.imag, type=2, axis=0)


def _inverse(s, nx):
    t = sfft.idct(s.real, type=2, axis=0) + 1j * sfft.idct(s.imag, type=2, axis=0)
    return sfft.irfft(t, n=nx, axis=1)


def ch_symbol(case: Case2D) -> np.ndarray:
    """Combined symbol of Eqs. Helmholtz1 + Helmholtz2 (reading R2)."""
    p = case.params
    lam = eigenvalues(case.nx, case.ny, case.h)
    eta2 = p.Cn * p.Cn
    return lam * lam - (p.S / eta2) * lam + GAMMA0 * p.Pe / (eta2 * p.dt)


def ch_solve(case: Case2D, Q: np.ndarray) -> np.ndarray:
    """Appendix A.1: solve (L^2 - (S/Cn^2) L + 1.5 Pe/(Cn^2 dt)) C = Q, L = laplacian."""
    return _inverse(_forward(Q) / ch_symbol(case), case.nx)


def ch_solve_two_stage(case: Case2D, Q: np.ndarray) -> np.ndarray:
    """Appendix A.1 literally: Eq. Helmholtz1 for Gamma, then Eq. Helmholtz2 for C, with
    alpha_s of the appendix (needs S >= Cn^2 sqrt(6 Pe / dt) so that alpha_s is real).
    In these variables lambda M = Cn^2 / Pe."""
    p = case.params
    eta2 = p.Cn * p.Cn
    lamM = eta2 / p.Pe
    disc = 1.0 - 6.0 * eta2 * eta2 / (lamM * p.dt * p.S * p.S)
    if disc < 0.0:
        raise ValueError("alpha_s is complex for this S")
    alpha_s = -(p.S / (2.0 * eta2)) * (1.0 + math.sqrt(disc))
    lam = eigenvalues(case.nx, case.ny, case.h)
    # Eq. Helmholtz1: (L - (alpha_s + S/Cn^2)) Gamma = Q; then Eq. Helmholtz2:
    # (L + alpha_s) C = Gamma.  The product of the two operators is the combined symbol.
    g = _forward(Q) / (lam - (alpha_s + p.S / eta2))
    c = g / (lam + alpha_s)
    return _inverse(c, case.nx)


def poisson_solve(case: Case2D, rhs: np.ndarray) -> np.ndarray:
    """laplacian(P) = rhs with the mean (k = 0) mode set to zero (Eq. PressurePoisson,
    solved by Fourier / cosine transforms as Sec. 4.4 allows)."""
    lam = eigenvalues(case.nx, case.ny, case.h)
    s = _forward(rhs)
    lam0 = lam.copy()
    lam0[0, 0] = 1.0
    s = s / lam0
    s[0, 0] = 0.0
    return _inverse(s, case.nx)


# ---------------------------------------------------------------------------- step
def _props(case: Case2D):
    p = case.params
    rho_l, rho_g = 1.0, 1.0 / p.rho_ratio
    mu_l, mu_g = 1.0, 1.0 / p.mu_ratio

    # reading R11: C is clamped to [-1, 1] in the property laws, so that rho never falls
    # below rho0 = min(rho_l, rho_g), the bound the Dodd-Ferrante split of Eq.
    # PressurePoisson is built on
    def rho(c):
        c = np.clip(c, -1.0, 1.0)
        return 0.5 * ((1.0 + c) * rho_l + (1.0 - c) * rho_g)

    def mu(c):
        c = np.clip(c, -1.0, 1.0)
        return 0.5 * ((1.0 + c) * mu_l + (1.0 - c) * mu_g)

    return rho, mu, min(rho_l, rho_g)


def ch_rhs(case: Case2D, geo: "Geometry2D", st: dict) -> np.ndarray:
    """a1: right-hand side Q of the combined CH solve (Appendix A.1, Eq. Helmholtz1 times
    Pe/Cn^2 in the nondimensional form of reading R1):
    Q = (Pe/Cn^2)(C_check/dt - div(u~ C~)) + lap[(psi'(C~) - S C~)/Cn^2]
        + lap[(phi~_wall - phi~)/Cn^2],
    C~ = 2C^n - C^{n-1}, C_check = 2C^n - C^{n-1}/2, u~ = 2u^n - u^{n-1}.
    The last term is reading R16: phi~ = psi'(C~) - Cn^2 lap(C~) is the chemical potential
    of C~ on every cell and phi~_wall the same field with the wall's no-flux condition
    d(phi)/dn = 0 (Eq. AllBCs) imposed by the ghost fill phi_G = phi_M of Sec. 4.2.2; the
    two differ only at the ghost cells.  With it the explicit part of the split is
    lap(phi~_wall)/Cn^2 and only the stabilisation of the increment C^{n+1} - C~ stays
    implicit across the wall."""
    p = case.params
    h = case.h
    ny = case.ny
    eta2 = p.Cn * p.Cn
    C, Co = st["C"], st["C_old"]
    Ct = 2.0 * C - Co
    Cc = 2.0 * C - 0.5 * Co
    ut = 2.0 * st["u"] - st["u_old"]
    vt = 2.0 * st["v"] - st["v_old"]
    Fx = ut * (0.5 * (_xm(Ct) + Ct))
    Fy = np.zeros((ny + 1, case.nx))
    Fy[1:ny] = vt[1:ny] * (0.5 * (Ct[:-1] + Ct[1:]))
    div = (_xp(Fx) - Fx) / h + (Fy[1:] - Fy[:-1]) / h
    g = ((Ct * Ct * Ct - Ct) - p.S * Ct) / eta2
    phi_t = (Ct * Ct * Ct - Ct) - eta2 * laplacian(Ct, h)
    phi_t_wall = chemical_potential(case, geo, Ct)
    return (p.Pe / eta2) * (Cc / p.dt - div) + laplacian(g, h) + laplacian((phi_t_wall - phi_t) / eta2, h)


def chemical_potential(case: Case2D, geo: "Geometry2D", C: np.ndarray) -> np.ndarray:
    """a4 (Eq. Chemical-Potential, reading R1): phi = psi'(C) - Cn^2 lap(C) on every cell, then
    the zero normal gradient at the wall, phi_G = phi_M (Sec. 4.2.2, last lines)."""
    eta = case.params.Cn
    phi = (C * C * C - C) - (eta * eta) * laplacian(C, case.h)
    phi_f = phi.reshape(-1)
    phi_f[geo.gcell] = mirror_value(phi_f.copy(), geo)
    return phi


def ch_flux_div(case: Case2D, C: np.ndarray, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """div(u C_f) with face means of C, no flux through the x2 walls (reading R8)."""
    h, ny = case.h, case.ny
    Fx = u * (0.5 * (_xm(C) + C))
    Fy = np.zeros((ny + 1, case.nx))
    Fy[1:ny] = v[1:ny] * (0.5 * (C[:-1] + C[1:]))
    return (_xp(Fx) - Fx) / h + (Fy[1:] - Fy[:-1]) / h


def ch_explicit(case: Case2D, geo: "Geometry2D", st: dict) -> np.ndarray:
    """a1 + a2, explicit variant (Eq. ExpCH, reading R15): the updated C on every cell,
    before the ghost fill."""
    p = case.params

    def F(C, u, v):
        return -ch_flux_div(case, C, u, v) + laplacian(chemical_potential(case, geo, C), case.h) / p.Pe

    Fn = F(st["C"], st["u"], st["v"])
    Fo = F(st["C_old"], st["u_old"], st["v_old"])
    return st["C"] + p.dt * (1.5 * Fn - 0.5 * Fo)


def _gather(field_flat, ap, w):
    """Omega_IP = sum_a W(a) Omega(AP_a) (Eq. weright averaged), per ghost."""
    acc = np.zeros(ap.shape[0])
    for a in range(ap.shape[1]):
        acc = acc + w[:, a] * field_flat[ap[:, a]]
    return acc


def mirror_value(field_flat, geo: Geometry2D):
    """Eq. extrapolation: Omega_M = 2 Omega_IP1 - Omega_IP2."""
    return 2.0 * _gather(field_flat, geo.ap1, geo.w1) - _gather(field_flat, geo.ap2, geo.w2)


def contact_angle_ghost(case: Case2D, C_M, gamma, dn):
    """a3 core, static angle (mu_f = 0), reading R4.  G, I and M lie on one normal line
    with I between them (dn from G, gamma dn from M), and Eqs. interpolationAtWall /
    UpdateC tie the three values by the linear relation C_G = ((gamma+1) C_I - C_M)/gamma.
    On that line the 3-point one-sided derivative of Eq. ProjectingToNT reduces to the
    slope dC/dn = (C_M - C_I)/(gamma dn) (the same reduction that turns Eq. UpdateVtan
    into its closed form).  The static wetting condition of Eq. WallBCS,
    F(C_I) = kappa Cn dC/dn + cos(theta) g'(C_I) = 0, with g'(C) = 3/4 (1 - C^2) on [-1, 1]
    and g' = 0 outside (g, the wall-energy switch of Eq. FreeEnergySolid, is constant beyond
    the pure phases), is solved as follows: if |C_M| >= 1, C_I = C_M; otherwise F changes sign
    on [-1, 1] and its one root there is a root of the quadratic a C_I^2 - k C_I + c = 0,
    a = -3/4 cos(theta), c = k C_M + 3/4 cos(theta), k = kappa Cn/(gamma dn): of
    r2 = 2c/(k + sqrt D) and r1 = (k + sqrt D)/(2a) (D = k^2 - 4ac) the one in [-1, 1] is
    taken (r2 when both qualify).  Eq. UpdateC then gives C_G.
    Returns (C_G, C_I, number of clamped discriminants)."""
    p = case.params
    ct = math.cos(math.radians(p.theta_deg))
    k = KAPPA * p.Cn / (gamma * dn)
    a = -0.75 * ct
    c = k * C_M + 0.75 * ct
    disc = k * k - 4.0 * a * c
    clamped = int(np.count_nonzero((disc < 0.0) & (np.abs(C_M) < 1.0)))
    sq = np.sqrt(np.maximum(disc, 0.0))
    r2 = 2.0 * c / (k + sq)
    if a != 0.0:
        r1 = (k + sq) / (2.0 * a)
        root = np.where(np.abs(r2) <= 1.0, r2, np.clip(r1, -1.0, 1.0))
    else:
        root = r2
    C_I = np.where(np.abs(C_M) >= 1.0, C_M, root)
    C_G = ((gamma + 1.0) * C_I - C_M) / gamma
    return C_G, C_I, clamped


def g_prime(C):
    """g'(C) = 3/4 (1 - C^2) of the wall-energy switch g(C) = (2 + 3C - C^3)/4 of Eq. WallBCS,
    zero beyond the pure phases (g constant there; reading R4)."""
    C = np.asarray(C, dtype=np.float64)
    return np.where(np.abs(C) < 1.0, 0.75 * (1.0 - C * C), 0.0)


def dynamic_contact_ghost(case: Case2D, C_M, gamma, dn, CI_n, adv):
    """a3 core, dynamic angle (mu_f > 0), reading R18.  Eq. WallBCS_recast integrated over
    one step for the per-ghost wall value C_I, implicitly in C_I:
      (C_I^{n+1} - C_I^n)/dt = -adv + (1/(mu_f Cn)) [kappa Cn dC/dn + cos(theta) g'(C_I^{n+1})],
    adv = v_t (dC/dx_t) at I (level-n velocity, gradient of C^{n+1} before the fill), the
    normal derivative the slope (C_M - C_I^{n+1})/(gamma dn) of reading R4.  With
    a = dt/(mu_f Cn), k = kappa Cn/(gamma dn) and R = C_I^n - dt adv + a k C_M this is
      F(C) = (1 + a k) C - a cos(theta) g'(C) - R = 0,
    linear where g' = 0 (|C| >= 1) and the quadratic (3/4) a cos C^2 + (1 + a k) C - (R + (3/4) a
    cos) = 0 on [-1, 1].  As in the static case (reading R4): if the linear solution
    R/(1 + a k) lies outside (-1, 1) it is taken; otherwise F(-1) < 0 < F(1) and the one root
    of the quadratic in [-1, 1] is taken (r2 = 2c/(b + sqrt(D)) when it qualifies, else
    r1 = -(b + sqrt(D))/(2a')).  As mu_f -> 0 this is R4's static quadratic (C_M for R/(1+ak));
    as mu_f -> infinity C_I^{n+1} = C_I^n - dt adv.  Then C_G by Eq. UpdateC and the wetting
    bracket B = kappa Cn dC/dn + cos(theta) g'(C_I) at the new level.
    Returns (C_G, C_I, B)."""
    p = case.params
    ct = math.cos(math.radians(p.theta_deg))
    k = KAPPA * p.Cn / (gamma * dn)
    a = p.dt / (p.mu_f * p.Cn)
    R = CI_n - p.dt * adv + a * k * C_M
    qb = 1.0 + a * k
    lin = R / qb
    qa = 0.75 * a * ct
    qc = R + 0.75 * a * ct
    sq = np.sqrt(np.maximum(qb * qb + 4.0 * qa * qc, 0.0))
    r2 = 2.0 * qc / (qb + sq)
    if qa != 0.0:
        r1 = -(qb + sq) / (2.0 * qa)
        root = np.where(np.abs(r2) <= 1.0, r2, np.clip(r1, -1.0, 1.0))
    else:
        root = r2
    C_I = np.where(np.abs(lin) >= 1.0, lin, root)
    C_G = ((gamma + 1.0) * C_I - C_M) / gamma
    B = k * (C_M - C_I) + ct * g_prime(C_I)
    return C_G, C_I, B


def cell_gradient(case: Case2D, C):
    """Central differences of a cell field at the cell centres (periodic x1; zero-gradient
    mirror rows at the x2 walls, reading R8)."""
    h = case.h
    return (_xp(C) - _xm(C)) / (2.0 * h), (_yp_mirror(C) - _ym_mirror(C)) / (2.0 * h)


def wall_advection(case: Case2D, geo: "Geometry2D", u, v, C_pre):
    """v_t (dC/dx_t) at the intersect points and (dC/dx_t)_I (Eq. ProjectingToNT, t = (n2, -n1)):
    the level-n cell-centred velocity and the central-difference gradient of C^{n+1} (before
    the fill), each at I as the gamma-weighted mean of the ghost's value and the mirror value
    (Eq. interpolationAtWall)."""
    g, gam = geo.gcell, geo.gamma
    at_I = lambda fld: (gam * fld.reshape(-1)[g] + mirror_value(fld.reshape(-1), geo)) / (gam + 1.0)
    uI = at_I(0.5 * (u + _xp(u)))
    vI = at_I(0.5 * (v[:-1] + v[1:]))
    gx, gy = cell_gradient(case, C_pre)
    gxI, gyI = at_I(gx), at_I(gy)
    n1, n2 = geo.n[:, 0], geo.n[:, 1]
    gt = gxI * n2 - gyI * n1
    return (uI * n2 - vI * n1) * gt, gt


def slip_ghost(case: Case2D, uM, vM, n, gamma, dn, B=None, gt=None, mu_I=None):
    """a6 core: Eq. NoPenetration for the normal component, Eq. UpdateVtan for the tangential
    one, Eq. UpdateVandW back to x1/x2 (reading R5).  With a dynamic angle the wetting bracket
    B and the tangential derivative gt = (dC/dx_t)_I enter through the term
    -(1/Ca) B gt l_s (gamma + 1) dn / (mu_I (l_s + gamma dn)) (reading R18); static: B = 0."""
    p = case.params
    n1, n2 = n[:, 0], n[:, 1]
    VnM = uM * n1 + vM * n2
    VtM = uM * n2 - vM * n1
    VnG = -VnM / gamma
    VtG = VtM * (p.l_s - dn) / (p.l_s + gamma * dn)
    if B is not None:
        VtG = VtG - (B * gt / p.Ca) * (p.l_s * (gamma + 1.0) * dn) / (mu_I * (p.l_s + gamma * dn))
    return VnG * n1 + VtG * n2, VnG * n2 - VtG * n1


def face_fix(case: Case2D, geo: "Geometry2D", uss, vss, ucen, vcen, uG, vG):
    """a6, last step (reading R10): the velocity on the faces of the face lists (alpha_f < 1,
    touching a ghost cell) becomes the mean of its two cells' centred values, where a ghost
    cell holds its filled value (uG, vG), a solid non-ghost cell 0 and a fluid cell its
    centred u** (ucen, vcen) from before the fill (the last sentence of Sec. 4.3).  x1-face
    (j, i) lies between cells (j, i-1) and (j, i); x2-face (j, i) between (j-1, i) and (j, i)."""
    nx = case.nx
    ucell = ucen.copy().reshape(-1)
    vcell = vcen.copy().reshape(-1)
    solid_flat = (geo.cls == CELL_SOLID).reshape(-1)
    ucell[solid_flat] = 0.0
    vcell[solid_flat] = 0.0
    ucell[geo.gcell] = uG
    vcell[geo.gcell] = vG
    uss_f = uss.copy()
    vss_f = vss.copy()
    fu_j, fu_i = np.divmod(geo.fu, nx)
    uss_f[fu_j, fu_i] = 0.5 * (ucell[fu_j * nx + (fu_i - 1) % nx] + ucell[fu_j * nx + fu_i])
    fv_j, fv_i = np.divmod(geo.fv, nx)
    vss_f[fv_j, fv_i] = 0.5 * (vcell[(fv_j - 1) * nx + fv_i] + vcell[fv_j * nx + fv_i])
    return uss_f, vss_f


def momentum_rhs(case: Case2D, C1: np.ndarray, u: np.ndarray, v: np.ndarray):
    """H = -div(u u) + div(mu (grad u + grad u^T)) / (Re rho) on the x1-faces (ny, nx) and the
    x2-faces (ny+1, nx; wall rows zero), with rho and mu from C1 (Eq. PredictionExp, the
    convective and viscous brackets; reading R8 for the discrete operators)."""
    Nu, Nv, Vu, Vv = momentum_terms(case, C1, u, v)
    return Nu + Vu, Nv + Vv


def momentum_terms(case: Case2D, C1: np.ndarray, u: np.ndarray, v: np.ndarray):
    """The two brackets of momentum_rhs separately: N = -div(u u) and
    V = div(mu (grad u + grad u^T)) / (Re rho) (x2-face wall rows zero)."""
    p = case.params
    nx, ny, h = case.nx, case.ny, case.h
    rho, mu, _ = _props(case)
    Cpad = np.vstack([C1[:1], C1, C1[-1:]])          # mirror rows j=-1, j=ny
    upad = np.vstack([-u[:1], u, -u[-1:]])           # no-slip ghost rows
    Cf_u = 0.5 * (_xm(C1) + C1)
    Cf_v = 0.5 * (C1[:-1] + C1[1:])                  # x2-faces j = 1..ny-1
    Ce = 0.25 * (((_xm(Cpad[:-1]) + Cpad[:-1]) + _xm(Cpad[1:])) + Cpad[1:])  # corners j=0..ny
    mu_c = mu(C1)
    mu_e = mu(Ce)
    tau_xx = 2.0 * mu_c * ((_xp(u) - u) / h)
    tau_yy = 2.0 * mu_c * ((v[1:] - v[:-1]) / h)
    dudy = (upad[1:] - upad[:-1]) / h                 # corners j = 0..ny
    dvdx = (v - _xm(v)) / h
    tau_xy = mu_e * (dudy + dvdx)
    visc_u = (tau_xx - _xm(tau_xx)) / h + (tau_xy[1:] - tau_xy[:-1]) / h
    visc_v = (_xp(tau_xy) - tau_xy)[1:ny] / h + (tau_yy[1:] - tau_yy[:-1]) / h
    uc = 0.5 * (u + _xp(u))
    vc = 0.5 * (v[:-1] + v[1:])
    uv = (0.5 * (upad[1:] + upad[:-1])) * (0.5 * (v + _xm(v)))
    conv_u = (uc * uc - _xm(uc * uc)) / h + (uv[1:] - uv[:-1]) / h
    conv_v = (_xp(uv) - uv)[1:ny] / h + (vc[1:] * vc[1:] - vc[:-1] * vc[:-1]) / h
    Nv = np.zeros((ny + 1, nx))
    Vv = np.zeros((ny + 1, nx))
    Nv[1:ny] = -conv_v
    Vv[1:ny] = visc_v / (p.Re * rho(Cf_v))
    return -conv_u, Nv, visc_u / (p.Re * rho(Cf_u)), Vv


def mass_flux_term(case: Case2D, C1, phi, u, v):
    """(rho'/(rho_f Pe)) (grad phi . grad) u on the x1- and x2-faces (the last term of Eq.
    predictionSemi, reading R19): rho' = (rho_l - rho_g)/2, the chemical potential's gradient
    by the face difference across the face and the mean of the two cells' central differences
    along it, the velocity's by central differences of its own faces (no-slip ghost rows -u
    at the x2 walls; v on the interior x2-faces, zero on the walls)."""
    p = case.params
    h, ny, nx = case.h, case.ny, case.nx
    rho, _, _ = _props(case)
    rp = 0.5 * (1.0 - 1.0 / p.rho_ratio)
    upad = np.vstack([-u[:1], u, -u[-1:]])
    phy_c = (_yp_mirror(phi) - _ym_mirror(phi)) / (2.0 * h)
    phx_c = (_xp(phi) - _xm(phi)) / (2.0 * h)
    mfu = (rp / (rho(0.5 * (_xm(C1) + C1)) * p.Pe)) * (
        ((phi - _xm(phi)) / h) * ((_xp(u) - _xm(u)) / (2.0 * h))
        + (0.5 * (phy_c + _xm(phy_c))) * ((upad[2:] - upad[:-2]) / (2.0 * h)))
    mfv = np.zeros((ny + 1, nx))
    vi = v[1:ny]
    mfv[1:ny] = (rp / (rho(0.5 * (C1[:-1] + C1[1:])) * p.Pe)) * (
        (0.5 * (phx_c[1:] + phx_c[:-1])) * ((_xp(vi) - _xm(vi)) / (2.0 * h))
        + ((phi[1:] - phi[:-1]) / h) * ((v[2:] - v[:-2]) / (2.0 * h)))
    return mfu, mfv


def velocity_eigenvalues(case: Case2D):
    """Eigenvalues of the 5-point Laplacian of the two velocity components with their x2
    boundary rows (periodic x1): x1-faces (no-slip ghost rows -u) in the real-Fourier x DST-II
    basis, modes m = 1..ny; x2-faces (interior faces, v = 0 on the walls) in the real-Fourier x
    DST-I basis, modes m = 1..ny-1; both -(4/h^2)(sin^2(pi k/nx) + sin^2(pi m/(2 ny)))."""
    nx, ny, h = case.nx, case.ny, case.h
    lx = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(nx // 2 + 1) / nx) ** 2
    lu = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(1, ny + 1) / (2.0 * ny)) ** 2
    lv = -(4.0 / (h * h)) * np.sin(np.pi * np.arange(1, ny) / (2.0 * ny)) ** 2
    return lu[:, None] + lx[None, :], lv[:, None] + lx[None, :]


def velocity_helmholtz(case: Case2D, ru, rv, a):
    """(1 - a L) d = r for both velocity components (Appendix A.2, Eq. predictionSemi, the
    implicit half of nu0 lap u), by the transforms of velocity_eigenvalues."""
    nx, ny = case.nx, case.ny
    lu, lv = velocity_eigenvalues(case)

    def solve(r, typ, lam):
        s = sfft.rfft(r, axis=1)
        t = sfft.dst(s.real, type=typ, axis=0) + 1j * sfft.dst(s.imag, type=typ, axis=0)
        t = t / (1.0 - a * lam)
        t = sfft.idst(t.real, type=typ, axis=0) + 1j * sfft.idst(t.imag, type=typ, axis=0)
        return sfft.irfft(t, n=nx, axis=1)

    du = solve(ru, 2, lu)
    dv = np.zeros((ny + 1, nx))
    dv[1:ny] = solve(rv[1:ny], 1, lv)
    return du, dv


def step(case: Case2D, geo: Geometry2D, st: dict) -> tuple[dict, dict]:
    """One full time step a1..a8.  Returns (new state, intermediates)."""
    p = case.params
    nx, ny, h = case.nx, case.ny, case.h
    eta = p.Cn
    rho, mu, rho0 = _props(case)
    info = {}

    # a1 + a2: semi-implicit CH (Appendix A.1), or the explicit variant (Eq. ExpCH)
    if getattr(p, "ch_scheme", 0) == 1:
        C_pre = ch_explicit(case, geo, st)
    else:
        Q = ch_rhs(case, geo, st)
        C_pre = ch_solve(case, Q)
        info["Q"] = Q
    info["C_pre"] = C_pre
    info["mass_pre"] = float(C_pre.sum())

    # a3: contact-angle ghost fill of C (Sec. 4.2.2)
    C1 = C_pre.copy()
    f = C1.reshape(-1)
    C_M = mirror_value(C_pre.reshape(-1), geo)
    B = gt = None
    if p.mu_f > 0.0:
        # dynamic angle (reading R18): the wall value C_I is state; unset (NaN) it starts as
        # the wall value of the level-n field, (gamma C^n_G + C^n_M)/(gamma + 1) (Eq.
        # interpolationAtWall at level n)
        g = geo.gcell
        gam = geo.gamma
        Cn_flat = st["C"].reshape(-1)
        CI_n = st.get("C_I")
        CI_n = np.full(len(g), np.nan) if CI_n is None else CI_n
        CI_n = np.where(np.isfinite(CI_n), CI_n,
                        (gam * Cn_flat[g] + mirror_value(Cn_flat, geo)) / (gam + 1.0))
        adv, gt = wall_advection(case, geo, st["u"], st["v"], C_pre)
        C_G, C_I, B = dynamic_contact_ghost(case, C_M, gam, geo.dn, CI_n, adv)
        clamped = 0
    else:
        C_G, C_I, clamped = contact_angle_ghost(case, C_M, geo.gamma, geo.dn)
    f[geo.gcell] = C_G
    info["C"] = C1
    info["C_I"] = C_I
    info["B"] = B
    info["disc_clamped"] = clamped
    info["mass"] = float(C1.sum())

    # a4: chemical potential, zero normal gradient at the wall (Sec. 4.2.2, last lines)
    phi = chemical_potential(case, geo, C1)
    info["phi"] = phi

    # a5: AB2 predictor + penalisation (Eq. PredictionExp, Eq. Penalization2), or the
    # semi-implicit predictor of Appendix A.2 (Eq. predictionSemi, reading R19)
    u, v = st["u"], st["v"]
    Cf_u = 0.5 * (_xm(C1) + C1)
    Cf_v = 0.5 * (C1[:-1] + C1[1:])                  # x2-faces j = 1..ny-1
    rho_u = rho(Cf_u)
    rho_v = rho(Cf_v)
    k_st = KAPPA / (p.Re * p.Ca * eta)
    st_u = k_st * (0.5 * (phi + _xm(phi))) * ((C1 - _xm(C1)) / h) / rho_u
    st_v = k_st * (0.5 * (phi[1:] + phi[:-1])) * ((C1[1:] - C1[:-1]) / h) / rho_v
    v_star = np.zeros((ny + 1, nx))
    if getattr(p, "ns_scheme", 0) == 1:
        Hu, Hv, Vu, Vv = momentum_terms(case, C1, u, v)     # history: the convective bracket
        mfu, mfv = mass_flux_term(case, C1, phi, u, v)
        Fu = (((1.5 * Hu - 0.5 * st["Hu"]) + st_u) + Vu) + mfu
        Fv = np.zeros((ny + 1, nx))
        Fv[1:ny] = (((1.5 * Hv[1:ny] - 0.5 * st["Hv"][1:ny]) + st_v) + Vv[1:ny]) + mfv[1:ny]
        nu0 = 0.5 * (1.0 + (1.0 / p.mu_ratio) / (1.0 / p.rho_ratio)) / p.Re
        du, dv = velocity_helmholtz(case, p.dt * Fu, p.dt * Fv, 0.5 * p.dt * nu0)
        u_star = u + du
        v_star[1:ny] = v[1:ny] + dv[1:ny]
    else:
        Hu, Hv = momentum_rhs(case, C1, u, v)
        u_star = u + p.dt * ((1.5 * Hu - 0.5 * st["Hu"]) + st_u)
        v_star[1:ny] = v[1:ny] + p.dt * ((1.5 * Hv[1:ny] - 0.5 * st["Hv"][1:ny]) + st_v)
    uss = geo.alpha_u * u_star
    vss = geo.alpha_v * v_star
    info["Hu"], info["Hv"] = Hu, Hv
    info["u_star"], info["v_star"] = u_star, v_star

    # a6: velocity ghost fill (Sec. 4.3) and face re-interpolation (reading R10)
    ucen = 0.5 * (uss + _xp(uss))
    vcen = 0.5 * (vss[:-1] + vss[1:])
    uM = mirror_value(ucen.reshape(-1), geo)
    vM = mirror_value(vcen.reshape(-1), geo)
    mu_I = mu(C_I) if B is not None else None
    uG, vG = slip_ghost(case, uM, vM, geo.n, geo.gamma, geo.dn, B, gt, mu_I)
    uss_f, vss_f = face_fix(case, geo, uss, vss, ucen, vcen, uG, vG)
    info["uG"], info["vG"] = uG, vG
    info["u_ss"], info["v_ss"] = uss_f, vss_f

    # a7: pressure Poisson (Eq. PressurePoisson)
    Ph = 2.0 * st["P"] - st["P_old"]
    gx = (1.0 - rho0 / rho_u) * ((Ph - _xm(Ph)) / h)
    gy = np.zeros((ny + 1, nx))
    gy[1:ny] = (1.0 - rho0 / rho_v) * ((Ph[1:] - Ph[:-1]) / h)
    div_g = (_xp(gx) - gx) / h + (gy[1:] - gy[:-1]) / h
    div_u = (_xp(uss_f) - uss_f) / h + (vss_f[1:] - vss_f[:-1]) / h
    rhs = div_g + (rho0 / p.dt) * div_u
    P1 = poisson_solve(case, rhs)
    info["rhs_p"] = rhs
    info["P"] = P1

    # a8: correction (Eq. correction)
    u1 = uss_f - p.dt * ((1.0 / rho0) * ((P1 - _xm(P1)) / h)
                         + (1.0 / rho_u - 1.0 / rho0) * ((Ph - _xm(Ph)) / h))
    v1 = np.zeros((ny + 1, nx))
    v1[1:ny] = vss_f[1:ny] - p.dt * ((1.0 / rho0) * ((P1[1:] - P1[:-1]) / h)
                                     + (1.0 / rho_v - 1.0 / rho0) * ((Ph[1:] - Ph[:-1]) / h))
    info["u"], info["v"] = u1, v1

    new = {"C": C1, "C_old": st["C"].copy(), "u": u1, "u_old": st["u"].copy(),
           "v": v1, "v_old": st["v"].copy(), "Hu": Hu, "Hv": Hv,
           "P": P1, "P_old": st["P"].copy()}
    if p.mu_f > 0.0:
        new["C_I"] = C_I.copy()
    return new, info


# --------------------------------------------------------------------- diagnostics
def divergence(u: np.ndarray, v: np.ndarray, h: float) -> np.ndarray:
    return (_xp(u) - u) / h + (v[1:] - v[:-1]) / h


def run(case: Case2D, st: dict, nsteps: int, geo: Geometry2D | None = None):
    geo = geo if geo is not None else build_geometry(case)
    for _ in range(nsteps):
        st, _ = step(case, geo, st)
    return st, geo
