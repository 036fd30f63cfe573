"""Seeded synthetic workloads for the hybrid immersed-boundary / phase-field step.

This module is the one piece shared by the CPU oracle (``oracle/``), the tests and
``bench.py``.  It holds *inputs only*: grid sizes, wall descriptors, physical
parameters and initial fields.  It contains none of the method's arithmetic
(no stencils, no solves, no ghost-cell formulas); the oracle and the CUDA library
each implement those independently.

Paper workloads used as the model for these inputs
  * 5.1 / 5.4 / 5.5: a 2D droplet on a flat or sinusoidal immersed wall, static
    contact angle, periodic in x1, walls in x2.
  * The initial interface is the tanh profile of Eq. InitializingC written in
    terms of the distance to the droplet centre:
    C = tanh((R - |x - x_c|) / (sqrt(2) Cn)); C = +1 is the liquid (droplet).
  * u = 0 and P = 0 at t = 0.

Wall descriptors (the solid is the set where the predicate is true)
  GEOM_FLAT      x2 < p0
  GEOM_SINUSOID  x2 < p0 + p1 * sin(2 pi p2 x1)
  GEOM_NONE      no solid anywhere (free droplet; used by closed-form tests)
  GEOM_MASK      the solid given by caller-supplied volume fractions (Case.alpha), 2D and 3D
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

GEOM_FLAT = 0
GEOM_SINUSOID = 1
GEOM_NONE = 3
GEOM_MASK = 6   # alpha = (alpha_c, alpha_u, alpha_v[, alpha_w]) arrays supplied with the case

# field ids shared by the C-ABI, the binding and the tests (inputs/outputs only)
FIELDS_2D = ("C", "C_old", "u", "u_old", "v", "v_old", "Hu", "Hv", "P", "P_old")


@dataclass(frozen=True)
class Params:
    """Nondimensional parameters (Sec. 5.1 definitions) plus the ghost-cell lengths.

    rho_ratio / mu_ratio are liquid/gas; the liquid has rho = mu = 1.
    d1 is the intersect-to-mirror distance, d2 the mirror-to-IP1 spacing (Sec. 4.1.2).
    """

    Re: float = 10.0
    Ca: float = 0.1
    Cn: float = 0.02
    Pe: float = 5.0e3
    S: float = 2.0
    rho_ratio: float = 10.0
    mu_ratio: float = 10.0
    theta_deg: float = 60.0
    l_s: float = 0.0
    mu_f: float = 0.0
    d1: float = 0.0
    d2: float = 0.0
    dt: float = 1.0e-4
    ch_scheme: int = 0   # 0: semi-implicit CH (Appendix A.1); 1: explicit AB2 (Eq. ExpCH)
    weights: int = 0     # averaging weights: 0 linear-exact (default), 1 plain inverse-distance
    ns_scheme: int = 0   # momentum predictor: 0 explicit AB2 (Eq. PredictionExp); 1 semi-implicit
                         # (Eq. predictionSemi, Appendix A.2)


@dataclass(frozen=True)
class Case2D:
    name: str
    nx: int
    ny: int
    lx: float
    ly: float
    geom_kind: int
    geom_p: tuple
    drop_c: tuple
    drop_r: float
    params: Params
    steps: int
    alpha: tuple = ()            # GEOM_MASK: (alpha_c, alpha_u, alpha_v) arrays

    @property
    def h(self) -> float:
        return self.lx / self.nx

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def _ghost_lengths(h: float, dim: int = 2) -> tuple[float, float]:
    # d1 larger than half a cell diagonal; d2 smaller than d1 (Sec. 4.1.2).
    d1 = math.sqrt(dim) * h
    return d1, 0.5 * d1


def flat_wall_case(nx: int = 128, ny: int = 64, theta_deg: float = 60.0, l_s: float = 0.0,
                   steps: int = 200, dt: float = 1.0e-4, Cn: float = 0.02, Pe: float = 5.0e3,
                   wall_y: float = 0.1, drop_r: float = 0.3, rho_ratio: float = 10.0,
                   mu_ratio: float = 10.0, name: str | None = None) -> Case2D:
    """Flat immersed wall x2 < wall_y on [0,2]x[0,1]; droplet centred on the wall."""
    h = 2.0 / nx
    d1, d2 = _ghost_lengths(h)
    p = Params(Re=10.0, Ca=0.1, Cn=Cn, Pe=Pe, S=2.0, rho_ratio=rho_ratio, mu_ratio=mu_ratio,
               theta_deg=theta_deg, l_s=l_s, d1=d1, d2=d2, dt=dt)
    return Case2D(name or f"flat_{nx}x{ny}", nx, ny, 2.0, 1.0, GEOM_FLAT, (wall_y, 0.0, 0.0, 0.0),
                  (1.0, wall_y), drop_r, p, steps)


def flat_wall_128x64() -> Case2D:
    """128x64 on [0,2]x[0,1], flat wall y=0.1, R=0.3 at (1,0.1), theta=60, Cn=0.02,
    Pe=5e3, Re=10, Ca=0.1, l_s=0, S=2, dt=1e-4, 200 steps (the small parity case)."""
    return flat_wall_case(name="flat_wall_128x64")


def sinusoid_wall_512x256(theta_deg: float = 45.0, l_s: float = 0.01, nx: int = 512,
                          ny: int = 256, steps: int = 5000) -> Case2D:
    """Sinusoidal wall y = 0.2 + 0.05 sin(4 pi x) on [0,2]x[0,1], 512x256, R=0.3 at (1,0.2),
    Cn=0.01, Re=10, Ca=0.1, Pe=1e4, dt from the viscous rule of Eq. timestep
    (0.25 Re h^2 / 6), 5000 steps.  theta in {45,90,135}, l_s in {0,0.01}."""
    h = 2.0 / nx
    d1, d2 = _ghost_lengths(h)
    dt = 0.25 * 10.0 * h * h / 6.0
    p = Params(Re=10.0, Ca=0.1, Cn=0.01 * (512 / nx), Pe=1.0e4, S=2.0, theta_deg=theta_deg,
               l_s=l_s, d1=d1, d2=d2, dt=dt)
    return Case2D(f"sinusoid_{nx}x{ny}_th{theta_deg:g}_ls{l_s:g}", nx, ny, 2.0, 1.0,
                  GEOM_SINUSOID, (0.2, 0.05, 2.0, 0.0), (1.0, 0.2), 0.3, p, steps)


def free_droplet_case(nx: int = 128, ny: int = 64, R: float = 0.3, Cn: float = 0.02,
                      rho_ratio: float = 1.0, mu_ratio: float = 1.0, dt: float = 1.0e-4) -> Case2D:
    """No solid at all; droplet in the middle of [0,2]x[0,1] (closed-form tests)."""
    h = 2.0 / nx
    d1, d2 = _ghost_lengths(h)
    p = Params(Cn=Cn, rho_ratio=rho_ratio, mu_ratio=mu_ratio, theta_deg=90.0, d1=d1, d2=d2, dt=dt)
    return Case2D(f"free_{nx}x{ny}", nx, ny, 2.0, 1.0, GEOM_NONE, (0.0, 0.0, 0.0, 0.0),
                  (1.0, 0.5), R, p, 1)


def ensemble_2d(n_instances: int = 64, seed: int = 2104) -> list[Case2D]:
    """Uneven 2D ensemble: grids drawn from {256x128, 512x256, 1024x512}; wall
    y = 0.2 + A sin(2 pi k x), A ~ U(0,0.08), k in {1..4}; theta ~ U(30,150) deg;
    l_s in {0, 0.005, 0.02}; R ~ U(0.2, 0.35).  Cn = 2.56 h, Re=10, Ca=0.1, Pe=5e3,
    dt = 0.25 Re h^2 / 6 per instance.  Seeded with numpy PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = [(256, 128), (512, 256), (1024, 512)]
    out = []
    for k in range(n_instances):
        nx, ny = sizes[int(rng.integers(0, 3))]
        A = float(rng.uniform(0.0, 0.08))
        kk = int(rng.integers(1, 5))
        theta = float(rng.uniform(30.0, 150.0))
        l_s = float((0.0, 0.005, 0.02)[int(rng.integers(0, 3))])
        R = float(rng.uniform(0.2, 0.35))
        h = 2.0 / nx
        d1, d2 = _ghost_lengths(h)
        p = Params(Re=10.0, Ca=0.1, Cn=2.56 * h, Pe=5.0e3, S=2.0, theta_deg=theta, l_s=l_s,
                   d1=d1, d2=d2, dt=0.25 * 10.0 * h * h / 6.0)
        out.append(Case2D(f"ens{k:02d}_{nx}x{ny}", nx, ny, 2.0, 1.0, GEOM_SINUSOID,
                          (0.2, A, float(kk), 0.0), (1.0, 0.2), R, p, 200))
    return out


def with_params(case: Case2D, **kw) -> Case2D:
    return replace(case, params=replace(case.params, **kw))


def initial_state(case: Case2D) -> dict:
    """Initial fields (FP64, row-major, x1 fastest).

    C: (ny, nx) cell centres; u: (ny, nx) x1-faces (face i is the left face of cell i);
    v: (ny+1, nx) x2-faces (rows 0 and ny are the domain walls); H*: like u/v; P: (ny, nx).
    The old time level equals the initial one (start-up reading of the scheme).
    """
    h = case.h
    xc = (np.arange(case.nx) + 0.5) * h
    yc = (np.arange(case.ny) + 0.5) * h
    X, Y = np.meshgrid(xc, yc)
    r = np.sqrt((X - case.drop_c[0]) ** 2 + (Y - case.drop_c[1]) ** 2)
    C = np.tanh((case.drop_r - r) / (math.sqrt(2.0) * case.params.Cn))
    z_c = np.zeros((case.ny, case.nx))
    z_v = np.zeros((case.ny + 1, case.nx))
    return {
        "C": C.copy(), "C_old": C.copy(),
        "u": z_c.copy(), "u_old": z_c.copy(),
        "v": z_v.copy(), "v_old": z_v.copy(),
        "Hu": z_c.copy(), "Hv": z_v.copy(),
        "P": z_c.copy(), "P_old": z_c.copy(),
    }


def random_state(case: Case2D, seed: int = 7, amp_u: float = 0.05) -> dict:
    """A perturbed state for single-step parity: the initial droplet with smooth
    random perturbations of every field, so every term of the step is exercised."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = initial_state(case)
    ny, nx = case.ny, case.nx

    def smooth(shape, amp):
        a = rng.standard_normal(shape)
        for _ in range(3):
            a = 0.25 * (np.roll(a, 1, 1) + np.roll(a, -1, 1)) + 0.5 * a
            a[1:-1] = 0.25 * (a[:-2] + a[2:]) + 0.5 * a[1:-1]
        return amp * a / max(1e-30, np.abs(a).max())

    s["C_old"] = s["C"] + smooth((ny, nx), 0.02)
    s["C"] = s["C"] + smooth((ny, nx), 0.02)
    for key in ("u", "u_old", "Hu"):
        s[key] = smooth((ny, nx), amp_u if key != "Hu" else 1.0)
    for key in ("v", "v_old", "Hv"):
        a = smooth((ny + 1, nx), amp_u if key != "Hv" else 1.0)
        a[0] = 0.0
        a[ny] = 0.0
        s[key] = a
    s["P"] = smooth((ny, nx), 1.0)
    s["P_old"] = s["P"] + smooth((ny, nx), 0.1)
    # the pressure is defined up to a constant; keep the gauge of the solver (zero mean)
    s["P"] -= s["P"].mean()
    s["P_old"] -= s["P_old"].mean()
    return s


# ============================================================================ 3D
# Layout: cell fields (nz, ny, nx), x fastest; u on x-faces (nz, ny, nx; face i is the left
# face of cell i), v on y-faces (nz, ny, nx), w on z-faces (nz+1, ny, nx; rows 0 and nz are
# the domain walls).  Periodic in x and y, walls in z.
#
# 3D solid descriptors
#   GEOM_FLAT     z < p0
#   GEOM_SPHERE   |x - (p0, p1, p2)| < p3
#   GEOM_SPHERES  union of the spheres (cx, cy, cz, r) of Case3D.spheres
#   GEOM_NONE     no solid
GEOM_SPHERE = 4
GEOM_SPHERES = 5


@dataclass(frozen=True)
class Case3D:
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    geom_kind: int
    geom_p: tuple
    drop_c: tuple
    drop_r: float
    params: Params
    steps: int
    spheres: tuple = ()          # ((cx, cy, cz, r), ...) for GEOM_SPHERES
    alpha: tuple = ()            # GEOM_MASK: (alpha_c, alpha_u, alpha_v, alpha_w) arrays

    @property
    def h(self) -> float:
        return self.lx / self.nx

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


def _dt_rule(h: float, Re: float) -> float:
    # viscous rule of Eq. timestep, 0.25 Re h^2 / 6
    return 0.25 * Re * h * h / 6.0


def sphere_case(n: int = 256, steps: int = 1000, name: str | None = None) -> Case3D:
    """Droplet on a solid sphere: n^3 cells on the unit cube, sphere R_s = 0.25 at the centre,
    droplet R = 0.2 centred on the sphere's top point (0.5, 0.5, 0.75), theta = 120 deg,
    Cn = 0.01 (scaled with h below 256), Re = 20, Ca = 0.05, l_s = 0.005, Pe = 1e4."""
    h = 1.0 / n
    d1, d2 = _ghost_lengths(h, 3)
    p = Params(Re=20.0, Ca=0.05, Cn=0.01 * 256 / n, Pe=1.0e4, S=2.0, theta_deg=120.0,
               l_s=0.005, d1=d1, d2=d2, dt=_dt_rule(h, 20.0))
    return Case3D(name or f"sphere_{n}", n, n, n, 1.0, 1.0, 1.0, GEOM_SPHERE,
                  (0.5, 0.5, 0.5, 0.25), (0.5, 0.5, 0.75), 0.2, p, steps)


def sphere_packing(seed: int = 350, r_lo: float = 0.03, r_hi: float = 0.06, z_top: float = 0.35,
                   solid_fraction: float = 0.4, max_fail: int = 1_000_000) -> tuple:
    """Random sequential addition of non-overlapping spheres, radii ~ U(r_lo, r_hi), centres
    uniform in [0,1)^2 x [0, z_top), periodic in x and y (overlap tested against the nearest
    periodic image), until the spheres' volume reaches solid_fraction of the slab
    [0,1]^2 x [0, z_top] or max_fail placements in a row fail.  Seeded PCG64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    target = solid_fraction * z_top
    out = []
    vol = 0.0
    fails = 0
    while vol < target and fails < max_fail:
        r = float(rng.uniform(r_lo, r_hi))
        c = (float(rng.uniform(0.0, 1.0)), float(rng.uniform(0.0, 1.0)),
             float(rng.uniform(0.0, z_top)))
        ok = True
        for (x, y, z, rr) in out:
            dx = abs(c[0] - x)
            dx = min(dx, 1.0 - dx)
            dy = abs(c[1] - y)
            dy = min(dy, 1.0 - dy)
            dz = c[2] - z
            if dx * dx + dy * dy + dz * dz < (r + rr) * (r + rr):
                ok = False
                break
        if ok:
            out.append((c[0], c[1], c[2], r))
            vol += 4.0 / 3.0 * math.pi * r ** 3
            fails = 0
        else:
            fails += 1
    return tuple(out)


def porous_case(n: int = 512, steps: int = 500, seed: int = 350, name: str | None = None,
                max_fail: int = 1_000_000) -> Case3D:
    """Droplet R = 0.15 at (0.5, 0.5, 0.5) above a random packing of spheres (sphere_packing)
    in z < 0.35, n^3 cells on the unit cube, theta = 60 deg, Cn = 0.005 (scaled with h below
    512), Re = 10, Ca = 0.1, l_s = 0.002, Pe = 1e4."""
    h = 1.0 / n
    d1, d2 = _ghost_lengths(h, 3)
    p = Params(Re=10.0, Ca=0.1, Cn=0.005 * 512 / n, Pe=1.0e4, S=2.0, theta_deg=60.0,
               l_s=0.002, d1=d1, d2=d2, dt=_dt_rule(h, 10.0))
    sph = sphere_packing(seed, max_fail=max_fail)
    return Case3D(name or f"porous_{n}", n, n, n, 1.0, 1.0, 1.0, GEOM_SPHERES, (0.0,) * 4,
                  (0.5, 0.5, 0.5), 0.15, p, steps, sph)


def flat_wall_case3d(nx: int = 32, ny: int = 16, nz: int = 16, wall_z: float = 0.2,
                     theta_deg: float = 60.0, l_s: float = 0.0, Cn: float | None = None,
                     drop_r: float = 0.35, rho_ratio: float = 10.0, mu_ratio: float = 10.0,
                     geom_kind: int | None = None, name: str | None = None) -> Case3D:
    """Flat immersed wall z < wall_z in [0, nx h] x [0, ny h] x [0, nz h] with h = 2/nx; a
    droplet centred on the wall at the box centre (small parity cases)."""
    h = 2.0 / nx
    d1, d2 = _ghost_lengths(h, 3)
    p = Params(Re=10.0, Ca=0.1, Cn=Cn if Cn is not None else 2.56 * h, Pe=5.0e3, S=2.0,
               rho_ratio=rho_ratio, mu_ratio=mu_ratio, theta_deg=theta_deg, l_s=l_s, d1=d1,
               d2=d2, dt=_dt_rule(h, 10.0))
    kind = GEOM_FLAT if geom_kind is None else geom_kind
    return Case3D(name or f"flat3d_{nx}x{ny}x{nz}", nx, ny, nz, 2.0, ny * h, nz * h, kind,
                  (wall_z, 0.0, 0.0, 0.0), (1.0, 0.5 * ny * h, wall_z), drop_r, p, 1)


def small_sphere_case(n: int = 32, theta_deg: float = 120.0, l_s: float = 0.005) -> Case3D:
    """The sphere workload on an n^3 grid (Cn = 2.56 h) for parity tests."""
    c = sphere_case(n, steps=1)
    return replace(c, params=replace(c.params, theta_deg=theta_deg, l_s=l_s))


def initial_state3d(case: Case3D) -> dict:
    """Initial fields (FP64): tanh droplet, zero velocity and pressure, old level = new."""
    h = case.h
    xc = (np.arange(case.nx) + 0.5) * h
    yc = (np.arange(case.ny) + 0.5) * h
    zc = (np.arange(case.nz) + 0.5) * h
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    r = np.sqrt((X - case.drop_c[0]) ** 2 + (Y - case.drop_c[1]) ** 2 + (Z - case.drop_c[2]) ** 2)
    C = np.tanh((case.drop_r - r) / (math.sqrt(2.0) * case.params.Cn))
    zc3 = np.zeros((case.nz, case.ny, case.nx))
    zw = np.zeros((case.nz + 1, case.ny, case.nx))
    return {"C": C.copy(), "C_old": C.copy(),
            "u": zc3.copy(), "u_old": zc3.copy(), "v": zc3.copy(), "v_old": zc3.copy(),
            "w": zw.copy(), "w_old": zw.copy(),
            "Hu": zc3.copy(), "Hv": zc3.copy(), "Hw": zw.copy(),
            "P": zc3.copy(), "P_old": zc3.copy()}


def random_state3d(case: Case3D, seed: int = 7, amp_u: float = 0.05) -> dict:
    """The initial droplet with smooth random perturbations of every field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s = initial_state3d(case)
    nz, ny, nx = case.nz, case.ny, case.nx

    def smooth(shape, amp):
        a = rng.standard_normal(shape)
        for _ in range(3):
            a = 0.25 * (np.roll(a, 1, 2) + np.roll(a, -1, 2)) + 0.5 * a
            a = 0.25 * (np.roll(a, 1, 1) + np.roll(a, -1, 1)) + 0.5 * a
            a[1:-1] = 0.25 * (a[:-2] + a[2:]) + 0.5 * a[1:-1]
        return amp * a / max(1e-30, np.abs(a).max())

    s["C_old"] = s["C"] + smooth((nz, ny, nx), 0.02)
    s["C"] = s["C"] + smooth((nz, ny, nx), 0.02)
    for key in ("u", "u_old", "Hu", "v", "v_old", "Hv"):
        s[key] = smooth((nz, ny, nx), 1.0 if key[0] == "H" else amp_u)
    for key in ("w", "w_old", "Hw"):
        a = smooth((nz + 1, ny, nx), 1.0 if key == "Hw" else amp_u)
        a[0] = 0.0
        a[nz] = 0.0
        s[key] = a
    s["P"] = smooth((nz, ny, nx), 1.0)
    s["P_old"] = s["P"] + smooth((nz, ny, nx), 0.1)
    s["P"] -= s["P"].mean()
    s["P_old"] -= s["P_old"].mean()
    return s


def droplet_C3d(case: Case3D, dtype=np.float32) -> np.ndarray:
    """The tanh droplet field of initial_state3d alone, built one z-plane at a time in the
    requested dtype (for grids whose full FP64 state would not fit comfortably on the host);
    the other initial fields are zero."""
    h = case.h
    xc = (np.arange(case.nx) + 0.5) * h
    yc = (np.arange(case.ny) + 0.5) * h
    Y, X = np.meshgrid(yc, xc, indexing="ij")
    r2xy = (X - case.drop_c[0]) ** 2 + (Y - case.drop_c[1]) ** 2
    out = np.empty((case.nz, case.ny, case.nx), dtype=dtype)
    s = math.sqrt(2.0) * case.params.Cn
    for k in range(case.nz):
        z = (k + 0.5) * h
        out[k] = np.tanh((case.drop_r - np.sqrt(r2xy + (z - case.drop_c[2]) ** 2)) / s)
    return out
