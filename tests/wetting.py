"""Measurements of a 2D droplet on a wall, used by the wetting tests (test helper).

Plain geometry only: the C = 0 level set is located by linear interpolation between cell
centres, a circle is fitted to it by linear least squares, and the circular-cap relations of
a droplet of area A at angle theta (measured through the liquid) give the expected shape:
r = sqrt(A / (theta - sin(theta) cos(theta))), base half-width r sin(theta), height
r (1 - cos(theta)).  No arithmetic of the method lives here.
"""
import math

import numpy as np


def level_points(case, C, wall_height, above):
    """Points of the C = 0 level set at least `above` over the wall, from crossings along
    rows and columns of cell centres."""
    h, nx, ny = case.h, case.nx, case.ny
    pts = []
    for j in range(ny):
        y = (j + 0.5) * h
        row = C[j]
        for i in range(nx):
            a, b = row[i], row[(i + 1) % nx]
            if a * b < 0:
                x = (i + 0.5 + a / (a - b)) * h
                if y > wall_height(x) + above:
                    pts.append((x, y))
    for i in range(nx):
        x = (i + 0.5) * h
        col = C[:, i]
        for j in range(ny - 1):
            a, b = col[j], col[j + 1]
            if a * b < 0:
                y = (j + 0.5 + a / (a - b)) * h
                if y > wall_height(x) + above:
                    pts.append((x, y))
    return np.array(pts)


def fit_circle(P):
    """Least-squares circle through the points P (k x 2): centre (xc, yc) and radius r."""
    A = np.c_[2 * P[:, 0], 2 * P[:, 1], np.ones(len(P))]
    xc, yc, c = np.linalg.lstsq(A, (P ** 2).sum(axis=1), rcond=None)[0]
    return xc, yc, math.sqrt(c + xc * xc + yc * yc)


def contact_angles(case, C, wall_height):
    """Apparent contact angles (deg, through the liquid) where the circle fitted to the
    C = 0 level set at least 3 Cn above the wall meets the wall: the angle between the
    circle's outward normal and the wall normal (pointing into the fluid)."""
    P = level_points(case, C, wall_height, 3.0 * case.params.Cn)
    xc, yc, r = fit_circle(P)
    xs = np.linspace(xc - r - 0.2, xc + r + 0.2, 40001)
    yw = np.array([wall_height(x) for x in xs])
    f = (xs - xc) ** 2 + (yw - yc) ** 2 - r * r
    roots = np.nonzero(np.sign(f[:-1]) != np.sign(f[1:]))[0]
    angles = []
    for k in roots:
        x0 = xs[k] - f[k] * (xs[k + 1] - xs[k]) / (f[k + 1] - f[k])
        y0 = wall_height(x0)
        dx = 1e-6
        slope = (wall_height(x0 + dx) - wall_height(x0 - dx)) / (2 * dx)
        nw = np.array([-slope, 1.0]) / math.hypot(slope, 1.0)
        nc = np.array([x0 - xc, y0 - yc]) / r
        angles.append(math.degrees(math.acos(np.clip(nc @ nw, -1.0, 1.0))))
    return np.array(angles)


def flat_wall_cap(case, C, yw):
    """Droplet on the flat wall x2 = yw: fitted angle (deg), fitted radius, droplet area
    (the area above the wall enclosed by the C = 0 level set: per column of centres, the
    length where C > 0 with linear interpolation at the crossings, from the wall up) and
    the height of the C = 0 crossing on the droplet's axis x1 = lx/2 above the wall (mean of
    the two centre columns next to the axis)."""
    P = level_points(case, C, lambda x: yw, 3.0 * case.params.Cn)
    xc, yc, r = fit_circle(P)
    theta = math.degrees(math.acos((yw - yc) / r))
    h, nx, ny = case.h, case.nx, case.ny
    j0 = int(math.floor(yw / h - 0.5)) + 1          # first row of centres above the wall
    area = 0.0
    for i in range(nx):
        col = C[:, i]
        y_prev, c_prev = yw, col[j0]                 # the wall takes the first centre's sign
        for j in range(j0, ny):
            y, c = (j + 0.5) * h, col[j]
            if c_prev > 0 and c > 0:
                area += (y - y_prev) * h
            elif c_prev > 0 >= c or c_prev <= 0 < c:
                yx = y_prev + (y - y_prev) * c_prev / (c_prev - c)
                area += ((yx - y_prev) if c_prev > 0 else (y - yx)) * h
            y_prev, c_prev = y, c
    tops = []
    for i in (nx // 2 - 1, nx // 2):
        col = C[:, i]
        for j in range(ny - 2, -1, -1):
            a, b = col[j], col[j + 1]
            if a > 0 >= b:
                tops.append((j + 0.5 + a / (a - b)) * h)
                break
    return theta, r, area, float(np.mean(tops)) - yw


def cap_shape(area, theta_deg):
    """Circular cap of the given area meeting a flat wall at theta: (r, base half-width,
    height)."""
    t = math.radians(theta_deg)
    r = math.sqrt(area / (t - math.sin(t) * math.cos(t)))
    return r, r * math.sin(t), r * (1.0 - math.cos(t))


def relax_flat_wall(spec):
    """Run the oracle for a droplet on the flat wall x2 = 0.1 of [0,2]x[0,1] (volume R = 0.3
    semicircle) from spec = dict(start='semi'|'cap', theta, weights, nx, Cn, dt, T) and return
    [(t, fitted angle, fitted r, area, axis height, all finite)] once per time unit.  'semi'
    starts from the semicircle centred on the wall (90 deg), 'cap' from the circular cap of
    the same area at theta.  Runs in a worker process of the wetting tests."""
    import dataclasses
    from oracle import ib_pf2d as O
    from workloads import cases
    th = spec["theta"]
    case = cases.flat_wall_case(nx=spec["nx"], ny=spec["nx"] // 2, theta_deg=th, Cn=spec["Cn"],
                                dt=spec["dt"])
    case = cases.with_params(case, weights=spec["weights"])
    if spec["start"] == "cap":
        r, _, _ = cap_shape(math.pi * 0.3 ** 2 / 2.0, th)
        case = dataclasses.replace(case, drop_c=(1.0, 0.1 - r * math.cos(math.radians(th))),
                                   drop_r=r)
    geo = O.build_geometry(case)
    st = cases.initial_state(case)
    per_unit = int(round(1.0 / case.params.dt))
    out = []
    for k in range(1, int(round(spec["T"] / case.params.dt)) + 1):
        st, _ = O.step(case, geo, st)
        if k % per_unit == 0:
            ok = all(np.isfinite(v).all() for v in st.values())
            out.append((k * case.params.dt,) + flat_wall_cap(case, st["C"], 0.1) + (ok,))
    return out
