"""GPU parity of the 3D path (through the C ABI) against the FP64 3D CPU oracle.

FP64: geometry integer tables identical, FP64 tables within 1e-12 (normals 1e-13); one step
from a common state within 1e-12 relative per field.  FP32 form: one step within the
rounding bounds of the 2D FP32 tests (C 5e-6; u, v, w, P 1e-5).
"""
import numpy as np
import pytest

from oracle import ib_pf3d as O3
from workloads import cases as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
FIELDS3 = ("C", "u", "v", "w", "P", "Hu", "Hv", "Hw", "C_old", "u_old", "v_old", "w_old", "P_old")


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _solver(ibpf, case, prec=None):
    s = ibpf.solver_from_cases([case], ibpf.FP64 if prec is None else prec)
    s.precompute_weights()
    return s


CASES = {
    "sphere32": lambda: W.small_sphere_case(32),
    "porous32": lambda: W.porous_case(32, steps=1),
    "flat3d": lambda: W.flat_wall_case3d(nx=32, ny=16, nz=16, wall_z=0.37, l_s=0.01),
    "free3d": lambda: W.flat_wall_case3d(nx=16, ny=16, nz=8, geom_kind=W.GEOM_NONE),
    # one long axis of 512 points each: the row transforms, the y transforms and the z
    # solve at the transform lengths of the 512^3 workload (and, in z, 32 windows of the
    # FP64 z-marching kernels; in the FP32 form, the wide y and z blocks)
    "xlong": lambda: _long(512, 16, 16),
    "ylong": lambda: _long(16, 512, 16),
    "zlong": lambda: _long(16, 16, 512),
}


def _long(nx, ny, nz):
    h = 2.0 / nx
    return W.flat_wall_case3d(nx=nx, ny=ny, nz=nz, wall_z=0.37 * min(nz, 16) * h, l_s=0.01)


_GEO = {}


def _geo(name):
    if name not in _GEO:
        c = CASES[name]()
        _GEO[name] = (c, O3.build_geometry3(c))
    return _GEO[name]


@pytest.mark.parametrize("name", ["sphere32", "porous32", "flat3d"])
def test_geometry_tables_3d(ibpf, name):
    case, geo = _geo(name)
    s = _solver(ibpf, case)
    nz, ny, nx = case.nz, case.ny, case.nx
    assert np.array_equal(s.table(ibpf.T_ALPHA_C).reshape(nz, ny, nx), geo.alpha_c)
    assert np.array_equal(s.table(ibpf.T_ALPHA_U).reshape(nz, ny, nx), geo.alpha_u)
    assert np.array_equal(s.table(ibpf.T_ALPHA_V).reshape(nz, ny, nx), geo.alpha_v)
    assert np.array_equal(s.table(ibpf.T_ALPHA_W).reshape(nz + 1, ny, nx), geo.alpha_w)
    assert np.array_equal(s.table(ibpf.T_CLASS).reshape(nz, ny, nx), geo.cls.astype(np.int32))
    assert np.array_equal(s.table(ibpf.T_GHOST_CELL), geo.gcell)
    ng = len(geo.gcell)
    assert ng > 0
    assert np.abs(s.table(ibpf.T_NORMAL).reshape(ng, 3) - geo.n).max() <= 1e-13
    assert _rel(s.table(ibpf.T_DN), geo.dn) <= 1e-12
    assert _rel(s.table(ibpf.T_GAMMA), geo.gamma) <= 1e-12
    assert np.array_equal(s.table(ibpf.T_AP1).reshape(ng, 7), geo.ap1)
    assert np.array_equal(s.table(ibpf.T_AP2).reshape(ng, 7), geo.ap2)
    assert np.abs(s.table(ibpf.T_W1).reshape(ng, 7) - geo.w1).max() <= 1e-12
    assert np.abs(s.table(ibpf.T_W2).reshape(ng, 7) - geo.w2).max() <= 1e-12
    assert np.array_equal(s.table(ibpf.T_FACE_U), geo.fu)
    assert np.array_equal(s.table(ibpf.T_FACE_V), geo.fv)
    assert np.array_equal(s.table(ibpf.T_FACE_W), geo.fw)
    s.close()


def _step_parity(ibpf, name, seed, prec=None):
    case, geo = _geo(name)
    st = W.random_state3d(case, seed=seed)
    ref, info = O3.step3(case, geo, st)
    s = _solver(ibpf, case, prec)
    s.write_state(st)
    s.step(1)
    out = s.read_state()
    if prec is not None and prec == ibpf.FP32:
        out = {k: v.astype(np.float64) for k, v in out.items()}
        out["C"] = out["C"] + s.read("C_lo").astype(np.float64)
    errs = {}
    for k in FIELDS3:
        a, b = out[k], ref[k]
        if k in ("P", "P_old"):
            a, b = a - a.mean(), b - b.mean()
        errs[k] = _rel(a, b)
    errs["phi"] = _rel(s.read("phi").astype(np.float64), info["phi"])
    mass = s.query(ibpf.Q_MASS)
    s.close()
    return errs, mass, ref


@pytest.mark.parametrize("name", list(CASES))
def test_step_parity_3d_fp64(ibpf, name):
    errs, mass, ref = _step_parity(ibpf, name, seed=len(name))
    bad = {k: e for k, e in errs.items() if not e <= TOL64}
    assert not bad, (name, bad)
    assert abs(mass - ref["C"].sum()) <= 1e-12 * np.abs(ref["C"]).sum()


@pytest.mark.parametrize("name", ["sphere32", "porous32", "xlong", "ylong", "zlong"])
def test_step_parity_3d_fp32(ibpf, name):
    errs, mass, ref = _step_parity(ibpf, name, seed=3, prec=ibpf.FP32)
    assert errs["C"] <= 5e-6, errs
    assert max(errs["u"], errs["v"], errs["w"], errs["P"]) <= 1e-5, errs
    # the FP64 mass of the compensated FP32 C: within the per-cell bound summed over cells
    c = ref["C"]
    assert abs(mass - c.sum()) <= 5e-6 * np.abs(c).max() * c.size


def test_multi_step_sphere_tracks_oracle(ibpf):
    case, geo = _geo("sphere32")
    st = W.initial_state3d(case)
    s = _solver(ibpf, case)
    s.write_state(st)
    for _ in range(20):
        st, _ = O3.step3(case, geo, st)
    s.step(20)
    out = s.read_state()
    assert s.query(ibpf.Q_STATUS) == 0.0
    s.close()
    for k in ("C", "u", "v", "w"):
        assert _rel(out[k], st[k]) <= 1e-10, k


@pytest.mark.parametrize("name,steps", [("sphere64", 400), ("porous64", 200)])
def test_fp32_run_bounds_vs_fp64_path_3d(ibpf, name, steps):
    # the FP32 form against the FP64 path (which tracks the oracle to round-off, see above)
    # from the initial droplet: C within 1e-5 and the velocity within 1e-4 (max-norm relative),
    # the bounds of the 2D mixed form
    case = W.small_sphere_case(64) if name == "sphere64" else W.porous_case(64, steps=1)
    st = W.initial_state3d(case)
    out = {}
    for prec in (ibpf.FP64, ibpf.FP32):
        s = _solver(ibpf, case, prec)
        s.write_state(st)
        s.step(steps)
        assert s.query(ibpf.Q_STATUS) == 0.0
        d = {k: v.astype(np.float64) for k, v in s.read_state().items()}
        if prec == ibpf.FP32:
            d["C"] = d["C"] + s.read("C_lo").astype(np.float64)
        out[prec] = d
        s.close()
    errs = {k: _rel(out[ibpf.FP32][k], out[ibpf.FP64][k]) for k in ("C", "u", "v", "w")}
    assert errs["C"] <= 1e-5 and max(errs["u"], errs["v"], errs["w"]) <= 1e-4, errs
