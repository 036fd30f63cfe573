"""GPU parity of the dynamic contact angle (mu_f > 0, Eq. WallBCS_recast with reading R18)
against the FP64 oracle: three steps from a common random state (the wall values C_I are
carried as state and compared too) within 1e-12 per field, in 2D (flat and sinusoidal walls,
with slip so that the wetting bracket enters the velocity fill) and 3D (sphere); a mixed
static / dynamic batched context; a bit-exact restart through the C_I field; and the FP32
form against the FP64 path."""
import dataclasses

import numpy as np
import pytest

from oracle import ib_pf2d as O
from oracle import ib_pf3d as O3
from workloads import cases as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _dyn(case, mu_f):
    return dataclasses.replace(case, params=dataclasses.replace(case.params, mu_f=mu_f))


CASES2 = {
    "flat": lambda: _dyn(W.flat_wall_case(l_s=0.02, theta_deg=60.0), 0.5),
    "sinusoid": lambda: _dyn(W.sinusoid_wall_512x256(theta_deg=135.0, l_s=0.01, nx=256, ny=128), 2.0),
}


@pytest.mark.parametrize("name", list(CASES2))
def test_dynamic_angle_parity_2d(ibpf, name):
    case = CASES2[name]()
    geo = O.build_geometry(case)
    st = W.random_state(case, seed=31)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(st)
    ref = st
    for n in range(3):
        ref, info = O.step(case, geo, ref)
        s.step(1)
        out = s.read_checkpoint()
        errs = {k: _rel(out[k], ref[k]) for k in ("C", "u", "v", "P", "Hu", "Hv", "C_I")}
        bad = {k: e for k, e in errs.items() if not e <= TOL64}
        assert not bad, (name, n, bad)
    assert np.abs(info["B"]).max() > 0.0          # the bracket is active
    s.close()


def test_dynamic_angle_parity_3d(ibpf):
    case = _dyn(W.small_sphere_case(32), 1.0)
    geo = O3.build_geometry3(case)
    st = W.random_state3d(case, seed=32)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(st)
    ref = st
    for n in range(2):
        ref, info = O3.step3(case, geo, ref)
        s.step(1)
        out = s.read_checkpoint()
        errs = {}
        for k in ("C", "u", "v", "w", "P", "C_I"):
            a, b = out[k], ref[k]
            if k == "P":
                a, b = a - a.mean(), b - b.mean()
            errs[k] = _rel(a, b)
        bad = {k: e for k, e in errs.items() if not e <= TOL64}
        assert not bad, (n, bad)
    s.close()


def test_mixed_static_and_dynamic_batch(ibpf):
    cs = [W.flat_wall_case(l_s=0.02), CASES2["flat"](), _dyn(W.flat_wall_case(nx=64, ny=32, l_s=0.01), 0.1)]
    st = [W.random_state(c, seed=40 + k) for k, c in enumerate(cs)]
    s = ibpf.solver_from_cases(cs, ibpf.FP64)
    s.precompute_weights()
    for k in range(len(cs)):
        s.write_state(st[k], k)
    s.step(2)
    for k, c in enumerate(cs):
        geo = O.build_geometry(c)
        ref = st[k]
        for _ in range(2):
            ref, _ = O.step(c, geo, ref)
        out = s.read_state(k)
        for f in ("C", "u", "v", "P"):
            assert _rel(out[f], ref[f]) <= TOL64, (k, f)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_restart_with_wall_values_is_bit_exact(ibpf, prec):
    p = ibpf.FP64 if prec == "fp64" else ibpf.FP32
    case = CASES2["flat"]()
    st = W.initial_state(case)
    a = ibpf.solver_from_cases([case], p)
    a.precompute_weights()
    a.write_state(st)
    a.step(30)
    ra = a.read_checkpoint()
    b = ibpf.solver_from_cases([case], p)
    b.precompute_weights()
    b.write_state(st)
    b.step(15)
    mid = b.read_checkpoint()
    assert np.isfinite(mid["C_I"]).all()
    b.close()
    c = ibpf.solver_from_cases([case], p)
    c.precompute_weights()
    c.write_checkpoint(mid)
    c.step(15)
    rc = c.read_checkpoint()
    for k in ra:
        assert np.array_equal(ra[k], rc[k]), k
    a.close()
    c.close()


def test_fp32_dynamic_run_tracks_fp64(ibpf):
    case = _dyn(W.flat_wall_case(theta_deg=120.0, l_s=0.02), 0.5)
    st = W.initial_state(case)
    out = {}
    for p in (ibpf.FP64, ibpf.FP32):
        s = ibpf.solver_from_cases([case], p)
        s.precompute_weights()
        s.write_state(st)
        s.step(2000)
        assert s.query(ibpf.Q_STATUS) == 0.0
        d = {k: v.astype(np.float64) for k, v in s.read_checkpoint().items()}
        if p == ibpf.FP32:
            d["C"] = d["C"] + d["C_lo"]
        out[p] = d
        s.close()
    e = {k: _rel(out[ibpf.FP32][k], out[ibpf.FP64][k]) for k in ("C", "u", "v", "C_I")}
    assert e["C"] <= 1e-5 and e["C_I"] <= 1e-5 and max(e["u"], e["v"]) <= 1e-4, e
