"""GPU parity of the explicit Cahn-Hilliard variant (Eq. ExpCH) through the C ABI against
the FP64 CPU oracle: one step from random states within 1e-12 relative (FP64), a multi-step
run from the droplet start, the batched uneven ensemble, and the FP32 form against the FP64
path over a run (C <= 1e-5, velocity <= 1e-4, the bounds of the semi-implicit FP32 form)."""
import dataclasses

import numpy as np
import pytest

from oracle import ib_pf2d as O
from workloads import cases as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
FIELDS = ("C", "u", "v", "P", "Hu", "Hv", "C_old", "u_old", "v_old", "P_old")


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _explicit(case):
    return dataclasses.replace(case, params=dataclasses.replace(case.params, ch_scheme=1))


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = {
    "flat128": lambda: _explicit(W.flat_wall_128x64()),
    "sinusoid512": lambda: _explicit(W.sinusoid_wall_512x256(theta_deg=135.0, l_s=0.01)),
    "ragged16x8": lambda: _explicit(W.flat_wall_case(nx=16, ny=8, wall_y=0.23, Cn=0.25, dt=1e-4)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_explicit_step_parity_fp64(ibpf, name):
    case = CASES[name]()
    geo = O.build_geometry(case)
    st = W.random_state(case, seed=17)
    ref, info = O.step(case, geo, st)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(st)
    s.step(1)
    out = s.read_state()
    if name == "flat128":   # ch_phi2, ch_fill2, ch_explicit replace the five a1/a2 launches
        assert s.query(ibpf.Q_LAUNCHES) == 15
    s.close()
    bad = {}
    for k in FIELDS:
        a, b = out[k], ref[k]
        if k in ("P", "P_old"):
            a, b = a - a.mean(), b - b.mean()
        e = _rel(a, b)
        if not e <= TOL64:
            bad[k] = e
    assert not bad, bad


def test_explicit_multi_step_tracks_oracle(ibpf):
    case = CASES["flat128"]()
    geo = O.build_geometry(case)
    st = W.initial_state(case)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(st)
    for _ in range(20):
        st, _ = O.step(case, geo, st)
    s.step(20)
    out = s.read_state()
    assert s.query(ibpf.Q_STATUS) == 0.0
    s.close()
    for k in ("C", "u", "v"):
        assert _rel(out[k], st[k]) <= 1e-10, k


def test_explicit_batched_ensemble_fp64(ibpf):
    ens = [_explicit(c) for c in W.ensemble_2d(64)[:6]]
    sts = [W.random_state(c, seed=40 + k) for k, c in enumerate(ens)]
    s = ibpf.solver_from_cases(ens, ibpf.FP64)
    s.precompute_weights()
    for k, st in enumerate(sts):
        s.write_state(st, k)
    s.step(1)
    for k, c in enumerate(ens):
        ref, _ = O.step(c, O.build_geometry(c), sts[k])
        out = s.read_state(k)
        for f in ("C", "u", "v"):
            assert _rel(out[f], ref[f]) <= TOL64, (k, f)
    s.close()


def test_explicit_fp32_run_bounds_vs_fp64_path(ibpf):
    case = CASES["sinusoid512"]()
    st = W.initial_state(case)
    out = {}
    for prec in (ibpf.FP64, ibpf.FP32):
        s = ibpf.solver_from_cases([case], prec)
        s.precompute_weights()
        s.write_state(st)
        s.step(1000)
        assert s.query(ibpf.Q_STATUS) == 0.0
        d = {k: v.astype(np.float64) for k, v in s.read_state().items()}
        if prec == ibpf.FP32:
            d["C"] = d["C"] + s.read("C_lo").astype(np.float64)
        out[prec] = d
        s.close()
    errs = {k: _rel(out[ibpf.FP32][k], out[ibpf.FP64][k]) for k in ("C", "u", "v")}
    assert errs["C"] <= 1e-5 and max(errs["u"], errs["v"]) <= 1e-4, errs


# ---------------------------------------------------------------------------- 3D
CASES3 = {
    "sphere32": lambda: _explicit(W.small_sphere_case(32)),
    "flat3d": lambda: _explicit(W.flat_wall_case3d(nx=32, ny=16, nz=16, wall_z=0.37, l_s=0.01)),
}
FIELDS3 = ("C", "u", "v", "w", "P", "Hu", "Hv", "Hw", "C_old", "w_old")


@pytest.mark.parametrize("name", list(CASES3))
def test_explicit_step_parity_3d_fp64(ibpf, name):
    from oracle import ib_pf3d as O3
    case = CASES3[name]()
    geo = O3.build_geometry3(case)
    st = W.random_state3d(case, seed=23)
    ref, _ = O3.step3(case, geo, st)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(st)
    s.step(1)
    out = s.read_state()
    s.close()
    bad = {}
    for k in FIELDS3:
        a, b = out[k], ref[k]
        if k == "P":
            a, b = a - a.mean(), b - b.mean()
        e = _rel(a, b)
        if not e <= TOL64:
            bad[k] = e
    assert not bad, bad


def test_explicit_3d_fp32_run_bounds_vs_fp64_path(ibpf):
    case = _explicit(W.small_sphere_case(64))
    st = W.initial_state3d(case)
    out = {}
    for prec in (ibpf.FP64, ibpf.FP32):
        s = ibpf.solver_from_cases([case], prec)
        s.precompute_weights()
        s.write_state(st)
        s.step(400)
        assert s.query(ibpf.Q_STATUS) == 0.0
        d = {k: v.astype(np.float64) for k, v in s.read_state().items()}
        if prec == ibpf.FP32:
            d["C"] = d["C"] + s.read("C_lo").astype(np.float64)
        out[prec] = d
        s.close()
    errs = {k: _rel(out[ibpf.FP32][k], out[ibpf.FP64][k]) for k in ("C", "u", "v", "w")}
    assert errs["C"] <= 1e-5 and max(errs["u"], errs["v"], errs["w"]) <= 1e-4, errs


def test_explicit_batched_ensemble_fp32_bounds_vs_fp64(ibpf):
    # the FP32 form of the explicit variant on an uneven batch, 200 steps from the droplet
    ens = [_explicit(c) for c in W.ensemble_2d(64)[:8]]
    out = {}
    for prec in (ibpf.FP64, ibpf.FP32):
        s = ibpf.solver_from_cases(ens, prec)
        s.precompute_weights()
        for k, c in enumerate(ens):
            s.write_state(W.initial_state(c), k)
        s.step(200)
        out[prec] = []
        for k in range(len(ens)):
            assert s.query(ibpf.Q_STATUS, k) == 0.0
            d = {f: v.astype(np.float64) for f, v in s.read_state(k).items()}
            if prec == ibpf.FP32:
                d["C"] = d["C"] + s.read("C_lo", k).astype(np.float64)
            out[prec].append(d)
        s.close()
    for k in range(len(ens)):
        a, b = out[ibpf.FP32][k], out[ibpf.FP64][k]
        assert _rel(a["C"], b["C"]) <= 1e-5, k
        assert max(_rel(a["u"], b["u"]), _rel(a["v"], b["v"])) <= 1e-4, k
