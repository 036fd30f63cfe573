"""GPU parity of the semi-implicit momentum predictor (ns_scheme = 1; Appendix A.2, Eq.
predictionSemi, reading R19) against the FP64 oracle: three steps from a common random
state within 1e-12 per field on the flat and the sinusoidal walls and in a batched context
of three grid sizes; the FP32 form against the FP64 path over 2000 steps."""
import dataclasses

import numpy as np
import pytest

from oracle import ib_pf2d as O
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


def _semi(case, **kw):
    return dataclasses.replace(case, params=dataclasses.replace(case.params, ns_scheme=1, **kw))


CASES = {
    "flat": lambda: _semi(W.flat_wall_case(l_s=0.01)),
    "sinusoid": lambda: _semi(W.sinusoid_wall_512x256(theta_deg=45.0, l_s=0.01, nx=256, ny=128)),
    "flat_dynamic": lambda: _semi(W.flat_wall_case(l_s=0.02), mu_f=0.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_semi_implicit_step_parity(ibpf, name):
    case = CASES[name]()
    geo = O.build_geometry(case)
    st = W.random_state(case, seed=17)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(st)
    ref = st
    for n in range(3):
        ref, info = O.step(case, geo, ref)
        s.step(1)
        out = s.read_state()
        errs = {k: _rel(out[k], ref[k]) for k in ("C", "u", "v", "P", "Hu", "Hv")}
        bad = {k: e for k, e in errs.items() if not e <= TOL64}
        assert not bad, (name, n, bad)
    s.close()


def test_semi_implicit_batched_sizes(ibpf):
    cs = [_semi(W.flat_wall_case(nx=nx, ny=nx // 2, Cn=2.56 * 2.0 / nx)) for nx in (64, 128, 256)]
    st = [W.random_state(c, seed=60 + k) for k, c in enumerate(cs)]
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


def test_fp32_semi_implicit_run_tracks_fp64(ibpf):
    case = _semi(W.sinusoid_wall_512x256(theta_deg=135.0, l_s=0.01))
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
    e = {k: _rel(out[ibpf.FP32][k], out[ibpf.FP64][k]) for k in ("C", "u", "v")}
    assert e["C"] <= 1e-5 and max(e["u"], e["v"]) <= 1e-4, e
