"""The FP32 form (FP32 fields, stencils, gathers and transforms; FP64 symbol denominators,
geometry weights and mass reduction; C held as a compensated FP32 pair) against the FP64
CPU oracle and the FP64 GPU path.

Bounds on the 512 x 256 sinusoidal-wall runs of 5000 steps: max|C - C_ref| / max|C_ref|
<= 1e-5, the same for u and v <= 1e-4, apparent contact angle within 0.1 deg.
One-step bounds follow from FP32 rounding (unit roundoff 2^-24 ~ 6e-8) of the inputs of a
step, amplified by the stencils of the random test state: C to 5e-6, the velocity and the
pressure (mean removed) to 1e-5.

"""
import math

import numpy as np
import pytest

from oracle import ib_pf2d as O
from workloads import cases

import wetting

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _solver(ibpf, case, prec):
    s = ibpf.solver_from_cases([case], prec)
    s.precompute_weights()
    return s


def _state64(ibpf, s):
    d = {k: v.astype(np.float64) for k, v in s.read_state().items()}
    if s.precision == ibpf.FP32:
        d["C"] = d["C"] + s.read("C_lo").astype(np.float64)
        d["C_old"] = d["C_old"] + s.read("C_old_lo").astype(np.float64)
    return d


def _errs(got, ref):
    out = {}
    for k in ("C", "u", "v"):
        out[k] = float(np.abs(got[k] - ref[k]).max() / np.abs(ref[k]).max())
    gp = got["P"] - got["P"].mean()
    rp = ref["P"] - ref["P"].mean()
    out["P"] = float(np.abs(gp - rp).max() / np.abs(rp).max())
    return out


def contact_angle(case, C):
    """Apparent contact angles (deg) at the two contact points of the circle fitted to the
    C = 0 level set (tests/wetting.py)."""
    return wetting.contact_angles(case, C, lambda x: float(O.wall_height(case, np.array([x]))[0]))


def test_fp32_one_step_vs_oracle(ibpf):
    case = cases.sinusoid_wall_512x256(theta_deg=45.0, l_s=0.01)
    st = cases.random_state(case, seed=5)
    geo = O.build_geometry(case)
    ref, _ = O.step(case, geo, st)
    s = _solver(ibpf, case, ibpf.FP32)
    s.write_state(st)
    s.step(1)
    e = _errs(_state64(ibpf, s), ref)
    s.close()
    assert e["C"] <= 5e-6 and e["u"] <= 1e-5 and e["v"] <= 1e-5 and e["P"] <= 1e-5, e


def test_fp32_run_bounds_vs_oracle(ibpf):
    # 5000 steps from the initial droplet, FP32 GPU against the FP64 CPU oracle
    case = cases.sinusoid_wall_512x256(theta_deg=45.0, l_s=0.01)
    st = cases.initial_state(case)
    s = _solver(ibpf, case, ibpf.FP32)
    s.write_state(st)
    s.step(case.steps)
    got = _state64(ibpf, s)
    s.close()
    geo = O.build_geometry(case)
    ref = st
    for _ in range(case.steps):
        ref, _ = O.step(case, geo, ref)
    e = _errs(got, ref)
    assert e["C"] <= 1e-5 and e["u"] <= 1e-4 and e["v"] <= 1e-4, e
    da = np.abs(contact_angle(case, got["C"]) - contact_angle(case, ref["C"]))
    assert da.shape == (2,) and da.max() < 0.1, da


@pytest.mark.parametrize("theta,l_s", [(t, l) for t in (45.0, 90.0, 135.0) for l in (0.0, 0.01)])
def test_fp32_run_bounds_vs_fp64_path(ibpf, theta, l_s):
    # the six sinusoidal-wall runs, 5000 steps each, FP32 form against the FP64 path
    # (which tracks the oracle to round-off, see test_gpu_parity)
    case = cases.sinusoid_wall_512x256(theta_deg=theta, l_s=l_s)
    st = cases.initial_state(case)
    steps = case.steps
    out = {}
    for prec in (ibpf.FP64, ibpf.FP32):
        s = _solver(ibpf, case, prec)
        s.write_state(st)
        s.step(steps)
        out[prec] = _state64(ibpf, s)
        s.close()
    e = _errs(out[ibpf.FP32], out[ibpf.FP64])
    assert e["C"] <= 1e-5 and e["u"] <= 1e-4 and e["v"] <= 1e-4, e
    da = np.abs(contact_angle(case, out[ibpf.FP32]["C"]) - contact_angle(case, out[ibpf.FP64]["C"]))
    assert da.shape == (2,) and da.max() < 0.1, da


def test_fp32_flat_wall_tracks_oracle(ibpf):
    case = cases.flat_wall_128x64()
    st = cases.initial_state(case)
    geo = O.build_geometry(case)
    s = _solver(ibpf, case, ibpf.FP32)
    s.write_state(st)
    s.step(case.steps)
    got = _state64(ibpf, s)
    s.close()
    ref = st
    for _ in range(case.steps):
        ref, _ = O.step(case, geo, ref)
    e = _errs(got, ref)
    assert e["C"] <= 1e-5 and e["u"] <= 1e-4 and e["v"] <= 1e-4, e


def test_fp32_checkpoint_restart_is_bit_exact(ibpf):
    case = cases.sinusoid_wall_512x256(theta_deg=135.0, l_s=0.0)
    st = cases.initial_state(case)
    a = _solver(ibpf, case, ibpf.FP32)
    a.write_state(st)
    a.step(40)
    ra = a.read_checkpoint()
    b = _solver(ibpf, case, ibpf.FP32)
    b.write_state(st)
    b.step(20)
    mid = b.read_checkpoint()
    b.close()
    c = _solver(ibpf, case, ibpf.FP32)
    c.write_checkpoint(mid)
    c.step(20)
    rc = c.read_checkpoint()
    for k in ra:
        assert np.array_equal(ra[k], rc[k]), k
    a.close()
    c.close()
