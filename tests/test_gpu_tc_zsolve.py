"""The split-BF16 tensor-core form (precision FP32_3XBF16): the FP32 form with the
wall-normal solve of the 3D Cahn-Hilliard and Poisson problems (Appendix A.1,
Eq. PressurePoisson) as dense cosine-transform products on the tensor cores.

Bounds.  Each operand is held as two BF16 parts (16 significant bits) and three products are
accumulated in FP32, so one transform carries a relative error of a few 2^-17 (about 1e-5 of
the column's largest value) against FP32's 2^-24.  Both solves are in increment form, so
that error scales the increment, not the field:
* one step from a perturbed state against the FP64 oracle: C within 1e-5, u, v, w, P within
  1e-4 (max-norm relative per field);
* runs from the initial droplet against the FP64 GPU path (which tracks the oracle to
  round-off per step): the mixed-precision bounds, C within 1e-5, velocity within 1e-4,
  and the sphere's apparent contact angle within 0.1 deg.
"""
import numpy as np
import pytest

from oracle import ib_pf3d as O3
from workloads import cases as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _flat(nx, ny, nz):
    h = 2.0 / nx
    return W.flat_wall_case3d(nx=nx, ny=ny, nz=nz, wall_z=0.37 * 16 * h, l_s=0.01)


CASES = {
    "z128": lambda: _flat(16, 16, 128),
    "z256": lambda: _flat(32, 8, 256),        # ragged: 8 x 18 spectrum columns
}


def _read64(ibpf, s):
    d = {k: v.astype(np.float64) for k, v in s.read_state().items()}
    d["C"] = d["C"] + s.read("C_lo").astype(np.float64)
    return d


@pytest.mark.parametrize("name", list(CASES))
def test_step_parity_split_bf16(ibpf, name):
    case = CASES[name]()
    geo = O3.build_geometry3(case)
    st = W.random_state3d(case, seed=5)
    ref, _ = O3.step3(case, geo, st)
    s = ibpf.solver_from_cases([case], ibpf.FP32_3XBF16)
    s.precompute_weights()
    s.write_state(st)
    s.step(1)
    assert s.query(ibpf.Q_STATUS) == 0.0
    out = _read64(ibpf, s)
    s.close()
    errs = {}
    for k in ("C", "u", "v", "w", "P"):
        a, b = out[k], ref[k]
        if k == "P":
            a, b = a - a.mean(), b - b.mean()
        errs[k] = _rel(a, b)
    assert errs["C"] <= 1e-5, errs
    assert max(errs["u"], errs["v"], errs["w"], errs["P"]) <= 1e-4, errs


def test_split_bf16_run_bounds_sphere128(ibpf):
    from test_gpu_scale_bounds import _sphere_angle
    case = W.small_sphere_case(128)
    st = W.initial_state3d(case)
    out, ang = {}, {}
    for prec in (ibpf.FP64, ibpf.FP32_3XBF16):
        s = ibpf.solver_from_cases([case], prec)
        s.precompute_weights()
        s.write_state(st)
        s.step(400)
        assert s.query(ibpf.Q_STATUS) == 0.0
        out[prec] = _read64(ibpf, s) if prec != ibpf.FP64 else s.read_state()
        ang[prec] = _sphere_angle(case, out[prec]["C"])
        s.close()
    errs = {k: _rel(out[ibpf.FP32_3XBF16][k], out[ibpf.FP64][k]) for k in ("C", "u", "v", "w")}
    assert errs["C"] <= 1e-5 and max(errs["u"], errs["v"], errs["w"]) <= 1e-4, errs
    assert abs(ang[ibpf.FP32_3XBF16] - ang[ibpf.FP64]) < 0.1, ang


def test_split_bf16_restart_is_bit_exact(ibpf):
    case = CASES["z128"]()
    st = W.random_state3d(case, seed=9)
    s = ibpf.solver_from_cases([case], ibpf.FP32_3XBF16)
    s.precompute_weights()
    s.write_state(st)
    s.step(3)
    ck = s.read_checkpoint()
    s.step(4)
    a = s.read_state()
    s.write_checkpoint(ck)
    s.step(4)
    b = s.read_state()
    s.close()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
