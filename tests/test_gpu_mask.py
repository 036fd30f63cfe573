"""GPU parity of the MASK geometry (caller-supplied volume fractions, reading R20): the
geometry tables and one step of the CUDA path against the FP64 oracle on MASK cases, 2D
(the fractions of the 512 x 256 sinusoidal wall) and 3D (those of the 32^3 sphere).
Integer tables identical, FP64 tables within 1e-12, fields within 1e-12 per step."""
from dataclasses import replace

import numpy as np
import pytest

from oracle import ib_pf2d as O
from oracle import ib_pf3d as O3
from workloads import cases as W

from test_gpu_parity import _geometry_parity, _step_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _mask2():
    case = W.sinusoid_wall_512x256(theta_deg=60.0, l_s=0.01)
    geo = O.build_geometry(case)
    return replace(case, geom_kind=W.GEOM_MASK, alpha=(geo.alpha_c, geo.alpha_u, geo.alpha_v))


def test_mask_geometry_and_step_2d(ibpf):
    case = _mask2()
    geo = _geometry_parity(ibpf, case)
    _step_parity(ibpf, case, W.random_state(case, seed=6), geo=geo)


def test_mask_geometry_and_step_3d(ibpf):
    base = W.small_sphere_case(32)
    g0 = O3.build_geometry3(base)
    case = replace(base, geom_kind=W.GEOM_MASK, alpha=(g0.alpha_c, g0.alpha_u, g0.alpha_v, g0.alpha_w))
    geo = O3.build_geometry3(case)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    nz, ny, nx = case.nz, case.ny, case.nx
    assert np.array_equal(s.table(ibpf.T_ALPHA_C).reshape(nz, ny, nx), geo.alpha_c)
    assert np.array_equal(s.table(ibpf.T_ALPHA_W).reshape(nz + 1, ny, nx), geo.alpha_w)
    assert np.array_equal(s.table(ibpf.T_CLASS).reshape(nz, ny, nx), geo.cls.astype(np.int32))
    assert np.array_equal(s.table(ibpf.T_GHOST_CELL), geo.gcell)
    ng = len(geo.gcell)
    assert ng > 0
    assert np.abs(s.table(ibpf.T_NORMAL).reshape(ng, 3) - geo.n).max() <= 1e-13
    assert _rel(s.table(ibpf.T_DN), geo.dn) <= 1e-12
    assert np.array_equal(s.table(ibpf.T_AP1).reshape(ng, 7), geo.ap1)
    assert np.array_equal(s.table(ibpf.T_AP2).reshape(ng, 7), geo.ap2)
    assert np.abs(s.table(ibpf.T_W1).reshape(ng, 7) - geo.w1).max() <= 1e-12
    assert np.abs(s.table(ibpf.T_W2).reshape(ng, 7) - geo.w2).max() <= 1e-12
    assert np.array_equal(s.table(ibpf.T_FACE_W), geo.fw)
    st = W.random_state3d(case, seed=4)
    ref, _ = O3.step3(case, geo, st)
    s.write_state(st)
    s.step(1)
    out = s.read_state()
    assert s.query(ibpf.Q_STATUS) == 0.0
    s.close()
    for k in ("C", "u", "v", "w", "P", "Hu", "Hv", "Hw"):
        a, b = out[k], ref[k]
        if k == "P":
            a, b = a - a.mean(), b - b.mean()
        assert _rel(a, b) <= 1e-12, k
