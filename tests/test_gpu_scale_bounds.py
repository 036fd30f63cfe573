"""The mixed-precision and batched forms at the scale of the stated workloads, against the
FP64 GPU path (which tracks the oracle to round-off per step, test_gpu_parity*):

* the six 512 x 256 sinusoidal-wall runs advanced in one batched context for 5000 steps are
  bit-identical to each run advanced alone (FP64 and FP32);
* the 64-instance FP32 ensemble over 200 steps: C within 1e-5, velocity within 1e-4
  (max-norm relative, per instance);
* the 256^3 droplet on a sphere over 1000 steps, FP32 and the split-BF16 tensor-core form:
  C within 1e-5, velocity within 1e-4, apparent contact angle within 0.1 deg;
* the 512^3 packing, FP32 over 500 steps: C within 1e-5, velocity within 1e-4.
"""
import math

import numpy as np
import pytest

from workloads import cases as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ibpf():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf as m
    return m


def _six():
    return [W.sinusoid_wall_512x256(theta_deg=t, l_s=s) for t in (45.0, 90.0, 135.0) for s in (0.0, 0.01)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_six_runs_equal_single_runs(ibpf, prec):
    p = ibpf.FP64 if prec == "fp64" else ibpf.FP32
    cs = _six()
    b = ibpf.solver_from_cases(cs, p)
    b.precompute_weights()
    for k, c in enumerate(cs):
        b.write_state(W.initial_state(c), k)
    b.step(5000)
    for k in range(len(cs)):
        assert b.query(ibpf.Q_STATUS, k) == 0.0
    for k, c in enumerate(cs):
        s = ibpf.solver_from_cases([c], p)
        s.precompute_weights()
        s.write_state(W.initial_state(c))
        s.step(5000)
        a, r = s.read_checkpoint(), b.read_checkpoint(k)
        for f in a:
            assert np.array_equal(a[f], r[f]), (k, f)
        s.close()
    b.close()


def _dev_fields(ibpf, s, torch, names, k=0):
    out = {}
    for n in names:
        t = torch.empty(s.field_shape(n, k), dtype=torch.float64 if s.precision == ibpf.FP64 else torch.float32,
                        device="cuda")
        s.read(n, k, out=t)
        out[n] = t.double()
    if s.precision != ibpf.FP64:
        lo = torch.empty(s.field_shape("C", k), dtype=torch.float32, device="cuda")
        s.read("C_lo", k, out=lo)
        out["C"] = out["C"] + lo.double()
    return out


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


def test_fp32_ensemble_bounds(ibpf):
    import torch
    cs = W.ensemble_2d(64)
    res = {}
    for p in (ibpf.FP64, ibpf.FP32):
        s = ibpf.solver_from_cases(cs, p)
        s.precompute_weights()
        for k, c in enumerate(cs):
            s.write_state(W.initial_state(c), k)
        s.step(200)
        res[p] = [_dev_fields(ibpf, s, torch, ("C", "u", "v"), k) for k in range(len(cs))]
        s.close()
    worst = {"C": 0.0, "u": 0.0, "v": 0.0}
    for k in range(len(cs)):
        for f in worst:
            worst[f] = max(worst[f], _rel(res[ibpf.FP32][k][f], res[ibpf.FP64][k][f]))
    assert worst["C"] <= 1e-5 and max(worst["u"], worst["v"]) <= 1e-4, worst


def _sphere_angle(case, C):
    """Angle (deg, through the liquid) between the droplet and the solid sphere where they
    meet: a sphere fitted to the C = 0 level set away from the solid, then the angle between
    the two spheres' outward normals on their circle of intersection."""
    h, n = case.h, case.nx
    Cz = C
    pts = []
    for axis in range(3):
        a = np.moveaxis(Cz, axis, 0)
        s0, s1 = a[:-1], a[1:]
        idx = np.nonzero(s0 * s1 < 0)
        frac = s0[idx] / (s0[idx] - s1[idx])
        coords = [None, None, None]
        rest = [d for d in range(3) if d != axis]
        coords[axis] = (idx[0] + 0.5 + frac) * h
        coords[rest[0]] = (idx[1] + 0.5) * h
        coords[rest[1]] = (idx[2] + 0.5) * h
        # moveaxis puts axis first and keeps the others in order: array dims (z, y, x)
        pts.append(np.stack([coords[2], coords[1], coords[0]], axis=1))
    P = np.concatenate(pts)
    cs, rs = np.array(case.geom_p[:3]), case.geom_p[3]
    P = P[np.linalg.norm(P - cs, axis=1) > rs + 3 * case.params.Cn]
    A = np.c_[2 * P, np.ones(len(P))]
    sol = np.linalg.lstsq(A, (P ** 2).sum(axis=1), rcond=None)[0]
    cd, r = sol[:3], math.sqrt(sol[3] + sol[:3] @ sol[:3])
    d = np.linalg.norm(cd - cs)
    cos_phi = (rs * rs + r * r - d * d) / (2 * rs * r)
    return 180.0 - math.degrees(math.acos(np.clip(cos_phi, -1.0, 1.0)))


def test_fp32_sphere_256_bounds_and_angle(ibpf):
    import torch
    case = W.sphere_case(256)
    res, ang = {}, {}
    # FP32 and the split-BF16 tensor-core form (the workload's stated transforms)
    for p in (ibpf.FP64, ibpf.FP32, ibpf.FP32_3XBF16):
        s = ibpf.solver_from_cases([case], p)
        s.precompute_weights()
        C0 = W.droplet_C3d(case, np.float64 if p == ibpf.FP64 else np.float32)
        s.write("C", C0)
        s.write("C_old", C0)
        s.step(1000)
        assert s.query(ibpf.Q_STATUS) == 0.0
        res[p] = _dev_fields(ibpf, s, torch, ("C", "u", "v", "w"))
        ang[p] = _sphere_angle(case, res[p]["C"].cpu().numpy())
        s.close()
        torch.cuda.empty_cache()
    for q in (ibpf.FP32, ibpf.FP32_3XBF16):
        e = {f: _rel(res[q][f], res[ibpf.FP64][f]) for f in ("C", "u", "v", "w")}
        assert e["C"] <= 1e-5 and max(e["u"], e["v"], e["w"]) <= 1e-4, (q, e)
        assert abs(ang[q] - ang[ibpf.FP64]) < 0.1, (q, ang)


def test_fp32_porous_512_bounds(ibpf):
    import torch
    case = W.porous_case(512)
    res = {}
    for p in (ibpf.FP64, ibpf.FP32):
        s = ibpf.solver_from_cases([case], p)
        s.precompute_weights()
        C0 = W.droplet_C3d(case, np.float64 if p == ibpf.FP64 else np.float32)
        s.write("C", C0)
        s.write("C_old", C0)
        del C0
        s.step(500)
        assert s.query(ibpf.Q_STATUS) == 0.0
        res[p] = _dev_fields(ibpf, s, torch, ("C", "u", "v", "w"))
        s.close()
        torch.cuda.empty_cache()
    e = {f: _rel(res[ibpf.FP32][f], res[ibpf.FP64][f]) for f in ("C", "u", "v", "w")}
    assert e["C"] <= 1e-5 and max(e["u"], e["v"], e["w"]) <= 1e-4, e
