"""Caller-owned field buffers (ib_pf_bind_fields): a context whose state lives in torch
tensors bound through the C ABI reproduces the library-owned context bit for bit, the
bound tensors hold the state the step advanced, and bad bindings are rejected."""
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


def _bind_all(ibpf, s, torch, dim, fp32):
    dt = torch.float32 if fp32 else torch.float64
    two = ["C", "u", "v", "P"] + (["w"] if dim == 3 else []) + (["C_lo"] if fp32 else [])
    one = ["Hu", "Hv"] + (["Hw"] if dim == 3 else [])
    held = {}
    for name in two:
        for lv in (0, 1):
            shp = s.field_shape("C" if name == "C_lo" else name)
            t = torch.full(shp, float("nan"), dtype=dt, device="cuda")
            s.bind(name, t, lv)
            held[(name, lv)] = t
    for name in one:
        t = torch.full(s.field_shape(name), float("nan"), dtype=dt, device="cuda")
        s.bind(name, t, 0)
        held[(name, 0)] = t
    return held


@pytest.mark.parametrize("dim,fp32", [(2, False), (2, True), (3, False), (3, True)])
def test_bound_tensors_reproduce_library_owned_run(ibpf, dim, fp32):
    import torch
    prec = ibpf.FP32 if fp32 else ibpf.FP64
    if dim == 2:
        case = W.sinusoid_wall_512x256(theta_deg=135.0, l_s=0.01, nx=256, ny=128)
        st = W.random_state(case, seed=9)
    else:
        case = W.small_sphere_case(32)
        st = W.random_state3d(case, seed=9)
    runs = []
    for bound in (False, True):
        s = ibpf.solver_from_cases([case], prec)
        s.precompute_weights()
        held = _bind_all(ibpf, s, torch, dim, fp32) if bound else None
        s.write_state(st)
        s.step(10)
        out = s.read_checkpoint()
        assert s.query(ibpf.Q_STATUS) == 0.0
        if bound:
            # after an even number of steps the level-0 buffers hold level n again
            assert np.array_equal(held[("C", 0)].cpu().numpy(), out["C"])
            assert np.array_equal(held[("C", 1)].cpu().numpy(), out["C_old"])
            assert np.array_equal(held[("Hu", 0)].cpu().numpy(), out["Hu"])
            s.step(1)       # odd: the roles have swapped
            assert np.array_equal(held[("C", 1)].cpu().numpy(), s.read("C"))
        runs.append(out)
        s.close()
        if bound:
            # the tensors survive the context (the caller owns them)
            assert torch.isfinite(held[("C", 0)]).all()
    for k in runs[0]:
        assert np.array_equal(runs[0][k], runs[1][k]), k


def test_bad_bindings_are_rejected(ibpf):
    import torch
    case = W.flat_wall_128x64()
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    good = torch.zeros(case.ny, case.nx, dtype=torch.float64, device="cuda")
    small = torch.zeros(case.ny, case.nx - 1, dtype=torch.float64, device="cuda")
    host = torch.zeros(case.ny, case.nx, dtype=torch.float64)
    flat = torch.zeros(case.ny * case.nx + 1, dtype=torch.float64, device="cuda")
    nb = good.numel() * 8
    for args in ((0, ibpf.F_C, 0, small.data_ptr(), small.numel() * 8),      # size
                 (0, ibpf.F_C, 2, good.data_ptr(), nb),                       # time level
                 (0, ibpf.F_HU, 1, good.data_ptr(), nb),                      # one-level field
                 (0, ibpf.F_PHI, 0, good.data_ptr(), nb),                     # not state
                 (0, ibpf.F_W, 0, good.data_ptr(), nb),                       # 2D has no w
                 (0, ibpf.F_C, 0, host.data_ptr(), nb),                       # host memory
                 (0, ibpf.F_C, 0, flat.data_ptr() + 8, nb),                   # misaligned
                 (1, ibpf.F_C, 0, good.data_ptr(), nb)):                      # instance
        with pytest.raises(ibpf.IbPfError) as ei:
            ibpf.ib_pf_bind_fields(s.ctx, *args)
        assert ei.value.status == ibpf.E_ARG
    ibpf.ib_pf_bind_fields(s.ctx, 0, ibpf.F_C, 0, good.data_ptr(), nb)
    with pytest.raises(ibpf.IbPfError):          # one buffer, two fields
        ibpf.ib_pf_bind_fields(s.ctx, 0, ibpf.F_P, 0, good.data_ptr(), nb)
    s.close()
