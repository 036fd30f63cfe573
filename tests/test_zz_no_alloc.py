"""The allocation-free Poisson entry point against the regular step.

ib_pf_poisson_solve_noalloc serves callers that cannot allocate device memory while they
run (their memory belongs to another framework's allocator, or an allocation in a timed
loop is not acceptable).  It must give the same solution as the Poisson solve inside
step a7 of ib_pf_step, which solves for the pressure increment P^{n+1} - (2P^n - P^{n-1}):
the step's Poisson right-hand side and its pressures are read back through the C ABI and
the allocation-free solve of that right-hand side is compared with the increment, on two
consecutive steps (the second call reuses the scratch the first one left behind), also at
the largest grids the fixed scratch accepts (1024 x 512 and 512 x 1024), and the device's
free memory is the same before and after a call.
"""
import numpy as np
import pytest

from workloads import cases

pytestmark = pytest.mark.gpu


def test_noalloc_poisson_matches_step_pressure():
    import torch
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf

    case = cases.sinusoid_wall_512x256(theta_deg=45.0, l_s=0.01)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(cases.random_state(case, seed=21))
    stream = torch.cuda.current_stream()
    out = torch.empty(case.ny, case.nx, dtype=torch.float64, device="cuda")
    for _ in range(2):
        p_hat = 2.0 * s.read("P") - s.read("P_old")
        s.step(1)
        rhs = torch.from_numpy(s.read("rhs_p")).cuda()
        p_step = s.read("P") - p_hat
        out.fill_(np.nan)
        ibpf.ib_pf_poisson_solve_noalloc(rhs.data_ptr(), out.data_ptr(), case.nx, case.ny,
                                         case.h, stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        err = np.abs(got - p_step).max() / np.abs(p_step).max()
        assert err <= 1e-12, err
    s.close()


def _grid_case(nx, ny):
    base = cases.flat_wall_case(nx=nx, ny=max(nx // 2, 8), wall_y=0.23, Cn=2.56 * 2.0 / nx)
    return cases.Case2D(f"flat_{nx}x{ny}", nx, ny, 2.0, ny * 2.0 / nx, base.geom_kind, base.geom_p,
                        (1.0, base.geom_p[0]), 0.3, base.params, 1)


@pytest.mark.parametrize("nx,ny", [(1024, 512), (512, 1024)])
def test_noalloc_largest_grids_allocate_nothing(nx, ny):
    import torch
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf

    case = _grid_case(nx, ny)
    s = ibpf.solver_from_cases([case], ibpf.FP64)
    s.precompute_weights()
    s.write_state(cases.random_state(case, seed=nx + ny))
    stream = torch.cuda.current_stream()
    out = torch.empty(ny, nx, dtype=torch.float64, device="cuda")
    for k in range(2):
        p_hat = 2.0 * s.read("P") - s.read("P_old")
        s.step(1)
        rhs = torch.from_numpy(s.read("rhs_p")).cuda()
        p_step = s.read("P") - p_hat
        out.fill_(np.nan)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        ibpf.ib_pf_poisson_solve_noalloc(rhs.data_ptr(), out.data_ptr(), nx, ny, case.h,
                                         stream.cuda_stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        if k == 1:      # the first call on the device may load the module
            assert free1 == free0, (free0, free1)
        err = np.abs(out.cpu().numpy() - p_step).max() / np.abs(p_step).max()
        assert err <= 1e-12, err
    s.close()


def test_noalloc_rejects_oversized_grid():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf
    with pytest.raises(ibpf.IbPfError) as ei:
        ibpf.ib_pf_poisson_solve_noalloc(1, 1, 2048, 512, 1.0 / 512)
    assert ei.value.status == ibpf.E_ARG
    assert "exceeds" in ibpf.ib_pf_last_error(None)
