"""The allocation-free Poisson entry point against the regular step.

ib_pf_poisson_solve_noalloc serves callers that cannot allocate device memory while they
run (their memory belongs to another framework's allocator, or an allocation in a timed
loop is not acceptable).  It must give the same solution as the Poisson solve inside
step a7 of ib_pf_step, which solves for the pressure increment P^{n+1} - (2P^n - P^{n-1}):
the step's Poisson right-hand side and its pressures are read back through the C ABI and
the allocation-free solve of that right-hand side is compared with the increment, on two
consecutive steps (the second call reuses the scratch the first one left behind).
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


def test_noalloc_rejects_oversized_grid():
    from paper_2104_00350_gb300 import build
    build.build()
    from paper_2104_00350_gb300 import ibpf
    with pytest.raises(ibpf.IbPfError) as ei:
        ibpf.ib_pf_poisson_solve_noalloc(1, 1, 2048, 512, 1.0 / 512)
    assert ei.value.status == ibpf.E_ARG
    assert "exceeds" in ibpf.ib_pf_last_error(None)
