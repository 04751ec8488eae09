"""Failure detection through the C ABI, made on the host (no GPU fault).

* A plan whose memory would exceed opts.mem_cap fails with ORI_ERR_OOM before
  it allocates past the cap, and a normal plan works afterwards.
* Non-finite data (a NaN right-hand side, a NaN impedance) end the solve
  with ORI_ERR_NONFINITE, detected by the device reductions; the plan keeps
  working for the next solve.
* maxit = 0 returns ORI_ERR_NOT_CONVERGED with the iterate (here u = 0).
"""

import math

import numpy as np
import pytest
import torch

from paper_1602_04691_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_mem_cap_gives_oom_and_leaves_the_device_usable():
    from paper_1602_04691_gb300 import OriError, Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_OOM
    n = 24
    h, N = inputs.random_h_N(n, 701)
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(OriError) as e:
        Plan(n, 2.0, to_dev(h), to_dev(N), mem_cap=1 << 20)
    assert e.value.status == ORI_ERR_OOM
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)     # nothing held back
    plan = Plan(n, 2.0, to_dev(h), to_dev(N))
    u, info = plan.solve(tol=1e-6)
    assert info["status"] == 0


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_nan_right_hand_side_is_reported_and_plan_recovers(precision):
    from paper_1602_04691_gb300 import Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_NONFINITE
    n = 12
    h, N = inputs.random_h_N(n, 702)
    plan = Plan(n, 2.0, to_dev(h), to_dev(N))
    rhs = inputs.random_complex(n ** 3, 703)
    rhs[17] = complex(math.nan, 0.0)
    u, info = plan.solve(rhs=to_dev(rhs), tol=1e-6, precision=precision, raise_on_failure=False)
    assert info["returned"] == ORI_ERR_NONFINITE
    u, info = plan.solve(tol=1e-6, precision=precision)
    assert info["status"] == 0 and info["relres"] <= 1e-6


def test_nan_impedance_is_reported():
    from paper_1602_04691_gb300 import Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_NONFINITE
    n = 10
    h, N = inputs.random_h_N(n, 704)
    h[33] = complex(math.nan, 1.0)
    plan = Plan(n, 2.0, to_dev(h), to_dev(N))
    u, info = plan.solve(tol=1e-6, raise_on_failure=False)
    assert info["returned"] == ORI_ERR_NONFINITE


def test_maxit_zero_returns_not_converged_with_zero_iterate():
    from paper_1602_04691_gb300 import Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_NOT_CONVERGED
    n = 8
    h, N = inputs.random_h_N(n, 705)
    plan = Plan(n, 1.0, to_dev(h), to_dev(N))
    u, info = plan.solve(tol=1e-6, precision="fp64", maxit=0, raise_on_failure=False)
    assert info["returned"] == ORI_ERR_NOT_CONVERGED and info["iters"] == 0
    assert float(u.abs().max()) == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cocg_breakdown_is_reported_with_finite_iterate(precision):
    """COCG's bilinear form r^T r is no norm: a nonzero residual can have
    r^T r = 0.  With h = 1 and N = 1 (S = 1 exactly) and b = e_0 + i e_1, the
    first residual S b has r^T r = 1 + i^2 = 0 exactly (also after the mixed
    solver scales it to unit norm in FP32), and rho = r^T r is the divisor of
    beta: the breakdown of COCG, found before the first step.  The solve
    reports ORI_ERR_BREAKDOWN and returns a finite iterate; the plan keeps
    working."""
    from paper_1602_04691_gb300 import Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_BREAKDOWN
    n = 6
    h, N = inputs.constant_h_N(n, 1.0, 1.0)
    plan = Plan(n, 2.0, to_dev(h), to_dev(N))
    rhs = np.zeros(n ** 3, dtype=np.complex128)
    rhs[0], rhs[1] = 1.0, 1j
    u, info = plan.solve(rhs=to_dev(rhs), tol=1e-8, precision=precision, raise_on_failure=False)
    assert info["returned"] == ORI_ERR_BREAKDOWN and info["status"] == ORI_ERR_BREAKDOWN
    assert torch.isfinite(torch.view_as_real(u)).all()
    u, info = plan.solve(tol=1e-8, precision=precision)
    assert info["status"] == 0 and info["relres"] <= 1e-8
