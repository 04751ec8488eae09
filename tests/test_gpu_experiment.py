"""Section 4's experiment on the GPU, and the field of Eq. 2.10.

* ori_field against the oracle's direct sum of Eq. 2.10 (off-grid points,
  points on the grid where it returns the effective field of Eq. 2.14).
* The Table 4 difference of GPU solutions of (RED, n = 20) and (IE, n = 40)
  with the Section 4 parameters against the oracle's solutions and metric,
  and against the printed value.
* A scaled (ORI) system (n = 240, nested with both) meeting relres 1e-6, its
  differences to (RED) and (IE) equal to the plane-wave estimate.
"""

import numpy as np
import pytest
import torch

import oracle as O
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


def test_field_matches_oracle_direct_sum():
    from paper_1602_04691_gb300 import Plan
    n, k, side, origin = 10, 2.2, 1.3, (0.2, -0.1, 0.05)
    h, N = inputs.random_h_N(n, 501)
    u = inputs.random_complex(n ** 3, 502)
    rng = np.random.default_rng(503)
    off = rng.uniform(-0.5, 2.0, size=(300, 3))
    on = O.cell_centres(n, origin, side)[rng.choice(n ** 3, 40, replace=False)]
    pts = np.concatenate([off, on])
    plan = Plan(n, k, to_dev(h), to_dev(N), side=side, origin=origin)
    alpha = (0.3, -0.4, 0.5)
    for a in (None, alpha):
        got = plan.field(to_dev(u), to_dev(pts), alpha=a).cpu().numpy()
        ref = O.field(pts, u, n, k, h, N, alpha=a, origin=origin, side=side)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_field_at_grid_points_is_the_solution():
    """At the cell points Eq. 2.10 (own cell left out) is Eq. 2.14, which the
    converged FP64 solution satisfies to its residual."""
    from paper_1602_04691_gb300 import Plan
    n, k = 9, 3.0
    h, N = inputs.random_h_N(n, 504)
    plan = Plan(n, k, to_dev(h), to_dev(N))
    u, info = plan.solve(tol=1e-12, precision="fp64", alpha=(0.0, 1.0, 0.0))
    pts = to_dev(O.cell_centres(n))
    f = plan.field(u, pts, alpha=(0.0, 1.0, 0.0))
    assert float((f - u).abs().max()) < 1e-9


def _oracle_solution(n):
    from paper_1602_04691_gb300 import experiment as E
    org = E.vertex_origin(n)
    u, _, _ = O.solve_red_cocg_fft(n, E.K, np.full(n ** 3, E.H), np.ones(n ** 3), alpha=E.ALPHA,
                                   origin=org, tol=1e-12)
    return u, O.cell_centres(n, org)


def test_section4_red_vs_ie_matches_oracle_and_table4():
    from paper_1602_04691_gb300 import experiment as E
    gpu = {}
    for n in (20, 40):
        u, info, plan = E.solve(n, DEV, tol=1e-11, precision="fp64")
        assert info["relres"] <= 1e-11
        gpu[n] = u
        plan.close()
    ored, pred = _oracle_solution(20)
    oie, pie = _oracle_solution(40)
    assert np.linalg.norm(gpu[20].cpu().numpy() - ored) / np.linalg.norm(ored) < 1e-9
    assert np.linalg.norm(gpu[40].cpu().numpy() - oie) / np.linalg.norm(oie) < 1e-9
    v_gpu = E.table4_difference(gpu[40], 40, gpu[20], 20)
    v_ora = O.table4_difference(oie, pie, ored, 20)
    assert abs(v_gpu - v_ora) < 1e-10
    assert abs(v_gpu - E.PRINTED_TABLE4["red_vs_ie"]) <= 1e-4
    # the vertex grid of the module is the oracle's grid with origin -d/2
    assert np.allclose(E.grid_points(40, DEV).cpu().numpy(), pie, atol=1e-15)


def test_section4_scaled_ori_against_red_and_ie():
    from paper_1602_04691_gb300 import experiment as E
    sols = {}
    for n in (20, 40, 240):
        u, info, plan = E.solve(n, DEV, tol=1e-6, precision="mixed")
        assert info["status"] == 0 and info["relres"] <= 1e-6
        sols[n] = u
        plan.close()
    for nf, nc in ((240, 20), (240, 40)):
        v = E.table4_difference(sols[nf], nf, sols[nc], nc)
        assert abs(v - E.plane_wave_estimate(nf, nc)) < 2e-5, (nf, nc, v)
