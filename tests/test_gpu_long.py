"""Padded length L = 2048: the pipelined FP32 passes, the shared-memory radix-8
passes of FP64 and paired FP32, and the radix-8 TILES schedules of FP32 Y and Z.

Grids of n >= 513 (up to the paper-scale n = 1000) pad to L = 2048.  The plan
option min_L forces that length on small grids, where the oracle's direct
sum and dense LU check every output; a natural n = 520 grid is checked on
rows per tile class in test_gpu_headline.py.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1602_04691_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def long_plan():
    from paper_1602_04691_gb300 import Plan
    n, k = 12, 2.4
    h, N = inputs.random_h_N(n, 601)
    plan = Plan(n, k, to_dev(h), to_dev(N), min_L=2048)
    assert plan.L == 2048
    yield n, k, h, N, plan
    plan.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision,form,bound", [("fp64", "A", 1e-12), ("df", "A", 1e-12), ("fp32", "A", 1e-5),
                                                  ("fp64", "B", 1e-12), ("fp32", "B", 1e-5)])
def test_L2048_matvec_vs_direct_sum(long_plan, precision, form, bound):
    n, k, h, N, plan = long_plan
    x = inputs.random_complex(n ** 3, 602)
    y = plan.matvec(to_dev(x), form=form, precision=precision).cpu().numpy()
    if form == "A":
        ref = O.red_matvec_direct(x, n, k, h, N)
    else:
        ref = O.symmetrised_matvec_direct(x, n, k, h, N)
    assert rel(y, ref) < bound


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-11, 1e-9), ("mixed", 1e-6, 2e-5)])
def test_L2048_solve_vs_lu(long_plan, precision, tol, bound):
    n, k, h, N, plan = long_plan
    u, info = plan.solve(tol=tol, precision=precision)
    assert info["status"] == 0 and info["relres"] <= tol
    u_lu = O.solve_dense(O.red_matrix(n, k, h, N), O.plane_wave(O.cell_centres(n), k))
    assert rel(u.cpu().numpy(), u_lu) < bound


def test_L2048_batch_vs_single(long_plan):
    n, k, h, N, plan = long_plan
    dirs = [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0)]
    ub, infos = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
    for j, a in enumerate(dirs):
        us, _ = plan.solve(tol=1e-10, precision="fp64", alpha=a)
        assert infos[j]["relres"] <= 1e-6
        assert rel(ub[0, j].cpu().numpy(), us.cpu().numpy()) < 1e-5


def test_L2048_fp32_pipelined_and_radix8_kernels_agree(long_plan):
    """At L = 2048 the FP32 Y forward, Z and Y inverse passes run the pipelined
    kernels (a 64-point stage with a zero-padded half or half its outputs kept,
    8-column tiles); the TILES schedule keeps the radix-8 shared-memory kernels.
    Both against the direct sum, and the default schedule restored afterwards."""
    from paper_1602_04691_gb300._lib import ORI_SCHED_TILES
    n, k, h, N, plan = long_plan
    x = inputs.random_complex(n ** 3, 606)
    ref = O.symmetrised_matvec_direct(x, n, k, h, N)
    xd = to_dev(x.astype(np.complex64))
    default = plan.schedule()
    y_pipe = plan.matvec32(xd, form="B").cpu().numpy()
    plan.set_schedule(dict(default, yfwd=ORI_SCHED_TILES, zconv=ORI_SCHED_TILES, yinv=ORI_SCHED_TILES))
    try:
        y_tiles = plan.matvec32(xd, form="B").cpu().numpy()
    finally:
        plan.set_schedule(default)
    assert rel(y_pipe, ref) < 1e-5
    assert rel(y_tiles, ref) < 1e-5
    assert rel(y_pipe, y_tiles) < 1e-5


def test_lean_plan_matches_full_plan_and_rejects_the_rest():
    """A lean plan (mixed solves only; the paper-scale memory budget) gives the
    full plan's solutions, holds less memory, and refuses what it cannot do."""
    from paper_1602_04691_gb300 import OriError, Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_UNSUPPORTED
    n, k = 16, 3.0
    h, N = inputs.random_h_N(n, 605)
    full = Plan(n, [k, 1.5], to_dev(h), to_dev(N))
    lean = Plan(n, [k, 1.5], to_dev(h), to_dev(N), lean=True)
    assert lean.bytes < full.bytes
    uf, _ = full.solve(tol=1e-6, precision="mixed")
    ul, il = lean.solve(tol=1e-6, precision="mixed")
    assert il["relres"] <= 1e-6
    assert rel(ul.cpu().numpy(), uf.cpu().numpy()) < 1e-13
    dirs = [(0.0, 0.0, 1.0), (0.0, 1.0, 1.0)]
    bf, _ = full.solve_batch(dirs, tol=1e-6, precision="mixed")
    bl, _ = lean.solve_batch(dirs, tol=1e-6, precision="mixed")
    assert rel(bl.cpu().numpy(), bf.cpu().numpy()) < 1e-13
    x = to_dev(inputs.random_complex(n ** 3, 606))
    for prec in ("fp32", "df"):
        assert rel(lean.matvec(x, form="B", precision=prec).cpu().numpy(),
                   full.matvec(x, form="B", precision=prec).cpu().numpy()) < 1e-15
    calls = [lambda: lean.matvec(x, form="A", precision="fp32"),
             lambda: lean.matvec(x, form="B", precision="fp64"),
             lambda: lean.solve(tol=1e-6, precision="fp64"),
             lambda: lean.solve(tol=1e-6, precision="mixed", residual="fp64"),
             lambda: lean.field(ul, to_dev(np.zeros((1, 3))))]
    for call in calls:
        with pytest.raises(OriError) as e:
            call()
        assert e.value.status == ORI_ERR_UNSUPPORTED
    full.close()
    lean.close()


def test_lean_plan_rejects_zero_impedance_cells():
    from paper_1602_04691_gb300 import OriError, Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_UNSUPPORTED
    n = 8
    h, N = inputs.random_h_N(n, 607)
    N[5] = 0.0
    with pytest.raises(OriError) as e:
        Plan(n, 1.0, to_dev(h), to_dev(N), lean=True)
    assert e.value.status == ORI_ERR_UNSUPPORTED
