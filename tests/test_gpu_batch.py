"""Batched solves: several wave numbers x several incidence directions in one batch.

Each system of a batch (wave number k_i, direction alpha_j) is the system of
Eq. 2.19 with the plane wave of Eq. 2.4; the batch must give what separate
solves give.  Checks: dense LU from the oracle at small n, the oracle's
direct-sum residual on sampled rows at n = 128 (16 directions x 4 wave
numbers), agreement with single-system solves, masking of systems that
converge early, and bitwise repeatability when the batch size changes in
between (the captured graphs are rebuilt).
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


def unit(a):
    a = np.asarray(a, dtype=np.float64)
    return a / np.linalg.norm(a)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def make_plan(n, k, h, N, **kw):
    from paper_1602_04691_gb300 import Plan
    return Plan(n, k, to_dev(h), to_dev(N), **kw)


@pytest.mark.parametrize("precision,tol,bound", [("fp64", 1e-12, 1e-9), ("mixed", 1e-6, 2e-5)])
def test_batch_plane_waves_vs_lu(precision, tol, bound):
    n, ks = 8, [1.0, 2.5]
    dirs = [(0.0, 0.0, 1.0), (1.0, 1.0, 0.0), (-0.3, 0.5, 0.8)]
    h, N = inputs.random_h_N(n, 81)
    plan = make_plan(n, ks, h, N)
    u, infos = plan.solve_batch(dirs, tol=tol, precision=precision)
    u = u.cpu().numpy()
    pos = O.cell_centres(n)
    for i, k in enumerate(ks):
        A = O.red_matrix(n, k, h, N)
        for j, a in enumerate(dirs):
            info = infos[i * len(dirs) + j]
            assert info["status"] == 0 and info["relres"] <= tol
            u_lu = O.solve_dense(A, O.plane_wave(pos, k, unit(a)))
            assert rel(u[i, j], u_lu) < bound, (i, j)


def test_batch_user_rhs_vs_lu():
    n, k = 10, 2.0
    h, N = inputs.random_h_N(n, 91)
    rhs = np.stack([inputs.random_complex(n ** 3, 910 + j) for j in range(3)])
    plan = make_plan(n, k, h, N)
    u, infos = plan.solve_batch(rhs=to_dev(rhs), tol=1e-12, precision="fp64")
    A = O.red_matrix(n, k, h, N)
    for j in range(3):
        assert rel(u[0, j].cpu().numpy(), O.solve_dense(A, rhs[j])) < 1e-9


def test_batch_matches_single_solves():
    """Every system of a mixed batch agrees with its own FP64 single solve."""
    n, ks = 20, [2.0, 5.0]
    dirs = inputs.fibonacci_directions(4)
    h, N = inputs.random_h_N(n, 92)
    plan = make_plan(n, ks, h, N)
    ub, infos = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
    for i, k in enumerate(ks):
        single = make_plan(n, k, h, N)
        for j, a in enumerate(dirs):
            us, _ = single.solve(tol=1e-10, precision="fp64", alpha=tuple(a))
            assert infos[i * len(dirs) + j]["relres"] <= 1e-6
            assert rel(ub[i, j].cpu().numpy(), us.cpu().numpy()) < 1e-5, (i, j)
        single.close()


def test_batch_masks_converged_systems():
    """A zero right-hand side stops at once (u = 0, no iterations) and systems
    of different difficulty stop at their own iteration counts, each meeting tol."""
    n = 16
    ks = [0.5, 6.0]
    h, N = inputs.random_h_N(n, 93)
    pos = O.cell_centres(n)
    rhs = np.zeros((2, 2, n ** 3), dtype=np.complex128)
    rhs[0, 0] = O.plane_wave(pos, ks[0])
    rhs[1, 0] = O.plane_wave(pos, ks[1])
    rhs[1, 1] = O.plane_wave(pos, ks[1], unit((1.0, 0.0, 0.0)))
    plan = make_plan(n, ks, h, N)
    for precision, tol in [("fp64", 1e-10), ("mixed", 1e-6)]:
        u, infos = plan.solve_batch(rhs=to_dev(rhs), tol=tol, precision=precision)
        u = u.cpu().numpy()
        assert infos[1]["iters"] == 0 and np.all(u[0, 1] == 0)
        iters = [infos[r]["iters"] for r in (0, 2, 3)]
        assert iters[0] < iters[1], iters
        for r in (0, 2, 3):
            assert infos[r]["status"] == 0 and infos[r]["relres"] <= tol
        A0 = O.red_matrix(n, ks[0], h, N)
        assert rel(u[0, 0], O.solve_dense(A0, rhs[0, 0])) < (1e-7 if precision == "fp64" else 2e-5)


def test_batch_repeatable_across_batch_sizes():
    n, ks = 12, [1.5, 3.0]
    dirs = [(0.0, 0.0, 1.0), (0.0, 1.0, 0.0)]
    h, N = inputs.random_h_N(n, 94)
    plan = make_plan(n, ks, h, N)
    u1, _ = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
    u1 = u1.cpu().numpy().copy()
    plan.solve(tol=1e-6, precision="mixed")
    plan.solve_batch(dirs[:1], tol=1e-6, precision="mixed")
    u2, _ = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
    assert np.array_equal(u1, u2.cpu().numpy())


def test_batch_graph_and_plain_launches_agree():
    n, ks = 12, [2.0, 4.0]
    dirs = inputs.fibonacci_directions(3)
    h, N = inputs.random_h_N(n, 95)
    plan = make_plan(n, ks, h, N)
    ug, ig = plan.solve_batch(dirs, tol=1e-6, precision="mixed", use_graph=True)
    up, ip = plan.solve_batch(dirs, tol=1e-6, precision="mixed", use_graph=False)
    assert np.array_equal(ug.cpu().numpy(), up.cpu().numpy())
    assert [i["iters"] for i in ig] == [i["iters"] for i in ip]


def test_batch_16_directions_4_wave_numbers_n128():
    """n = 128, 16 directions spread on the sphere x k in {1, 2, 4, 8}: one
    mixed batch of 64 systems, each meeting relres 1e-6.  Sampled rows of
    Eq. 2.19 by direct summation (oracle) for three systems, and two systems
    against their own FP64 single solves."""
    n, ks = 128, [1.0, 2.0, 4.0, 8.0]
    dirs = inputs.fibonacci_directions(16)
    h, N = inputs.random_h_N(n, 4)
    plan = make_plan(n, ks, h, N)
    u, infos = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
    assert len(infos) == 64
    for r, info in enumerate(infos):
        assert info["status"] == 0 and info["relres"] <= 1e-6, (r, info)
    pos_rows = np.random.default_rng(128).choice(n ** 3, 48, replace=False)
    centres = O.cell_centres(n)
    for (i, j) in [(0, 0), (2, 7), (3, 15)]:
        k = ks[i]
        ui = u[i, j].cpu().numpy()
        Au = O.red_matvec_rows(ui, pos_rows, n, k, h, N)
        u0 = O.plane_wave(centres[pos_rows], k, unit(dirs[j]))
        assert np.linalg.norm(Au - u0) / np.linalg.norm(u0) < 1e-4, (i, j)
    for (i, j) in [(1, 3), (3, 9)]:
        single = make_plan(n, ks[i], h, N)
        us, _ = single.solve(tol=1e-9, precision="fp64", alpha=tuple(dirs[j]))
        assert rel(u[i, j].cpu().numpy(), us.cpu().numpy()) < 1e-5, (i, j)
        single.close()


def test_every_schedule_matches_oracle_and_autotune_caches(tmp_path):
    """Each launch schedule of the FP32 passes gives the FP32 operator within
    its tolerance of the oracle's direct sum and a batch that meets tol; the
    autotuner keeps one of them and a second call reads it from the cache."""
    n, ks = 24, [2.0, 3.0]                    # L = 64: both kernels exist per pass
    h, N = inputs.random_h_N(n, 96)
    x = inputs.random_complex(n ** 3, 97)
    ref = O.red_matvec_direct(x, n, ks[0], h, N)
    plan = make_plan(n, ks, h, N)
    default = plan.schedule()
    assert default == {"yfwd": 0, "zconv": 0, "yinv": 0, "ctas_per_sm": 0, "vec_ctas_per_sm": 8,
                       "yfwd_variant": 0, "zconv_variant": 0, "yinv_variant": 0}
    dirs = [(0.0, 0.0, 1.0), (0.6, 0.8, 0.0)]
    for y in (0, 1):
        for z in (0, 1):
            for yi in (0, 1):
                for cap, vec in ((0, 8), (1, 4), (2, 16)):
                    plan.set_schedule(dict(default, yfwd=y, zconv=z, yinv=yi, ctas_per_sm=cap, vec_ctas_per_sm=vec))
                    y32 = plan.matvec(to_dev(x), form="A", precision="fp32").cpu().numpy()
                    assert rel(y32, ref) < 1e-5, (y, z, yi, cap)
                    _, infos = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
                    assert all(i["status"] == 0 and i["relres"] <= 1e-6 for i in infos)
    path = str(tmp_path / "tune.json")
    r1 = plan.autotune(nrhs=4, path=path)
    assert not r1["cached"] and r1["ms"] > 0
    assert plan.schedule() == r1["schedule"]
    other = make_plan(n, ks, h, N)
    r2 = other.autotune(nrhs=4, path=path)
    assert r2["cached"] and other.schedule() == r1["schedule"]
    u, infos = other.solve_batch(dirs, tol=1e-6, precision="mixed")
    assert all(i["relres"] <= 1e-6 for i in infos)


def bulk_staged(sch):
    """1 when the FP32 Z pass runs the persistent kernel with 16-column tiles."""
    return int(sch["zconv"] == 0 and sch["zconv_variant"] != 1)


@pytest.mark.parametrize("n", [100, 200, 260])
def test_every_launch_variant_matches_oracle(n):
    """The tile-width and radix-split variants of the persistent FP32 Y-forward,
    Z and Y-inverse kernels at L = 256, 512 and 1024 (n = 100, 200, 260): each
    alone, and all at once, give the FP32 operator within 1e-5 of the oracle's
    direct sums on rows of every tile class; a mixed solve meets tol with
    them.  The 16-column Z tiles are staged by bulk copies (TMA): the plan's
    counters show it for every such variant and for every FP32 operator
    application of the solve."""
    k = 3.0
    h, N = inputs.random_h_N(n, 90 + n)
    x = inputs.random_complex(n ** 3, 91 + n).astype(np.complex64)
    plan = make_plan(n, k, h, N)
    assert plan.L in (256, 512, 1024)
    default = plan.schedule()
    rng = np.random.default_rng(n)
    rows = np.unique(np.concatenate([[0, n - 1, n * n - 1, n ** 3 - 1, n ** 3 - n, (n // 2) * (n * n + n + 1)],
                                     rng.choice(n ** 3, 24, replace=False)]))
    S = O.sqrt_hN(h, N)
    G = O.kernel_octant(n, k)
    ref = x[rows] + S[rows] * (O.C_S_SPHERE / n ** 3) * O.offdiag_sum_rows_octant(
        S * x.astype(np.complex128), rows, n, k, octant=G)
    xd = to_dev(x)
    schedules = [dict(default, **{f: v}) for f in ("yfwd_variant", "zconv_variant", "yinv_variant") for v in (1, 2)]
    schedules += [dict(default, yfwd_variant=v, zconv_variant=v, yinv_variant=v) for v in (1, 2)]
    for sch in [default] + schedules:
        plan.set_schedule(sch)
        plan.reset_stats()
        y = plan.matvec32(xd, form="B").cpu().numpy()
        assert rel(y[rows], ref) < 1e-5, sch
        # 16-column Z tiles stage their rows and spectrum slices by bulk copies
        st = plan.stats()
        assert st["fp32_matvecs"] == 1
        assert st["fp32_bulk_matvecs"] == bulk_staged(sch), sch
    plan.set_schedule(default)
    plan.reset_stats()
    _, info = plan.solve(tol=1e-6, precision="mixed")
    assert info["status"] == 0 and info["relres"] <= 1e-6
    st = plan.stats()
    assert st["fp32_matvecs"] > 0 and st["fp32_bulk_matvecs"] == st["fp32_matvecs"] * bulk_staged(default)
    plan.close()


def test_set_schedule_rejects_bad_fields():
    from paper_1602_04691_gb300 import OriError
    n = 8
    h, N = inputs.random_h_N(n, 98)
    plan = make_plan(n, 1.0, h, N)
    for bad in ({"yfwd": 2, "zconv": 0, "yinv": 0, "ctas_per_sm": 0, "vec_ctas_per_sm": 8},
                {"yfwd": 0, "zconv": 0, "yinv": 3, "ctas_per_sm": 0, "vec_ctas_per_sm": 8},
                {"yfwd": 0, "zconv": 0, "yinv": 0, "ctas_per_sm": -1, "vec_ctas_per_sm": 8},
                {"yfwd": 0, "zconv": 0, "yinv": 0, "ctas_per_sm": 0, "vec_ctas_per_sm": 17},
                {"yfwd": 0, "zconv": 0, "yinv": 0, "ctas_per_sm": 0, "vec_ctas_per_sm": 8, "zconv_variant": 1}):
        with pytest.raises(OriError):                # n = 8 pads to L = 16: variant 0 only
            plan.set_schedule(bad)
    assert plan.schedule()["vec_ctas_per_sm"] == 8


def test_warm_start_from_solution_and_from_a_perturbed_guess():
    """x0 (initial guess of u): the exact solution needs no refinement step;
    a perturbed solution converges to the same u in fewer iterations than a
    cold start; a zero right-hand side still gives u = 0."""
    n, k = 20, 4.0
    h, N = inputs.random_h_N(n, 97)
    plan = make_plan(n, k, h, N)
    for precision, tol in (("mixed", 1e-6), ("fp64", 1e-10)):
        uc, ic = plan.solve(tol=tol, precision=precision)
        ue, ie = plan.solve(tol=tol, precision=precision, x0=uc.clone())
        assert ie["relres"] <= tol and ie["fp64_matvecs"] >= 1
        if precision == "mixed":
            assert ie["iters"] == 0
        assert rel(ue.cpu().numpy(), uc.cpu().numpy()) < 10 * tol
        noise = torch.from_numpy(inputs.random_complex(n ** 3, 98)).to(DEV) * 1e-3
        up, ip = plan.solve(tol=tol, precision=precision, x0=uc + noise * uc.abs().mean())
        assert ip["relres"] <= tol and ip["iters"] < ic["iters"]
        assert rel(up.cpu().numpy(), uc.cpu().numpy()) < 100 * tol
    zero = torch.zeros(n ** 3, dtype=torch.complex128, device=DEV)
    uz, iz = plan.solve(rhs=zero, tol=1e-6, x0=torch.ones_like(zero))
    assert float(uz.abs().max()) == 0.0


def test_batch_warm_start_and_one_call_solve():
    from paper_1602_04691_gb300 import solve
    n, ks = 12, [1.5, 3.0]
    dirs = [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0)]
    h, N = inputs.random_h_N(n, 99)
    plan = make_plan(n, ks, h, N)
    ub, ib = plan.solve_batch(dirs, tol=1e-6, precision="mixed")
    uw, iw = plan.solve_batch(dirs, tol=1e-6, precision="mixed", x0=ub.reshape(-1).clone())
    assert all(i["iters"] == 0 and i["relres"] <= 1e-6 for i in iw)
    assert rel(uw.cpu().numpy(), ub.cpu().numpy()) < 1e-5
    u1, i1 = solve(to_dev(h), to_dev(N), ks[0], tol=1e-6, alpha=dirs[1])
    assert rel(u1.cpu().numpy(), ub[0, 1].cpu().numpy()) < 1e-5
