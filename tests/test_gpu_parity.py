"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle.

Tolerances (relative L2):
* FP64 operator vs the oracle's direct sum: 1e-12.
* FP32 operator vs the oracle: 1e-5 (complex64 FFTs of length L <= 1024 with
  correctly rounded twiddles: a few units of 6e-8 times log2(L) per pass).
* Solves: compared with dense LU at n <= 12, the difference bounded by the
  residual tolerance times the condition number (checked with a margin).
"""

import math

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


def make_plan(n, k, h, N, side=1.0, origin=(0.0, 0.0, 0.0)):
    from paper_1602_04691_gb300 import Plan
    return Plan(n, k, to_dev(h), to_dev(N), side=side, origin=origin)


# ---------------------------------------------------------------------------
# Operator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [2, 3, 4, 5, 7, 8, 12, 16, 17])
def test_fp64_matvec_A_vs_direct_sum(n):
    k, side = 2.3, 1.0
    h, N = inputs.random_h_N(n, 1000 + n)
    x = inputs.random_complex(n ** 3, 2000 + n)
    plan = make_plan(n, k, h, N, side)
    y = plan.matvec(to_dev(x), form="A", precision="fp64").cpu().numpy()
    ref = O.red_matvec_direct(x, n, k, h, N, side=side)
    assert rel(y, ref) < 1e-12


@pytest.mark.parametrize("n", [3, 8, 13])
def test_fp64_matvec_B_vs_direct_sum(n):
    k = 1.7
    h, N = inputs.random_h_N(n, 300 + n)
    x = inputs.random_complex(n ** 3, 400 + n)
    plan = make_plan(n, k, h, N, side=0.8, origin=(0.1, -0.2, 0.3))
    y = plan.matvec(to_dev(x), form="B", precision="fp64").cpu().numpy()
    ref = O.symmetrised_matvec_direct(x, n, k, h, N, side=0.8, origin=(0.1, -0.2, 0.3))
    assert rel(y, ref) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 8, 13, 16])
def test_df_matvec_vs_direct_sum(n):
    """Paired-FP32 (double-float) operator: held to the FP64 bar (1e-12)."""
    k = 3.3
    h, N = inputs.random_h_N(n, 700 + n)
    x = inputs.random_complex(n ** 3, 800 + n)
    plan = make_plan(n, k, h, N)
    yA = plan.matvec(to_dev(x), form="A", precision="df").cpu().numpy()
    yB = plan.matvec(to_dev(x), form="B", precision="df").cpu().numpy()
    assert rel(yA, O.red_matvec_direct(x, n, k, h, N)) < 1e-12
    assert rel(yB, O.symmetrised_matvec_direct(x, n, k, h, N)) < 1e-12


def test_df_matvec_sampled_rows_n64():
    n, k = 64, 5.0
    h, N = inputs.random_h_N(n, 3)
    x = inputs.random_complex(n ** 3, 17)
    plan = make_plan(n, k, h, N)
    y = plan.matvec(to_dev(x), form="A", precision="df").cpu().numpy()
    y64 = plan.matvec(to_dev(x), form="A", precision="fp64").cpu().numpy()
    rows = np.random.default_rng(18).choice(n ** 3, 64, replace=False)
    assert rel(y[rows], O.red_matvec_rows(x, rows, n, k, h, N)) < 1e-12
    assert rel(y, y64) < 1e-12


@pytest.mark.parametrize("n", [70, 130, 260])
def test_df_matvec_matches_fp64_large(n):
    """Paired-FP32 operator against the native FP64 one at L = 256, 512, 1024."""
    k = 5.0
    h, N = inputs.random_h_N(n, 40 + n)
    x = inputs.random_complex(n ** 3, 50 + n)
    plan = make_plan(n, k, h, N)
    xd = to_dev(x)
    for form in ("A", "B"):
        y = plan.matvec(xd, form=form, precision="df")
        y64 = plan.matvec(xd, form=form, precision="fp64")
        err = float(torch.linalg.vector_norm(y - y64) / torch.linalg.vector_norm(y64))
        assert err < 1e-12, (form, err)
    plan.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [4, 9, 16, 24])
def test_fp32_matvec_vs_direct_sum(n):
    k = 5.0
    h, N = inputs.random_h_N(n, 500 + n)
    x = inputs.random_complex(n ** 3, 600 + n)
    plan = make_plan(n, k, h, N)
    refA = O.red_matvec_direct(x, n, k, h, N)
    refB = O.symmetrised_matvec_direct(x, n, k, h, N)
    yA = plan.matvec(to_dev(x), form="A", precision="fp32").cpu().numpy()
    yB = plan.matvec(to_dev(x), form="B", precision="fp32").cpu().numpy()
    assert rel(yA, refA) < 1e-5
    assert rel(yB, refB) < 1e-5
    y32 = plan.matvec32(to_dev(x.astype(np.complex64)), form="B").cpu().numpy()
    assert rel(y32, refB) < 1e-5


def test_fp64_matvec_sampled_rows_n64():
    """Config-2 grid (n = 64, 128^3 FFT buffers): 256 sampled rows of the
    direct sum (each an O(N) sum in the oracle)."""
    n, k = 64, 2.0
    h, N = inputs.random_h_N(n, 2)
    x = inputs.random_complex(n ** 3, 7)
    plan = make_plan(n, k, h, N)
    y = plan.matvec(to_dev(x), form="A", precision="fp64").cpu().numpy()
    rows = np.random.default_rng(8).choice(n ** 3, 256, replace=False)
    ref = O.red_matvec_rows(x, rows, n, k, h, N)
    assert rel(y[rows], ref) < 1e-12


@pytest.mark.parametrize("n", [128])
def test_fp32_matvec_sampled_rows_large(n):
    """FP32 B-form operator at n = 128 (configurations 4 and 5) on sampled rows
    the oracle computes one by one (n = 512: test_gpu_headline.py)."""
    k = 5.0
    h, N = inputs.random_h_N(n, 3)
    x = inputs.random_complex(n ** 3, 9).astype(np.complex64)
    plan = make_plan(n, k, h, N)
    y = plan.matvec32(to_dev(x), form="B").cpu().numpy()
    rng = np.random.default_rng(10)
    rows = np.concatenate([[0, n ** 3 - 1, n * n * (n // 2) + n * (n // 2) + n // 2],
                           rng.choice(n ** 3, 5 if n > 128 else 40, replace=False)])
    S = O.sqrt_hN(h, N)
    xs = S * x.astype(np.complex128)
    d = 1.0 / n
    Kxs = (O.C_S_SPHERE * d ** 3) * O.offdiag_sum_rows_grid(xs, rows, n, k)
    ref = x[rows] + S[rows] * Kxs
    assert rel(y[rows], ref) < 1e-5
    del plan
    torch.cuda.empty_cache()


def test_matvec_linear_and_deterministic():
    n, k = 10, 3.0
    h, N = inputs.random_h_N(n, 11)
    x = inputs.random_complex(n ** 3, 12)
    z = inputs.random_complex(n ** 3, 13)
    plan = make_plan(n, k, h, N)
    a = plan.matvec(to_dev(x), "A", "fp64").cpu().numpy()
    b = plan.matvec(to_dev(z), "A", "fp64").cpu().numpy()
    c = plan.matvec(to_dev(2 * x - 1j * z), "A", "fp64").cpu().numpy()
    assert rel(c, 2 * a - 1j * b) < 1e-13
    a2 = plan.matvec(to_dev(x), "A", "fp64").cpu().numpy()
    assert np.array_equal(a, a2)


# ---------------------------------------------------------------------------
# Solves
# ---------------------------------------------------------------------------

def test_config1_fp64_solve_vs_lu():
    """n = 12 (P = 1728), unit cube, k = 1, h = 1+1i, N = 1, alpha = (0,0,1):
    GPU FP64 COCG to relres 1e-12 against dense LU."""
    n, k = 12, 1.0
    h, N = inputs.constant_h_N(n, 1 + 1j, 1.0)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-12, precision="fp64")
    u_lu = O.solve_dense(O.red_matrix(n, k, h, N), O.plane_wave(O.cell_centres(n), k))
    assert info["relres"] <= 1e-11
    assert rel(u.cpu().numpy(), u_lu) < 1e-9


@pytest.mark.parametrize("precision,tol,bound,residual", [("fp64", 1e-11, 1e-9, "df"), ("mixed", 1e-6, 2e-5, "df"),
                                                          ("mixed", 1e-6, 2e-5, "fp64"), ("mixed", 1e-10, 1e-8, "df")])
def test_variable_medium_solve_vs_lu(precision, tol, bound, residual):
    n, k = 10, 2.0
    h, N = inputs.random_h_N(n, 2)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=tol, precision=precision, residual=residual)
    u_lu = O.solve_dense(O.red_matrix(n, k, h, N), O.plane_wave(O.cell_centres(n), k))
    assert info["relres"] <= tol
    assert rel(u.cpu().numpy(), u_lu) < bound


def test_config2_fp64_solve_rows_n64():
    """n = 64, k = 2, seeded h and N, FP64 to relres 1e-10: the oracle checks the
    residual of Eq. 2.19 on sampled rows by direct summation."""
    n, k = 64, 2.0
    h, N = inputs.random_h_N(n, 2)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-10, precision="fp64")
    u = u.cpu().numpy()
    assert info["relres"] <= 1e-10
    rows = np.random.default_rng(22).choice(n ** 3, 128, replace=False)
    u0 = O.plane_wave(O.cell_centres(n), k)
    Au = O.red_matvec_rows(u, rows, n, k, h, N)
    # |S|-weighted residual of the original system on the sampled rows
    assert np.linalg.norm(Au - u0[rows]) / np.linalg.norm(u0[rows]) < 1e-8


def test_fp64_solve_vs_oracle_fft_cocg_n24():
    n, k = 24, 2.0
    h, N = inputs.random_h_N(n, 24)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-10, precision="fp64")
    u_or, it, rr = O.solve_red_cocg_fft(n, k, h, N, tol=1e-10)
    assert rel(u.cpu().numpy(), u_or) < 1e-8


@pytest.mark.parametrize("residual", ["df", "fp64"])
def test_mixed_vs_fp64_n32(residual):
    n, k = 32, 5.0
    h, N = inputs.random_h_N(n, 3)
    plan = make_plan(n, k, h, N)
    u64, i64 = plan.solve(tol=1e-10, precision="fp64")
    um, im = plan.solve(tol=1e-6, precision="mixed", residual=residual)
    assert im["relres"] <= 1e-6
    assert im["outer_iters"] >= 1 and im["fp64_matvecs"] >= 1
    assert rel(um.cpu().numpy(), u64.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("resid_update", [True, False])
def test_mixed_residual_is_certified(resid_update):
    """The mixed solve's reported residual (and bound) agrees with an independent
    FP64 evaluation of ||S u0 - B (S u)|| / ||S u0|| from the returned u."""
    n, k = 40, 5.0
    h, N = inputs.random_h_N(n, 41)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-6, precision="mixed", resid_update=resid_update)
    S = O.sqrt_hN(h, N)
    u0 = O.plane_wave(O.cell_centres(n), k)
    w = S * u.cpu().numpy()
    Bw = plan.matvec(to_dev(w), form="B", precision="fp64").cpu().numpy()
    true_rel = np.linalg.norm(S * u0 - Bw) / np.linalg.norm(S * u0)
    assert true_rel <= 1e-6
    assert abs(true_rel - info["relres"]) <= info["relres_bound"] + 1e-12
    if resid_update:
        assert info["resid_updates"] >= 1 and info["fp64_matvecs"] == 1
    else:
        assert info["resid_updates"] == 0


def test_zero_impedance_returns_incident_field():
    n, k = 6, 1.5
    h, N = inputs.constant_h_N(n, 0.0, 1.0)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-8, precision="mixed")
    u0 = O.plane_wave(O.cell_centres(n), k)
    assert info["iters"] == 0
    assert rel(u.cpu().numpy(), u0) < 1e-15


def test_zero_density_cells_recovered():
    n, k = 6, 1.3
    h, N = inputs.random_h_N(n, 61)
    N[::3] = 0.0
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-12, precision="fp64")
    u_lu = O.solve_dense(O.red_matrix(n, k, h, N), O.plane_wave(O.cell_centres(n), k))
    assert rel(u.cpu().numpy(), u_lu) < 1e-9


def test_user_rhs_and_direction():
    n, k = 8, 2.5
    h, N = inputs.random_h_N(n, 71)
    plan = make_plan(n, k, h, N, side=2.0, origin=(-1.0, -1.0, -1.0))
    alpha = np.array([0.48, 0.6, 0.64])
    pos = O.cell_centres(n, (-1.0, -1.0, -1.0), 2.0)
    u1, _ = plan.solve(tol=1e-12, precision="fp64", alpha=tuple(alpha))
    u2, _ = plan.solve(rhs=to_dev(O.plane_wave(pos, k, alpha)), tol=1e-12, precision="fp64")
    A = O.red_matrix(n, k, h, N, origin=(-1.0, -1.0, -1.0), side=2.0)
    u_lu = O.solve_dense(A, O.plane_wave(pos, k, alpha))
    assert rel(u1.cpu().numpy(), u_lu) < 1e-9
    assert rel(u2.cpu().numpy(), u_lu) < 1e-9


def test_maxit_reports_not_converged_with_iterate():
    from paper_1602_04691_gb300._lib import ORI_ERR_NOT_CONVERGED
    n, k = 10, 4.0
    h, N = inputs.random_h_N(n, 81)
    plan = make_plan(n, k, h, N)
    u, info = plan.solve(tol=1e-14, precision="fp64", maxit=3, raise_on_failure=False)
    assert info["returned"] == ORI_ERR_NOT_CONVERGED
    assert info["iters"] <= 3 + 8
    assert np.all(np.isfinite(u.cpu().numpy()))


def test_solve_is_deterministic():
    n, k = 12, 3.0
    h, N = inputs.random_h_N(n, 91)
    plan = make_plan(n, k, h, N)
    a, ia = plan.solve(tol=1e-8, precision="mixed")
    b, ib = plan.solve(tol=1e-8, precision="mixed")
    assert ia["iters"] == ib["iters"]
    assert torch.equal(a, b)


def test_graph_and_plain_launches_agree():
    n, k = 12, 3.0
    h, N = inputs.random_h_N(n, 92)
    plan = make_plan(n, k, h, N)
    a, ia = plan.solve(tol=1e-9, precision="fp64", use_graph=True)
    b, ib = plan.solve(tol=1e-9, precision="fp64", use_graph=False)
    assert ia["iters"] == ib["iters"]
    assert torch.equal(a, b)


# ---------------------------------------------------------------------------
# Adjoint gradient
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,bound", [("fp64", 1e-8), ("mixed", 1e-4)])
def test_adjoint_gradient_vs_dense_oracle(precision, bound):
    n, k = 5, 1.6
    h, N = inputs.random_h_N(n, 71)
    obs = inputs.observation_cells(n, 12, 5)
    target = O.plane_wave(O.cell_centres(n), k)[obs]
    u_ref, J, gh_ref, gN_ref = O.adjoint_gradient_dense(n, k, h, N, obs, target)
    plan = make_plan(n, k, h, N)
    tol = 1e-12 if precision == "fp64" else 1e-8
    u, _ = plan.solve(tol=tol, precision=precision)
    un = u.cpu().numpy()
    ec = np.zeros(n ** 3, dtype=np.complex128)
    ec[obs] = np.conj(un[obs] - target)
    gh, gN, info = plan.adjoint(u, to_dev(ec), tol=tol, precision=precision)
    assert rel(gh.cpu().numpy(), gh_ref) < bound
    assert rel(gN.cpu().numpy(), gN_ref) < bound


def test_adjoint_and_solve_take_lazy_conjugate_views():
    """Plan.adjoint with econj = e.conj() (a lazy view over e's memory) and
    Plan.solve with rhs = v.conj() give the results of materialised inputs."""
    n, k = 5, 1.6
    h, N = inputs.random_h_N(n, 71)
    obs = inputs.observation_cells(n, 12, 5)
    target = O.plane_wave(O.cell_centres(n), k)[obs]
    u_ref, J, gh_ref, gN_ref = O.adjoint_gradient_dense(n, k, h, N, obs, target)
    plan = make_plan(n, k, h, N)
    u, _ = plan.solve(tol=1e-12, precision="fp64")
    e = torch.zeros_like(u)
    e[torch.from_numpy(obs).to(DEV)] = u[torch.from_numpy(obs).to(DEV)] - to_dev(target)
    lazy = e.conj()
    assert lazy.is_conj()
    gh, gN, _ = plan.adjoint(u, lazy, tol=1e-12, precision="fp64")
    assert rel(gh.cpu().numpy(), gh_ref) < 1e-8
    assert rel(gN.cpu().numpy(), gN_ref) < 1e-8
    v = to_dev(np.random.default_rng(8).standard_normal(n ** 3) + 1j)
    a, _ = plan.solve(rhs=v.conj(), tol=1e-12, precision="fp64")
    b, _ = plan.solve(rhs=v.conj().resolve_conj(), tol=1e-12, precision="fp64")
    assert torch.equal(a, b)
    with pytest.raises(ValueError):
        plan.solve(out=torch.empty(n ** 3, dtype=torch.complex128, device=DEV).conj())


def test_autograd_function_matches_oracle():
    from paper_1602_04691_gb300 import solve_autograd
    n, k = 4, 2.0
    h, N = inputs.random_h_N(n, 33)
    obs = np.array([0, 5, 21, 40, 63])
    target = np.zeros(obs.size, dtype=np.complex128)
    u_ref, J_ref, gh_ref, gN_ref = O.adjoint_gradient_dense(n, k, h, N, obs, target)
    plan = make_plan(n, k, h, N)
    ht = to_dev(h).requires_grad_(True)
    Nt = to_dev(N).requires_grad_(True)
    u = solve_autograd(plan, ht, Nt, tol=1e-12, precision="fp64")
    J = (u[torch.from_numpy(obs).to(DEV)].abs() ** 2).sum()
    J.backward()
    assert abs(J.item() - J_ref) < 1e-10 * abs(J_ref)
    assert rel(ht.grad.cpu().numpy(), gh_ref) < 1e-8
    assert rel(Nt.grad.cpu().numpy(), gN_ref) < 1e-8


def test_autograd_backward_uses_its_own_forward_medium():
    """Two differentiable solves on one plan with different media, then the
    backward of the first: its gradients are those of a lone forward-backward
    with the first medium (the backward restores the medium it needs)."""
    from paper_1602_04691_gb300 import solve_autograd
    n, k = 4, 2.0
    h1, N1 = inputs.random_h_N(n, 33)
    h2, N2 = inputs.random_h_N(n, 34)
    obs = torch.tensor([0, 5, 21, 40, 63], device=DEV)
    plan = make_plan(n, k, h1, N1)
    ha = to_dev(h1).requires_grad_(True)
    Na = to_dev(N1).requires_grad_(True)
    ua = solve_autograd(plan, ha, Na, tol=1e-12, precision="fp64")
    (ua[obs].abs() ** 2).sum().backward()
    ref_h, ref_N = ha.grad.clone(), Na.grad.clone()
    hb = to_dev(h1).requires_grad_(True)
    Nb = to_dev(N1).requires_grad_(True)
    ub = solve_autograd(plan, hb, Nb, tol=1e-12, precision="fp64")
    hc = to_dev(h2).requires_grad_(True)
    Nc = to_dev(N2).requires_grad_(True)
    uc = solve_autograd(plan, hc, Nc, tol=1e-12, precision="fp64")
    (ub[obs].abs() ** 2).sum().backward()
    assert rel(hb.grad.cpu().numpy(), ref_h.cpu().numpy()) < 1e-12
    assert rel(Nb.grad.cpu().numpy(), ref_N.cpu().numpy()) < 1e-12
    (uc[obs].abs() ** 2).sum().backward()
    _, _, gh2, gN2 = O.adjoint_gradient_dense(n, k, h2, N2, obs.cpu().numpy(), np.zeros(5, dtype=np.complex128))
    assert rel(hc.grad.cpu().numpy(), gh2) < 1e-8
    assert rel(Nc.grad.cpu().numpy(), gN2) < 1e-8
