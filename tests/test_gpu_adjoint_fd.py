"""Adjoint gradient against central finite differences at n = 128.

Configuration: n = 128, k = 2, h and N drawn with seed 5, J = sum over 1024
observation cells of |u_o - t_o|^2 with t = u0 (the scattered-field energy),
64 random cells checked in the three directions Re h, Im h and N.

One cell changes J by ~1e-11 relative, so perturbed solves are not
differenced directly.  For a change of cell p, A(h') - A(h) = K diag(delta_p)
has a single column, c_S |Delta| G_off(:, p) times the change of h_p N_p,
which one FP64 A-form matvec of the unit vector e_p gives without
cancellation: A e_p - e_p.  The perturbed solution is u + d with
A(h') d = -(A(h') - A(h)) u (the base residual drops out of the central
difference to first order), and J(h') - J(h) = sum_obs 2 Re(conj(e) d) + |d|^2.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1602_04691_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_adjoint_gradient_vs_central_differences_n128():
    from paper_1602_04691_gb300 import Plan
    n, k = 128, 2.0
    h_np, N_np = inputs.random_h_N(n, 5)
    h = torch.from_numpy(h_np).to(DEV)
    N = torch.from_numpy(N_np).to(DEV)
    obs = torch.from_numpy(inputs.observation_cells(n, 1024, 5)).to(DEV)
    cells = np.random.default_rng(55).choice(n ** 3, 64, replace=False)
    plan = Plan(n, k, h, N)
    u, info = plan.solve(tol=1e-12, precision="fp64")
    assert info["relres"] <= 1e-12
    # target: the incident wave on the observation cells (J = scattered-field energy)
    u0 = torch.from_numpy(O.plane_wave(O.cell_centres(n), k)).to(DEV)
    e = torch.zeros_like(u)
    e[obs] = u[obs] - u0[obs]
    econj = e.conj().contiguous()
    gh, gN, ia = plan.adjoint(u, econj, tol=1e-12, precision="fp64")
    gh_m, gN_m, _ = plan.adjoint(u, econj, tol=1e-8, precision="mixed")
    # mixed-precision gradients against FP64 gradients
    assert float(torch.linalg.vector_norm(gh_m - gh) / torch.linalg.vector_norm(gh)) < 1e-4
    assert float(torch.linalg.vector_norm(gN_m - gN) / torch.linalg.vector_norm(gN)) < 1e-4

    def dJ(d):
        dd = d[obs]
        return float((2.0 * (econj[obs] * dd).real + dd.abs() ** 2).sum())

    fd_h, fd_N, ad_h, ad_N = [], [], [], []
    for p in cells:
        ep = torch.zeros_like(u)
        ep[p] = 1.0
        col = plan.matvec(ep, form="A", precision="fp64") - ep   # c_S |Delta| G_off(:, p) h_p N_p
        hp, Np, up = h[p].item(), N[p].item(), u[p].item()
        grads = []
        for direction in ("re", "im", "N"):
            step = 1e-4 * (abs(hp) if direction != "N" else Np)
            diffs = []
            for s in (+1.0, -1.0):
                h2, N2 = h.clone(), N.clone()
                if direction == "re":
                    h2[p] = hp + s * step
                elif direction == "im":
                    h2[p] = hp + 1j * s * step
                else:
                    N2[p] = Np + s * step
                dw = h2[p].item() * N2[p].item() - hp * Np          # change of h_p N_p
                rhs = -(col * (dw / (hp * Np) * up)).contiguous()
                plan.set_medium(h2, N2)
                d, di = plan.solve(rhs=rhs, tol=1e-10, precision="mixed")
                assert di["status"] == 0
                diffs.append(dJ(d))
            grads.append((diffs[0] - diffs[1]) / (2.0 * step))
        plan.set_medium(h, N)
        fd_h.append(complex(grads[0], grads[1]))
        fd_N.append(grads[2])
        ad_h.append(gh[p].item())
        ad_N.append(gN[p].item())
    fd_h, ad_h, fd_N, ad_N = map(np.array, (fd_h, ad_h, fd_N, ad_N))
    assert np.linalg.norm(fd_h - ad_h) / np.linalg.norm(ad_h) < 1e-4
    assert np.linalg.norm(fd_N - ad_N) / np.linalg.norm(ad_N) < 1e-4
