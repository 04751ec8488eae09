"""Pins of the CPU oracle against things other than itself.

Each test fixes a part of the oracle to a value printed in the paper, a
closed form, an invariant, a library routine that the special case reduces
to, or brute force on a tiny grid, so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from paper_1602_04691_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# --------------------------------------------------------------------------
# Section 3 padding example (printed integers)
# --------------------------------------------------------------------------

def test_padding_example_section3():
    g = _golden("padding_example.json")
    src = np.array(g["input"])
    G_pad = np.array([O.pad_kernel_mirror(row) for row in src])
    u_pad = O.pad_field_zero(src)
    assert np.array_equal(G_pad, np.array(g["G_padded"]))
    assert np.array_equal(u_pad, np.array(g["u_padded"]))
    # the padded G is a periodic, even signal: c[j] = c[L - j]
    L = G_pad.shape[1]
    for j in range(1, L):
        assert np.array_equal(G_pad[:, j], G_pad[:, L - j])


# --------------------------------------------------------------------------
# Section 4 recipe (printed values, 6 significant digits)
# --------------------------------------------------------------------------

def test_recipe_section4_values():
    g = _golden("recipe_section4.json")
    k = g["k"]
    assert abs(2 * math.pi * g["frequency_hz"] / g["speed_cm_per_s"] - k) < 5e-7
    h = complex(g["h_re"], g["h_im"])
    n = O.refraction_from_h(h, k, O.C_S_SPHERE, g["N"], complex(g["n0_re"], g["n0_im"]))
    assert abs(n - complex(g["n_re"], g["n_im"])) < 2e-6
    # the inverse recipe (Eq. 2.25-2.26) recovers h to the printed digits
    h_back = O.h_from_refraction(complex(g["n_re"], g["n_im"]), k)
    assert abs(h_back.real - h.real) / h.real < 2e-5
    assert abs(h_back.imag - h.imag) / h.imag < 2e-5
    # the branch matters: numpy's principal root gives the other sign
    principal = np.sqrt(1.0 - O.C_S_SPHERE * h / k ** 2)
    assert abs(principal + n) < 2e-6


def test_branch_of_eq_4_2():
    # arg in [0, 2 pi): z on the positive imaginary axis -> phi = pi/2
    assert abs(O.branch_sqrt_cut_positive_axis(1j) - complex(math.cos(math.pi / 4), math.sin(math.pi / 4))) < 1e-15
    # just below the cut [0, inf): phi -> 2 pi, so the root is near -1
    z = complex(4.0, -1e-12)
    assert abs(O.branch_sqrt_cut_positive_axis(z) + 2.0) < 1e-9
    # negative real axis: phi = pi -> root = i |z|^(1/2)
    assert abs(O.branch_sqrt_cut_positive_axis(-9.0) - 3j) < 1e-14


# --------------------------------------------------------------------------
# Green's function (Eq. 2.6a): Helmholtz equation, source strength, radiation
# --------------------------------------------------------------------------

def test_greens_function_is_outgoing_helmholtz_fundamental_solution():
    k = 1.7
    # (lap + k^2) G = 0 away from the source, by central differences in 3D
    x0 = np.array([0.4, -0.3, 0.5])
    hstep = 1e-3
    f = lambda p: O.greens_function(np.linalg.norm(p), k)  # noqa: E731
    lap = 0.0
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = hstep
        lap += (f(x0 + e) - 2 * f(x0) + f(x0 - e)) / hstep ** 2
    assert abs(lap + k * k * f(x0)) < 1e-5 * abs(f(x0)) * k * k + 1e-6
    # unit source: flux of -grad G through a small sphere -> 1  (lap G = -delta)
    r = 1e-6
    dGdr = (O.greens_function(r * 1.001, k) - O.greens_function(r * 0.999, k)) / (0.002 * r)
    assert abs(-4 * math.pi * r * r * dGdr - 1.0) < 1e-5
    # radiation condition (Eq. 2.5): r (dG/dr - i k G) -> 0 for large r
    R = 1e5
    dG = (O.greens_function(R + 1e-3, k) - O.greens_function(R - 1e-3, k)) / 2e-3
    assert abs(R * (dG - 1j * k * O.greens_function(R, k))) < 1e-5


def test_plane_wave_matches_table6_phase():
    """Table 6 (RED, paper's parameters): samples equal exp(i k x) to within
    the weak scattering (|h| ~ 5e-6): this fixes the sign of the phase of u0."""
    g = _golden("table6_red_samples.json")
    k = 0.182651
    xs = np.array(g["x_samples"])
    pos = np.stack([xs, np.zeros_like(xs), np.zeros_like(xs)], axis=1)
    u0 = O.plane_wave(pos, k, (1.0, 0.0, 0.0))
    table = np.array(g["values_re"]) + 1j * np.array(g["values_im"])
    assert np.max(np.abs(u0 - table)) < 2e-5
    # the opposite sign of the phase is far off
    assert np.max(np.abs(np.conj(u0) - table)) > 0.2


# --------------------------------------------------------------------------
# The operator
# --------------------------------------------------------------------------

def test_two_particle_closed_form():
    """Eq. 2.19 with only two occupied cells (N = 0 elsewhere) is a 2x2 system
    solved by Cramer's rule; the cells with N = 0 then carry the explicit sum."""
    n, k, side = 4, 2.3, 1.0
    d = side / n
    h = np.zeros(n ** 3, dtype=np.complex128)
    N = np.zeros(n ** 3)
    i1, i2 = 5, 42
    h[i1], h[i2] = 3.0 + 1.5j, 0.7 - 2.2j
    N[i1], N[i2] = 1.3, 0.6
    A = O.red_matrix(n, k, h, N, side=side)
    pos = O.cell_centres(n, side=side)
    u0 = O.plane_wave(pos, k, (0.3, 0.4, math.sqrt(0.75)))
    u = O.solve_dense(A, u0)
    r12 = np.linalg.norm(pos[i1] - pos[i2])
    g = np.exp(1j * k * r12) / (4 * math.pi * r12)
    w1 = 4 * math.pi * h[i1] * N[i1] * d ** 3
    w2 = 4 * math.pi * h[i2] * N[i2] * d ** 3
    u1, u2 = O.two_particle_solution(u0[i1], u0[i2], g, w1, w2)
    assert abs(u[i1] - u1) < 1e-14 and abs(u[i2] - u2) < 1e-14
    # unoccupied cells: u_q = u0_q - sum_i G(x_q, x_i) w_i u_i
    for q in (0, 17, 63):
        s = 0
        for i, wi, ui in ((i1, w1, u1), (i2, w2, u2)):
            r = np.linalg.norm(pos[q] - pos[i])
            s += np.exp(1j * k * r) / (4 * math.pi * r) * wi * ui
        assert abs(u[q] - (u0[q] - s)) < 1e-14


def test_zero_impedance_gives_incident_field():
    n, k = 5, 1.0
    h, N = inputs.constant_h_N(n, 0.0)
    u, it, rr = O.solve_red_cocg_fft(n, k, h, N, tol=1e-12)
    u0 = O.plane_wave(O.cell_centres(n), k)
    assert it == 0
    assert np.array_equal(u, u0)


def test_first_order_born_limit():
    """For |h| -> 0 the solution is u0 - K D u0 + O(|h|^2)."""
    n, k = 4, 1.5
    h, N = inputs.random_h_N(n, 11)
    u0 = O.plane_wave(O.cell_centres(n), k)
    errs = []
    for eps in (1e-3, 1e-4):
        A = O.red_matrix(n, k, eps * h, N)
        u = O.solve_dense(A, u0)
        errs.append(np.linalg.norm(u - O.born_first_order(u0, n, k, eps * h, N)) / np.linalg.norm(u - u0))
    # relative error of the first-order term scales like eps
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 5


def test_direct_sum_rows_equal_dense_matrix():
    n, k = 3, 2.0
    h, N = inputs.random_h_N(n, 3)
    x = inputs.random_complex(n ** 3, 4)
    A = O.red_matrix(n, k, h, N)
    assert rel(O.red_matvec_direct(x, n, k, h, N, chunk=5), A @ x) < 1e-14
    rows = np.array([0, 7, 26])
    assert rel(O.red_matvec_rows(x, rows, n, k, h, N), (A @ x)[rows]) < 1e-14


def test_grid_row_sums_equal_dense_rows():
    """The memory-light row sums used at large n agree with the dense matrix."""
    n, k, side = 6, 2.7, 1.4
    h, N = inputs.random_h_N(n, 5)
    x = inputs.random_complex(n ** 3, 6)
    w = O.red_weights(h, N, side / n)
    rows = np.array([0, 17, 100, 215])
    A = O.red_matrix(n, k, h, N, side=side)
    got = x[rows] + O.offdiag_sum_rows_grid(w * x, rows, n, k, side, planes_per_chunk=4)
    assert rel(got, (A @ x)[rows]) < 1e-14


def test_octant_row_sums_equal_dense_rows_everywhere():
    """The table-driven row sums (used at n = 512) against the dense matrix on
    every row of an n = 6 grid (corners, edges, faces, interior), and against
    the per-row direct evaluation on an odd n = 9 grid."""
    n, k, side = 6, 2.7, 1.4
    h, N = inputs.random_h_N(n, 5)
    x = inputs.random_complex(n ** 3, 6)
    w = O.red_weights(h, N, side / n)
    A = O.red_matrix(n, k, h, N, side=side)
    rows = np.arange(n ** 3)
    got = x + O.offdiag_sum_rows_octant(w * x, rows, n, k, side)
    assert rel(got, A @ x) < 1e-14
    n = 9
    v = inputs.random_complex(n ** 3, 7)
    rows = np.array([0, n - 1, n * n - 1, n ** 3 - 1, n ** 3 - n, 4 * n * n + 4 * n + 4, 123, 500])
    a = O.offdiag_sum_rows_octant(v, rows, n, 4.1, 0.9)
    b = O.offdiag_sum_rows_grid(v, rows, n, 4.1, 0.9, planes_per_chunk=2)
    assert rel(a, b) < 1e-14


def test_kernel_octant_values():
    """The table holds G(d |offset|) with the origin left out (p = q excluded)."""
    n, k, side = 5, 3.3, 2.0
    G = O.kernel_octant(n, k, side)
    d = side / n
    assert G[0, 0, 0] == 0
    for a, b, c in [(0, 0, 1), (1, 2, 3), (4, 4, 4), (3, 0, 2)]:
        r = d * math.sqrt(a * a + b * b + c * c)
        assert abs(G[a, b, c] - np.exp(1j * k * r) / (4 * math.pi * r)) < 1e-15
    # G depends on |offset| only: any permutation of the three axes gives the same table
    assert np.array_equal(G, G.transpose(1, 0, 2)) and np.array_equal(G, G.transpose(2, 1, 0))


def test_brute_force_tiny_grid():
    """n = 2 (8 cells) summed pair by pair in plain Python."""
    n, k, side = 2, 3.1, 0.7
    h, N = inputs.random_h_N(n, 21)
    x = inputs.random_complex(n ** 3, 22)
    d = side / n
    pts = [((ix + 0.5) * d, (iy + 0.5) * d, (iz + 0.5) * d)
           for iz in range(n) for iy in range(n) for ix in range(n)]
    y = []
    for q in range(8):
        s = x[q]
        for p in range(8):
            if p == q:
                continue
            r = math.dist(pts[q], pts[p])
            s += (complex(math.cos(k * r), math.sin(k * r)) / (4 * math.pi * r)) \
                * 4 * math.pi * h[p] * N[p] * d ** 3 * x[p]
        y.append(s)
    assert rel(O.red_matvec_direct(x, n, k, h, N, side=side), np.array(y)) < 1e-14


@pytest.mark.parametrize("n", [2, 3, 4, 7])
def test_fft_convolution_equals_direct_sum(n):
    """Section 3: mirror padding to (2n-2)^3 and zero embedding at any
    L >= 2n - 1 give the same crop as the direct sum."""
    k, side = 2.5, 1.3
    h, N = inputs.random_h_N(n, 100 + n)
    x = inputs.random_complex(n ** 3, 200 + n)
    ref = O.red_matvec_direct(x, n, k, h, N, side=side)
    assert rel(O.red_matvec_fft(x, n, k, h, N, side=side), ref) < 1e-13
    L2 = 1 << int(math.ceil(math.log2(2 * n)))
    for L in sorted({2 * n - 1, 2 * n, L2}):
        assert rel(O.red_matvec_fft(x, n, k, h, N, side=side, L=L, embedding="zero"), ref) < 1e-13


def test_kernel_cube_is_even_and_self_term_zero():
    n, k, d = 5, 1.1, 0.2
    for c in (O.kernel_cube(n, k, d), O.kernel_cube(n, k, d, L=16, embedding="zero")):
        L = c.shape[0]
        assert c[0, 0, 0] == 0
        m = (-np.arange(L)) % L
        assert np.array_equal(c, c[np.ix_(m, m, m)])
    # spectrum of an even cube is even along each axis
    Gh = np.fft.fftn(O.kernel_cube(n, k, d, L=16, embedding="zero"))
    m = (-np.arange(16)) % 16
    assert np.allclose(Gh, Gh[np.ix_(m, m, m)], rtol=0, atol=1e-12 * np.abs(Gh).max())


def test_complex_symmetry_and_similarity():
    n, k = 3, 1.8
    h, N = inputs.random_h_N(n, 31)
    x = inputs.random_complex(n ** 3, 32)
    y = inputs.random_complex(n ** 3, 33)
    B = O.symmetrised_matrix(n, k, h, N)
    A = O.red_matrix(n, k, h, N)
    assert abs(x @ (B @ y) - y @ (B @ x)) < 1e-14 * abs(x @ (B @ y))
    S = O.sqrt_hN(h, N)
    assert rel(np.diag(S) @ A @ np.diag(1 / S), B) < 1e-14
    # A itself is not symmetric when h N varies ...
    assert abs(x @ (A @ y) - y @ (A @ x)) > 1e-6
    # ... but is when h N is constant
    hc, Nc = inputs.constant_h_N(n, 1 + 1j, 1.0)
    Ac = O.red_matrix(n, k, hc, Nc)
    assert abs(x @ (Ac @ y) - y @ (Ac @ x)) < 1e-14 * abs(x @ (Ac @ y))
    # matrix-free symmetrised products agree with the dense B
    assert rel(O.symmetrised_matvec_direct(x, n, k, h, N), B @ x) < 1e-14
    assert rel(O.symmetrised_matvec_fft(x, n, k, h, N), B @ x) < 1e-13


def test_translation_gives_global_phase():
    """G depends on differences only, so shifting the cube by delta multiplies
    u by exp(i k alpha . delta)."""
    n, k = 3, 2.2
    alpha = np.array([0.0, 0.6, 0.8])
    h, N = inputs.random_h_N(n, 41)
    delta = np.array([0.31, -0.12, 0.05])
    u_a = O.solve_dense(O.red_matrix(n, k, h, N), O.plane_wave(O.cell_centres(n), k, alpha))
    u_b = O.solve_dense(O.red_matrix(n, k, h, N, origin=tuple(delta)),
                        O.plane_wave(O.cell_centres(n, tuple(delta)), k, alpha))
    assert rel(u_b, np.exp(1j * k * alpha @ delta) * u_a) < 1e-13


# --------------------------------------------------------------------------
# Solver
# --------------------------------------------------------------------------

def test_cocg_reduces_to_cg_on_real_spd():
    """On a real symmetric positive-definite system COCG is CG: compare iterates
    with scipy's CG after the same number of steps."""
    rng = np.random.default_rng(7)
    M = rng.standard_normal((30, 30))
    A = M @ M.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    for m in (1, 3, 6):
        x_cocg, it, _ = O.cocg(lambda v: A @ v, b.astype(complex), tol=0.0, maxit=m)
        x_cg, _ = spla.cg(A, b, rtol=1e-30, atol=0.0, maxiter=m)
        assert it == m
        assert rel(x_cocg.real, x_cg) < 1e-12 and np.max(np.abs(x_cocg.imag)) == 0


def test_cocg_finite_termination():
    """In exact arithmetic COCG ends in at most N steps on an N x N complex symmetric system."""
    n, k = 2, 1.0
    h, N = inputs.random_h_N(n, 51)
    B = O.symmetrised_matrix(n, k, h, N)
    b = inputs.random_complex(8, 52)
    x, it, rr = O.cocg(lambda v: B @ v, b, tol=0.0, maxit=8)
    assert rel(B @ x, b) < 1e-12


def test_config1_lu_vs_cocg():
    """n = 12 (1728 cells), unit cube, k = 1, h = 1 + 1i, N = 1, alpha = (0,0,1):
    dense LU against COCG run to relres 1e-12 (kappa = 0.9 does not enter, Eq. 2.18)."""
    n, k = 12, 1.0
    h, N = inputs.constant_h_N(n, 1 + 1j, 1.0)
    A = O.red_matrix(n, k, h, N)
    u0 = O.plane_wave(O.cell_centres(n), k)
    u_lu = O.solve_dense(A, u0)
    u_cg, it, rr = O.solve_red_cocg_fft(n, k, h, N, tol=1e-12)
    assert rr <= 1e-12
    assert rel(u_cg, u_lu) < 1e-9
    assert O.relative_residual(lambda v: A @ v, u_cg, u0) < 1e-11


def test_symmetrised_cocg_matches_lu_variable_hN():
    n, k = 6, 2.0
    h, N = inputs.random_h_N(n, 2)
    A = O.red_matrix(n, k, h, N)
    u0 = O.plane_wave(O.cell_centres(n), k)
    u_lu = O.solve_dense(A, u0)
    u_cg, it, rr = O.solve_red_cocg_fft(n, k, h, N, tol=1e-12)
    assert rel(u_cg, u_lu) < 1e-10


@pytest.mark.parametrize("L", [None, 11, 16])
def test_spectrum_matvec_equals_direct_sum(L):
    """The CPU-baseline matvec (zero-embedded spectrum built plane by plane,
    scipy.fft on threads) against brute-force direct summation of B x, in
    complex128 (1e-13) and complex64 (1e-5), at odd and power-of-two L."""
    n, k, side = 6, 2.9, 1.2
    h, N = inputs.random_h_N(n, 31)
    x = inputs.random_complex(n ** 3, 32)
    ref = O.symmetrised_matvec_direct(x, n, k, h, N, side=side)
    S = O.sqrt_hN(h, N)
    for dtype, bound in ((np.complex128, 1e-13), (np.complex64, 1e-5)):
        spec = O.kernel_spectrum_zero(n, k, side, L=L, dtype=dtype, workers=2)
        assert spec.dtype == dtype
        y = O.symmetrised_matvec_spectrum(x.astype(dtype), S.astype(dtype), spec, n, workers=2)
        assert y.dtype == dtype
        assert rel(y, ref) < bound
    with pytest.raises(ValueError):
        O.kernel_spectrum_zero(n, k, side, L=2 * n - 2)


def test_cpu_fft_cocg_matches_lu():
    """The timed CPU solver (the paper's algorithm, Section 3-4) against dense LU:
    complex128 to relres 1e-12, and complex64 (the paper's arithmetic) to 1e-5."""
    n, k = 6, 2.0
    h, N = inputs.random_h_N(n, 2)
    u_lu = O.solve_dense(O.red_matrix(n, k, h, N), O.plane_wave(O.cell_centres(n), k))
    seen = []
    u, it, rr = O.solve_cocg_fft_cpu(n, k, h, N, tol=1e-12, dtype=np.complex128, workers=2,
                                     callback=seen.append)
    assert rr <= 1e-12 and seen == list(range(1, it + 1))
    assert rel(u, u_lu) < 1e-10
    u, it, rr = O.solve_cocg_fft_cpu(n, k, h, N, tol=1e-5, dtype=np.complex64, workers=2)
    assert rr <= 1e-5
    assert rel(u, u_lu) < 1e-4


def test_zero_density_cells_recovered():
    """Cells with N = 0 (S = 0) get u = u0 - K(S w) instead of w / S."""
    n, k = 4, 1.3
    h, N = inputs.random_h_N(n, 61)
    N[::3] = 0.0
    A = O.red_matrix(n, k, h, N)
    u0 = O.plane_wave(O.cell_centres(n), k)
    u_cg, it, rr = O.solve_red_cocg_fft(n, k, h, N, tol=1e-13)
    assert rel(u_cg, O.solve_dense(A, u0)) < 1e-11


def test_paper_parameters_weak_scattering():
    """Section 4 parameters on the RED grid P = 8000 (n = 20): the solution stays
    within 2e-5 of u0, as in Tables 5-7 (|u| = 1 to the printed digits)."""
    n = 20
    k = 0.182651
    h, N = inputs.constant_h_N(n, 2.65481e-9 + 5.30961e-6j, 1.0)
    u, it, rr = O.solve_red_cocg_fft(n, k, h, N, alpha=(1.0, 0.0, 0.0), tol=1e-12)
    u0 = O.plane_wave(O.cell_centres(n), k, (1.0, 0.0, 0.0))
    assert np.max(np.abs(u - u0)) < 2e-5
    assert np.max(np.abs(np.abs(u) - 1.0)) < 2e-5


# --------------------------------------------------------------------------
# Gradient
# --------------------------------------------------------------------------

def test_adjoint_gradient_vs_central_differences():
    n, k = 3, 1.6
    h, N = inputs.random_h_N(n, 71)
    obs = np.array([1, 8, 20])
    target = np.array([0.3 + 0.1j, -0.2j, 0.5])
    u, J, gh, gN = O.adjoint_gradient_dense(n, k, h, N, obs, target)
    u0 = O.plane_wave(O.cell_centres(n), k)

    def J_of(hh, NN):
        return O.objective(O.solve_dense(O.red_matrix(n, k, hh, NN), u0), obs, target)

    step = 1e-6
    for p in (0, 13, 26):
        e = np.zeros(n ** 3)
        e[p] = step
        dre = (J_of(h + e, N) - J_of(h - e, N)) / (2 * step)
        dim = (J_of(h + 1j * e, N) - J_of(h - 1j * e, N)) / (2 * step)
        dN = (J_of(h, N + e) - J_of(h, N - e)) / (2 * step)
        assert abs(gh[p] - complex(dre, dim)) < 1e-7 * max(1.0, abs(gh[p]))
        assert abs(gN[p] - dN) < 1e-7 * max(1.0, abs(gN[p]))


# --------------------------------------------------------------------------
# Charges, the field off the grid (Eq. 2.10, 2.13) and the Table 4 metric
# --------------------------------------------------------------------------

SECTION4_K = 0.182651
SECTION4_H = 2.65481e-9 + 5.30961e-6j


def test_field_at_cell_points_is_the_solution():
    """Eq. 2.10 evaluated at the particle points, leaving out each particle's
    own term, is the effective field of Eq. 2.14; the solution of Eq. 2.19
    (dense LU) must satisfy it.  A wrong sign or scale of the charges Q_m
    (Eq. 2.13) breaks the identity."""
    n, k = 5, 2.0
    h, N = inputs.random_h_N(n, 404)
    pos = O.cell_centres(n, (0.1, -0.2, 0.3), 0.9)
    A = O.red_matrix(n, k, h, N, origin=(0.1, -0.2, 0.3), side=0.9)
    u0 = O.plane_wave(pos, k, (0.0, 0.6, 0.8))
    u = O.solve_dense(A, u0)
    f = O.field(pos, u, n, k, h, N, alpha=(0.0, 0.6, 0.8), origin=(0.1, -0.2, 0.3), side=0.9)
    assert np.max(np.abs(f - u)) < 1e-13
    # the scattered part alone is u - u0
    fs = O.field(pos, u, n, k, h, N, origin=(0.1, -0.2, 0.3), side=0.9)
    assert np.max(np.abs(fs - (u - u0))) < 1e-13


def test_field_of_one_particle_closed_form():
    """One occupied cell (N = 0 elsewhere): u_1 = u0(x_1), Q_1 = -c_S h N |Delta| u_1,
    and off the grid u(x) = u0(x) + Q_1 exp(ik r) / (4 pi r), r = |x - x_1|."""
    n, k, side = 3, 1.7, 1.2
    h = np.zeros(n ** 3, dtype=np.complex128)
    N = np.zeros(n ** 3)
    j = 13                                   # the centre cell
    h[j], N[j] = 0.8 - 0.3j, 1.5
    pos = O.cell_centres(n, side=side)
    u = O.solve_dense(O.red_matrix(n, k, h, N, side=side), O.plane_wave(pos, k))
    assert abs(u[j] - O.plane_wave(pos[j:j + 1], k)[0]) < 1e-15
    Q1 = -4 * math.pi * h[j] * N[j] * (side / n) ** 3 * u[j]
    x = np.array([[0.1, 1.7, -0.4], [2.0, 0.3, 0.9]])
    r = np.linalg.norm(x - pos[j], axis=1)
    expect = np.exp(1j * k * x[:, 2]) + Q1 * np.exp(1j * k * r) / (4 * math.pi * r)
    got = O.field(x, u, n, k, h, N, alpha=(0.0, 0.0, 1.0), side=side)
    assert np.max(np.abs(got - expect)) < 1e-15


def test_table4_metric_by_hand():
    """One coarse cube holding 8 fine points: the mean of |x_i - y|.  Values
    chosen so the mean is 0.375 exactly: |diffs| = 0,0,0,0,1,0.5,1.5,0."""
    fine_pts = O.cell_centres(2)
    y = 1.0 + 1.0j
    diffs = np.array([0, 0, 0, 0, 1.0, 0.5j, -1.5, 0])
    assert O.table4_difference(y + diffs, fine_pts, np.array([y]), 1) == 0.375
    # two coarse cubes along x (n_coarse = 2 uses 8 cubes; fill only those with points)
    fine_pts = O.cell_centres(4)
    coarse = np.arange(8) * (1.0 + 0.5j)
    q = ((fine_pts[:, 2] // 0.5) * 4 + (fine_pts[:, 1] // 0.5) * 2 + fine_pts[:, 0] // 0.5).astype(int)
    fine = coarse[q].copy()
    fine[np.argmax(q == 5)] += 0.8           # one of the 8 points of cube 5
    assert abs(O.table4_difference(fine, fine_pts, coarse, 2) - 0.1) < 1e-15


def test_table4_metric_zero_for_nested_constant_fields():
    """A fine field equal to the coarse value of its sub-cube differs by 0, also
    when fine points lie exactly on sub-cube faces (vertex points)."""
    nc, nf = 3, 6
    coarse = np.exp(1j * np.arange(nc ** 3))
    for origin in ((0.0, 0.0, 0.0), (-0.5 / nf,) * 3):      # centres, vertices
        pts = O.cell_centres(nf, origin)
        m = np.rint((pts - origin[0]) * nf - 0.5).astype(int)   # fine cell indices
        qc = m * nc // nf
        q = (qc[:, 2] * nc + qc[:, 1]) * nc + qc[:, 0]
        assert O.table4_difference(coarse[q], pts, coarse, nc) == 0.0


def test_table4_reproduces_printed_red_vs_ie():
    """Section 4: (RED) with P = 8000 sub-cubes against (IE) with C = 64000
    collocation points, the paper's parameters.  Points at the grid vertices
    d*m (Eq. 3.3.5), each unknown owning the sub-cube [m d, (m+1) d).  The
    metric matches the printed 0.0022 to one unit of its last digit, and the
    plane-wave estimate (the scattered part is ~1e-5 here)."""
    g = _golden("table4_differences.json")
    sol = {}
    for n in (g["n_red"], g["n_ie"]):
        d = 1.0 / n
        org = (-d / 2,) * 3
        h = np.full(n ** 3, SECTION4_H)
        u, it, rr = O.solve_red_cocg_fft(n, SECTION4_K, h, np.ones(n ** 3), alpha=(1.0, 0.0, 0.0),
                                        origin=org, tol=1e-10)
        sol[n] = (u, O.cell_centres(n, org))
    v = O.table4_difference(sol[40][0], sol[40][1], sol[20][0], 20)
    assert abs(v - g["red_vs_ie"]) <= g["printed_resolution"]
    est = np.mean([abs(np.exp(1j * SECTION4_K * j / 40) - 1) for j in range(2)])
    assert abs(v - est) < 1e-6
