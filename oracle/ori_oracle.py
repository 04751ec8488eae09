"""CPU FP64 oracle for the RED/ORI linear system of Ramm & Tran (test infrastructure).

What it computes (the plain definitions; nothing is blocked, fused or reordered
beyond what the paper states):

* Eq. 2.19 (RED), with the sum moved to the left-hand side:
      u_q + c_S * sum_{p != q} G(x_q, x_p) h_p N_p |Delta_p| u_p = u0_q,
  G(x, y) = exp(ik|x-y|) / (4 pi |x-y|)                          (Eq. 2.6a, Eq. 3.3.2)
  u0(x)   = exp(ik alpha.x)                                        (Eq. 2.4)
  With one particle per cell and N = 1 this is also ORI, Eq. 2.15, because
  a^(2-kappa) * #(Delta_p) = N(x_p)|Delta_p| (Eq. 2.18); kappa therefore never
  enters the matrix.
* Cells: a cube [origin, origin + side]^3 cut into n^3 equal sub-cubes; the
  point x_p of a cell is its centre (Eq. 2.19 "for example, the center of
  Delta_p"; Section 4 collocates at centres).  Arrays are C-ordered [z][y][x]
  with x fastest.
* The FFT matvec of Section 3: the off-diagonal sum is a 3D convolution
  (Eq. 3.3.6-3.3.7) of the kernel cube with the field cube; it is evaluated by
  the convolution theorem (Eq. 3.3.8) after padding G by mirroring and u by
  zeros (the padding example of Section 3; padded size (2b-2)^3).
* COCG, the conjugate orthogonal conjugate gradient method the paper uses
  (Section 1, Section 3), as published by van der Vorst & Melissen: CG with the
  unconjugated bilinear form <a, b> = sum a_i b_i.  The paper states the stop
  test ||r|| / ||RHS|| (Section 4).
* Complex symmetry.  A = I + K D with K = c_S |Delta| G_off (symmetric) and
  D = diag(h N) is complex symmetric only when h N is constant (the paper's
  experiment, Section 4).  For variable h, N the oracle also provides
  B = I + S K S, S = diag(sqrt(h N)) (principal root), which is symmetric and
  similar to A: B = S A S^-1.  Solving B w = S u0 and setting u = w / S gives
  the same u.
* The refraction recipe of Eq. 2.24-2.26 / Eq. 4.1-4.2.
* The gradient of J = sum_obs |u_o - t_o|^2 with respect to h and N by the
  dense adjoint (derived from Eq. 2.19; the paper has no gradient).
* The cell charges of Eq. 2.13, the field off the grid of Eq. 2.10, and the
  solution-difference metric of Section 4 (Table 4).

Floating point is numpy float64 / complex128 throughout, except that the
timed CPU solver (solve_cocg_fft_cpu, the paper's algorithm as Section 4 ran
it on CPU cores) can also run in complex64, the paper's arithmetic.  numpy's
and scipy's FFTs, dense LU (``numpy.linalg.solve``) and matrix products serve
as library steps.

This module is test infrastructure.  Only tests, the package smoke check and
the CPU-baseline leg of the benchmark may call it.
"""

from __future__ import annotations

import math
import numpy as np

__all__ = [
    "C_S_SPHERE", "cell_size", "cell_centres", "plane_wave", "greens_function",
    "red_weights", "red_matrix", "red_matvec_direct", "red_matvec_rows", "offdiag_sum_rows_grid",
    "kernel_octant", "offdiag_sum_rows_octant",
    "symmetrised_matrix", "symmetrised_matvec_direct", "sqrt_hN",
    "pad_kernel_mirror", "pad_field_zero", "kernel_cube",
    "fft_convolution", "red_matvec_fft", "symmetrised_matvec_fft",
    "cocg", "solve_dense", "solve_red_cocg_fft", "relative_residual",
    "kernel_spectrum_zero", "symmetrised_matvec_spectrum", "solve_cocg_fft_cpu",
    "two_particle_solution", "refraction_from_h", "h_from_refraction",
    "branch_sqrt_cut_positive_axis", "adjoint_gradient_dense", "objective",
    "born_first_order", "charges", "field", "table4_difference",
]

# Surface constant c_S for a sphere: |S_m| = c_S a^2 (Eq. 2.13 and the remark after it).
C_S_SPHERE = 4.0 * math.pi


# ----------------------------------------------------------------------------
# Geometry and the continuous ingredients
# ----------------------------------------------------------------------------

def cell_size(n: int, side: float = 1.0) -> float:
    """Side d of one sub-cube Delta_p when the cube of side `side` is cut n ways.
    |Delta_p| = d^3 (Eq. 2.18)."""
    return side / n


def cell_centres(n: int, origin=(0.0, 0.0, 0.0), side: float = 1.0) -> np.ndarray:
    """Centres x_p of the n^3 cells, shape (n^3, 3) with columns (x, y, z),
    rows in C-order [z][y][x] (x fastest).  Eq. 2.19 takes x_p at the centre
    of Delta_p; Eq. 3.3.5 writes the uniform grid as d*(m1, m2, m3)."""
    d = cell_size(n, side)
    c = (np.arange(n) + 0.5) * d
    zz, yy, xx = np.meshgrid(c + origin[2], c + origin[1], c + origin[0], indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)


def plane_wave(positions: np.ndarray, k: float, alpha=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Incident field u0(x) = exp(i k alpha . x), |alpha| = 1 (Eq. 2.4)."""
    a = np.asarray(alpha, dtype=np.float64)
    a = a / np.linalg.norm(a)
    return np.exp(1j * k * (positions @ a))


def greens_function(r, k: float):
    """G = exp(ikr) / (4 pi r) for r > 0 (Eq. 2.6a, Eq. 3.3.2)."""
    r = np.asarray(r, dtype=np.float64)
    return np.exp(1j * k * r) / (4.0 * math.pi * r)


def red_weights(h, N, d: float, c_S: float = C_S_SPHERE) -> np.ndarray:
    """Per-cell factor c_S h_p N_p |Delta_p| that multiplies G_qp u_p in Eq. 2.19."""
    return c_S * np.asarray(h, dtype=np.complex128).ravel() * \
        np.asarray(N, dtype=np.float64).ravel() * d ** 3


def sqrt_hN(h, N) -> np.ndarray:
    """S_p = sqrt(h_p N_p), principal branch (numpy's complex sqrt)."""
    return np.sqrt(np.asarray(h, dtype=np.complex128).ravel() *
                   np.asarray(N, dtype=np.float64).ravel())


# ----------------------------------------------------------------------------
# Dense and direct-sum forms of the operator (Eq. 2.19)
# ----------------------------------------------------------------------------

def _offdiag_greens_matrix(pos: np.ndarray, k: float) -> np.ndarray:
    """G_qp for q != p and 0 on the diagonal (the sum in Eq. 2.19 excludes p = q)."""
    diff = pos[:, None, :] - pos[None, :, :]
    r = np.sqrt((diff ** 2).sum(axis=2))
    G = np.zeros(r.shape, dtype=np.complex128)
    off = r > 0
    G[off] = greens_function(r[off], k)
    return G


def red_matrix(n, k, h, N, origin=(0.0, 0.0, 0.0), side=1.0, c_S=C_S_SPHERE) -> np.ndarray:
    """Dense A with A u = u0 equivalent to Eq. 2.19:  A_qp = delta_qp + G_qp w_p,
    w_p = c_S h_p N_p |Delta_p|, G_qq = 0."""
    pos = cell_centres(n, origin, side)
    w = red_weights(h, N, cell_size(n, side), c_S)
    A = _offdiag_greens_matrix(pos, k) * w[None, :]
    A[np.diag_indices_from(A)] += 1.0
    return A


def symmetrised_matrix(n, k, h, N, origin=(0.0, 0.0, 0.0), side=1.0, c_S=C_S_SPHERE) -> np.ndarray:
    """Dense B = I + S K S with K = c_S |Delta| G_off and S = diag(sqrt(h N))."""
    pos = cell_centres(n, origin, side)
    d = cell_size(n, side)
    S = sqrt_hN(h, N)
    B = (c_S * d ** 3) * _offdiag_greens_matrix(pos, k) * S[:, None] * S[None, :]
    B[np.diag_indices_from(B)] += 1.0
    return B


def red_matvec_rows(x, rows, n, k, h, N, origin=(0.0, 0.0, 0.0), side=1.0,
                    c_S=C_S_SPHERE, chunk=64):
    """Rows `rows` of A x by the plain O(N) sum per row (Eq. 2.19):
    (A x)_q = x_q + sum_{p != q} G(|x_q - x_p|) c_S h_p N_p |Delta_p| x_p."""
    pos = cell_centres(n, origin, side)
    w = red_weights(h, N, cell_size(n, side), c_S)
    wx = w * np.asarray(x, dtype=np.complex128).ravel()
    rows = np.asarray(rows, dtype=np.int64).ravel()
    out = np.empty(rows.size, dtype=np.complex128)
    for s in range(0, rows.size, chunk):
        q = rows[s:s + chunk]
        diff = pos[q][:, None, :] - pos[None, :, :]
        r = np.sqrt((diff ** 2).sum(axis=2))
        G = np.zeros(r.shape, dtype=np.complex128)
        off = r > 0
        G[off] = greens_function(r[off], k)
        out[s:s + chunk] = x.ravel()[q] + G @ wx
    return out


def offdiag_sum_rows_grid(v, rows, n, k, side=1.0, planes_per_chunk=32):
    """sum_{p != q} G(|x_q - x_p|) v_p for the cells q in `rows`, by direct
    summation over the grid one slab of z-planes at a time (memory O(n^2 *
    planes_per_chunk) instead of the O(N) positions of red_matvec_rows).  Cell
    centres differ by d times integer offsets (Eq. 3.3.5), so the distance of a
    cell from q needs only the three 1D offset arrays."""
    d = side / n
    vv = np.asarray(v, dtype=np.complex128).reshape(n, n, n)
    rows = np.asarray(rows, dtype=np.int64).ravel()
    out = np.empty(rows.size, dtype=np.complex128)
    idx = np.arange(n)
    for t, q in enumerate(rows):
        qz, rem = divmod(int(q), n * n)
        qy, qx = divmod(rem, n)
        dy2 = ((idx - qy) * d) ** 2
        dx2 = ((idx - qx) * d) ** 2
        acc = 0j
        for z0 in range(0, n, planes_per_chunk):
            zs = idx[z0:z0 + planes_per_chunk]
            dz2 = ((zs - qz) * d) ** 2
            r = np.sqrt(dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :])
            G = np.zeros(r.shape, dtype=np.complex128)
            nz = r > 0
            G[nz] = greens_function(r[nz], k)
            acc += np.sum(G * vv[z0:z0 + planes_per_chunk])
        out[t] = acc
    return out


def kernel_octant(n, k, side=1.0) -> np.ndarray:
    """G(d |(a, b, c)|) for cell offsets 0 <= a, b, c < n, indexed [a][b][c], and 0
    at the origin (the sum of Eq. 2.19 / Eq. 3.3.7 excludes p = q).  Cell points
    differ by d times integer offsets (Eq. 3.3.5), so these n^3 values are every
    value G takes in the off-diagonal sum; G depends on |offset| only."""
    d = side / n
    b2 = (np.arange(n, dtype=np.float64) * d) ** 2
    out = np.empty((n, n, n), dtype=np.complex128)
    for a in range(n):
        r = np.sqrt((a * d) ** 2 + b2[:, None] + b2[None, :])
        plane = np.zeros((n, n), dtype=np.complex128)
        nz = r > 0
        plane[nz] = greens_function(r[nz], k)
        out[a] = plane
    return out


def _axis_pieces(q: int, n: int):
    """Cover the cells 0..n-1 of one axis by two runs: cells q..n-1 sit at offsets
    0..n-1-q from q, cells q-1..0 (taken downwards) at offsets 1..q."""
    pieces = [(slice(0, n - q), slice(q, n))]
    if q > 0:
        pieces.append((slice(1, q + 1), slice(q - 1, None, -1)))
    return pieces


def offdiag_sum_rows_octant(v, rows, n, k, side=1.0, octant=None):
    """sum_{p != q} G(|x_q - x_p|) v_p for the cells q in `rows` (the same sums as
    offdiag_sum_rows_grid): every cell p of the grid, taken as a product of one run
    per axis (_axis_pieces), multiplies v_p by the table value G(d |offset|) of
    kernel_octant.  No evaluation of G per row, so large grids (n = 512) take well
    under a second per row.  `octant` may pass a kernel_octant(n, k, side) table."""
    G = kernel_octant(n, k, side) if octant is None else octant
    vv = np.asarray(v, dtype=np.complex128).reshape(n, n, n)
    rows = np.asarray(rows, dtype=np.int64).ravel()
    out = np.empty(rows.size, dtype=np.complex128)
    for t, q in enumerate(rows):
        qz, rem = divmod(int(q), n * n)
        qy, qx = divmod(rem, n)
        acc = 0j
        for gz, vz in _axis_pieces(qz, n):
            for gy, vy in _axis_pieces(qy, n):
                for gx, vx in _axis_pieces(qx, n):
                    acc += np.einsum("ijk,ijk->", G[gz, gy, gx], vv[vz, vy, vx])
        out[t] = acc
    return out


def red_matvec_direct(x, n, k, h, N, origin=(0.0, 0.0, 0.0), side=1.0, c_S=C_S_SPHERE, chunk=64):
    """All rows of A x by direct O(N^2) summation (Eq. 2.19)."""
    return red_matvec_rows(x, np.arange(n ** 3), n, k, h, N, origin, side, c_S, chunk)


def symmetrised_matvec_direct(x, n, k, h, N, origin=(0.0, 0.0, 0.0), side=1.0,
                              c_S=C_S_SPHERE, chunk=64):
    """B x = x + S K (S x) by direct summation; K = c_S |Delta| G_off."""
    S = sqrt_hN(h, N)
    x = np.asarray(x, dtype=np.complex128).ravel()
    ones = np.ones(n ** 3)
    # (A' y)_q = y_q + sum_{p!=q} G_qp c_S |Delta| y_p with h N := 1
    Ky_plus_y = red_matvec_rows(S * x, np.arange(n ** 3), n, k, ones, ones, origin, side, c_S, chunk)
    return x + S * (Ky_plus_y - S * x)


# ----------------------------------------------------------------------------
# Section 3: the convolution form and its padding
# ----------------------------------------------------------------------------

def pad_kernel_mirror(row) -> np.ndarray:
    """Padding of G along one axis from the Section 3 example:
    copy every entry except the first and the last, in reverse order, after
    the last one:  [1 2 3 4] -> [1 2 3 4 3 2]  (length 2b - 2)."""
    row = np.asarray(row)
    return np.concatenate([row, row[-2:0:-1]])


def pad_field_zero(row, length=None) -> np.ndarray:
    """Padding of u along one axis from the Section 3 example:
    [1 2 3 4] -> [1 2 3 4 0 0]; `length` defaults to 2b - 2."""
    row = np.asarray(row)
    b = row.shape[-1]
    if length is None:
        length = 2 * b - 2
    out = np.zeros(row.shape[:-1] + (length,), dtype=row.dtype)
    out[..., :b] = row
    return out


def kernel_cube(n, k, d, L=None, embedding="mirror") -> np.ndarray:
    """Kernel cube c[j3, j2, j1] of size L^3 whose cyclic convolution with a
    zero-padded field gives the off-diagonal sum of Eq. 3.3.7.

    The b^3 cube G(j1, j2, j3) = G(d |(j1, j2, j3)|) for 0 <= j_i < b (b = n),
    with G(0, 0, 0) = 0 because the sum excludes m = j (Eq. 3.3.7), is padded
    on each axis in turn (Section 3: pad x, pad y, pad z).

    embedding="mirror": the paper's padding, L = 2n - 2 (the default for L).
    embedding="zero":   entries 0 <= j < n and L - n < j < L carry
                        G(|signed offset|); the rest are 0; any L >= 2n - 1.
    """
    idx = np.arange(n)
    g1 = idx * d
    Z, Y, X = np.meshgrid(g1, g1, g1, indexing="ij")
    r = np.sqrt(X ** 2 + Y ** 2 + Z ** 2)
    G = np.zeros((n, n, n), dtype=np.complex128)
    nz = r > 0
    G[nz] = greens_function(r[nz], k)
    if embedding == "mirror":
        if L is not None and L != 2 * n - 2:
            raise ValueError("the mirror padding has length 2n - 2")
        c = G
        for ax in range(3):
            c = np.apply_along_axis(pad_kernel_mirror, ax, c)
        return c
    if embedding == "zero":
        if L is None or L < 2 * n - 1:
            raise ValueError("zero embedding needs L >= 2n - 1")
        # signed offset s in (-(n-1), ..., n-1) sits at index s mod L
        sidx = np.concatenate([np.arange(n), np.arange(-(n - 1), 0)]) % L
        src = np.concatenate([np.arange(n), np.arange(n - 1, 0, -1)])
        c = np.zeros((L, L, L), dtype=np.complex128)
        c[np.ix_(sidx, sidx, sidx)] = G[np.ix_(src, src, src)]
        return c
    raise ValueError(embedding)


def fft_convolution(field, c) -> np.ndarray:
    """Crop of the cyclic convolution of the zero-padded n^3 field with the
    L^3 kernel cube c, by the convolution theorem G*u = F^-1(F(G) . F(u))
    (Eq. 3.3.8); entries past the n-th on each axis are discarded (Section 3)."""
    field = np.asarray(field, dtype=np.complex128)
    n = field.shape[0]
    L = c.shape[0]
    padded = np.zeros((L, L, L), dtype=np.complex128)
    padded[:n, :n, :n] = field
    conv = np.fft.ifftn(np.fft.fftn(c) * np.fft.fftn(padded))
    return conv[:n, :n, :n]


def red_matvec_fft(x, n, k, h, N, side=1.0, c_S=C_S_SPHERE, L=None, embedding="mirror"):
    """A x = x + c_S (G_off * (h N |Delta| x)) with the convolution done by FFT
    (Section 3).  Result flattened in C-order."""
    d = cell_size(n, side)
    c = kernel_cube(n, k, d, L, embedding)
    w = red_weights(h, N, d, c_S).reshape(n, n, n)
    xx = np.asarray(x, dtype=np.complex128).reshape(n, n, n)
    return (xx + fft_convolution(w * xx, c)).ravel()


def symmetrised_matvec_fft(x, n, k, h, N, side=1.0, c_S=C_S_SPHERE, L=None, embedding="mirror",
                           _c=None):
    """B x = x + S (c_S |Delta| G_off * (S x)) with the FFT convolution."""
    d = cell_size(n, side)
    c = kernel_cube(n, k, d, L, embedding) if _c is None else _c
    S = sqrt_hN(h, N).reshape(n, n, n)
    xx = np.asarray(x, dtype=np.complex128).reshape(n, n, n)
    return (xx + S * (c_S * d ** 3) * fft_convolution(S * xx, c)).ravel()


# ----------------------------------------------------------------------------
# Solvers
# ----------------------------------------------------------------------------

def relative_residual(apply_A, u, rhs) -> float:
    """||r|| / ||RHS||, r = RHS - A u (the convergence measure of Section 4)."""
    r = rhs - apply_A(u)
    return float(np.linalg.norm(r) / np.linalg.norm(rhs))


def cocg(apply_A, b, tol=1e-12, maxit=1000, x0=None, dtype=np.complex128, callback=None):
    """Conjugate orthogonal conjugate gradient (van der Vorst & Melissen), the
    solver named in Section 1 and Section 3, for complex-symmetric A.

    Vectors and scalars are kept in `dtype` (complex128; complex64 is the
    arithmetic of the paper's runs, Section 4).  `callback(it)`, if given, is
    called after each iteration.  Returns (x, iterations, recursive relative
    residual)."""
    b = np.asarray(b, dtype=dtype)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=dtype)
    r = b - apply_A(x) if x0 is not None else b.copy()
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0, 0.0
    p = r.copy()
    rho = np.sum(r * r)             # <r, r>, no conjugate
    it = 0
    relres = np.linalg.norm(r) / nb
    while relres > tol and it < maxit:
        q = apply_A(p)
        mu = np.sum(p * q)          # <p, A p>
        alpha = rho / mu
        x = x + alpha * p
        r = r - alpha * q
        rho_new = np.sum(r * r)
        beta = rho_new / rho
        rho = rho_new
        p = r + beta * p
        it += 1
        relres = np.linalg.norm(r) / nb
        if callback is not None:
            callback(it)
    return x, it, float(relres)


def solve_dense(A, b) -> np.ndarray:
    """Direct solve by LU with partial pivoting (numpy.linalg.solve)."""
    return np.linalg.solve(A, b)


def solve_red_cocg_fft(n, k, h, N, alpha=(0.0, 0.0, 1.0), side=1.0, origin=(0.0, 0.0, 0.0),
                       c_S=C_S_SPHERE, tol=1e-10, maxit=2000, rhs=None, L=None, embedding="mirror"):
    """The paper's algorithm on the CPU: COCG on the symmetrised system
    B w = S u0 with the Section 3 FFT matvec, then u = w / S (u = u0 - K(S w)
    where S = 0).  Returns (u, iterations, recursive relres of w)."""
    d = cell_size(n, side)
    if embedding == "mirror" and n < 2:
        raise ValueError("n >= 2")
    c = kernel_cube(n, k, d, L, embedding)
    S = sqrt_hN(h, N)
    if rhs is None:
        rhs = plane_wave(cell_centres(n, origin, side), k, alpha)
    apply_B = lambda v: symmetrised_matvec_fft(v, n, k, h, N, side, c_S, L, embedding, _c=c)  # noqa: E731
    w, it, rr = cocg(apply_B, S * rhs, tol=tol, maxit=maxit)
    u = np.empty_like(w)
    nz = S != 0
    u[nz] = w[nz] / S[nz]
    if not np.all(nz):
        Kw = (c_S * d ** 3) * fft_convolution((S * w).reshape(n, n, n), c).ravel()
        u[~nz] = rhs[~nz] - Kw[~nz]
    return u, it, rr


# ----------------------------------------------------------------------------
# The paper's algorithm on CPU cores (the timed CPU baseline): Section 3's FFT
# convolution inside COCG, as Section 4 ran it with FFTW on CPU cores.  The
# FFTs are scipy.fft's, on `workers` threads; the spectrum F(G) is computed
# once (Eq. 3.3.9 counts it per matvec: the result is the same).
# ----------------------------------------------------------------------------

def kernel_spectrum_zero(n, k, side=1.0, c_S=C_S_SPHERE, L=None, dtype=np.complex128, workers=None):
    """F(c) for the kernel cube c = c_S |Delta| G_off zero-embedded in L^3 (the
    zero embedding of kernel_cube; L >= 2n - 1, default the smallest power of
    two >= 2n), filled plane by plane from kernel_octant so that no L^3
    complex128 temporary is needed, then transformed in place in `dtype`."""
    import scipy.fft as sfft
    if L is None:
        L = 1
        while L < 2 * n:
            L *= 2
    if L < 2 * n - 1:
        raise ValueError("zero embedding needs L >= 2n - 1")
    d = cell_size(n, side)
    G = kernel_octant(n, k, side)
    # wrapped index j of one axis holds |signed offset| = j for j < n, L - j for j > L - n
    wrapped = np.concatenate([np.arange(n), np.arange(L - n + 1, L)])
    offset = np.concatenate([np.arange(n), np.arange(n - 1, 0, -1)])
    c = np.zeros((L, L, L), dtype=dtype)
    scale = c_S * d ** 3
    for jz, az in zip(wrapped, offset):
        c[jz][np.ix_(wrapped, wrapped)] = (scale * G[az][np.ix_(offset, offset)]).astype(dtype)
    return sfft.fftn(c, overwrite_x=True, workers=workers)


def symmetrised_matvec_spectrum(x, S, spec, n, workers=None):
    """B x = x + S (c_S |Delta| G_off * (S x)) with the kernel's spectrum `spec`
    (kernel_spectrum_zero): zero-pad S x to L^3, FFT, multiply, inverse FFT,
    keep the first n entries per axis (Eq. 3.3.8, Section 3).  Arithmetic in
    the spectrum's dtype."""
    import scipy.fft as sfft
    L = spec.shape[0]
    pad = np.zeros((L, L, L), dtype=spec.dtype)
    pad[:n, :n, :n] = (S * x).reshape(n, n, n)
    f = sfft.fftn(pad, overwrite_x=True, workers=workers)
    f *= spec
    conv = sfft.ifftn(f, overwrite_x=True, workers=workers)
    return x + S * conv[:n, :n, :n].ravel()


def solve_cocg_fft_cpu(n, k, h, N, alpha=(0.0, 0.0, 1.0), side=1.0, origin=(0.0, 0.0, 0.0),
                       c_S=C_S_SPHERE, tol=1e-6, maxit=2000, dtype=np.complex64, workers=None,
                       spec=None, callback=None):
    """COCG on B w = S u0 with the FFT matvec of symmetrised_matvec_spectrum in
    `dtype`, then u = w / S; every cell needs S != 0.  `spec` may pass a
    kernel_spectrum_zero of the same dtype.  Returns (u, iterations, recursive
    relres)."""
    S = sqrt_hN(h, N)
    if np.any(S == 0):
        raise ValueError("solve_cocg_fft_cpu needs h N != 0 in every cell")
    if spec is None:
        spec = kernel_spectrum_zero(n, k, side, c_S, dtype=dtype, workers=workers)
    S_t = S.astype(dtype)
    rhs = plane_wave(cell_centres(n, origin, side), k, alpha)
    apply_B = lambda v: symmetrised_matvec_spectrum(v, S_t, spec, n, workers)  # noqa: E731
    w, it, rr = cocg(apply_B, (S * rhs).astype(dtype), tol=tol, maxit=maxit, dtype=dtype, callback=callback)
    return w.astype(np.complex128) / S, it, rr


def two_particle_solution(u01, u02, g, w1, w2):
    """Closed form of Eq. 2.15 / 2.19 with two particles:
        u1 + g w2 u2 = u01,   u2 + g w1 u1 = u02
    (g = G(|x1 - x2|), w_i = c_S h_i N_i |Delta|), solved by Cramer's rule."""
    det = 1.0 - g * g * w1 * w2
    return (u01 - g * w2 * u02) / det, (u02 - g * w1 * u01) / det


def born_first_order(u0, n, k, h, N, side=1.0, c_S=C_S_SPHERE):
    """First term of the Neumann series of Eq. 2.19: u ~ u0 - K D u0 (error O(|h|^2))."""
    Au0 = red_matvec_direct(u0, n, k, h, N, side=side, c_S=c_S)
    return u0 - (Au0 - u0)


# ----------------------------------------------------------------------------
# Refraction recipe (Eq. 2.24 - 2.26, Eq. 4.1 - 4.2)
# ----------------------------------------------------------------------------

def branch_sqrt_cut_positive_axis(z):
    """z^(1/2) = |z|^(1/2) exp(i phi / 2), phi = arg z taken in [0, 2 pi) (Eq. 4.2)."""
    z = complex(z)
    phi = math.atan2(z.imag, z.real)
    if phi < 0.0:
        phi += 2.0 * math.pi
    return math.sqrt(abs(z)) * complex(math.cos(phi / 2.0), math.sin(phi / 2.0))


def refraction_from_h(h, k, c_S=C_S_SPHERE, N=1.0, n0=1.0 + 0.0j):
    """n = [n0^2 - k^-2 c_S h N]^(1/2) with the branch of Eq. 4.2 (Eq. 4.1)."""
    return branch_sqrt_cut_positive_axis(n0 * n0 - c_S * h * N / (k * k))


def h_from_refraction(n_desired, k, c_S=C_S_SPHERE, N=1.0, n0=1.0 + 0.0j):
    """p = k^2 (n0^2 - n^2) (Eq. 2.25);  h = p / (c_S N) (Eq. 2.26)."""
    p = k * k * (n0 * n0 - n_desired * n_desired)
    return p / (c_S * N)


# ----------------------------------------------------------------------------
# Gradient of a field objective (dense adjoint; the paper has no gradient)
# ----------------------------------------------------------------------------

def objective(u, obs, target) -> float:
    """J = sum over observation cells of |u_o - t_o|^2."""
    e = u[obs] - target
    return float(np.sum(np.abs(e) ** 2))


def adjoint_gradient_dense(n, k, h, N, obs, target, alpha=(0.0, 0.0, 1.0), side=1.0,
                           origin=(0.0, 0.0, 0.0), c_S=C_S_SPHERE):
    """Gradient of J(h, N) with u solving A(h, N) u = u0 (Eq. 2.19).

    A = I + K D, K = c_S |Delta| G_off (symmetric), D = diag(h N).  For a change
    of h_p:  A du = -K e_p N_p u_p dh_p, so with psi = A^-T conj(e)
    (e = u - t on obs cells, 0 elsewhere):
        dJ = 2 Re(g_p dh_p),  g_p = -(K psi)_p N_p u_p.
    Returned gradients use the convention dJ/dRe h + i dJ/dIm h = 2 conj(g_p),
    and dJ/dN_p = 2 Re(-(K psi)_p h_p u_p).  Returns (u, J, grad_h, grad_N)."""
    h = np.asarray(h, dtype=np.complex128).ravel()
    N = np.asarray(N, dtype=np.float64).ravel()
    pos = cell_centres(n, origin, side)
    d = cell_size(n, side)
    K = (c_S * d ** 3) * _offdiag_greens_matrix(pos, k)
    A = np.eye(n ** 3, dtype=np.complex128) + K * (h * N)[None, :]
    u0 = plane_wave(pos, k, alpha)
    u = np.linalg.solve(A, u0)
    e = np.zeros_like(u)
    e[obs] = u[obs] - target
    psi = np.linalg.solve(A.T, np.conj(e))
    Kpsi = K @ psi
    g_h = -Kpsi * N * u
    g_N = -Kpsi * h * u
    return u, objective(u, obs, target), 2.0 * np.conj(g_h), 2.0 * np.real(g_N)


# ----------------------------------------------------------------------------
# Charges, the field off the grid, and the solution-difference metric
# (Section 2, Section 4)
# ----------------------------------------------------------------------------

def charges(u, n, h, N, side=1.0, c_S=C_S_SPHERE) -> np.ndarray:
    """Total charge of the particles of each cell, Eq. 2.13 summed over a cell:
    every particle of Delta_p carries Q = -c_S a^(2-kappa) h(x_p) u_e(x_p), and
    a^(2-kappa) * #(Delta_p) = N_p |Delta_p| (Eq. 2.18), so the cell carries
    -c_S h_p N_p |Delta_p| u_p with u_p the solution of Eq. 2.19."""
    return -red_weights(h, N, cell_size(n, side), c_S) * np.asarray(u, dtype=np.complex128).ravel()


def field(points, u, n, k, h, N, alpha=None, origin=(0.0, 0.0, 0.0), side=1.0,
          c_S=C_S_SPHERE, chunk=256) -> np.ndarray:
    """The field of Eq. 2.10, u(x) = u0(x) + sum_m G(x, x_m) Q_m, by direct
    summation over the n^3 cells (Q from `charges`).  A point that coincides
    with a cell point x_j leaves out m = j: the sum is then the effective field
    of Eq. 2.14, which the solution u_j of Eq. 2.19 satisfies.  alpha = None
    returns the scattered part alone (no u0)."""
    pts = np.atleast_2d(np.asarray(points, dtype=np.float64))
    pos = cell_centres(n, origin, side)
    Q = charges(u, n, h, N, side, c_S)
    d = cell_size(n, side)
    out = np.empty(len(pts), dtype=np.complex128)
    for s in range(0, len(pts), chunk):
        diff = pts[s:s + chunk, None, :] - pos[None, :, :]
        r = np.sqrt((diff ** 2).sum(axis=2))
        G = np.zeros(r.shape, dtype=np.complex128)
        far = r > 1e-9 * d
        G[far] = greens_function(r[far], k)
        out[s:s + chunk] = G @ Q
    if alpha is not None:
        out += plane_wave(pts, k, alpha)
    return out


def table4_difference(fine, fine_points, coarse, n_coarse, origin=(0.0, 0.0, 0.0), side=1.0) -> float:
    """Solution difference of Section 4 (Table 4): the cube [origin, origin +
    side)^3 is cut into n_coarse^3 sub-cubes Delta_q, the coarse solution holds
    one value y_q per sub-cube, and the fine solution values x_i sit at the
    points fine_points[i].  For each Delta_q, average |x_i - y_q| over the fine
    points lying in Delta_q (sub-cubes are half-open, [q d, (q+1) d) per axis);
    return the largest average."""
    pts = np.asarray(fine_points, dtype=np.float64)
    dc = side / n_coarse
    # half-open sub-cubes [q dc, (q+1) dc): a point on a face belongs to the
    # sub-cube above it (the relative 1e-9 absorbs rounding of the coordinates)
    idx = np.floor((pts - np.asarray(origin, dtype=np.float64)) / dc + 1e-9).astype(np.int64)
    inside = np.all((idx >= 0) & (idx < n_coarse), axis=1)
    q = (idx[:, 2] * n_coarse + idx[:, 1]) * n_coarse + idx[:, 0]
    diff = np.abs(np.asarray(fine, dtype=np.complex128).ravel() - np.asarray(coarse).ravel()[np.where(inside, q, 0)])
    sums = np.bincount(q[inside], weights=diff[inside], minlength=n_coarse ** 3)
    counts = np.bincount(q[inside], minlength=n_coarse ** 3)
    has = counts > 0
    return float(np.max(sums[has] / counts[has]))
