"""Parity at the benchmark's sizes, through the C ABI, against the CPU oracle.

* The n = 512 operator (1024^3 padded FFTs) in the two arithmetics the mixed
  solve of the benchmark runs: the FP32 operator (fifteen applications per
  solve) and the paired-FP32 operator of the refinement residual, on output
  rows chosen per tile class, against the oracle's direct sums (Eq. 2.19).
* The FP64 and paired-FP32 operators at L = 1024 (n = 260) against oracle rows.
* Configuration 3 of the benchmark (k = 5, seeded h and N): the mixed solve to
  relres 1e-6 against the FP64 solve to 1e-10, at n = 256 and n = 512.

Output cell (z, y, x) of the operator: the X-inverse pass writes whole lines
(z, y) in tiles of consecutive lines, the Y-inverse pass writes y < n of one z
plane in tiles of 16 frequency columns, and the Z pass mixes every (ky, kx)
tile into every output cell.  Rows are therefore taken on a grid of z, y and x
classes (first, second, middle, last lines and planes; x at both sides of a
16-column boundary and at the end of a line) plus random cells.

Tolerances: FP32 operator 1e-5 relative L2 (also the bar of the solver's
residual-update bound), and each row's error at most 3e-5 of the rows' RMS;
FP64 and paired FP32 1e-12; mixed vs FP64 solutions 1e-5.
"""

from concurrent.futures import ThreadPoolExecutor

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


def max_row_err(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(np.abs(b) ** 2)))


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def tile_class_rows(n, seed, extra=16):
    zs = [0, 1, n // 2, n - 1]
    ys = [0, 1, n // 2 - 1, n - 1]
    xs = [0, 15, 16, n - 1]
    rows = [(z * n + y) * n + x for z in zs for y in ys for x in xs]
    rng = np.random.default_rng(seed)
    rows += [int(r) for r in rng.choice(n ** 3, extra, replace=False)]
    return np.array(sorted(set(rows)), dtype=np.int64)


def oracle_offdiag_rows(v, rows, n, k):
    """sum_{p != q} G v_p on `rows` by the oracle, the rows spread over host threads."""
    G = O.kernel_octant(n, k)
    with ThreadPoolExecutor(16) as ex:
        parts = list(ex.map(lambda q: O.offdiag_sum_rows_octant(v, [q], n, k, octant=G)[0], rows))
    return np.array(parts)


def test_n512_fp32_and_paired_operators_on_tile_class_rows():
    """y = B x = x + S c_S |Delta| K (S x) at n = 512 (config 3): the FP32
    operator the inner COCG iterates with (the persistent pipelined passes the
    benchmark times) and the paired-FP32 operator of the refinement residual."""
    from paper_1602_04691_gb300 import Plan
    n, k = 512, 5.0
    h, N = inputs.random_h_N(n, 3)
    x32 = inputs.random_complex(n ** 3, 9).astype(np.complex64)
    x64 = x32.astype(np.complex128)
    plan = Plan(n, k, to_dev(h), to_dev(N))
    assert plan.L == 1024
    y32 = plan.matvec32(to_dev(x32), form="B").cpu().numpy()
    ydf = plan.matvec(to_dev(x64), form="B", precision="df").cpu().numpy()
    plan.close()
    del plan
    torch.cuda.empty_cache()
    rows = tile_class_rows(n, 10)
    assert rows.size >= 64
    S = O.sqrt_hN(h, N)
    d = 1.0 / n
    ref = x64[rows] + S[rows] * (O.C_S_SPHERE * d ** 3) * oracle_offdiag_rows(S * x64, rows, n, k)
    assert rel(y32[rows], ref) < 1e-5
    assert max_row_err(y32[rows], ref) < 3e-5
    assert rel(ydf[rows], ref) < 1e-12


def test_n520_fp32_operator_on_tile_class_rows():
    """n = 520 pads to L = 2048 (the paper-scale passes); 8-column tiles there."""
    from paper_1602_04691_gb300 import Plan
    n, k = 520, 5.0
    h, N = inputs.random_h_N(n, 603)
    x = inputs.random_complex(n ** 3, 604).astype(np.complex64)
    plan = Plan(n, k, to_dev(h), to_dev(N))
    assert plan.L == 2048
    y = plan.matvec32(to_dev(x), form="B").cpu().numpy()
    plan.close()
    del plan
    torch.cuda.empty_cache()
    rows = tile_class_rows(n, 11)
    S = O.sqrt_hN(h, N)
    xs = S * x.astype(np.complex128)
    ref = x[rows] + S[rows] * (O.C_S_SPHERE / n ** 3) * oracle_offdiag_rows(xs, rows, n, k)
    assert rel(y[rows], ref) < 1e-5
    assert max_row_err(y[rows], ref) < 3e-5


@pytest.mark.parametrize("precision", ["fp64", "df"])
def test_n260_fp64_class_operators_vs_oracle_rows(precision):
    """A form y = x + c_S |Delta| K (h N x) at L = 1024 (n = 260), 1e-12."""
    from paper_1602_04691_gb300 import Plan
    n, k = 260, 5.0
    h, N = inputs.random_h_N(n, 40 + n)
    x = inputs.random_complex(n ** 3, 50 + n)
    plan = Plan(n, k, to_dev(h), to_dev(N))
    assert plan.L == 1024
    y = plan.matvec(to_dev(x), form="A", precision=precision).cpu().numpy()
    plan.close()
    del plan
    torch.cuda.empty_cache()
    rows = tile_class_rows(n, 12)
    w = O.red_weights(h, N, 1.0 / n)
    ref = x[rows] + oracle_offdiag_rows(w * x, rows, n, k)
    assert rel(y[rows], ref) < 1e-12


@pytest.mark.parametrize("n", [256, 512])
def test_config3_mixed_solve_agrees_with_fp64(n):
    """k = 5, seeded h and N (seed 3): mixed to relres 1e-6 against FP64 to
    1e-10; both report ORI_OK and the solutions agree within 1e-5."""
    from paper_1602_04691_gb300 import Plan
    k = 5.0
    h, N = inputs.random_h_N(n, 3)
    plan = Plan(n, k, to_dev(h), to_dev(N))
    u64, i64 = plan.solve(tol=1e-10, precision="fp64")
    um, im = plan.solve(tol=1e-6, precision="mixed")
    assert i64["status"] == 0 and i64["relres"] <= 1e-10
    assert im["status"] == 0 and im["relres"] + im["relres_bound"] <= 1e-6
    err = float(torch.linalg.vector_norm(um - u64) / torch.linalg.vector_norm(u64))
    assert err < 1e-5
    plan.close()
    del plan
    torch.cuda.empty_cache()
