"""ori_matvec_noalloc: the operator for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: their device memory belongs to another
framework's pool, or they must not risk the device-wide synchronisation an
allocation can cause, or they run under a no-allocation rule.  The entry
point keeps every intermediate in one static device array; this test checks
it against the oracle's direct sum (Eq. 2.19) and against the plan-based
entry point ori_matvec (FP64 A form) within the FP64 operator tolerance, on
two calls in a row (the array keeps the previous call's contents, which must
not leak into the next result), and checks that a call after the first one
leaves the device's free memory unchanged.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_1602_04691_gb300 import inputs

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1602_04691_gb300 import _lib
    return _lib


def _noalloc_into(_lib, n, k, side, h, N, x, y):
    dom = _lib.Domain()
    dom.side = side
    st = _lib.load().ori_matvec_noalloc(n, k, ctypes.byref(dom), 0.0, h.data_ptr(), N.data_ptr(),
                                        x.data_ptr(), y.data_ptr(),
                                        int(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, "ori_matvec_noalloc")
    torch.cuda.synchronize()


def _noalloc(_lib, n, k, side, h, N, x):
    y = torch.empty_like(x)
    _noalloc_into(_lib, n, k, side, h, N, x, y)
    return y.cpu().numpy()


@pytest.mark.parametrize("n", [5, 16])
def test_noalloc_matches_plan_matvec_twice(lib, n):
    from paper_1602_04691_gb300 import Plan
    k, side = 2.7, 1.3
    results = []
    for call in range(2):
        h, N = inputs.random_h_N(n, 900 + 10 * n + call)
        x = inputs.random_complex(n ** 3, 950 + 10 * n + call)
        hd, Nd, xd = (torch.from_numpy(a).to(DEV) for a in (h, N, x))
        plan = Plan(n, k, hd, Nd, side=side)
        ref = plan.matvec(xd, form="A", precision="fp64").cpu().numpy()
        plan.close()
        y = _noalloc(lib, n, k, side, hd, Nd, xd)
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err < 1e-12, f"call {call}: rel err {err}"
        direct = O.red_matvec_direct(x, n, k, h, N, side=side)
        err = np.linalg.norm(y - direct) / np.linalg.norm(direct)
        assert err < 1e-12, f"call {call}: rel err vs the oracle {err}"
        results.append(y)
    assert not np.array_equal(results[0], results[1])


def test_noalloc_call_allocates_nothing(lib):
    """After the first call's set-up, a call leaves the device's free memory as it was."""
    n, k, side = 16, 1.9, 1.0
    h, N = inputs.random_h_N(n, 977)
    x = inputs.random_complex(n ** 3, 978)
    hd, Nd, xd = (torch.from_numpy(a).to(DEV) for a in (h, N, x))
    y = torch.empty_like(xd)
    _noalloc_into(lib, n, k, side, hd, Nd, xd, y)
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc_into(lib, n, k, side, hd, Nd, xd, y)
    assert torch.cuda.mem_get_info()[0] == free0
    ref = O.red_matvec_direct(x, n, k, h, N, side=side)
    yn = y.cpu().numpy()
    assert np.linalg.norm(yn - ref) / np.linalg.norm(ref) < 1e-12


def test_noalloc_rejects_overlapping_buffers(lib):
    n = 4
    h = torch.ones(n ** 3, dtype=torch.complex128, device=DEV)
    N = torch.ones(n ** 3, dtype=torch.float64, device=DEV)
    buf = torch.zeros(2 * n ** 3, dtype=torch.complex128, device=DEV)
    dom = lib.Domain()
    dom.side = 1.0
    x, y = buf[:n ** 3], buf[n ** 3 // 2:n ** 3 // 2 + n ** 3]   # y starts inside x
    st = lib.load().ori_matvec_noalloc(n, 1.0, ctypes.byref(dom), 0.0, h.data_ptr(), N.data_ptr(),
                                       x.data_ptr(), y.data_ptr(), None)
    assert st == lib.ORI_ERR_INVALID_ARG
    assert b"overlap" in lib.load().ori_last_error()


def test_noalloc_rejects_oversize_grid(lib):
    n = 17
    h = torch.zeros(n ** 3, dtype=torch.complex128, device=DEV)
    N = torch.zeros(n ** 3, dtype=torch.float64, device=DEV)
    x = torch.zeros(n ** 3, dtype=torch.complex128, device=DEV)
    y = torch.empty_like(x)
    dom = lib.Domain()
    dom.side = 1.0
    st = lib.load().ori_matvec_noalloc(n, 1.0, ctypes.byref(dom), 0.0, h.data_ptr(), N.data_ptr(),
                                       x.data_ptr(), y.data_ptr(), None)
    assert st == lib.ORI_ERR_INVALID_ARG
    assert b"ORI_NOALLOC_MAX_N" in lib.load().ori_last_error()
