"""The C ABI library loads and exports every function include/ori.h declares
(no compute calls: these run without a GPU)."""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ori.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ori_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1602_04691_gb300 import build as b
    if not os.path.exists(b.LIB) and shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no nvcc to build libori.so")
    return b.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ori_plan", "ori_matvec", "ori_cocg_solve", "ori_adjoint_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_export(libpath):
    from paper_1602_04691_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()
    lib = _lib.load()
    assert lib.ori_abi_version() == 6
    assert lib.ori_status_string(0) == b"ok"
    assert lib.ori_status_string(5) == b"COCG breakdown"


def test_default_options_host_only(libpath):
    from paper_1602_04691_gb300 import _lib
    lib = _lib.load()
    o = _lib.SolveOpts()
    lib.ori_default_solve_opts(ctypes.byref(o))
    assert o.tol == 1e-6 and o.precision == _lib.ORI_MIXED and o.check_every == 8
    assert tuple(o.alpha) == (0.0, 0.0, 1.0)


def test_invalid_arguments_rejected_before_device_work(libpath):
    """Argument checks run on the host and return a status (no GPU needed)."""
    from paper_1602_04691_gb300 import _lib
    lib = _lib.load()
    dom = _lib.Domain()
    dom.side = 1.0
    h = ctypes.c_void_p()
    st = lib.ori_plan(1, 1.0, ctypes.byref(dom), 1, 1, None, None, ctypes.byref(h))
    assert st == _lib.ORI_ERR_INVALID_ARG and b"n must be" in lib.ori_last_error()
    st = lib.ori_plan(8, -1.0, ctypes.byref(dom), 1, 1, None, None, ctypes.byref(h))
    assert st == _lib.ORI_ERR_INVALID_ARG
    st = lib.ori_plan(8, float("nan"), ctypes.byref(dom), 1, 1, None, None, ctypes.byref(h))
    assert st == _lib.ORI_ERR_INVALID_ARG
    st = lib.ori_plan(8, 1.0, ctypes.byref(dom), None, 1, None, None, ctypes.byref(h))
    assert st == _lib.ORI_ERR_INVALID_ARG
    dom.side = 0.0
    st = lib.ori_plan(8, 1.0, ctypes.byref(dom), 1, 1, None, None, ctypes.byref(h))
    assert st == _lib.ORI_ERR_INVALID_ARG
    assert lib.ori_matvec(None, 1, 2, 0, 0, None) == _lib.ORI_ERR_INVALID_ARG
    assert lib.ori_cocg_solve(None, None, 1, None, None, None) == _lib.ORI_ERR_INVALID_ARG


def test_binding_resolves_lazy_conjugate_and_negative_views():
    """torch.conj() and negation can return views whose memory still holds the
    original values (a conjugate or negative bit), and .contiguous() keeps
    them lazy.  The binding hands raw pointers to C, so every input must be
    made plain first and no output may carry such a bit."""
    import torch
    from paper_1602_04691_gb300.ori import _plain
    x = torch.tensor([1 + 2j, 3 - 4j, -0.5 + 0.25j], dtype=torch.complex128)
    c = x.conj()
    assert c.contiguous().is_conj()                  # the trap: memory still holds x
    p = _plain(c)
    assert not p.is_conj() and not p.is_neg()
    assert torch.equal(torch.view_as_real(p), torch.view_as_real(x).mul(torch.tensor([1.0, -1.0], dtype=torch.float64)))
    q = _plain(torch._neg_view(c))
    assert not q.is_conj() and not q.is_neg()
    assert torch.equal(torch.view_as_real(q), torch.view_as_real(x).mul(torch.tensor([-1.0, 1.0], dtype=torch.float64)))


def test_build_stamp_covers_every_included_file():
    """Every local file a translation unit includes (directly or through another
    header) is hashed into the build stamp, so editing it rebuilds libori.so."""
    from paper_1602_04691_gb300 import build as b
    hashed = {os.path.realpath(f) for f in b.stamped_files()}
    seen, todo = set(), [os.path.realpath(os.path.join(b.CSRC, f)) for f in b.SOURCES]
    while todo:
        f = todo.pop()
        if f in seen:
            continue
        seen.add(f)
        with open(f) as fh:
            for inc in re.findall(r'^\s*#\s*include\s+"([^"]+)"', fh.read(), flags=re.M):
                path = os.path.realpath(os.path.join(os.path.dirname(f), inc))
                if os.path.exists(path):
                    todo.append(path)
    missing = sorted(seen - hashed)
    assert not missing, missing
    assert os.path.realpath(os.path.join(b.CSRC, "dfft.cuh")) in hashed
