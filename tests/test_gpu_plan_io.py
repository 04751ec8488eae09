"""Saved kernel spectra and residual histories, through the C ABI.

* A plan built from another plan's saved spectra (ori_plan_save_spectrum,
  ori_plan_from_spectrum) applies the same operators bit for bit and solves
  to the same solutions; a lean plan can be built from a full plan's spectra
  and saves its own; a saved form for another grid, c_S or cube side, or a
  truncated one, is refused.
* The residual history of a solve (ori_solve_opts.history) holds COCG's
  recursive residual after every iteration: it falls to the tolerance, its
  last value matches the info of an FP64 solve, and a mixed solve records
  every FP32 iteration of its refinement steps.
"""

import numpy as np
import pytest
import torch

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


def test_plan_from_saved_spectrum_is_identical(tmp_path):
    from paper_1602_04691_gb300 import Plan
    n, ks, side = 20, [2.0, 3.5], 1.3
    h, N = inputs.random_h_N(n, 301)
    a = Plan(n, ks, to_dev(h), to_dev(N), side=side)
    saved = a.save_spectrum(str(tmp_path / "spec.bin"))
    assert len(saved) == 576 + 2 * (a.L // 2 + 1) ** 3 * 16
    b = Plan(n, 0.0, to_dev(h), to_dev(N), side=side, spectrum=str(tmp_path / "spec.bin"))
    assert b.ks == ks
    x = to_dev(inputs.random_complex(n ** 3, 302))
    for form in ("A", "B"):
        for prec in ("fp64", "fp32", "df"):
            assert torch.equal(a.matvec(x, form, prec), b.matvec(x, form, prec)), (form, prec)
    ua, ia = a.solve(tol=1e-8, precision="mixed")
    ub, ib = b.solve(tol=1e-8, precision="mixed")
    assert torch.equal(ua, ub) and ia["iters"] == ib["iters"]
    # a lean plan from the full plan's spectra, and back from the lean plan's own save
    lean = Plan(n, 0.0, to_dev(h), to_dev(N), side=side, spectrum=saved, lean=True)
    ul, _ = lean.solve(tol=1e-8, precision="mixed")
    # the same spectra; a lean plan recovers u = w / S by division (no stored 1 / S)
    assert float(torch.linalg.vector_norm(ul - ua) / torch.linalg.vector_norm(ua)) < 1e-13
    resaved = lean.save_spectrum()
    c = Plan(n, 0.0, to_dev(h), to_dev(N), side=side, spectrum=resaved)
    y64 = a.matvec(x, "B", "fp64")
    err = float(torch.linalg.vector_norm(c.matvec(x, "B", "fp64") - y64) / torch.linalg.vector_norm(y64))
    assert err < 1e-13                      # paired FP32 keeps about 48 bits of the FP64 spectrum


def test_saved_spectrum_for_another_plan_is_refused():
    from paper_1602_04691_gb300 import OriError, Plan
    from paper_1602_04691_gb300._lib import ORI_ERR_INVALID_ARG
    n = 12
    h, N = inputs.random_h_N(n, 303)
    saved = Plan(n, 1.5, to_dev(h), to_dev(N)).save_spectrum()
    h2, N2 = inputs.random_h_N(n + 1, 304)
    bad = [dict(n=n + 1, h=h2, N=N2),                  # another grid (n and L differ)
           dict(side=2.0), dict(c_S=3.0), dict(min_L=64)]
    for b in bad:
        nn = b.get("n", n)
        with pytest.raises(OriError) as e:
            Plan(nn, 0.0, to_dev(b.get("h", h)), to_dev(b.get("N", N)), side=b.get("side", 1.0),
                 c_S=b.get("c_S"), min_L=b.get("min_L", 0), spectrum=saved)
        assert e.value.status == ORI_ERR_INVALID_ARG, b
    with pytest.raises(OriError) as e:
        Plan(n, 0.0, to_dev(h), to_dev(N), spectrum=saved[:-16])
    assert e.value.status == ORI_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        Plan(n, 0.0, to_dev(h), to_dev(N), spectrum=b"not a spectrum" * 64)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-6)])
def test_residual_history_records_every_iteration(precision, tol):
    from paper_1602_04691_gb300 import Plan
    n, k = 24, 3.0
    h, N = inputs.random_h_N(n, 305)
    plan = Plan(n, k, to_dev(h), to_dev(N))
    _, info = plan.solve(tol=tol, precision=precision, history=True)
    hist = info["history"]
    assert len(hist) == info["iters"]
    assert all(np.isfinite(hist)) and hist[-1] < hist[0]
    if precision == "fp64":
        assert hist[-1] <= tol
        assert abs(hist[-1] - info["relres_recur"]) <= 1e-12 + 1e-6 * hist[-1]
    else:
        assert hist[-1] <= 10 * tol                  # the recursive estimate of the last FP32 step
    _, info2 = plan.solve(tol=tol, precision=precision)   # history off: the last recorded stays readable
    assert plan.residual_history(0) == hist
