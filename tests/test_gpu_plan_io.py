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
* Plan.solve_media (media and solutions in host memory, the copies
  overlapping the solves) gives each medium's solution as set_medium and
  solve one by one do, and matches the oracle's LU solution (Eq. 2.19).
"""

import numpy as np
import pytest
import torch

import oracle as O
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


@pytest.mark.parametrize("precision,tol,bound", [("mixed", 1e-6, 2e-5), ("fp64", 1e-11, 1e-9)])
def test_solve_media_matches_one_by_one_and_oracle(precision, tol, bound):
    """Three media through solve_media with an output buffer used twice (it
    ends with the third solution) against set_medium + solve per medium, and
    each solution against dense LU of the oracle."""
    from paper_1602_04691_gb300 import Plan
    n, k = 10, 2.5
    media = [inputs.random_h_N(n, 700 + i) for i in range(3)]
    hs = [torch.from_numpy(h).pin_memory() for h, _ in media]
    Ns = [torch.from_numpy(N).pin_memory() for _, N in media]
    a = torch.empty(n ** 3, dtype=torch.complex128).pin_memory()
    b = torch.empty(n ** 3, dtype=torch.complex128).pin_memory()
    plan = Plan(n, k, to_dev(media[0][0]), to_dev(media[0][1]))
    infos = plan.solve_media(hs, Ns, [a, b, a], tol=tol, precision=precision)
    got = [a.numpy().copy(), b.numpy().copy()]
    want = []
    for h, N in media:
        plan.set_medium(to_dev(h), to_dev(N))
        u, _ = plan.solve(tol=tol, precision=precision)
        want.append(u.cpu().numpy())
    plan.close()
    assert all(i["returned"] == 0 for i in infos)
    for g, w in ((got[0], want[2]), (got[1], want[1])):
        assert np.linalg.norm(g - w) / np.linalg.norm(w) <= 1e-13
    u0 = O.plane_wave(O.cell_centres(n), k)
    for i, (h, N) in enumerate(media):
        ref = O.solve_dense(O.red_matrix(n, k, h, N), u0)
        assert np.linalg.norm(want[i] - ref) / np.linalg.norm(ref) <= bound, i


def test_solve_media_rejects_device_or_mistyped_entries():
    from paper_1602_04691_gb300 import Plan
    n = 4
    h, N = inputs.random_h_N(n, 9)
    plan = Plan(n, 1.0, to_dev(h), to_dev(N))
    u = torch.empty(n ** 3, dtype=torch.complex128)
    with pytest.raises(TypeError):
        plan.solve_media([to_dev(h)], [torch.from_numpy(N)], [u])
    with pytest.raises(TypeError):
        plan.solve_media([torch.from_numpy(h)], [torch.from_numpy(N).float()], [u])
    with pytest.raises(ValueError):
        plan.solve_media([torch.from_numpy(h)], [], [u])
    plan.close()
