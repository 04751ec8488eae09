"""Python face of the C ABI: a Plan object over torch CUDA tensors.

Every operation runs in libori.so on the GPU; this module only checks tensor
types and passes pointers and the current CUDA stream.  The system is Eq. 2.19
of the paper (RED; ORI when each cell holds one particle and N = 1):
    u_q + c_S sum_{p != q} G(x_q, x_p) h_p N_p |Delta_p| u_p = u0_q.
"""

from __future__ import annotations

import ctypes as C
import math
import os

import torch

from . import _lib
from ._lib import ORI_DF, ORI_FORM_A, ORI_FORM_B, ORI_FP32, ORI_FP64, ORI_MIXED, OriError  # noqa: F401

_FORMS = {"A": ORI_FORM_A, "B": ORI_FORM_B}
_PREC = {"fp64": ORI_FP64, "fp32": ORI_FP32, "mixed": ORI_MIXED, "df": ORI_DF}


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _plain(t: torch.Tensor) -> torch.Tensor:
    """A dense tensor whose memory holds its values.  torch.conj() and negation
    can return lazy views (a conjugate or negative bit over the original
    memory) that stay lazy under .contiguous(); C reads the memory, so the bits
    are resolved first."""
    return t.resolve_conj().resolve_neg().contiguous()


def _need(t: torch.Tensor, dtype, numel: int, name: str) -> torch.Tensor:
    """An input argument: checked, then made plain (see _plain)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return _plain(t)


def _out(t: torch.Tensor, dtype, numel: int, name: str) -> torch.Tensor:
    """An output argument: written in place, so it must already be dense memory
    of the right type and size (a copy would leave the caller's tensor unwritten)."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    if not t.is_contiguous() or t.is_conj() or t.is_neg():
        raise ValueError(f"{name} must be contiguous, without a lazy conjugate or negative bit")
    return t


def solve_opts(tol=1e-6, precision="mixed", maxit=1000, inner_tol=1e-5, max_outer=8,
               check_every=8, alpha=(0.0, 0.0, 1.0), use_graph=True, residual="df",
               resid_update=True, x0=None, history=False) -> _lib.SolveOpts:
    lib = _lib.load()
    o = _lib.SolveOpts()
    lib.ori_default_solve_opts(C.byref(o))
    o.tol = float(tol)
    o.precision = _PREC[precision]
    o.maxit = int(maxit)
    o.inner_tol = float(inner_tol)
    o.max_outer = int(max_outer)
    o.check_every = int(check_every)
    for i in range(3):
        o.alpha[i] = float(alpha[i])
    o.use_graph = 1 if use_graph else 0
    o.residual = _PREC[residual]
    o.resid_update = 1 if resid_update else 0
    o.history = 1 if history else 0
    if x0 is not None:
        if not (isinstance(x0, torch.Tensor) and x0.is_cuda and x0.dtype == torch.complex128
                and x0.is_contiguous() and not x0.is_conj() and not x0.is_neg()):
            raise TypeError("x0 must be a contiguous complex128 CUDA tensor without a lazy conjugate or negative bit")
        o.x0 = x0.data_ptr()
    return o


class Plan:
    """Operator for one grid (n^3 cells of a cube), wave number k and medium (h, N).

    h: complex128 CUDA tensor of n^3 impedances, N: float64 CUDA tensor of n^3
    densities, both C-ordered [z][y][x].  c_S defaults to 4 pi (spheres).
    k may be a sequence of wave numbers: the plan then holds one spectrum per
    entry, ``solve_batch`` solves for all of them, and the single-system
    calls use the first.  ``spectrum``: the bytes of ``save_spectrum`` of a
    plan with the same n, padded length, c_S and side (or a path to a file of
    them); the plan then takes its spectra from there instead of computing
    them, and its wave numbers are the saved ones (k is ignored)."""

    def __init__(self, n: int, k, h: torch.Tensor, N: torch.Tensor, side: float = 1.0,
                 origin=(0.0, 0.0, 0.0), c_S: float | None = None, mem_cap: int = 0, min_L: int = 0,
                 lean: bool = False, stream=None, spectrum=None):
        lib = _lib.load()
        self.n = int(n)
        if spectrum is not None:
            if isinstance(spectrum, (str, os.PathLike)):
                with open(spectrum, "rb") as f:
                    spectrum = f.read()
            spectrum = bytes(spectrum)
            k = list(_saved_wave_numbers(spectrum))
        self.ks = [float(v) for v in k] if hasattr(k, "__len__") else [float(k)]
        if not self.ks:
            raise ValueError("k must hold at least one wave number")
        self.k = self.ks[0]
        self.side = float(side)
        self.origin = tuple(float(v) for v in origin)
        self.c_S = 4.0 * math.pi if c_S is None else float(c_S)
        m = self.n ** 3
        h = _need(h, torch.complex128, m, "h")
        N = _need(N, torch.float64, m, "N")
        self.device = h.device
        dom = _lib.Domain()
        for i in range(3):
            dom.origin[i] = self.origin[i]
        dom.side = self.side
        po = _lib.PlanOpts()
        lib.ori_default_plan_opts(C.byref(po))
        po.c_S = self.c_S
        po.mem_cap = int(mem_cap)
        po.min_L = int(min_L)
        po.lean = 1 if lean else 0
        ks_arr = (C.c_double * len(self.ks))(*self.ks)
        if len(self.ks) > 1:
            po.n_k = len(self.ks)
            po.ks = C.cast(ks_arr, C.POINTER(C.c_double))
        handle = C.c_void_p()
        with torch.cuda.device(self.device):
            if spectrum is not None:
                st = lib.ori_plan_from_spectrum(self.n, C.byref(dom), h.data_ptr(), N.data_ptr(), C.byref(po),
                                                spectrum, len(spectrum), _stream_ptr(stream), C.byref(handle))
            else:
                st = lib.ori_plan(self.n, self.k, C.byref(dom), h.data_ptr(), N.data_ptr(), C.byref(po),
                                  _stream_ptr(stream), C.byref(handle))
        _lib.check(st, "ori_plan_from_spectrum" if spectrum is not None else "ori_plan")
        self._h = handle
        nn, LL, by = C.c_int64(), C.c_int64(), C.c_size_t()
        lib.ori_plan_info(self._h, C.byref(nn), C.byref(LL), C.byref(by))
        self.L = int(LL.value)
        self.bytes = int(by.value)
        self.medium_version = 0   # counts set_medium calls (OriSolve checks it in backward)

    # -- lifetime ------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _lib.load().ori_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    # -- accounting ------------------------------------------------------------
    def set_timing(self, on: bool = True):
        """Bracket every kernel of this plan with CUDA events (summed per pass kind)."""
        _lib.check(_lib.load().ori_plan_set_timing(self.handle, 1 if on else 0), "ori_plan_set_timing")

    def stats(self) -> dict:
        st = _lib.PlanStats()
        _lib.check(_lib.load().ori_plan_get_stats(self.handle, C.byref(st)), "ori_plan_get_stats")
        return st.as_dict()

    def reset_stats(self):
        _lib.check(_lib.load().ori_plan_reset_stats(self.handle), "ori_plan_reset_stats")

    # -- launch schedule -------------------------------------------------------
    def schedule(self) -> dict:
        sc = _lib.Schedule()
        _lib.check(_lib.load().ori_plan_get_schedule(self.handle, C.byref(sc)), "ori_plan_get_schedule")
        return sc.as_dict()

    def set_schedule(self, schedule: dict):
        sc = _lib.Schedule.from_dict(schedule)
        _lib.check(_lib.load().ori_plan_set_schedule(self.handle, C.byref(sc)), "ori_plan_set_schedule")

    def autotune_now(self, nrhs: int = 1, reps: int = 3, stream=None):
        """Time the candidate schedules for a batch of nrhs systems and keep the
        fastest; returns (schedule dict, FP32 operator ms for the batch)."""
        sc = _lib.Schedule()
        ms = C.c_float()
        with torch.cuda.device(self.device):
            st = _lib.load().ori_plan_autotune(self.handle, int(nrhs), int(reps), C.byref(sc), C.byref(ms),
                                               _stream_ptr(stream))
        _lib.check(st, "ori_plan_autotune")
        return sc.as_dict(), float(ms.value)

    def autotune(self, nrhs: int = 1, path: str | None = None, reps: int = 3, force: bool = False) -> dict:
        """Schedule for this GPU, n and batch size from the JSON cache, else timed and cached."""
        from . import autotune as _at
        name = torch.cuda.get_device_name(self.device)
        return _at.tune(self, nrhs, name, path=path, reps=reps, force=force)

    # -- saved spectra and residual histories --------------------------------------
    def save_spectrum(self, path: str | None = None, stream=None) -> bytes:
        """The plan's kernel spectra in their saved form (ori_plan_save_spectrum);
        written to `path` as well when given.  Plan(..., spectrum=...) reuses them."""
        lib = _lib.load()
        nb = C.c_size_t()
        _lib.check(lib.ori_plan_spectrum_bytes(self.handle, C.byref(nb)), "ori_plan_spectrum_bytes")
        buf = C.create_string_buffer(nb.value)
        with torch.cuda.device(self.device):
            _lib.check(lib.ori_plan_save_spectrum(self.handle, buf, nb.value, _stream_ptr(stream)),
                       "ori_plan_save_spectrum")
        data = buf.raw
        if path is not None:
            with open(path, "wb") as f:
                f.write(data)
        return data

    def residual_history(self, system: int = 0) -> list:
        """COCG's residual estimates ||r|| / ||RHS|| after each iteration of the last
        solve run with history=True (refinement steps one after another)."""
        lib = _lib.load()
        cnt = C.c_int()
        _lib.check(lib.ori_plan_residual_history(self.handle, int(system), None, 0, C.byref(cnt)),
                   "ori_plan_residual_history")
        out = (C.c_double * max(1, cnt.value))()
        _lib.check(lib.ori_plan_residual_history(self.handle, int(system), out, cnt.value, C.byref(cnt)),
                   "ori_plan_residual_history")
        return [float(out[i]) for i in range(cnt.value)]

    # -- medium ----------------------------------------------------------------
    def set_medium(self, h: torch.Tensor, N: torch.Tensor, stream=None):
        m = self.n ** 3
        h = _need(h, torch.complex128, m, "h")
        N = _need(N, torch.float64, m, "N")
        _lib.check(_lib.load().ori_plan_set_medium(self.handle, h.data_ptr(), N.data_ptr(),
                                                   _stream_ptr(stream)), "ori_plan_set_medium")
        self.medium_version += 1

    # -- operator ----------------------------------------------------------------
    def matvec(self, x: torch.Tensor, form: str = "A", precision: str = "fp64", stream=None):
        """y = A x (form "A", Eq. 2.19) or B x = x + S K (S x) (form "B")."""
        x = _need(x, torch.complex128, self.n ** 3, "x")
        y = torch.empty_like(x)
        _lib.check(_lib.load().ori_matvec(self.handle, x.data_ptr(), y.data_ptr(), _FORMS[form],
                                          _PREC[precision], _stream_ptr(stream)), "ori_matvec")
        return y

    def matvec32(self, x: torch.Tensor, form: str = "B", out: torch.Tensor | None = None, stream=None):
        """The FP32 operator on complex64 vectors (what the mixed solver iterates with)."""
        x = _need(x, torch.complex64, self.n ** 3, "x")
        y = torch.empty_like(x) if out is None else _out(out, torch.complex64, self.n ** 3, "out")
        _lib.check(_lib.load().ori_matvec32(self.handle, x.data_ptr(), y.data_ptr(), _FORMS[form],
                                            _stream_ptr(stream)), "ori_matvec32")
        return y

    # -- solves ------------------------------------------------------------------
    def solve(self, rhs: torch.Tensor | None = None, out: torch.Tensor | None = None,
              raise_on_failure: bool = True, stream=None, **kw):
        """Solve A u = rhs (rhs None: plane wave exp(ik alpha . x)); returns (u, info dict)."""
        m = self.n ** 3
        if rhs is not None:
            rhs = _need(rhs, torch.complex128, m, "rhs")
        if kw.get("x0") is not None:
            kw["x0"] = _need(kw["x0"], torch.complex128, m, "x0")
        u = torch.empty(m, dtype=torch.complex128, device=self.device) if out is None else _out(out, torch.complex128, m, "out")
        o = solve_opts(**kw)
        info = _lib.SolveInfo()
        st = _lib.load().ori_cocg_solve(self.handle, rhs.data_ptr() if rhs is not None else None,
                                        u.data_ptr(), C.byref(o), C.byref(info), _stream_ptr(stream))
        if raise_on_failure:
            _lib.check(st, "ori_cocg_solve")
        d = info.as_dict()
        d["returned"] = st
        if kw.get("history"):
            d["history"] = self.residual_history(0)
        return u, d

    def solve_media(self, hs, Ns, us, raise_on_failure: bool = True, **kw):
        """Solve for a sequence of media held in host memory: for each i, set
        the medium (hs[i], Ns[i]), solve, and copy the solution into us[i].

        hs[i] (complex128), Ns[i] (float64) and us[i] (complex128) are CPU
        tensors of n^3 values; pinned ones (``pin_memory()``) let the copies
        run on the copy engines while the GPU solves: the inputs of the next
        media travel to the device and the solutions of the previous ones to
        the host during the solve of medium i, through three device buffers
        of each.
        An entry of us may repeat (the copies into it follow one another).
        ``kw`` are the options of ``solve``.  Returns the info dicts."""
        count = len(hs)
        if len(Ns) != count or len(us) != count:
            raise ValueError("hs, Ns and us must have the same length")
        m = self.n ** 3
        for name, seq, dt in (("hs", hs, torch.complex128), ("Ns", Ns, torch.float64), ("us", us, torch.complex128)):
            for t in seq:
                if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != dt or t.numel() != m \
                        or not t.is_contiguous():
                    raise TypeError(f"every entry of {name} must be a contiguous CPU {dt} tensor of {m} values")
        dev = self.device
        main = torch.cuda.current_stream(dev)
        cin, cout = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        # three device buffers of each: the inputs of two media ahead are on
        # their way while one is solved, and a solution has two solves' time
        # to reach the host before its buffer is reused (host-link copy rates
        # vary from run to run; the slack absorbs slow copies)
        nb = min(3, count)
        ahead = max(1, nb - 1)
        hb = [torch.empty(m, dtype=torch.complex128, device=dev) for _ in range(nb)]
        Nb = [torch.empty(m, dtype=torch.float64, device=dev) for _ in range(nb)]
        ub = [torch.empty(m, dtype=torch.complex128, device=dev) for _ in range(nb)]
        # an event that was never recorded is complete for a waiting stream
        uploaded = [torch.cuda.Event() for _ in range(nb)]
        consumed = [torch.cuda.Event() for _ in range(nb)]
        solved = [torch.cuda.Event() for _ in range(nb)]
        downloaded = [torch.cuda.Event() for _ in range(nb)]

        def upload(i):
            b = i % nb
            cin.wait_event(consumed[b])          # set_medium of medium i - nb has read the buffers
            with torch.cuda.stream(cin):
                hb[b].copy_(hs[i], non_blocking=True)
                Nb[b].copy_(Ns[i], non_blocking=True)
            uploaded[b].record(cin)

        def download(i):
            b = i % nb
            cout.wait_event(solved[b])
            with torch.cuda.stream(cout):
                us[i].copy_(ub[b], non_blocking=True)
            downloaded[b].record(cout)

        infos = []
        for i in range(min(ahead, count)):
            upload(i)
        for i in range(count):
            b = i % nb
            main.wait_event(uploaded[b])
            self.set_medium(hb[b], Nb[b], stream=main)
            consumed[b].record(main)
            if i + ahead < count:
                upload(i + ahead)
            main.wait_event(downloaded[b])       # the solution of medium i - nb has left ub[b]
            _, info = self.solve(out=ub[b], raise_on_failure=raise_on_failure, stream=main, **kw)
            solved[b].record(main)
            download(i)
            infos.append(info)
        cout.synchronize()
        # the caller's stream is ordered after the copies into us
        for b in range(nb):
            main.wait_event(downloaded[b])
        return infos

    def solve_batch(self, alphas=None, rhs: torch.Tensor | None = None, out: torch.Tensor | None = None,
                    raise_on_failure: bool = True, stream=None, **kw):
        """Solve for every wave number of the plan and every incidence direction at once.

        alphas: sequence of ndir directions (x, y, z) for plane-wave right-hand sides, or
        None with rhs: complex128 tensor of shape (n_k, ndir, n^3) (or anything of that
        size).  Returns (u of shape (n_k, ndir, n^3), list of n_k * ndir info dicts with
        system r = i * ndir + j)."""
        m = self.n ** 3
        nk = len(self.ks)
        if rhs is not None:
            if rhs.numel() % (nk * m) != 0:
                raise ValueError(f"rhs must hold n_k * ndir * {m} elements")
            ndir = rhs.numel() // (nk * m)
            rhs = _need(rhs, torch.complex128, nk * ndir * m, "rhs")
            al = None
        else:
            if alphas is None:
                raise ValueError("give alphas or rhs")
            dirs = [tuple(float(c) for c in a) for a in alphas]
            if not dirs or any(len(a) != 3 for a in dirs):
                raise ValueError("alphas must be a non-empty sequence of 3-vectors")
            ndir = len(dirs)
            al = (C.c_double * (3 * ndir))(*[c for a in dirs for c in a])
        u = (torch.empty(nk * ndir * m, dtype=torch.complex128, device=self.device)
             if out is None else _out(out, torch.complex128, nk * ndir * m, "out"))
        if kw.get("x0") is not None:
            kw["x0"] = _need(kw["x0"], torch.complex128, nk * ndir * m, "x0")
        o = solve_opts(**kw)
        infos = (_lib.SolveInfo * (nk * ndir))()
        st = _lib.load().ori_cocg_solve_batch(self.handle, ndir, C.cast(al, C.c_void_p) if al is not None else None,
                                              rhs.data_ptr() if rhs is not None else None, u.data_ptr(),
                                              C.byref(o), C.cast(infos, C.c_void_p), _stream_ptr(stream))
        if raise_on_failure:
            _lib.check(st, "ori_cocg_solve_batch")
        out_infos = []
        for i in range(nk * ndir):
            d = infos[i].as_dict()
            d["returned"] = st
            out_infos.append(d)
        return u.view(nk, ndir, m), out_infos

    def field(self, u: torch.Tensor, points: torch.Tensor, alpha=None, stream=None) -> torch.Tensor:
        """Field of Eq. 2.10 at `points` (float64 CUDA tensor of shape (npts, 3)) for the
        solution u: the scattered part, plus the incident wave when alpha is given."""
        u = _need(u, torch.complex128, self.n ** 3, "u")
        if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float64
                and points.dim() == 2 and points.shape[1] == 3):
            raise TypeError("points must be a float64 CUDA tensor of shape (npts, 3)")
        points = _plain(points)
        out = torch.empty(points.shape[0], dtype=torch.complex128, device=self.device)
        al = None if alpha is None else (C.c_double * 3)(*[float(v) for v in alpha])
        _lib.check(_lib.load().ori_field(self.handle, u.data_ptr(), int(points.shape[0]), points.data_ptr(),
                                         C.cast(al, C.c_void_p) if al is not None else None, out.data_ptr(),
                                         _stream_ptr(stream)), "ori_field")
        return out

    def adjoint(self, u: torch.Tensor, econj: torch.Tensor, raise_on_failure: bool = True,
                stream=None, **kw):
        """Gradient of J = sum_obs |u_o - t_o|^2 w.r.t. h and N; econj = conj(u - t) on the
        observation cells and 0 elsewhere.  Returns (grad_h, grad_N, info)."""
        m = self.n ** 3
        u = _need(u, torch.complex128, m, "u")
        econj = _need(econj, torch.complex128, m, "econj")
        gh = torch.empty(m, dtype=torch.complex128, device=self.device)
        gN = torch.empty(m, dtype=torch.float64, device=self.device)
        o = solve_opts(**kw)
        info = _lib.SolveInfo()
        st = _lib.load().ori_adjoint_solve(self.handle, u.data_ptr(), econj.data_ptr(), gh.data_ptr(),
                                           gN.data_ptr(), C.byref(o), C.byref(info), _stream_ptr(stream))
        if raise_on_failure:
            _lib.check(st, "ori_adjoint_solve")
        d = info.as_dict()
        d["returned"] = st
        return gh, gN, d


def _saved_wave_numbers(data: bytes):
    """Wave numbers stored in a saved spectrum's header (the library checks the rest)."""
    import struct
    if len(data) < 576 or data[:8] != b"ORISPEC\0":
        raise ValueError("not a saved spectrum")
    n_k = struct.unpack_from("<i", data, 20)[0]
    if not 1 <= n_k <= 64:
        raise ValueError("saved spectrum: bad wave-number count")
    return struct.unpack_from(f"<{n_k}d", data, 48)


def solve(h: torch.Tensor, N: torch.Tensor, k, side: float = 1.0, origin=(0.0, 0.0, 0.0), rhs=None,
          c_S: float | None = None, lean: bool = False, **kw):
    """One call: build a plan for the n^3 grid of h (complex128) and N (float64), solve
    Eq. 2.19 (rhs None: the plane wave of direction `alpha`), free the plan.  Returns
    (u, info).  Keep a Plan instead when solving repeatedly on one medium."""
    n = int(round(h.numel() ** (1.0 / 3.0)))
    if n ** 3 != h.numel():
        raise ValueError("h must hold n^3 values")
    with Plan(n, k, h, N, side=side, origin=origin, c_S=c_S, lean=lean) as plan:
        return plan.solve(rhs=rhs, **kw)


class OriSolve(torch.autograd.Function):
    """u = A(h, N)^-1 rhs with a hand-written adjoint backward.

    The forward solution is kept for the backward (one checkpoint, no
    per-iteration storage); the backward is one more COCG solve on the same
    plan (A^T = S B S^-1) plus elementwise products.  The medium of the
    forward (h, N) is saved too: if the plan's medium changed in between (a
    later forward or set_medium on the same plan), the backward puts it back
    before the adjoint solve, so each graph gets the gradient of its own
    forward."""

    @staticmethod
    def forward(ctx, h, N, plan: Plan, rhs, kw):
        hd, Nd = h.detach(), N.detach()
        plan.set_medium(hd, Nd)
        u, info = plan.solve(rhs, **kw)
        ctx.plan = plan
        ctx.kw = kw
        ctx.info = info
        ctx.medium_version = plan.medium_version
        ctx.save_for_backward(u, hd, Nd)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        u, hd, Nd = ctx.saved_tensors
        if ctx.plan.medium_version != ctx.medium_version:
            ctx.plan.set_medium(hd, Nd)
            ctx.medium_version = ctx.plan.medium_version
        # grad_u = dL/dRe u + i dL/dIm u; dL = Re(conj(grad_u) du) = 2 Re(conj(e) du), e = grad_u / 2
        econj = torch.conj(grad_u).contiguous() * 0.5
        gh, gN, _ = ctx.plan.adjoint(u, econj.to(torch.complex128), **ctx.kw)
        return gh, gN, None, None, None


def solve_autograd(plan: Plan, h: torch.Tensor, N: torch.Tensor, rhs=None, **kw):
    """Differentiable solve: gradients flow to h (complex) and N (real)."""
    return OriSolve.apply(h, N, plan, rhs, kw)
