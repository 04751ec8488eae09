#!/usr/bin/env python
"""Benchmark of the hot path: the mixed-precision COCG solve of Eq. 2.19.

Workload (one step = one solve): n = 512 cells per axis (P = 134,217,728 cells,
1024^3 padded FFTs), unit cube, k = 5, plane wave alpha = (0, 0, 1), seeded
h, N ~ U[0.5, 1.5] (inputs.random_h_N, seed 3), FP32 COCG with FP64 scalars
inside FP64 iterative refinement, to relative residual 1e-6.  The plan (the
kernel spectrum) is built once, outside the timed region, and reported apart.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
paper's algorithm restated in numpy/scipy, on the host cores) instead.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Solve time to rel-res 1e-6 + FFT-matvec HBM GB/s at n=512, mixed vs FP64"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--k", type=float, default=5.0)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-cpu-legs", action="store_true",
                    help="CPU baseline: only the full solve of the workload, not the smaller legs")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--matvec-reps", type=int, default=20)
    ap.add_argument("--no-cufft", action="store_true",
                    help="skip the cuFFT comparator (the same matvec through torch.fft on the full padded cube)")
    ap.add_argument("--lean", action="store_true",
                    help="lean plan (mixed solves only; needed for the largest grids, e.g. --n 1000)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch schedule (no autotuning before the timed region)")
    ap.add_argument("--schedule", default=None,
                    help="JSON object of ori_schedule fields to run with instead of autotuning (for example the "
                         "schedule a bench line reports, to profile the same kernels)")
    ap.add_argument("--experiment", action="store_true",
                    help="run the Section 4 experiment scaled to one GPU (RED n=20, IE n=40, ORI n=480) "
                         "and print its JSON line instead of the benchmark")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched leg (n=128, 16 directions x 4 wave numbers)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "source": "measured"}
    except Exception:
        return dict(PEAKS_FALLBACK, source="fallback")


# ---------------------------------------------------------------------------
# Algorithmic bytes per launch of each pass (complex element = 8 B in FP32,
# 16 B in FP64; N = n^3 cells; H = L/2 + 1).  COCG-mode prologue/epilogue.
# ---------------------------------------------------------------------------
def alg_bytes(kind: str, n: int, L: int, cb: int) -> float:
    N = n ** 3
    T1 = n * n * L
    T2 = n * L * L
    H3 = (L // 2 + 1) ** 3
    table = {}
    # exact per-kind counts (the zero halves of the padded cubes are never read):
    table["xfwd"] = (3 * N + N + T1) * cb        # read r, p, S; write p, T1 = [n][n][L]
    table["yfwd"] = (T1 + T2) * cb               # read T1 = [n][n][L]; write T2 = [n][L][L]
    table["zconv"] = (T2 + T2 + H3) * cb         # read and write T2 in place; spectrum once
    table["yinv"] = (T2 + T1) * cb               # read T2; write T1
    table["xinv"] = (T1 + 3 * N) * cb            # read T1, p, S; write q
    table["update"] = 6 * N * cb                 # read x, p, r, q; write x, r
    return float(table[kind])


def matvec_alg_bytes(n: int, L: int, cb: int) -> float:
    """Bytes of one standalone B-form matvec (y = x + S K(S x)): X fwd reads x, S and
    writes T1; Y fwd; Z conv; Y inv; X inv reads T1, x, S and writes y."""
    N, T1, T2, H3 = n ** 3, n * n * L, n * L * L, (L // 2 + 1) ** 3
    return float(((2 * N + T1) + (T1 + T2) + (2 * T2 + H3) + (T2 + T1) + (T1 + 3 * N)) * cb)


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1602_04691_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kind: str, n: int, variant: int = 0):
    """DRAM bytes per launch of pass `kind` (launch variant `variant`) from the
    committed ncu summary, only if the kernel sources are unchanged since it
    was taken and its figure is for this grid size (other sizes may pad to
    another L and run other kernels)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("source_hash") != source_hash():
        return None
    ent = d.get("kernels", {}).get(kind, {}).get(str(variant))
    if not ent or ent.get("n") != n:
        return None
    return ent["dram_bytes_per_launch"]


def split_L1(L: int) -> int:
    """First-stage radix of the default split L = L1 * L2 (Split<L> in the sources)."""
    lg = L.bit_length() - 1
    return 1 << ((lg + 1) // 2)


def fp32_kernel_name(kind: str, L: int, sched: dict) -> str:
    """The FP32 kernel that runs a pass of the B-form matvec at padded length L
    (L >= 64) under a launch schedule (1 = ORI_SCHED_TILES; *_variant: tile
    width and radix split of the persistent Y and Z kernels at L = 256..1024)."""
    tiles = {key: sched.get(key, 0) == 1 for key in ("yfwd", "zconv", "yinv")}
    if kind == "update":
        return "k_cocg_update<float>"
    L1 = split_L1(L)

    def pipe(key):
        v = sched.get(key + "_variant", 0) if 256 <= L <= 1024 else 0
        C, l1 = {0: (16, L1), 1: (8, L1), 2: (16, 2 * L1)}[v] if L <= 1024 else (8, L1)
        return C, l1

    if L <= 1024:
        (cy, ly), (cz, lz), (ci, li) = pipe("yfwd"), pipe("zconv"), pipe("yinv")
        return {"xfwd": f"k_xfwd_pipe<{L}, 4>", "xinv": f"k_xinv_pipe<{L}, 4>",
                "yfwd": f"k_strided<float, {L}>(FWD)" if tiles["yfwd"] else f"k_yfwd_pipe<float, {L}, {cy}, {ly}>",
                "zconv": f"k_strided<float, {L}>(ZCONV)" if tiles["zconv"] else f"k_zconv_pipe<float, {L}, {cz}, {lz}>",
                "yinv": f"k_strided<float, {L}>(INV)" if tiles["yinv"] else f"k_yinv_pipe<{L}, {ci}, {li}>"}[kind]
    return {"xfwd": f"k_xfwd_pipe<{L}, 4>", "xinv": f"k_xinv_pipe<{L}, 4>",
            "yfwd": f"k_strided_smem<float, {L}, 4>(FWD)" if tiles["yfwd"] else f"k_yfwd_pipe<float, {L}, 8, {L1}>",
            "zconv": f"k_zconv_smem<float, {L}, 8>" if tiles["zconv"] else f"k_zconv_pipe<float, {L}, 8, {L1}>",
            "yinv": f"k_strided_smem<float, {L}, 4>(INV)" if tiles["yinv"] else f"k_yinv_pipe<{L}, 8, {L1}>"}[kind]


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix=f"ori_clocks_rank{index}_", suffix=".csv")
        os.close(fd)

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                try:
                    rows.append({"sm": float(parts[1]), "max": float(parts[2]), "util": float(parts[4]),
                                 "hw": parts[6], "hwt": parts[7], "swt": parts[8], "pcap": parts[9]})
                except ValueError:
                    continue
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in load:
            if r["hw"].lower() == "active":
                reasons.add("hw_slowdown")
            if r["hwt"].lower() == "active":
                reasons.add("hw_thermal_slowdown")
            if r["swt"].lower() == "active":
                reasons.add("sw_thermal_slowdown")
            if r["pcap"].lower() == "active":
                reasons.add("sw_power_cap")
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


# ---------------------------------------------------------------------------
# CPU baseline: the oracle's restatement of the paper's algorithm (COCG with
# the Section 3 FFT convolution, complex64 as in Section 4) on the host cores
# ---------------------------------------------------------------------------
def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


class CpuSolve:
    """One CPU solve of the benchmark's workload, split into its plan (the
    kernel spectrum) and COCG iterations so that callers can time either."""

    def __init__(self, n, k, seed, dtype_name="complex64", workers=None):
        import numpy as np
        import oracle as O
        from paper_1602_04691_gb300 import inputs
        self.O, self.np = O, np
        self.n, self.k = n, k
        self.dtype = np.dtype(dtype_name).type
        self.workers = workers or os.cpu_count()
        self.h, self.N = inputs.random_h_N(n, seed)
        t0 = time.perf_counter()
        self.spec = O.kernel_spectrum_zero(n, k, dtype=self.dtype, workers=self.workers)
        self.plan_s = time.perf_counter() - t0

    def solve(self, tol, maxit=2000, callback=None):
        t0 = time.perf_counter()
        u, it, rr = self.O.solve_cocg_fft_cpu(self.n, self.k, self.h, self.N, tol=tol, maxit=maxit,
                                              dtype=self.dtype, workers=self.workers, spec=self.spec,
                                              callback=callback)
        return u, it, rr, time.perf_counter() - t0


def cpu_solve_leg(n, k, seed, tol, dtype_name="complex64", workers=None):
    cs = CpuSolve(n, k, seed, dtype_name, workers)
    u, it, rr, solve_s = cs.solve(tol)
    del cs.spec
    return {"n": n, "dtype": dtype_name, "plan_s": cs.plan_s, "solve_s": solve_s, "iters": it,
            "relres_recur": rr}, u


def cpu_legs(k, seed, tol, workers):
    """The other CPU legs, each measured: the oracle's direct-sum matvec (numpy,
    O(N^2)), dense LU at n = 12, and full CPU FFT-COCG solves at smaller n in
    complex64 and complex128."""
    import numpy as np
    import oracle as O
    from paper_1602_04691_gb300 import inputs
    legs = {"direct_sum_matvec_s": {}, "fft_cocg": []}
    for n in (12, 16, 24):
        h, N = inputs.random_h_N(n, seed)
        x = inputs.random_complex(n ** 3, seed + 1)
        t0 = time.perf_counter()
        O.red_matvec_direct(x, n, k, h, N)
        legs["direct_sum_matvec_s"][str(n)] = time.perf_counter() - t0
    t24 = legs["direct_sum_matvec_s"]["24"]
    legs["direct_sum_matvec_n512_extrapolated_s"] = t24 * (512 / 24) ** 6
    n = 12
    h, N = inputs.random_h_N(n, seed)
    t0 = time.perf_counter()
    A = O.red_matrix(n, k, h, N)
    u_lu = O.solve_dense(A, O.plane_wave(O.cell_centres(n), k))
    legs["dense_lu_n12_s"] = time.perf_counter() - t0
    del A, u_lu
    for n in (64, 128, 256):
        for dt in ("complex64", "complex128"):
            leg, _ = cpu_solve_leg(n, k, seed, tol, dt, workers)
            legs["fft_cocg"].append(leg)
    return legs


def cpu_baseline(n, k, seed, tol, u_gpu=None, legs=True):
    """Full CPU solve of the benchmark workload (measured, not scaled), and
    the smaller legs.  u_gpu: the GPU solution, compared with the CPU one."""
    import numpy as np
    workers = os.cpu_count()
    leg, u = cpu_solve_leg(n, k, seed, tol, "complex64", workers)
    out = {"value": leg["solve_s"], "unit": "s", "cores": workers, "kind": "oracle",
           "sample": (f"one full solve of this workload on the host: the oracle's COCG with the zero-padded "
                      f"FFT convolution (Section 3) in complex64 (Section 4's arithmetic), scipy.fft on "
                      f"{workers} threads (elementwise numpy on one), {leg['iters']} iterations to recursive "
                      f"relres {leg['relres_recur']:.2e}; plan (kernel spectrum) {leg['plan_s']:.1f} s not "
                      f"included; CPU {cpu_model()}"),
           "plan_s": leg["plan_s"], "iters": leg["iters"]}
    if u_gpu is not None:
        out["cpu_vs_gpu_rel_l2"] = float(np.linalg.norm(u - u_gpu) / np.linalg.norm(u_gpu))
    del u
    if legs:
        out["legs"] = cpu_legs(k, seed, tol, workers)
    return out


# ---------------------------------------------------------------------------
# Arms
# ---------------------------------------------------------------------------
def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reference_arm(args, world, rank):
    """The oracle (the paper's algorithm on the host cores, complex64 as in
    Section 4) on this workload.  The kernel spectrum is built once, untimed.
    A step is one COCG iteration of the CPU solve; warm-up and timed steps
    continue one solve to convergence, then start the next.  value = the wall
    time of the first complete solve in this run (measured); if no solve
    completes within the run, value = the mean iteration time x the iterations
    so far, marked as a lower bound."""
    if rank != 0:
        return
    cs = CpuSolve(args.n, args.k, args.seed, "complex64")
    total = args.warmup + args.steps
    marks = []                      # wall-clock time at the end of each iteration
    solves = []                     # (start, end, iterations) of each completed solve

    def note(it):
        marks.append(time.perf_counter())

    t_start = time.perf_counter()
    while len(marks) < total:
        t0 = time.perf_counter()
        _, it, rr, _ = cs.solve(args.tol, maxit=total - len(marks), callback=note)
        if rr <= args.tol:
            solves.append((t0, time.perf_counter(), it, rr))
        if it == 0:
            break
    timed = marks[args.warmup:total]
    starts = [marks[args.warmup - 1] if args.warmup > 0 else t_start] + timed[:-1]
    per_iter = [b - a for a, b in zip(starts, timed)]
    ms_step = 1e3 * statistics.mean(per_iter)
    if solves:
        s0 = solves[0]
        v = s0[1] - s0[0]
        how = (f"wall time of a complete CPU solve in this run ({s0[2]} iterations, recursive relres "
               f"{s0[3]:.2e})")
    else:
        v = ms_step / 1e3 * len(marks)
        how = f"no solve completed in {len(marks)} iterations: mean iteration x {len(marks)} (lower bound)"
    cpu = {"value": v, "unit": "s", "cores": cs.workers, "kind": "oracle",
           "sample": (f"oracle COCG + zero-padded FFT convolution (Section 3), complex64, scipy.fft on "
                      f"{cs.workers} threads; a step = one COCG iteration at the full size; value = {how}; "
                      f"plan {cs.plan_s:.1f} s not included; CPU {cpu_model()}")}
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
           "config": workload_config(args), "cpu_baseline": cpu,
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def workload_config(args):
    n = args.n
    L = 4
    while L < 2 * n:
        L *= 2
    return {"workload": (f"mixed-precision COCG solve of Eq. 2.19 to relres {args.tol:g}, n={n} "
                         f"(P={n ** 3:,} cells), {L}^3 padded FFTs, k={args.k:g}, unit cube, alpha=(0,0,1), "
                         f"h,N ~ U[0.5,1.5] seed {args.seed}"),
            "n": n, "L": L, "k": args.k, "tol": args.tol, "precision": "mixed FP32/FP64",
            "l2": "inputs larger than L2 (each complex64 vector is n^3*8 B)",
            "parallelism": f"replicas x{args.gpus}"}


def ours_arm(args, world, rank, local):
    import numpy as np
    import torch
    from paper_1602_04691_gb300 import Plan, inputs

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n, k = args.n, args.k
    h_np, N_np = inputs.random_h_N(n, args.seed)
    h_host = torch.from_numpy(h_np).pin_memory()
    N_host = torch.from_numpy(N_np).pin_memory()
    del h_np, N_np
    h_dev = h_host.to(dev, non_blocking=True)
    N_dev = N_host.to(dev, non_blocking=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = Plan(n, k, h_dev, N_dev, lean=args.lean)
    plan_s = time.perf_counter() - t0
    L = plan.L
    if args.lean and args.no_e2e and (args.no_cufft or args.matvec_reps <= 0):
        # a lean plan keeps no reference to h and N, and no later leg reads them:
        # give their 24 bytes a cell back to the solver's vectors (n = 1000)
        h_dev = N_dev = None
        torch.cuda.empty_cache()
    tune_path = os.path.join(tempfile.gettempdir(), f"ori_autotune_bench_{os.getpid()}.json")
    if args.schedule:
        plan.set_schedule(dict(plan.schedule(), **json.loads(args.schedule)))
        tuned = {"schedule": plan.schedule(), "ms": None}
    elif args.no_autotune:
        tuned = {"schedule": plan.schedule(), "ms": None}
    else:
        tuned = plan.autotune(nrhs=1, path=tune_path)
    kw = dict(tol=args.tol, precision="mixed")
    u = torch.empty(n ** 3, dtype=torch.complex128, device=dev)

    for _ in range(args.warmup):
        plan.solve(out=u, **kw)
    torch.cuda.synchronize()

    # ---- timed region: K solves, inputs resident ---------------------------
    plan.reset_stats()
    plan.set_timing(True)
    clocks = ClockSampler(local)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    infos = []
    for _ in range(args.steps):
        _, info = plan.solve(out=u, **kw)
        infos.append(info)
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ck = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    stats = plan.stats()
    plan.set_timing(False)
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_per_step = ms_total / args.steps
    value = ms_total / 1e3 / (args.steps * world)

    # ---- roofline of the dominant kernel (FP32 pass with the largest time) --
    pk = peaks()
    fp32_kinds = ["xfwd", "yfwd", "zconv", "yinv", "xinv", "update"]
    pm, pc = stats["pass_ms"], stats["pass_count"]
    dom = max(fp32_kinds, key=lambda kk: pm.get(kk + "_f32", 0.0))
    dom_ms = pm[dom + "_f32"] / max(1, pc[dom + "_f32"])
    ab = alg_bytes(dom, n, L, 8)
    achieved = ab / (dom_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": fp32_kernel_name(dom, L, plan.schedule()), "achieved": achieved,
            "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
            "traffic": traffic_from_profiles(dom, n, plan.schedule().get(dom + "_variant", 0)),
            "alg_bytes_per_launch": ab,
            "ms_per_launch": dom_ms, "peak_source": pk["source"] + " (burst copy)"}
    passes = {}
    for kk in fp32_kinds:
        key = kk + "_f32"
        if pc.get(key):
            per = pm[key] / pc[key]
            b = alg_bytes(kk, n, L, 8)
            passes[kk] = {"launches": pc[key], "ms_total": pm[key], "ms_per_launch": per,
                          "alg_GBps": b / (per * 1e-3) / 1e9}
    for kk, v in pm.items():
        if kk.endswith("_f64") or kk.endswith("_df") or kk.startswith("vector"):
            passes[kk] = {"launches": pc[kk], "ms_total": v, "ms_per_launch": v / max(1, pc[kk])}

    # ---- standalone FP32 matvec (the operator the inner COCG applies) -------
    matvec = None
    if args.matvec_reps > 0:
        x32 = torch.randn(n ** 3, dtype=torch.complex64, device=dev)
        y32 = torch.empty_like(x32)
        for _ in range(3):
            plan.matvec32(x32, "B", out=y32)
        torch.cuda.synchronize()
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        m0.record()
        for _ in range(args.matvec_reps):
            plan.matvec32(x32, "B", out=y32)
        m1.record()
        torch.cuda.synchronize()
        mv_ms = m0.elapsed_time(m1) / args.matvec_reps
        mv_bytes = matvec_alg_bytes(n, L, 8)
        matvec = {"fp32_ms": mv_ms, "alg_bytes": mv_bytes, "alg_GBps": mv_bytes / (mv_ms * 1e-3) / 1e9,
                  "frac_of_hbm": mv_bytes / (mv_ms * 1e-3) / 1e9 / pk["hbm_gbs"]}
        if not args.no_cufft and rank == 0:
            _last_ms[:] = [mv_ms]
            matvec["cufft_comparator"] = cufft_comparator(plan, h_dev, N_dev, x32, y32, n, k, L, dev)
        del x32, y32

    # ---- plain FP64 GPU solve (comparator), once -------------------------------
    fp64 = None
    if not args.no_fp64 and rank == 0:
        u64 = torch.empty_like(u)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        _, i64 = plan.solve(out=u64, tol=args.tol, precision="fp64", maxit=2000)
        f1.record()
        torch.cuda.synchronize()
        diff = float(torch.linalg.vector_norm(u - u64) / torch.linalg.vector_norm(u64))
        fp64 = {"s": f0.elapsed_time(f1) / 1e3, "iters": i64["iters"], "relres": i64["relres"],
                "mixed_vs_fp64_rel_l2": diff, "speedup_mixed": f0.elapsed_time(f1) / ms_per_step}
        del u64

    # ---- mixed solve with the refinement residual in native FP64 (comparison) ---
    mixed_native = None
    if not args.no_fp64 and rank == 0:
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        _, im = plan.solve(out=u, tol=args.tol, precision="mixed", residual="fp64")
        f1.record()
        torch.cuda.synchronize()
        mixed_native = {"s": f0.elapsed_time(f1) / 1e3, "iters": im["iters"], "outer_iters": im["outer_iters"],
                        "relres": im["relres"]}

    # ---- end to end through the public API with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        u_host = torch.empty(n ** 3, dtype=torch.complex128).pin_memory()
        parts_ms = {"h2d": 0.0, "set_medium": 0.0, "solve": 0.0, "d2h": 0.0}

        def e2e_step():
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record()
            h_dev.copy_(h_host, non_blocking=True)
            N_dev.copy_(N_host, non_blocking=True)
            ev[1].record()
            plan.set_medium(h_dev, N_dev)
            ev[2].record()
            plan.solve(out=u, **kw)
            ev[3].record()
            u_host.copy_(u, non_blocking=True)
            ev[4].record()
            return ev

        # untimed warm-up: the first transfers from freshly pinned pages run slower
        for _ in range(min(args.warmup, 2)):
            e2e_step()
        torch.cuda.synchronize()
        # the host link alone: the same pinned buffers copied with nothing else running
        link = {}
        for key, fn, nbytes in (("h2d", lambda: h_dev.copy_(h_host, non_blocking=True), h_host.numel() * 16),
                                ("d2h", lambda: u_host.copy_(u, non_blocking=True), u_host.numel() * 16)):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            fn()
            c0.record()
            for _ in range(3):
                fn()
            c1.record()
            torch.cuda.synchronize()
            link[key + "_GBps"] = 3 * nbytes / (c0.elapsed_time(c1) * 1e-3) / 1e9
        # the same steps one after another (no overlap): where the time goes
        steps_e2e = max(1, min(args.steps, 3))
        evs = []
        for _ in range(steps_e2e):
            evs.append(e2e_step())
        torch.cuda.synchronize()
        for ev in evs:
            for key, a, b in (("h2d", 0, 1), ("set_medium", 1, 2), ("solve", 2, 3), ("d2h", 3, 4)):
                parts_ms[key] += ev[a].elapsed_time(ev[b]) / steps_e2e
        serial_s = evs[0][0].elapsed_time(evs[-1][4]) / 1e3 / steps_e2e
        # the timed e2e: Plan.solve_media over args.steps media in pinned host
        # memory (the same medium each step), the copies of the next medium's
        # inputs and of the previous solution overlapping each solve
        u_host2 = torch.empty(n ** 3, dtype=torch.complex128).pin_memory()
        outs = [u_host, u_host2] * ((args.steps + 1) // 2)
        plan.solve_media([h_host] * 2, [N_host] * 2, [u_host, u_host2], **kw)   # warm-up (buffers, graphs)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        plan.solve_media([h_host] * args.steps, [N_host] * args.steps, outs[:args.steps], **kw)
        g1.record()
        torch.cuda.synchronize()
        e2e_s = g0.elapsed_time(g1) / 1e3 / args.steps
        e2e_s = max_over_ranks(e2e_s * 1e3, world, dev) / 1e3
        h2d_bytes = h_host.numel() * 16 + N_host.numel() * 8
        d2h_bytes = u_host.numel() * 16
        e2e = {"value": e2e_s / world, "unit": "s",
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
               "how": (f"Plan.solve_media over {args.steps} media in pinned host memory: per medium the "
                       f"host->device copy of h and N, set_medium, the mixed solve and the device->host copy "
                       f"of u, the copies on their own streams overlapping the neighbouring solves"),
               "serial_s": serial_s,
               "parts_ms_serial": parts_ms,
               "h2d_GBps": h2d_bytes / (parts_ms["h2d"] * 1e-3) / 1e9 if parts_ms["h2d"] > 0 else None,
               "d2h_GBps": d2h_bytes / (parts_ms["d2h"] * 1e-3) / 1e9 if parts_ms["d2h"] > 0 else None,
               "host_link_alone": link}
        del u_host2, outs

    cpu = None
    if not args.no_cpu and rank == 0:
        plan.solve(out=u, **kw)
        u_np = u.cpu().numpy()
        cpu = cpu_baseline(n, k, args.seed, args.tol, u_gpu=u_np, legs=not args.no_cpu_legs)
        del u_np

    stats_main = stats
    plan.close()
    del u
    torch.cuda.empty_cache()
    batched = None
    if not args.no_batch and rank == 0:
        batched = batched_leg(args, dev)

    last = infos[-1]
    out = {
        "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "config": workload_config(args),
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(stats_main["kernel_launches"]) * world,
        "clocks": ck,
        "solve": {"iters": last["iters"], "outer_iters": last["outer_iters"], "relres": last["relres"],
                  "fp64_matvecs": last["fp64_matvecs"], "status": last["status"]},
        "plan_s": plan_s, "fp64_solve": fp64, "mixed_fp64_residual": mixed_native,
        "residual_arith": "paired FP32 (double-float) FFT passes, complex128 vectors",
        "matvec": matvec, "passes": passes,
        "schedule": tuned["schedule"], "schedule_operator_ms": tuned["ms"],
        "fp32_matvecs_per_step": stats_main["fp32_matvecs"] / args.steps,
        "fp64_matvecs_per_step": stats_main["fp64_matvecs"] / args.steps,
        "batched": batched,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)


_last_ms = []   # our standalone matvec time, for the comparator's ratio


def cufft_comparator(plan, h_dev, N_dev, x32, y_ours, n, k, L, dev, reps=5):
    """The same FP32 B-form matvec y = x + S K (S x) through cuFFT (torch.fft) as a
    library comparator, the way it is usually written: zero-pad S x into the full
    L^3 cube, 3D FFT, multiply by the full spectrum, inverse 3D FFT, crop, add x.
    Its spectrum is the FP64 FFT of the kernel cube, rounded to complex64 once
    (outside the timing).  Not part of the library."""
    import torch
    d = 1.0 / n
    idx = torch.arange(L, device=dev, dtype=torch.float64)
    s = torch.where(idx <= L // 2, idx, idx - L)                       # signed offsets
    s = torch.where(s.abs() <= n - 1, s, torch.full_like(s, float("inf")))
    r = d * torch.sqrt(s[:, None, None] ** 2 + s[None, :, None] ** 2 + s[None, None, :] ** 2)
    del s
    c = torch.zeros(L, L, L, dtype=torch.complex128, device=dev)
    ok = torch.isfinite(r) & (r > 0)
    rr = r[ok]
    c[ok] = (4 * math.pi * d ** 3) * torch.exp(1j * k * rr) / (4 * math.pi * rr)
    del r, ok, rr
    ghat = torch.fft.fftn(c).to(torch.complex64)
    del c
    torch.cuda.empty_cache()
    S = torch.sqrt(h_dev * N_dev).to(torch.complex64)
    pad = torch.zeros(L, L, L, dtype=torch.complex64, device=dev)

    def matvec(x):
        pad.zero_()
        pad[:n, :n, :n] = (S * x).view(n, n, n)
        f = torch.fft.fftn(pad)
        f *= ghat
        conv = torch.fft.ifftn(f)
        return x + S * conv[:n, :n, :n].reshape(-1)

    for _ in range(2):
        y = matvec(x32)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        y = matvec(x32)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    plan.matvec32(x32, "B", out=y_ours)
    # compare the operator parts y - x (for random x the identity term dominates y)
    diff = float(torch.linalg.vector_norm(y - y_ours) / torch.linalg.vector_norm(y_ours - x32))
    del pad, ghat, S, y
    torch.cuda.empty_cache()
    return {"ms": ms, "speedup_of_ours": ms / max(1e-9, float(_last_ms[0])) if _last_ms else None,
            "rel_l2_vs_ours_of_K_part": diff,
            "how": "torch.fft.fftn/ifftn (cuFFT C2C, complex64) on the zero-padded L^3 cube + elementwise pad, "
                   "spectrum multiply, crop and axpy"}


def batched_leg(args, dev, n=128, ks=(1.0, 2.0, 4.0, 8.0), ndir=16, reps=3):
    """Multi-direction, multi-frequency data of the inverse problem: 16
    directions spread on the sphere x 4 wave numbers at n = 128, one mixed
    batch of 64 systems, against the same 64 systems solved one by one."""
    import torch
    from paper_1602_04691_gb300 import Plan, inputs

    h_np, N_np = inputs.random_h_N(n, 4)
    h = torch.from_numpy(h_np).to(dev)
    N = torch.from_numpy(N_np).to(dev)
    dirs = inputs.fibonacci_directions(ndir)
    plan = Plan(n, list(ks), h, N)
    tune_path = os.path.join(tempfile.gettempdir(), f"ori_autotune_bench_{os.getpid()}.json")
    tuned = plan.autotune(nrhs=len(ks) * ndir, path=tune_path)
    kw = dict(tol=1e-6, precision="mixed")
    plan.solve_batch(dirs, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        u, infos = plan.solve_batch(dirs, **kw)
    e1.record()
    torch.cuda.synchronize()
    batch_s = e0.elapsed_time(e1) / 1e3 / reps
    worst = max(i["relres"] for i in infos)
    iters = [i["iters"] for i in infos]
    del u
    plan.close()
    # the same systems, one solve at a time (one plan per wave number)
    seq_s = 0.0
    for k in ks:
        single = Plan(n, k, h, N)
        single.solve(alpha=tuple(dirs[0]), **kw)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for a in dirs:
            single.solve(alpha=tuple(a), **kw)
        s1.record()
        torch.cuda.synchronize()
        seq_s += s0.elapsed_time(s1) / 1e3
        single.close()
    nsys = len(ks) * ndir
    return {"workload": f"n={n}, {ndir} directions x k in {list(ks)}, mixed to relres 1e-6",
            "systems": nsys, "batch_s": batch_s, "systems_per_s": nsys / batch_s,
            "sequential_s": seq_s, "speedup_vs_sequential": seq_s / batch_s,
            "max_relres": worst, "iters_min": min(iters), "iters_max": max(iters),
            "schedule": tuned["schedule"], "schedule_operator_ms": tuned["ms"]}


def experiment_arm(args, rank, local):
    """Section 4's experiment (Table 4 differences, Eq. 2.10 samples) on one GPU."""
    import torch
    from paper_1602_04691_gb300 import experiment
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    out = experiment.run(device=dev)
    out["experiment"] = "Section 4 scaled: RED n=20, IE n=40, ORI n=480, mixed to relres 1e-6"
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.experiment:
        experiment_arm(args, rank, local)
    elif args.impl == "reference":
        reference_arm(args, world, rank)
    else:
        ours_arm(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
