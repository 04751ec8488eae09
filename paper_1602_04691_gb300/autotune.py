"""Schedule cache for the plan autotuner (ori_plan_autotune).

The library times the candidate launch schedules of the FP32 passes on a
plan; this module keeps the winners in a JSON file keyed by GPU name, grid
size n, batch size and arithmetic, so that later plans for the same key take
the cached schedule without timing anything.  The file maps

    "<gpu name>|n=<n>|nrhs=<nrhs>|arith=fp32|sched=2"  ->  {"schedule": {...}, "ms": t}

where "schedule" holds the ori_schedule fields (kernel choice, launch variant
(tile width and radix split) and CTA cap of the FP32 Y-forward, Z and
Y-inverse passes, and the vector-kernel grid) and "ms" the FP32 operator time
of the whole batch measured when the entry was written.  "sched" numbers the
set of fields the tuner searches: entries written for an older set are tuned
again.

Cache location: the ``path`` argument, else the ORI_AUTOTUNE_CACHE
environment variable, else ``~/.cache/ori_autotune.json``.
"""

from __future__ import annotations

import json
import os
import tempfile

ARITH = "fp32"   # the tuned schedules are those of the FP32 passes
SCHED_FIELDS_VERSION = 2   # 2: launch variants (tile width, radix split) added


def cache_path(path: str | None = None) -> str:
    if path:
        return path
    env = os.environ.get("ORI_AUTOTUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "ori_autotune.json")


def cache_key(gpu_name: str, n: int, nrhs: int, arith: str = ARITH) -> str:
    return f"{gpu_name}|n={int(n)}|nrhs={int(nrhs)}|arith={arith}|sched={SCHED_FIELDS_VERSION}"


def load(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def store(path: str, key: str, schedule: dict, ms: float) -> None:
    """Add one entry, rewriting the file atomically (write to a temporary file, rename)."""
    data = load(path)
    data[key] = {"schedule": dict(schedule), "ms": float(ms)}
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".ori_autotune.", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


_FIELDS = ("yfwd", "zconv", "yinv", "ctas_per_sm", "vec_ctas_per_sm", "yfwd_variant", "zconv_variant",
           "yinv_variant")


def valid_schedule(s) -> bool:
    return isinstance(s, dict) and all(isinstance(s.get(f), int) for f in _FIELDS)


def tune(plan, nrhs: int, gpu_name: str, path: str | None = None, reps: int = 3,
         force: bool = False) -> dict:
    """Give `plan` the schedule for (gpu_name, plan.n, nrhs): from the cache when
    present (and `force` is false), else by timing on the plan and storing the
    result.  Returns {"schedule": ..., "ms": ..., "cached": bool, "key": ...}."""
    p = cache_path(path)
    key = cache_key(gpu_name, plan.n, nrhs)
    if not force:
        entry = load(p).get(key)
        if isinstance(entry, dict) and valid_schedule(entry.get("schedule")):
            plan.set_schedule(entry["schedule"])
            return {"schedule": dict(entry["schedule"]), "ms": entry.get("ms"), "cached": True, "key": key}
    sched, ms = plan.autotune_now(nrhs, reps)
    store(p, key, sched, ms)
    return {"schedule": sched, "ms": ms, "cached": False, "key": key}
