"""Host logic of the schedule cache (no GPU): keys, hits, misses, bad files."""

import json

from paper_1602_04691_gb300 import autotune as AT


class FakePlan:
    def __init__(self, n):
        self.n = n
        self.applied = []
        self.tuned = 0

    def set_schedule(self, s):
        self.applied.append(dict(s))

    def autotune_now(self, nrhs, reps):
        self.tuned += 1
        return {"yfwd": 1, "zconv": 0, "yinv": 1, "ctas_per_sm": 1, "vec_ctas_per_sm": 4,
                "yfwd_variant": 0, "zconv_variant": 2, "yinv_variant": 1}, 1.25 * nrhs


def test_key_names_gpu_n_batch_arithmetic_and_field_set():
    assert AT.cache_key("GPU X", 512, 64) == "GPU X|n=512|nrhs=64|arith=fp32|sched=2"


def test_miss_tunes_and_stores_then_hit_applies(tmp_path):
    path = str(tmp_path / "cache.json")
    p = FakePlan(128)
    r1 = AT.tune(p, 64, "GPU X", path=path)
    assert not r1["cached"] and p.tuned == 1 and r1["ms"] == 80.0
    data = json.load(open(path))
    entry = data["GPU X|n=128|nrhs=64|arith=fp32|sched=2"]["schedule"]
    assert entry["yfwd"] == 1 and entry["zconv_variant"] == 2 and entry["yinv_variant"] == 1
    q = FakePlan(128)
    r2 = AT.tune(q, 64, "GPU X", path=path)
    assert r2["cached"] and q.tuned == 0 and q.applied == [r1["schedule"]]
    # another batch size, grid or GPU is another key
    for plan, nrhs, gpu in [(FakePlan(128), 16, "GPU X"), (FakePlan(64), 64, "GPU X"), (FakePlan(128), 64, "GPU Y")]:
        assert not AT.tune(plan, nrhs, gpu, path=path)["cached"]
    assert len(json.load(open(path))) == 4


def test_force_retunes(tmp_path):
    path = str(tmp_path / "c.json")
    p = FakePlan(32)
    AT.tune(p, 1, "G", path=path)
    AT.tune(p, 1, "G", path=path, force=True)
    assert p.tuned == 2


def test_corrupt_or_invalid_cache_is_ignored(tmp_path):
    path = tmp_path / "bad.json"
    path.write_text("{not json")
    p = FakePlan(16)
    assert not AT.tune(p, 2, "G", path=str(path))["cached"]
    assert json.load(open(path))  # rewritten as valid JSON
    path.write_text(json.dumps({AT.cache_key("G", 16, 2): {"schedule": {"yfwd": "x"}}}))
    q = FakePlan(16)
    assert not AT.tune(q, 2, "G", path=str(path))["cached"] and q.tuned == 1


def test_entry_without_launch_variants_is_tuned_again(tmp_path):
    """An entry of the older field set (no launch variants) is neither applied nor trusted."""
    path = tmp_path / "old.json"
    old = {"yfwd": 0, "zconv": 0, "yinv": 0, "ctas_per_sm": 0, "vec_ctas_per_sm": 8}
    path.write_text(json.dumps({"G|n=16|nrhs=2|arith=fp32": {"schedule": old, "ms": 1.0},
                                AT.cache_key("G", 16, 2): {"schedule": old, "ms": 1.0}}))
    q = FakePlan(16)
    assert not AT.tune(q, 2, "G", path=str(path))["cached"] and q.tuned == 1 and q.applied == []


def test_env_variable_names_default_path(tmp_path, monkeypatch):
    monkeypatch.setenv("ORI_AUTOTUNE_CACHE", str(tmp_path / "env.json"))
    assert AT.cache_path() == str(tmp_path / "env.json")
    assert AT.cache_path("explicit.json") == "explicit.json"
