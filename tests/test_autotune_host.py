"""The autotuner's cache (paper_2510_20870_gb300/autotune.py) on the host: save records the
fastest candidate and the default's time under the GPU / workload-class key, load reads it back,
apply sets the cached configuration through rox_set_launch_config (a host-only call) and falls
back to the library default for an unknown class. The committed cache holds an entry for every
class bench.py applies, each a valid configuration. The GPU-side sweep (CUDA events) is
exercised by `bench.py --autotune`."""
import json
import os

import pytest

import paper_2510_20870_gb300 as rox
from paper_2510_20870_gb300 import autotune

DEFAULT = {"warps_per_cta": 8, "ctas_per_sm": 0, "split_rounds": 1}


@pytest.fixture
def fake_gpu(monkeypatch):
    # key() names the GPU; without one, stand in a fixed name
    monkeypatch.setattr(autotune, "key", lambda cls, device=None: "TEST GPU|1 SMs|%s" % cls)
    yield
    rox.rox_reset_launch_config()


def test_save_load_apply_roundtrip(tmp_path, fake_gpu):
    path = str(tmp_path / "tuning.json")
    results = [(autotune._as_dict(c), ms) for c, ms in zip(autotune.CANDIDATES, [10.0, 9.5, 12.0, 30.0, 9.0, 9.2, 11.0, 13.0])]
    best = autotune.save("demo", results, path=path, note="unit test")
    assert best == {"warps_per_cta": 4, "ctas_per_sm": 0, "split_rounds": 1}       # the 9.0 ms candidate
    entry = autotune.load(path)["TEST GPU|1 SMs|demo"]
    assert entry["best_ms"] == 9.0 and entry["default_ms"] == 10.0 and len(entry["results"]) == 8
    cfg, cached = autotune.apply("demo", path=path)
    assert cached and cfg == best and rox.rox_get_launch_config() == best
    cfg, cached = autotune.apply("unknown class", path=path)
    assert not cached and cfg == DEFAULT and rox.rox_get_launch_config() == DEFAULT


def test_save_keeps_other_entries_and_missing_cache_is_empty(tmp_path, fake_gpu):
    path = str(tmp_path / "tuning.json")
    assert autotune.load(path) == {}
    autotune.save("a", [(DEFAULT, 5.0)], path=path)
    autotune.save("b", [(DEFAULT, 6.0)], path=path)
    assert set(autotune.load(path)) == {"TEST GPU|1 SMs|a", "TEST GPU|1 SMs|b"}


def test_committed_cache_covers_the_bench_classes():
    with open(autotune.CACHE) as f:
        cache = json.load(f)
    classes = {k.split("|")[-1] for k in cache}
    assert {"large", "exomol", "batch"} <= classes
    for entry in cache.values():
        b = entry["best"]
        rox.rox_set_launch_config(b["warps_per_cta"], b["ctas_per_sm"], b["split_rounds"])   # valid knobs
        assert min(r["ms"] for r in entry["results"]) == entry["best_ms"]
    rox.rox_reset_launch_config()
    assert os.path.dirname(autotune.CACHE) == os.path.dirname(os.path.abspath(rox.__file__))
