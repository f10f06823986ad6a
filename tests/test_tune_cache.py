"""Host logic of the autotuner cache (no GPU): keys, the JSON file's round trip
and robustness, and the tune-or-reuse flow of tuned_plan with a stand-in plan
whose autotune records that it ran."""
import json

import numpy as np

from paper_2605_01086_gb300 import codec, tune_cache


def _domains(shapes):
    return [codec.Domain(N, E, min(2, E), E, 50.0, 0.004, (1.0, 1.0, 0.0), 12, np.full(256, 8, np.uint8))
            for N, E in shapes]


def _segments(lengths):
    n = len(lengths)
    return codec.segments_array(np.zeros(n, np.uint64), np.ones(n, np.uint64), lengths, np.zeros(n, np.uint64),
                                np.zeros(n, np.uint32))


class FakePlan:
    tuned = 0

    def __init__(self, domains, segments, device=None, **kw):
        self.kw = kw

    def empty_out(self):
        return None

    def autotune(self, words, symlen, out, trials=3):
        FakePlan.tuned += 1
        return {"idct": 0, "schedule": 0, "tile_samples": 4096, "threads": 768, "ctas_per_sm": 1, "kernel": 3}, 1.5


def test_key_classes():
    d = _domains([(32, 16)])
    k1 = tune_cache.cache_key("GB300", d, 6_000_000_000, 10_000)
    assert k1 == tune_cache.cache_key("GB300", d, 5_000_000_000, 9_000)        # same power-of-two classes
    assert k1 != tune_cache.cache_key("GB300", d, 1_000_000_000, 10_000)       # other size class
    assert k1 != tune_cache.cache_key("GB200", d, 6_000_000_000, 10_000)       # other GPU
    assert k1 != tune_cache.cache_key("GB300", d, 6_000_000_000, 10_000, "bf16x3")
    assert k1 != tune_cache.cache_key("GB300", _domains([(64, 32)]), 6_000_000_000, 10_000)
    # the set of shapes, not their order or multiplicity
    assert tune_cache.cache_key("g", _domains([(32, 16), (64, 8)]), 100, 4) == \
        tune_cache.cache_key("g", _domains([(64, 8), (32, 16), (32, 16)]), 100, 4)


def test_plan_kwargs_names():
    kw = tune_cache.plan_kwargs({"idct": 2, "schedule": 0, "kernel": 4, "threads": 640, "tile_samples": 4096,
                                 "ctas_per_sm": 0})
    assert kw == {"idct": "bf16x3", "schedule": "persistent", "kernel": "tensor", "threads": 640,
                  "tile_samples": 4096, "ctas_per_sm": 0}


def test_tune_then_reuse(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    doms, segs = _domains([(32, 16)]), _segments([100000, 200000])
    FakePlan.tuned = 0
    p1, o1, hit1 = tune_cache.tuned_plan(doms, segs, None, None, path, plan_cls=FakePlan, gpu_name="GB300")
    assert not hit1 and FakePlan.tuned == 1 and p1.kw == {"idct": "fp32"}
    p2, o2, hit2 = tune_cache.tuned_plan(doms, segs, None, None, path, plan_cls=FakePlan, gpu_name="GB300")
    assert hit2 and FakePlan.tuned == 1 and o2 == o1
    assert p2.kw == tune_cache.plan_kwargs(o1)
    # another precision is another entry
    _, _, hit3 = tune_cache.tuned_plan(doms, segs, None, None, path, idct="tf32", plan_cls=FakePlan,
                                       gpu_name="GB300")
    assert not hit3 and FakePlan.tuned == 2
    data = json.load(open(path))
    assert len(data) == 2 and all(v["ms"] == 1.5 for v in data.values())


def test_unreadable_file_means_tuning_again(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    assert tune_cache.TuneCache(str(path)).entries == {}
    path.write_text(json.dumps({"k": {"options": "nope"}, "j": {"options": {"threads": 256}, "ms": 1.0}}))
    c = tune_cache.TuneCache(str(path))
    assert c.get("k") is None and c.get("j") == {"threads": 256}
    FakePlan.tuned = 0
    tune_cache.tuned_plan(_domains([(16, 8)]), _segments([5000]), None, None, str(path), plan_cls=FakePlan,
                          gpu_name="x")
    assert FakePlan.tuned == 1 and len(json.load(open(path))) == 2
