"""Host logic of the launch-shape autotuner: cache keys, candidates, the
choice, the cache file and the shipped GB300 entries (no GPU)."""
import json

import pytest

import workloads
from paper_1908_01762_gb300 import autotune, sisph

DEV = "GPU sm_103 x152"


def test_workload_key_classes():
    tg = workloads.taylor_green(100)            # 10,000 particles, no walls
    k = autotune.workload_key([tg], sisph.MIXED, DEV)
    assert k == autotune.workload_key([workloads.taylor_green(104)], sisph.MIXED, DEV)  # 10,816
    assert k != autotune.workload_key([workloads.taylor_green(200)], sisph.MIXED, DEV)
    assert k != autotune.workload_key([tg], sisph.FP64, DEV)
    assert k != autotune.workload_key([tg], sisph.MIXED, "other GPU")
    assert k != autotune.workload_key([tg, tg], sisph.MIXED, DEV)
    tank = workloads.still_tank_2d(90, 90)
    assert "walls1" in autotune.workload_key([tank], sisph.MIXED, DEV) and "walls0" in k
    assert "dim3" in autotune.workload_key([workloads.dam_break_3d(dx=0.06)], sisph.MIXED, DEV)


def test_candidates():
    small = [workloads.taylor_green(50)]        # 10 fluid tiles of 256
    c = autotune.candidates(small, 152)
    assert {o["block"] for o in c} == set(autotune.BLOCKS)
    assert {o["skin"] for o in c} == set(autotune.SKINS)
    assert {o["ppe_sync"] for o in c} == {0, 1}
    assert len(c) == len({json.dumps(o, sort_keys=True) for o in c})
    # more fluid tiles than 8 per SM: the automatic form is the barrier form,
    # so the barrier is not tried a second time
    big = [workloads.taylor_green(400)]         # 625 tiles of 256, 1250 of 128
    c = autotune.candidates(big, 64)
    assert all(o["ppe_sync"] == 0 for o in c)
    for o in c:
        assert o["block"] % 32 == 0 and 64 <= o["block"] <= 256 and 0 <= o["skin"] <= 1


def test_pick():
    t = [{"options": {"a": 0}, "ms_per_step": 2.0}, {"options": {"a": 1}, "ms_per_step": None},
         {"options": {"a": 2}, "ms_per_step": 1.5}, {"options": {"a": 3}, "ms_per_step": 1.5}]
    assert autotune.pick(t)["options"] == {"a": 2}
    # within 1 % of the defaults (the first trial): the defaults stay
    near = [{"options": {"a": 0}, "ms_per_step": 1.0}, {"options": {"a": 1}, "ms_per_step": 0.995}]
    assert autotune.pick(near)["options"] == {"a": 0}
    assert autotune.pick(near, margin=0.0)["options"] == {"a": 1}
    # defaults that cannot run: the fastest of the rest
    assert autotune.pick([{"options": {"a": 0}, "ms_per_step": None}] + near[1:])["options"] == {"a": 1}
    with pytest.raises(RuntimeError):
        autotune.pick([{"options": {}, "ms_per_step": None}])


def test_tune_with_a_timer_and_the_cache(tmp_path):
    case = workloads.taylor_green(50)
    path = str(tmp_path / "cache.json")
    seen = []

    def timer(o):
        seen.append(dict(o))
        if o["block"] == 128 and o["skin"] == 0.25:
            return None                          # a candidate that cannot run
        return 1.0 + 0.01 * o["block"] / 128 - o["skin"] + 0.1 * o["ppe_sync"]

    e = autotune.tune([case], sisph.MIXED, path=path, timer=timer, device=DEV, sms=152)
    assert seen[0] == autotune.DEFAULTS and len(seen) == len({json.dumps(o, sort_keys=True) for o in seen})
    assert e["options"] == {"block": 256, "skin": 0.25, "ppe_sync": 0}
    assert e["default_ms_per_step"] == pytest.approx(1.0 + 0.02 - 0.15)
    assert autotune.lookup([case], sisph.MIXED, path, device=DEV) == e["options"]
    assert autotune.lookup([case], sisph.FP64, path, device=DEV) is None
    # a second workload class is merged into the same file
    tank = workloads.still_tank_2d(20, 20)
    autotune.tune([tank], sisph.MIXED, path=path, timer=lambda o: 1.0, device=DEV, sms=152)
    assert len(autotune.load_cache(path)) == 2
    assert autotune.lookup([case], sisph.MIXED, path, device=DEV) == e["options"]
    assert autotune.lookup([tank], sisph.MIXED, path, device=DEV) == autotune.DEFAULTS


def test_shipped_cache_is_valid():
    data = autotune.load_cache(autotune.DEFAULT_CACHE)
    for key, e in data.items():
        o = e["options"]
        assert set(o) == {"block", "skin", "ppe_sync"}, key
        assert o["block"] % 32 == 0 and 64 <= o["block"] <= 256
        assert 0.0 <= o["skin"] <= 1.0 and o["ppe_sync"] in (0, 1, 2)
        assert e["ms_per_step"] <= e["default_ms_per_step"]
        assert e["options"] == autotune.DEFAULTS or e["ms_per_step"] < 0.99 * e["default_ms_per_step"]
        assert any(t["options"] == o and t["ms_per_step"] == e["ms_per_step"] for t in e["trials"])
