"""Host logic of the schedule autotuner: search, selection, cache write and reuse, and the choice
between the time-blocked and the plain kernels (a fake solver and a fake timer; no GPU)."""
import json

from paper_1907_11771_gb300 import autotune as A
from paper_1907_11771_gb300 import binding as B

FUSED, PLAIN = B.GBS_KERNEL_FUSED, B.GBS_KERNEL_PLAIN


class FakeSolver:
    def __init__(self, fused=True):
        self.opts = {"hseg": 256, "tmax": 4, "schedule": 0, "kernel": B.GBS_KERNEL_AUTO}
        self.fused = fused

    def uses_fused(self):
        return self.fused

    def set_option(self, k, v):
        self.opts[k] = v


def _cost(o, plain_cost=10.0):
    if o["kernel"] == PLAIN:
        return plain_cost
    return abs(o["hseg"] - 192) / 100.0 + (0.5 if o["tmax"] == 2 else 0.0) + 0.1 * o["schedule"]


def test_autotune_picks_the_fastest_applies_and_caches(tmp_path):
    cache = str(tmp_path / "tune.json")
    s = FakeSolver()
    calls = []
    timer = lambda: (calls.append(dict(s.opts)), _cost(s.opts))[1]
    r = A.autotune(s, cache=cache, timer=timer, key="w1")
    assert not r["cached"]
    assert r["options"] == {"hseg": 192, "tmax": 4, "schedule": 0, "kernel": FUSED}
    assert s.opts == r["options"]
    space = A.DEFAULT_SPACE
    assert len(calls) == len(space["hseg"]) * len(space["tmax"]) * len(space["schedule"]) + 1   # + plain
    assert len({json.dumps(c, sort_keys=True) for c in calls}) == len(calls)   # every candidate once
    with open(cache) as f:
        assert json.load(f)["w1"]["options"] == r["options"]
    # same key: applied from the cache without timing
    s2, calls2 = FakeSolver(), []
    r2 = A.autotune(s2, cache=cache, timer=lambda: (calls2.append(1), 0.0)[1], key="w1")
    assert r2["cached"] and not calls2 and s2.opts == r["options"]
    # another key, a restricted space, and a forced re-tune
    s3 = FakeSolver()
    r3 = A.autotune(s3, space={"hseg": [64, 512], "tmax": [4], "schedule": [1]}, cache=cache,
                    timer=lambda: _cost(s3.opts), key="w2")
    assert r3["options"] == {"hseg": 64, "tmax": 4, "schedule": 1, "kernel": FUSED}
    r4 = A.autotune(FakeSolver(), cache=cache, timer=lambda: 1.0, key="w1", retune=True)
    assert not r4["cached"]
    with open(cache) as f:
        assert set(json.load(f)) == {"w1", "w2"}


def test_autotune_skips_problems_without_the_time_blocked_kernel(tmp_path):
    assert A.autotune(FakeSolver(fused=False), cache=str(tmp_path / "t.json"), timer=lambda: 1.0, key="k") is None


def test_autotune_picks_the_plain_kernels_when_faster(tmp_path):
    cache = str(tmp_path / "tune.json")
    s = FakeSolver()
    r = A.autotune(s, cache=cache, timer=lambda: _cost(s.opts, plain_cost=-1.0), key="few-sequences")
    assert r["options"]["kernel"] == PLAIN
    assert {k: r["options"][k] for k in A.KNOBS} == {"hseg": 192, "tmax": 4, "schedule": 0}   # best schedule kept
    assert s.opts["kernel"] == PLAIN
    s2 = FakeSolver()
    r2 = A.autotune(s2, cache=cache, timer=lambda: 1.0, key="few-sequences")
    assert r2["cached"] and s2.opts["kernel"] == PLAIN
    s3 = FakeSolver()
    r3 = A.autotune(s3, cache=False, timer=lambda: _cost(s3.opts, plain_cost=-1.0), key="x", plain=False)
    assert r3["options"]["kernel"] == FUSED


def test_autotune_3d_varies_only_the_z_segment(tmp_path):
    s = FakeSolver()
    s.ndim = 3
    s.opts["zseg"] = 128
    calls = []
    cost = lambda o: 10.0 if o["kernel"] == PLAIN else abs(o["zseg"] - 64) / 64.0
    timer = lambda: (calls.append(dict(s.opts)), cost(s.opts))[1]
    r = A.autotune(s, cache=str(tmp_path / "t.json"), timer=timer, key="w3")
    assert r["options"] == {"zseg": 64, "kernel": FUSED}
    assert len(calls) == len(A.DEFAULT_SPACE_3D["zseg"]) + 1
    assert all(c["hseg"] == 256 and c["tmax"] == 4 for c in calls)   # the 2D knobs stay untouched
