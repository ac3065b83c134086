"""Host logic of the launch-shape autotuner, on the CPU: the fastest candidate is
chosen, stored under its workload-class key, reused without timing, re-timed
when forced, and an unreadable cache counts as empty.  Stand-ins replace the
plan, the batch and the CUDA-event timer; the GPU test of the same module
(tests/test_gpu_batch.py) times real launches."""
import json

import pytest

from paper_1003_4984_gb300 import autotune
from paper_1003_4984_gb300.api import LaunchCfg

# made-up launch times (ms) per shape: (4, 1, 16) is the fastest
TIMES = {(2, 0, 8): 5.0, (4, 1, 16): 1.5, (8, 2, 8): 3.0}
CANDS = [LaunchCfg(*k) for k in TIMES]
LAUNCHED = []  # the shape of every stand-in launch, in order


class _Plan:
    def __init__(self, nside=64, K=32, spin=2, precision="mixed"):
        self.nside, self.K, self.spin, self.precision = nside, K, spin, precision
        self.cfg = None
        self.lens_calls = 0

    def set_launch(self, cfg):
        self.cfg = cfg

    def lens(self, map_, defl, out, var, first=0, count=None):
        self.lens_calls += 1
        LAUNCHED.append(self.cfg)


class _Batch:
    def __init__(self):
        self.staged_tile = None
        self.cfg = None
        self.launches = 0

    def stage(self, jobs, tile_points):
        self.staged_tile = tile_points

    def launch(self, cfg):
        self.cfg = cfg
        self.launches += 1
        LAUNCHED.append(cfg)


@pytest.fixture
def seen(monkeypatch):
    """The shapes the tuner timed, in order.  The stand-in timer runs the call once and
    reports the made-up time of the shape it launched; the device key is fixed."""
    timed = []

    def timer(fn, reps):
        fn()
        timed.append(LAUNCHED[-1])
        return TIMES[LAUNCHED[-1].key()]

    monkeypatch.setattr(autotune, "_device_key", lambda: "GB300-test|152")
    monkeypatch.setattr(autotune, "_time", timer)
    return timed


def test_plan_tuner_picks_the_fastest_shape_and_caches_it(tmp_path, seen):
    import torch

    plan = _Plan()
    cache = str(tmp_path / "tune.json")
    m, d = torch.zeros(10), torch.zeros((4, 2))
    cfg = autotune.tune_plan(plan, m, d, 0, 4, cache=cache, cands=CANDS)
    assert cfg.key() == (4, 1, 16) and plan.cfg.key() == (4, 1, 16)
    assert [c.key() for c in seen] == list(TIMES)
    data = json.load(open(cache))
    entry = data[autotune.plan_key(plan)]
    assert entry["cfg"] == [4, 1, 16] and entry["ms"] == 1.5 and entry["points"] == 4
    assert sorted(tuple(k) for k, _ in entry["tried"]) == sorted(TIMES)
    # a second plan of the same class reuses the stored shape without timing
    plan2 = _Plan()
    seen.clear()
    cfg2 = autotune.tune_plan(plan2, m, d, 0, 4, cache=cache, cands=[LaunchCfg(1, 1, 1)])
    assert cfg2.key() == (4, 1, 16) and plan2.cfg.key() == (4, 1, 16) and not seen and plan2.lens_calls == 0
    # another class (other K) is tuned on its own; forcing re-times a known class
    plan3 = _Plan(K=16)
    autotune.tune_plan(plan3, m, d, 0, 4, cache=cache, cands=CANDS)
    assert len(seen) == len(TIMES)
    seen.clear()
    autotune.tune_plan(_Plan(), m, d, 0, 4, cache=cache, cands=CANDS[:1], force=True)
    assert len(seen) == 1
    data = json.load(open(cache))
    assert data[autotune.plan_key(plan)]["cfg"] == [2, 0, 8]  # the forced re-tune replaced the entry
    assert data[autotune.plan_key(plan3)]["cfg"] == [4, 1, 16]


def test_batch_tuner_stages_the_winner_and_keys_by_class_mix(tmp_path, seen):
    batch = _Batch()
    staged = []
    batch.stage = lambda jobs, tile: (staged.append(tile), setattr(batch, "staged_tile", tile))
    cache = tmp_path / "sub" / "tune.json"  # the directory is created on save
    jobs = [(_Plan(K=32, spin=2), 0, 8, None, None, None, None, None),
            (_Plan(K=16, spin=0), 0, 8, None, None, None, None, None),
            (_Plan(K=32, spin=2), 8, 8, None, None, None, None, None)]
    cfg = autotune.tune_batch(batch, jobs, cache=str(cache), cands=CANDS)
    assert cfg.key() == (4, 1, 16) and batch.staged_tile == 16  # the winner is left staged
    # each candidate is staged with its own tile size before it is launched
    assert staged[:len(TIMES)] == [k[2] for k in TIMES] and [c.key() for c in seen] == list(TIMES)
    key = autotune.batch_key(jobs)
    assert key == "batch|GB300-test|152|K16s0mixed,K32s2mixed"  # classes, not job count or order
    assert autotune.batch_key(list(reversed(jobs))) == key
    assert json.load(open(cache))[key]["cfg"] == [4, 1, 16]
    seen.clear()
    assert autotune.tune_batch(_Batch(), jobs[:2], cache=str(cache), cands=CANDS).key() == (4, 1, 16)
    assert not seen


def test_unreadable_cache_counts_as_empty(tmp_path, seen):
    import torch

    plan = _Plan()
    cache = tmp_path / "tune.json"
    cache.write_text("{not json")
    cfg = autotune.tune_plan(plan, torch.zeros(4), torch.zeros((2, 2)), 0, 2, cache=str(cache), cands=CANDS)
    assert cfg.key() == (4, 1, 16) and len(seen) == len(TIMES)
    assert json.load(open(cache))[autotune.plan_key(plan)]["cfg"] == [4, 1, 16]
    assert not list(tmp_path.glob("*.tmp*"))  # written through a temporary file, then renamed


def test_candidates_respect_the_warp_limit():
    assert {c.warps_per_block for c in autotune.candidates(4)} == {2, 4}
    assert len(autotune.candidates()) == 18
