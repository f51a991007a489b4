"""Host logic of the autotuner without a GPU: the timed work and the CUDA
events are replaced by fakes whose time depends on the applied tuning, and the
real threshold setter of the library (a host-side value) is used.  Checks that
the fastest candidate is applied and cached, that a cached entry is applied on
the next call without timing, that a candidate whose result differs is never
applied or cached, and that the cache key separates graphs and parameters."""
import json

import pytest
import torch

import paper_1404_4797_gb300 as S
from paper_1404_4797_gb300 import autotune as A
from paper_1404_4797_gb300 import build as B
from paper_1404_4797_gb300 import inputs as I

CANDS = [(32, 256, 2048, 6144), (16, 256, 2048, 6144), (32, 128, 1024, 4096)]
FAST = (16, 256, 2048, 6144)


class _Clock:
    """Fake device clock: each timed call of the work advances it by the
    applied tuning's cost."""
    def __init__(self, cost):
        self.t = 0.0
        self.cost = cost
        self.calls = 0

    def work(self, *args, **kw):
        self.calls += 1
        t = S.get_tuning()
        key = (t["small_max"], t["med_max"], t["mid_max"], t["seg_smem"])
        self.t += self.cost(key)
        return self.result(key)

    def result(self, key):
        return (torch.arange(8, dtype=torch.int32),)


class _Event:
    clock = None

    def __init__(self, enable_timing=True):
        self.at = None

    def record(self, stream=None):
        self.at = _Event.clock.t

    def elapsed_time(self, other):
        return other.at - self.at


@pytest.fixture
def fake(monkeypatch):
    B.build()
    S.lib()  # the tuning setter is a host-side value: no GPU needed
    saved = S.get_tuning()
    clock = _Clock(lambda key: 1.0 if key == FAST else 2.0 + 0.1 * key[0] / 32)
    _Event.clock = clock
    monkeypatch.setattr(A, "_multilevel", lambda g, p: clock.work())
    monkeypatch.setattr(A, "_sweeps", lambda *a: clock.work())
    monkeypatch.setattr(A, "_device_name", lambda: "fake-gpu")
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    yield clock
    S.set_tuning(**saved)


def _graph(n=300, m=1200, seed=3):
    return I.random_graph(n, m, seed=seed)


def test_fastest_candidate_is_applied_and_cached(fake, tmp_path):
    cache = str(tmp_path / "tuning.json")
    g = _graph()
    res = A.autotune(g, 4, candidates=CANDS, reps=2, cache=cache, ml_params={"k": 4})
    assert res["identical"] and res["workload"] == "multilevel"
    assert tuple(res["best"].values()) == FAST
    assert tuple(S.get_tuning().values()) == FAST
    assert res["ms"]["16/256/2048/6144"] == pytest.approx(1.0)
    assert fake.calls == len(CANDS) * 3  # one untimed check and two timed reps each
    data = json.load(open(cache))
    key = "fake-gpu|" + A.signature(g, 4, 0.03, 3, 6, 4, {"k": 4})
    assert list(data) == [key] and data[key]["best"] == res["best"]


def test_cached_entry_is_applied_without_timing(fake, tmp_path):
    cache = str(tmp_path / "tuning.json")
    g = _graph()
    first = A.load_or_tune(g, 4, cache=cache, ml_params={"k": 4})
    assert first["cached"] is False
    S.set_tuning(*CANDS[0])
    calls = fake.calls
    again = A.load_or_tune(g, 4, cache=cache, ml_params={"k": 4})
    assert again["cached"] is True and fake.calls == calls
    assert again["best"] == first["best"]
    assert S.get_tuning() == first["best"]


def test_a_candidate_with_another_result_is_never_applied(fake, tmp_path, monkeypatch):
    cache = str(tmp_path / "tuning.json")
    monkeypatch.setattr(fake, "result", lambda key: (torch.full((8,), 1 if key == FAST else 0,
                                                                dtype=torch.int32),))
    S.set_tuning(*CANDS[2])
    res = A.autotune(_graph(), 4, candidates=CANDS, reps=1, cache=cache)
    assert res["identical"] is False
    assert tuple(S.get_tuning().values()) == CANDS[2]  # the setting before the call
    assert not (tmp_path / "tuning.json").exists()


def test_signature_separates_graphs_and_parameters():
    g, h = _graph(seed=3), _graph(seed=4)
    base = A.signature(g, 4, 0.03, 3, 6, 4)
    assert base == A.signature(_graph(seed=3), 4, 0.03, 3, 6, 4)
    others = [A.signature(h, 4, 0.03, 3, 6, 4), A.signature(g, 8, 0.03, 3, 6, 4),
              A.signature(g, 4, 0.05, 3, 6, 4), A.signature(g, 4, 0.03, 2, 6, 4),
              A.signature(g, 4, 0.03, 3, 5, 4), A.signature(g, 4, 0.03, 3, 6, 2),
              A.signature(g, 4, 0.03, 3, 6, 4, {"k": 4})]
    assert base not in others and len(set(others)) == len(others)


def test_unreadable_cache_is_retuned(fake, tmp_path):
    cache = tmp_path / "tuning.json"
    cache.write_text("{not json")
    res = A.load_or_tune(_graph(), 4, cache=str(cache), ml_params={"k": 4})
    assert res["cached"] is False and tuple(res["best"].values()) == FAST
    assert json.loads(cache.read_text())  # rewritten
