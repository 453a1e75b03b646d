"""Host logic of the batched-view autotuner on the CPU: the split of a batch
into contiguous partitions, the candidates it times (no more partitions than
views), the choice of the fastest, and the per-configuration cache.  The
renderer and the timer are replaced by fakes, so no GPU is needed."""
import json
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2412_04459_gb300 import autotune  # noqa: E402


@pytest.mark.parametrize("n,parts", [(1, 1), (2, 4), (10, 3), (16, 4), (7, 7)])
def test_split_covers_the_views_contiguously(n, parts):
    sp = autotune._split(n, parts)
    assert len(sp) == min(parts, n)
    assert sp[0][0] == 0 and sp[-1][1] == n
    assert all(b > a for a, b in sp)
    assert all(sp[i][1] == sp[i + 1][0] for i in range(len(sp) - 1))
    sizes = [b - a for a, b in sp]
    assert max(sizes) - min(sizes) <= 1


class _FakeRenderer:
    built = []

    def __init__(self, scene, cams, K=3, t_stop=1e-4, tile=16, partitions=1, backward=True):
        self.tile, self.partitions = tile, partitions
        _FakeRenderer.built.append((tile, partitions))

    def capture(self):
        return self

    def step(self):
        pass


def _scene():
    return types.SimpleNamespace(n_vox=1000, grid=types.SimpleNamespace(shape=(1500,)), max_level=6,
                                 centre=types.SimpleNamespace(device="cuda:0"))


def _cams(sizes):
    return [types.SimpleNamespace(width=w, height=h) for w, h in sizes]


@pytest.fixture
def fakes(monkeypatch, tmp_path):
    _FakeRenderer.built = []
    monkeypatch.setattr(autotune, "BatchedRenderer", _FakeRenderer)
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda d=None: "fake-gpu")
    monkeypatch.setattr(autotune.torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setenv("SVR_TUNE_CACHE", str(tmp_path / "tune.json"))
    return tmp_path / "tune.json"


def test_tune_times_each_candidate_and_keeps_the_fastest(monkeypatch, fakes):
    # tile 16 with 2 partitions is fastest
    cost = {(8, 1): 3.0, (8, 2): 2.5, (16, 1): 2.0, (16, 2): 1.5, (32, 1): 4.0, (32, 2): 3.5}
    monkeypatch.setattr(autotune, "_time", lambda fn, reps: cost[(fn.__self__.tile, fn.__self__.partitions)])
    res = autotune.tune(_scene(), _cams([(64, 48), (32, 32)]), partitions=(1, 2, 4))
    assert (res["tile"], res["partitions"]) == (16, 2)
    # 4 partitions exceed the 2 views: never built
    assert sorted(_FakeRenderer.built) == sorted(cost)
    assert set(res["ms"]) == {f"{t}/{p}" for t, p in cost}
    # the result is cached under the configuration's key
    cached = json.loads(fakes.read_text())
    assert list(cached.values()) == [res]


def test_cached_result_is_reused_and_keyed_by_configuration(monkeypatch, fakes):
    monkeypatch.setattr(autotune, "_time", lambda fn, reps: float(fn.__self__.tile))
    first = autotune.tune(_scene(), _cams([(64, 48)]), partitions=(1,))
    assert first["tile"] == 8
    # another timing now, but the same configuration: the cache answers
    _FakeRenderer.built = []
    monkeypatch.setattr(autotune, "_time", lambda fn, reps: -float(fn.__self__.tile))
    assert autotune.tune(_scene(), _cams([(64, 48)]), partitions=(1,)) == first
    assert _FakeRenderer.built == []
    # another image size is another configuration; use_cache=False ignores the cache
    other = autotune.tune(_scene(), _cams([(64, 64)]), partitions=(1,))
    assert other["tile"] == 32 and _FakeRenderer.built
    assert autotune.tune(_scene(), _cams([(64, 48)]), partitions=(1,), use_cache=False)["tile"] == 32
    assert len(json.loads(fakes.read_text())) == 2
