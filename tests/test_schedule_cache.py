"""The persistent schedule cache (checkpoint / resume of the search), on the
CPU: nk_tune is replaced by a fake that records its calls, so only the
cache logic runs; the schedule space it checks entries against is the
library's own (host logic)."""
import json

import pytest

nt = pytest.importorskip("paper_2307_16080_gb300.nk_tune")
from paper_2307_16080_gb300 import schedule_cache as sc  # noqa: E402

DEV = "GB300|sm_103|152"


class FakeTune:
    def __init__(self):
        self.calls = []

    def __call__(self, p, mode, topk, params, reps, stream):
        self.calls.append((p.op, p.M, p.n, mode))
        best = nt.nk_enumerate_schedules(p)[0]
        rep = nt.nk_tune_report(candidates=10, timed=10, best_ms=0.5, default_ms=0.6)
        return best, rep


@pytest.fixture
def fake(monkeypatch):
    f = FakeTune()
    monkeypatch.setattr(nt, "nk_tune", f)
    return f


def _cache(path, fp="fp-1", dev=DEV):
    return sc.ScheduleCache(str(path), device=dev, fingerprint=fp)


def test_miss_then_hit_across_processes(tmp_path, fake):
    path = tmp_path / "schedules.json"
    p = nt.conv_problem(8, 56, 56, 64, 64, 3, 3, 1, 1)
    s1, rep = sc.tune_cached(p, cache=_cache(path))
    assert rep is not None and len(fake.calls) == 1
    assert s1 in nt.nk_enumerate_schedules(p)
    # a new cache object reading the same file (another process, a restart)
    s2, rep2 = sc.tune_cached(p, cache=_cache(path))
    assert s2 == s1 and rep2 is None and len(fake.calls) == 1
    # another problem, another search mode: misses
    sc.tune_cached(nt.matmul_problem(512, 512, 512), cache=_cache(path))
    sc.tune_cached(p, mode=nt.NK_TUNE_EVOLUTION, topk=5, cache=_cache(path))
    assert len(fake.calls) == 3
    assert len(_cache(path)) == 3


def test_stale_fingerprint_or_device_is_ignored(tmp_path, fake):
    path = tmp_path / "schedules.json"
    p = nt.matmul_problem(1000, 700, 3000)
    sc.tune_cached(p, cache=_cache(path))
    assert _cache(path).get(p) is not None
    assert _cache(path, fp="fp-2").get(p) is None          # rebuilt library
    assert _cache(path, dev="other|sm_100|148").get(p) is None
    sc.tune_cached(p, cache=_cache(path, fp="fp-2"))        # re-tuned and replaced
    assert len(fake.calls) == 2
    assert _cache(path, fp="fp-2").get(p) is not None


def test_corrupt_or_foreign_file_reads_as_empty(tmp_path, fake):
    path = tmp_path / "schedules.json"
    p = nt.matmul_problem(256, 256, 256)
    path.write_text("{ not json")
    assert len(_cache(path)) == 0
    sc.tune_cached(p, cache=_cache(path))
    doc = json.loads(path.read_text())
    assert doc["format"] == sc.FORMAT and len(doc["entries"]) == 1
    path.write_text(json.dumps({"format": 999, "entries": doc["entries"]}))
    assert _cache(path).get(p) is None


def test_illegal_stored_schedule_is_ignored(tmp_path, fake):
    path = tmp_path / "schedules.json"
    p = nt.conv_problem(8, 28, 28, 128, 128, 3, 3, 2, 1)
    c = _cache(path)
    c.put(p, nt.NK_TUNE_EXHAUSTIVE, 5, (128, 64, 192, 1, 1, 1))   # stacked rows: stride 1 only
    assert _cache(path).get(p) is None
    c.put(p, nt.NK_TUNE_EXHAUSTIVE, 5, (1, 2, 3))
    assert _cache(path).get(p) is None


def test_writers_merge_instead_of_clobbering(tmp_path, fake):
    path = tmp_path / "schedules.json"
    a, b = _cache(path), _cache(path)        # both read the empty file
    pa, pb = nt.matmul_problem(384, 384, 384), nt.matmul_problem(640, 640, 640)
    a.put(pa, nt.NK_TUNE_EXHAUSTIVE, 5, nt.nk_enumerate_schedules(pa)[0])
    b.put(pb, nt.NK_TUNE_EXHAUSTIVE, 5, nt.nk_enumerate_schedules(pb)[0])
    c = _cache(path)
    assert c.get(pa) is not None and c.get(pb) is not None


def test_model_search_keys_on_the_parameters(tmp_path, fake):
    import numpy as np
    path = tmp_path / "schedules.json"
    p = nt.matmul_problem(1024, 1024, 1024)
    w1 = np.zeros(10, np.float32).tobytes()
    w2 = np.ones(10, np.float32).tobytes()
    sc.tune_cached(p, mode=nt.NK_TUNE_MODEL_TOPK, topk=5, params=w1, cache=_cache(path))
    assert _cache(path).get(p, nt.NK_TUNE_MODEL_TOPK, 5, w1) is not None
    assert _cache(path).get(p, nt.NK_TUNE_MODEL_TOPK, 5, w2) is None
    assert _cache(path).get(p, nt.NK_TUNE_MODEL_TOPK, 3, w1) is None


def test_cache_dir_from_environment(tmp_path, monkeypatch):
    monkeypatch.setenv("NK_CACHE_DIR", str(tmp_path / "nkc"))
    assert sc.default_path() == str(tmp_path / "nkc" / "schedules.json")


def test_source_fingerprint_is_stable():
    assert sc.source_fingerprint() == sc.source_fingerprint()
    assert len(sc.source_fingerprint()) == 16
