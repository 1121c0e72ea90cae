"""Host logic of the autotune cache (paper_1908_00041_gb300.tune_cache) with a stand-in
plan: miss -> tune and record, hit -> apply without timing, keys separate degree, batch,
precision, I/O type and GPU, a stale entry is retuned, an unreadable file is a miss, the
environment variable selects the file.  The C setter's argument checks run on the host."""
import ctypes
import json

import pytest

from paper_1908_00041_gb300 import api, tune_cache


class FakePlan:
    def __init__(self, L=255, batch=8, precision=api.FAVEST_BF16X6, io_type=api.FAVEST_IO_C64,
                 best=(32, 2, 1)):
        self.L, self.batch, self.precision, self.io_type = L, batch, precision, io_type
        self.best, self.shape, self.tuned, self.applied = best, (128, 1, 2), 0, []

    def tune(self, stream=None):
        self.tuned += 1
        self.shape = self.best

    def gen_shape(self):
        return self.shape[0], self.shape[1]

    def gen_chains(self):
        return self.shape[2]

    def set_gen_shape(self, lt, mb, nj):
        if (lt, mb, nj) == (7, 7, 7):
            raise api.FavestError(api.FAVEST_EINVAL, "favest_plan_set_gen_shape")
        self.applied.append((lt, mb, nj))
        self.shape = (lt, mb, nj)


def test_miss_then_hit(tmp_path):
    path = str(tmp_path / "t.json")
    p = FakePlan()
    assert tune_cache.tune(p, "GB300", path) == (32, 2, 1, False) and p.tuned == 1
    q = FakePlan(best=(64, 1, 2))
    assert tune_cache.tune(q, "GB300", path) == (32, 2, 1, True)
    assert q.tuned == 0 and q.applied == [(32, 2, 1)]
    assert json.load(open(path)) == {"L255/B8/p1/io1/GB300": [32, 2, 1]}


def test_keys_separate_workloads(tmp_path):
    path = str(tmp_path / "t.json")
    tune_cache.tune(FakePlan(), "GB300", path)
    for p, dev in ((FakePlan(L=511), "GB300"), (FakePlan(batch=16), "GB300"),
                   (FakePlan(io_type=api.FAVEST_IO_R32), "GB300"), (FakePlan(), "other GPU")):
        assert tune_cache.tune(p, dev, path)[3] is False and p.tuned == 1
    assert len(json.load(open(path))) == 5


def test_stale_entry_is_retuned(tmp_path):
    path = str(tmp_path / "t.json")
    k = tune_cache.key(255, 8, api.FAVEST_BF16X6, api.FAVEST_IO_C64, "GB300")
    json.dump({k: [7, 7, 7], "other": [1, 2, 3]}, open(path, "w"))
    p = FakePlan()
    assert tune_cache.tune(p, "GB300", path) == (32, 2, 1, False) and p.tuned == 1
    d = json.load(open(path))
    assert d[k] == [32, 2, 1] and d["other"] == [1, 2, 3]


def test_unreadable_file_is_a_miss(tmp_path):
    path = tmp_path / "t.json"
    path.write_text("{not json")
    p = FakePlan()
    assert tune_cache.tune(p, "GB300", str(path))[3] is False
    assert json.loads(path.read_text())


def test_environment_selects_the_file(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "cache.json"
    monkeypatch.setenv("FAVEST_TUNE_CACHE", str(path))
    assert tune_cache.cache_path() == str(path)
    tune_cache.tune(FakePlan(), "GB300")
    assert path.exists() and not [f for f in path.parent.iterdir() if f.name.startswith(".tune-")]


def test_set_gen_shape_rejects_null_plan():
    from paper_1908_00041_gb300 import build
    build.build()
    L = api.lib()
    assert L.favest_plan_set_gen_shape(None, 128, 1, 2) == api.FAVEST_EINVAL
    assert L.favest_plan_set_gen_shape(ctypes.c_void_p(0), 5, 5, 5) == api.FAVEST_EINVAL
