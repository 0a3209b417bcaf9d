"""The launch-shape cache of `autotune` (JSON per geometry class), on the CPU:
the library is replaced by a fake that records the native calls, so the test
checks which calls a cached or an uncached geometry makes and what the file
holds."""
import json
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2211_14212_gb300 import cbct


class FakeLib:
    """Stands in for libcbct.so: autotune picks (4, 5) and fills the times;
    set/get_launch keep the shapes per handle."""

    def __init__(self):
        self.calls = []
        self.launch = {}

    def cbct_geometry_autotune(self, h, max_angles, t, stream):
        self.calls.append(("autotune", h, max_angles))
        for i in range(cbct.TUNE_TIMES):
            t[i] = 1.0 + i
        self.launch[h] = (4, 5)
        return cbct.CBCT_OK

    def cbct_geometry_set_launch(self, h, f, b):
        self.calls.append(("set_launch", h, f, b))
        self.launch[h] = (f, b)
        return cbct.CBCT_OK

    def cbct_geometry_get_launch(self, h, f, b):
        f._obj.value, b._obj.value = self.launch.get(h, (1, 0))
        return cbct.CBCT_OK

    def cbct_last_error(self):
        return b""


PARAMS = dict(nx=32, ny=32, nz=32, dx=1.0, dy=1.0, dz=1.0, nu=64, nv=64, du=1.2, dv=1.2, dso=1000.0, dsd=1500.0)


def geometry(handle, **over):
    p = dict(PARAMS, **over)
    return SimpleNamespace(handle=handle, params=p, angles=np.linspace(0, 2 * np.pi, 60, endpoint=False))


@pytest.fixture
def fake(monkeypatch):
    lib = FakeLib()
    monkeypatch.setattr(cbct, "_lib", lib)
    monkeypatch.setattr(cbct, "_stream_handle", lambda stream: None)   # no CUDA stream on the CPU
    monkeypatch.delenv("CBCT_TUNE_CACHE", raising=False)
    return lib


def test_second_geometry_of_a_class_takes_the_cached_shapes(fake, tmp_path):
    path = tmp_path / "tune.json"
    r1 = cbct.autotune(geometry(11), max_angles=8, cache=path)
    assert r1["cached"] is False and (r1["fwd_rows"], r1["bwd_config"]) == (4, 5)
    assert [c[0] for c in fake.calls] == ["autotune"]
    data = json.loads(path.read_text())
    assert data["version"] == cbct.TUNE_CACHE_VERSION and len(data["entries"]) == 1
    entry = next(iter(data["entries"].values()))
    assert entry["fwd_rows"] == 4 and entry["bwd_config"] == 5 and entry["max_angles"] == 8
    assert entry["backward_ms"][cbct.BWD_CONFIGS[7]] == float(len(cbct.FWD_ROWS) + 7 + 1)

    fake.calls.clear()
    r2 = cbct.autotune(geometry(12), max_angles=8, cache=path)
    assert r2["cached"] is True and r2["bwd_shape"] == cbct.BWD_CONFIGS[5]
    assert fake.calls == [("set_launch", 12, 4, 5)]          # no timing
    assert cbct.get_launch(geometry(12)) == (4, 5)


def test_other_geometry_classes_are_tuned_and_added(fake, tmp_path):
    path = tmp_path / "tune.json"
    cbct.autotune(geometry(1), cache=path)
    cbct.autotune(geometry(2, nz=64), cache=path)
    cbct.autotune(geometry(3, dsd=1536.0), cache=path)
    assert [c[0] for c in fake.calls] == ["autotune"] * 3
    assert len(json.loads(path.read_text())["entries"]) == 3


def test_key_separates_what_the_choice_depends_on():
    base = cbct.tune_key(PARAMS, 60, "dev")
    assert cbct.tune_key(dict(PARAMS), 60, "dev") == base
    for change in (dict(nx=33), dict(dz=0.5), dict(nu=65), dict(dv=1.0), dict(dso=900.0)):
        assert cbct.tune_key(dict(PARAMS, **change), 60, "dev") != base
    assert cbct.tune_key(PARAMS, 61, "dev") != base
    assert cbct.tune_key(PARAMS, 60, "other") != base


@pytest.mark.parametrize("content", [
    "not json",
    json.dumps({"version": 999, "entries": {}}),
    json.dumps([1, 2, 3]),
])
def test_unreadable_or_foreign_files_are_ignored_and_replaced(fake, tmp_path, content):
    path = tmp_path / "tune.json"
    path.write_text(content)
    r = cbct.autotune(geometry(5), cache=path)
    assert r["cached"] is False
    assert json.loads(path.read_text())["version"] == cbct.TUNE_CACHE_VERSION


def test_invalid_cached_shapes_are_retuned(fake, tmp_path):
    path = tmp_path / "tune.json"
    key = cbct.tune_key(PARAMS, 60, cbct._device_name())
    path.write_text(json.dumps({"version": cbct.TUNE_CACHE_VERSION,
                                "entries": {key: {"fwd_rows": 3, "bwd_config": 0}}}))
    r = cbct.autotune(geometry(6), cache=path)
    assert r["cached"] is False and [c[0] for c in fake.calls] == ["autotune"]
    assert json.loads(path.read_text())["entries"][key]["fwd_rows"] == 4


def test_environment_variable_names_the_cache(fake, tmp_path, monkeypatch):
    path = tmp_path / "env.json"
    monkeypatch.setenv("CBCT_TUNE_CACHE", str(path))
    cbct.autotune(geometry(7))
    assert path.exists()
    fake.calls.clear()
    assert cbct.autotune(geometry(8))["cached"] is True
    assert fake.calls == [("set_launch", 8, 4, 5)]


def test_no_cache_always_times(fake):
    cbct.autotune(geometry(9))
    cbct.autotune(geometry(10))
    assert [c[0] for c in fake.calls] == ["autotune", "autotune"]
