"""CPU checks of the autotuner's cache file: save/load round trip, merging, and
rejection of files it did not write (no GPU needed: the cache is host state)."""
import json

import pytest

from paper_2403_16665_gb300 import _build, adfft


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return adfft.load()


ENTRY = {"device": "NVIDIA GB300|sm_103|cuda-driver 13000", "N": 16384, "M": 131072, "batch": 4096,
         "dtype": 0, "precision": 0, "algo": 1, "fft_len": 8192, "cluster": 4, "staged": 1, "grid": 0,
         "ms": 2.33}


def write(path, obj):
    path.write_text(json.dumps(obj) if not isinstance(obj, str) else obj)
    return str(path)


def test_round_trip_and_merge(lib, tmp_path):
    adfft.autotune_clear()
    e2 = dict(ENTRY, N=8192, M=20480, dtype=1, algo=3, fft_len=0, cluster=0, staged=0, grid=-1, four_step_a=1024,
              ms=0.5)
    e3 = dict(ENTRY, device='other "gpu"\\x', batch=7)
    adfft.autotune_load(write(tmp_path / "a.json", {"adfft_autotune": 1, "entries": [ENTRY, e2]}))
    adfft.autotune_load(write(tmp_path / "b.json", {"adfft_autotune": 1, "entries": [e3]}))
    out = tmp_path / "out.json"
    adfft.autotune_save(str(out))
    got = json.loads(out.read_text())
    assert got["adfft_autotune"] == 1
    key = lambda e: (e["device"], e["N"], e["M"], e["batch"], e["dtype"], e["precision"])  # noqa: E731
    entries = {key(e): e for e in got["entries"]}
    assert len(entries) == 3
    for want in (ENTRY, e2, e3):
        e = entries[key(want)]
        for k in ("algo", "fft_len", "cluster", "staged", "grid"):
            assert e[k] == want[k], (k, e, want)
        assert e["four_step_a"] == want.get("four_step_a", 0)
        assert abs(e["ms"] - want["ms"]) <= 1e-5 * want["ms"]
    # the saved file loads again; a later entry for the same key replaces the earlier one
    adfft.autotune_clear()
    adfft.autotune_load(str(out))
    adfft.autotune_load(write(tmp_path / "c.json", {"adfft_autotune": 1, "entries": [dict(ENTRY, cluster=8)]}))
    adfft.autotune_save(str(out))
    entries = {key(e): e for e in json.loads(out.read_text())["entries"]}
    assert len(entries) == 3 and entries[key(ENTRY)]["cluster"] == 8
    adfft.autotune_clear()
    adfft.autotune_save(str(out))
    assert json.loads(out.read_text()) == {"adfft_autotune": 1, "entries": []}


@pytest.mark.parametrize("text", [
    "",
    "{}",
    "[]",
    '{"adfft_autotune": 2, "entries": []}',                              # unknown version
    '{"adfft_autotune": 1}',                                             # no entries
    '{"adfft_autotune": 1, "entries": [{}]}',
    '{"adfft_autotune": 1, "entries": [' + json.dumps(dict(ENTRY, algo=2)) + ']}',        # chirp-z is not tuned
    '{"adfft_autotune": 1, "entries": [' + json.dumps({k: v for k, v in ENTRY.items() if k != "cluster"}) + ']}',
    '{"adfft_autotune": 1, "entries": [' + json.dumps(ENTRY) + ']} trailing',
    '{"adfft_autotune": 1, "entries": [' + json.dumps(ENTRY)[:-3] + ']}',                 # truncated
    '{"adfft_autotune": 1, "entries": [' + json.dumps(dict(ENTRY, staged=5)) + ']}',
    '{"adfft_autotune": 1, "entries": [' + json.dumps(dict(ENTRY, grid=-2)) + ']}',
    '{"adfft_autotune": 1, "entries": [' + json.dumps(dict(ENTRY, four_step_a=-4)) + ']}',
])
def test_rejects_malformed_files_and_merges_nothing(lib, tmp_path, text):
    adfft.autotune_clear()
    with pytest.raises(adfft.AdfftError) as ei:
        adfft.autotune_load(write(tmp_path / "bad.json", text))
    assert ei.value.code == -1
    out = tmp_path / "out.json"
    adfft.autotune_save(str(out))
    assert json.loads(out.read_text())["entries"] == []


def test_grid_field_is_optional(lib, tmp_path):
    adfft.autotune_clear()
    e = {k: v for k, v in ENTRY.items() if k != "grid"}
    adfft.autotune_load(write(tmp_path / "g.json", {"adfft_autotune": 1, "entries": [e]}))
    out = tmp_path / "out.json"
    adfft.autotune_save(str(out))
    assert json.loads(out.read_text())["entries"][0]["grid"] == 0
    adfft.autotune_clear()


def test_missing_file_and_null_arguments(lib, tmp_path):
    with pytest.raises(adfft.AdfftError):
        adfft.autotune_load(str(tmp_path / "does_not_exist.json"))
    assert lib.adfft_autotune_load(None) == -1
    assert lib.adfft_autotune_save(None) == -1
    assert lib.adfft_plan_autotune(None, None, None, None, 0, 0) == -1
    assert lib.adfft_plan_set_launch_shape(None, 0, 0, -1, 0) == -1
