"""The C-ABI library on the host: it builds, loads, exports what the header
declares, and validates arguments before touching a device."""

import ctypes
import os
import re

import pytest

from paper_1401_8288_gb300 import build as libbuild
from paper_1401_8288_gb300 import xcorr

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "xcorr.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return xcorr.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(xcorr_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("xcorr_plan_create", "xcorr_execute", "xcorr_dump", "xcorr_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (xcorr_\w+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(xcorr.EXPORTS) <= exported


def test_config_struct_layout_matches_c():
    # six ints then a size_t
    assert ctypes.sizeof(xcorr.xcorr_config) == 32
    assert xcorr.xcorr_config.hbm_budget_bytes.offset == 24


@pytest.mark.parametrize("kwargs,status", [
    (dict(n_stations=0, n_channels=4, max_time_per_exec=16), 1),
    (dict(n_stations=4, n_channels=0, max_time_per_exec=16), 1),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=0), 1),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=16, n_pols=1), 1),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=16, fmt=7), 1),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=16, engine=9), 1),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=16, fmt=xcorr.XCORR_IN_CF32,
          engine=xcorr.XCORR_ENGINE_CUDA_CORE), 2),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=16777217, fmt=xcorr.XCORR_IN_CF32), 4),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=70000, fmt=xcorr.XCORR_IN_CI8), 4),
    (dict(n_stations=4, n_channels=4, max_time_per_exec=16777216), 4),
])
def test_plan_create_rejects_before_touching_the_device(lib, kwargs, status):
    with pytest.raises(xcorr.XcorrError) as e:
        xcorr.xcorr_plan_create(**kwargs)
    assert e.value.status == status
    assert xcorr.xcorr_last_error()


def test_null_plan_is_rejected(lib):
    with pytest.raises(xcorr.XcorrError) as e:
        xcorr.xcorr_execute(None, 0, 1, 0)
    assert e.value.status == 1
    xcorr.xcorr_destroy(None)  # a no-op


def test_baseline_index_matches_the_packed_triangle(lib):
    ns = 5
    seen = {}
    for a in range(ns):
        for b in range(a + 1):
            for p in range(2):
                for q in range(2):
                    idx, conj = xcorr.xcorr_baseline_index(ns, a, b, p, q)
                    i, j = 2 * a + p, 2 * b + q
                    if j > i:
                        assert conj and a == b and p < q
                        i, j = j, i
                    else:
                        assert not conj
                    assert idx == i * (i + 1) // 2 + j
                    seen.setdefault(idx, []).append((a, b, p, q))
    # every stored pair is reachable; only the auto XY/YX pair is reached twice
    assert sorted(seen) == list(range(2 * ns * (2 * ns + 1) // 2))
    assert all(len(v) == 1 or (v[0][0] == v[0][1]) for v in seen.values())
    with pytest.raises(xcorr.XcorrError):
        xcorr.xcorr_baseline_index(ns, 1, 2, 0, 0)  # b > a


def test_tuning_cache_file_round_trip(lib, tmp_path):
    # the autotuners' cache in JSON lines: every field read back, unreadable lines skipped
    import json
    good = {"scope": "plan", "device": "NVIDIA GB300", "sms": 152, "fmt": 0, "n_inputs": 512,
            "n_channels": 512, "n_time": 2048, "stage_variant": 4, "groups": 1, "x_streams": 1,
            "unfused": 0, "us": 501, "shape_table": 2}
    batch = dict(good, scope="batch", n_inputs=64, n_channels=64, n_time=1024, stage_variant=3, us=12)
    path = tmp_path / "tuning.jsonl"
    lines = [json.dumps(good), "not json at all", json.dumps(dict(good, stage_variant=99)),
             json.dumps({k: v for k, v in good.items() if k != "groups"}), json.dumps(batch),
             json.dumps(dict(good, shape_table=1)), ""]  # a line of another shape-table revision
    path.write_text("\n".join(lines) + "\n")
    xcorr.xcorr_tuning_cache_clear()
    assert xcorr.xcorr_tuning_cache_load(str(path)) == (2, 4)
    out = tmp_path / "saved.jsonl"
    assert xcorr.xcorr_tuning_cache_save(str(out)) == 2
    saved = [json.loads(line) for line in out.read_text().splitlines()]
    assert sorted(saved, key=lambda d: d["scope"]) == [batch, good]
    # the same problem loaded again replaces its entry; clear empties the cache
    path.write_text(json.dumps(dict(good, stage_variant=8, us=512)) + "\n")
    assert xcorr.xcorr_tuning_cache_load(str(path)) == (1, 0)
    assert xcorr.xcorr_tuning_cache_save(str(out)) == 2
    assert {d["scope"]: d["stage_variant"] for d in map(json.loads, out.read_text().splitlines())} == \
        {"plan": 8, "batch": 3}
    xcorr.xcorr_tuning_cache_clear()
    assert xcorr.xcorr_tuning_cache_save(str(out)) == 0
    with pytest.raises(xcorr.XcorrError):
        xcorr.xcorr_tuning_cache_load(str(tmp_path / "missing.jsonl"))
