"""Host logic of bench.py's roofline inputs (no GPU).

The DRAM traffic a bench line reports comes from profiles/traffic.json only
while every source file the captured launch depends on is unchanged (its
hash); otherwise the line carries null.  The peaks come from
MEASURED_PEAKS.json, else the stated fallbacks.  The GAS bindings refuse
mismatched argument lengths before calling the library.
"""
import hashlib
import json
import os

import pytest

import bench


def _h(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def test_traffic_only_while_every_source_is_unchanged(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    a = tmp_path / "k.cuh"
    b = tmp_path / "w.cu"
    a.write_text("kernel v1\n")
    b.write_text("work list v1\n")
    entry = {"sources": {"k.cuh": _h(a), "w.cu": _h(b)}, "dram_bytes_per_launch": 1234, "capture": "x.md"}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"key": entry}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("key")[0] == 1234.0
    assert bench.profile_traffic("other") == (None, None)
    b.write_text("work list v2\n")  # a dependency changed: the counters no longer describe the launch
    assert bench.profile_traffic("key")[0] is None
    b.write_text("work list v1\n")
    os.remove(a)  # a dependency missing
    assert bench.profile_traffic("key")[0] is None


def test_committed_traffic_entries_name_existing_sources():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)
    for key, ent in d.items():
        if not isinstance(ent, dict):  # a comment
            continue
        assert ent["dram_bytes_per_launch"] > 0, key
        srcs = list(ent.get("sources", {})) + ([ent["source"]] if "source" in ent else [])
        assert srcs, key
        for src in srcs:
            assert os.path.exists(os.path.join(bench.ROOT, src)), (key, src)
        cap = ent.get("capture")
        if cap:
            assert os.path.exists(os.path.join(bench.ROOT, cap)), (key, cap)


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    hbm, src = bench.measured_peaks()
    assert hbm == bench.FALLBACK_HBM_GBS and src == "fallback"
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.5}))
    assert bench.measured_peaks() == (6000.5, "measured")


def test_gas_bindings_check_lengths():
    from paper_1609_07757_gb300 import _lib as L
    with pytest.raises(ValueError):
        L.iscsi_set_gas((2, 3), (0,), (4, 4))
    with pytest.raises(ValueError):
        L.iscsi_init_gas(5, 2, 2, (2, 3), (0, 4), (4,), [[0.0]], None, 0.0)
    with pytest.raises(ValueError):
        L.iscsi_init_gas(5, 2, 2, (), (), (), [[0.0]], None, 0.0)
