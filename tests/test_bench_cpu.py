"""Host logic of bench.py that needs no GPU: the wording of the oracle sample,
the calibration of the CPU baseline's stride toward its time target and the
parsing of pinned launch knobs."""
import sys
import types

import bench


def test_ordinal():
    assert [bench.ordinal(k) for k in (1, 2, 3, 4, 11, 12, 13, 21, 22, 23, 101, 111, 112)] == \
        ["1st", "2nd", "3rd", "4th", "11th", "12th", "13th", "21st", "22nd", "23rd", "101st", "111th", "112th"]


def _fake_oracle(monkeypatch, per_ray_s, overhead_s, calls):
    def fake(wl, stride, n_threads=0):
        n = 4194304 // stride
        calls.append(stride)
        return n, overhead_s + n * per_ray_s
    monkeypatch.setattr(bench, "time_oracle", fake)
    monkeypatch.setattr(bench, "oracle_segments_per_ray", lambda wl: {"value": 0.0, "sample": ""})
    monkeypatch.setattr(bench, "oracle_single_core", lambda wl: {"value": 0.0, "sample": ""})
    m = types.ModuleType("oracle")
    m.threads = lambda: 16
    monkeypatch.setitem(sys.modules, "oracle", m)


def test_cpu_baseline_reaches_its_target(monkeypatch):
    """A small calibration sample overstates the time per ray (fixed
    overhead); the refinement still lands within a factor of two of the
    target, or takes every ray when that is below it."""
    for per_ray in (2.2e-6, 1e-5, 5e-5):
        calls = []
        _fake_oracle(monkeypatch, per_ray, 0.3, calls)
        out = bench.cpu_baseline(None, target_s=15.0)
        n = 4194304 // calls[-1]
        dt = 0.3 + n * per_ray
        assert calls[-1] == 1 or dt >= 7.5, (per_ray, calls, dt)
        assert dt <= 30.0, (per_ray, calls, dt)
        assert out["value"] == n / dt and out["cores"] == 16 and out["kind"] == "oracle"
        assert ("every ray" in out["sample"]) == (calls[-1] == 1)
        assert len(calls) <= 4


def test_emit_appends_jsonl(monkeypatch, capsys):
    import json
    import os
    scratch = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build")
    os.makedirs(scratch, exist_ok=True)
    log = os.path.join(scratch, f"bench_{os.getpid()}.jsonl")
    if os.path.exists(log):
        os.remove(log)
    monkeypatch.setattr(bench, "_LOG", log)
    bench.emit({"metric": "m", "value": 1.0})
    bench.emit({"metric": "m", "value": 2.0})
    with open(log) as f:
        lines = f.read().splitlines()
    os.remove(log)
    assert [json.loads(x)["value"] for x in lines] == [1.0, 2.0]
    assert capsys.readouterr().out.splitlines() == lines


def test_pinned_launches_parse_the_printed_form():
    import pytest
    spec = '{"cone": [[128, 8, 0], [128, 16, 1]], "parallel": [[128, 8, 0], [128, 8, 0]]}'
    assert bench.pinned_launches(spec, ["cone", "parallel"]) == [((128, 8, 0), (128, 16, 1)),
                                                                  ((128, 8, 0), (128, 8, 0))]
    with pytest.raises(SystemExit):
        bench.pinned_launches('{"cone": [[128, 8, 0], [128, 8, 1]]}', ["cone", "parallel"])
    with pytest.raises(SystemExit):
        bench.pinned_launches('{"cone": [[128, 8], [128, 8, 1]]}', ["cone"])
