"""Host logic of the autotuner (no GPU): coordinate descent, the settings table, signatures."""

import json

import pytest

import paper_2509_19162_gb300 as cgp

cgp.build()
from paper_2509_19162_gb300 import tune  # noqa: E402  (needs the built library)


def test_coordinate_descent_finds_separable_minimum():
    knobs = (("a", (0, 1, 2, 3)), ("b", ("x", "y", "z")), ("c", (False, True)))
    cost = {"a": {0: 5, 1: 3, 2: 1, 3: 4}, "b": {"x": 2, "y": 0, "z": 1}, "c": {False: 1, True: 0}}
    calls = []

    def measure(s):
        calls.append(dict(s))
        return sum(cost[k][v] for k, v in s.items())

    best, t, trials = tune.coordinate_descent(knobs, measure)
    assert best == {"a": 2, "b": "y", "c": True} and t == 1 + 0 + 0
    # the start plus each other value of each knob once
    assert len(calls) == 1 + 3 + 2 + 1 and len(trials) == len(calls)


def test_coordinate_descent_skips_inapplicable_settings():
    knobs = (("s", ("auto", "sort", "hash")), ("g", (0, 1)))

    def measure(s):
        if s["s"] == "sort":
            return None
        return {"auto": 2.0, "hash": 1.0}[s["s"]] + (0.5 if s["g"] else 0.0)

    best, t, trials = tune.coordinate_descent(knobs, measure)
    assert best == {"s": "hash", "g": 0} and t == 1.0
    with pytest.raises(ValueError):
        tune.coordinate_descent(knobs, lambda s: None)


def test_table_roundtrip(tmp_path):
    path = str(tmp_path / "tune.json")
    t = tune.TuneTable(path)
    assert t.get("batch:x") is None
    t.put("batch:x", {"ilp": 2, "graph": True}, 0.25, 0.3, [1, 2, 3])
    t2 = tune.TuneTable(path)
    assert t2.get("batch:x") == {"ilp": 2, "graph": True}
    assert json.load(open(path))["batch:x"]["default_seconds"] == 0.3


def test_signatures_depend_on_workload_and_device():
    jobs = [(6, [[1, 0, 2, 3, 4, 5]], True, -1), (7, [[1, 2, 0, 3, 4, 5, 6]], False, -1)]
    a = tune.batch_signature(jobs, device="dev0")
    assert a == tune.batch_signature(list(reversed(jobs)), device="dev0")   # order-free multiset
    assert a != tune.batch_signature(jobs, device="dev1")
    assert a != tune.batch_signature(jobs[:1], device="dev0")
    g = tune.growth_signature(6, [[1, 0, 2, 3, 4, 5]], device="d", max_radius=-1)
    assert g != tune.growth_signature(6, [[1, 0, 2, 3, 4, 5]], device="d", max_radius=3)


def test_batch_options_translation():
    s = {"visited": "hash", "ilp": 2, "grid_per_sm": 3, "wave_l2": -1, "max_active": 512, "unit": 2,
         "graph": True}
    assert tune.batch_options(s, 152) == {"visited": "hash", "ilp": 2, "grid": 456, "wave_l2": -1,
                                          "max_active": 512, "unit": 2, "graph": True}


def test_batch_knobs_cover_visited_set_kind_chunking_and_graph():
    names = [k for k, _ in tune.BATCH_KNOBS]
    assert names == ["visited", "ilp", "grid_per_sm", "wave_l2", "max_active", "unit", "graph"]
    values = dict(tune.BATCH_KNOBS)
    assert set(values["visited"]) == {"auto", "hash", "bitmap"}
    assert values["graph"][0] is True                   # the library default comes first
    assert values["unit"][0] == 4 and values["max_active"][0] == 0
