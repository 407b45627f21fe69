"""GPU checks of the batch launch settings, the CUDA-graph replay of a batch run and the
autotuner: every setting gives the results of the default run and of the oracle."""

import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg():
    import torch
    assert torch.cuda.is_available()
    import paper_2509_19162_gb300 as p
    p.build()
    return p


@pytest.fixture(scope="module")
def spec():
    jobs = w.batch_groups(count=192)
    return [(j.n, j.gens, j.inverse_closed, -1) for j in jobs]


@pytest.fixture(scope="module")
def reference(cg, spec):
    with cg.Batch(spec) as b:
        return [r.layers for r in b.run()]


def test_default_batch_matches_oracle(spec, reference):
    for (n, gens, inv, rad), layers in list(zip(spec, reference))[::16]:
        assert layers == oracle.growth(n, gens)[0]


@pytest.mark.parametrize("opts", [
    {"graph": False},
    {"visited": "hash"},
    {"visited": "bitmap", "ilp": 2},
    {"ilp": 3, "grid": 152},
    {"wave_l2": 1 << 16, "graph": True},
    {"wave_l2": -1, "grid": 300},
    {"max_active": 7},
    {"max_active": 1, "unit": 4},
    {"unit": 2, "graph": False},
    {"unit": 8, "visited": "hash"},
])
def test_settings_do_not_change_results(cg, spec, reference, opts):
    with cg.Batch(spec, **opts) as b:
        for _ in range(3):              # first run plans (and captures), later runs replay
            assert [r.layers for r in b.run()] == reference
        st = b.stats()
        assert st["launches"] >= 2


def test_graph_replay_after_option_change(cg, spec, reference):
    with cg.Batch(spec, graph=True) as b:
        assert [r.layers for r in b.run()] == reference
        b.set_options(ilp=2)            # drops the plan and the graph
        assert [r.layers for r in b.run()] == reference
        assert [r.layers for r in b.run(cap=600)] == reference   # another capacity: replanned


def test_tune_batch(cg, spec, reference, tmp_path):
    from paper_2509_19162_gb300 import tune
    table = tune.TuneTable(str(tmp_path / "t.json"))
    res = tune.tune_batch(spec, table=table, reps=1)
    assert res["seconds"] <= res["default_seconds"]
    assert table.get(res["signature"]) == res["settings"]
    with cg.Batch(spec, **res["options"]) as b:
        assert [r.layers for r in b.run()] == reference


def test_tune_growth(cg):
    from paper_2509_19162_gb300 import tune
    res = tune.tune_growth(8, w.coxeter(8), reps=1)
    assert res["seconds"] <= res["default_seconds"]
    assert res["settings"]["strategy"] in ("auto", "bitmap", "hash", "sweep", "sort")
