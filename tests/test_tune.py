"""Tuning table and tuner bookkeeping (no GPU: the table lives on the host)."""
import json

import pytest

from paper_1802_08483_gb300 import mapdec, synth, tune


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1802_08483_gb300 import build
    build.build()
    mapdec.load()
    yield
    mapdec.mapdec_tune_clear()


def test_table_set_get_remove():
    mapdec.mapdec_tune_clear()
    t = {"P": 8, "nsub": 4, "chain_budget_kb": 72, "chain_stages": 2, "store_metric": 1,
         "tensor_cores": 2, "chain_threads": 512}
    mapdec.mapdec_tune_set(64, 12, 2, t)
    assert mapdec.mapdec_tune_get(64, 12, 2) == t
    assert mapdec.mapdec_tune_get(64, 12, 3) is None
    t2 = dict(t, P=4)
    mapdec.mapdec_tune_set(64, 12, 2, t2)  # replaces
    assert mapdec.mapdec_tune_get(64, 12, 2) == t2
    mapdec.mapdec_tune_set(64, 12, 2, None)
    assert mapdec.mapdec_tune_get(64, 12, 2) is None


def test_table_rejects_bad_class():
    with pytest.raises(mapdec.MapDecError):
        mapdec.mapdec_tune_set(1, 12, 2, {"P": 8})
    with pytest.raises(mapdec.MapDecError):
        mapdec.mapdec_tune_set(4, 2, 0, {"P": 8})


def test_json_round_trip(tmp_path):
    mapdec.mapdec_tune_clear()
    table = {"entries": [
        {"q": 16, "n": 10, "I": 2, "tune": {"P": 16, "nsub": 8, "chain_budget_kb": 100,
                                            "chain_stages": 2, "store_metric": 0}, "ms": 1.0},
        {"q": 2, "n": 4, "I": 2, "tune": {"P": 32, "nsub": 0, "chain_budget_kb": 0,
                                          "chain_stages": 0, "store_metric": 1}, "ms": 2.0}]}
    path = tmp_path / "t.json"
    tune.save(table, str(path))
    assert json.loads(path.read_text()) == table
    mapdec.mapdec_tune_clear()
    tune.load(str(path))
    assert mapdec.mapdec_tune_get(16, 10, 2)["P"] == 16
    assert mapdec.mapdec_tune_get(2, 4, 2)["store_metric"] == 1
    # fields missing from an older table read as the planner's choice
    assert mapdec.mapdec_tune_get(2, 4, 2)["tensor_cores"] == 0
    assert mapdec.mapdec_tune_get(2, 4, 2)["chain_threads"] == 0
    mapdec.mapdec_tune_clear()


def test_classes_and_samples():
    frames = [synth.config_frame(3, k) for k in range(40)]
    cls = tune.classes(frames)
    assert sum(len(v) for v in cls.values()) == 40
    for key, idx in cls.items():
        assert all(tune.class_of(frames[k]) == key for k in idx)
    idx = list(range(100))
    s = tune.sample_indices(idx, 7)
    assert len(s) == 7 and s[0] == 0 and s[-1] == 99 and s == sorted(set(s))
    assert tune.sample_indices(idx[:5], 7) == idx[:5]


def test_sample_indices_spread_and_all():
    from paper_1802_08483_gb300 import tune
    idx = list(range(100, 110))
    assert tune.sample_indices(idx, 0) == idx          # 0: every frame
    assert tune.sample_indices(idx, 20) == idx         # fewer frames than asked: all
    s = tune.sample_indices(idx, 3)
    assert s[0] == 100 and s[-1] == 109 and len(s) == 3
