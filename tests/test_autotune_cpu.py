"""Host logic of the autotuner: choice under a budget, tie-breaking, cache round trip."""
import pytest

from paper_2508_19138_gb300 import autotune


def test_choose_fastest_within_budget_and_ties():
    cost = {4: 0.5, 8: 0.3, 16: 0.3, 32: 0.1}
    res = autotune.choose(lambda c: cost[c], [32, 4, 8, 16], fits=lambda c: c <= 16)
    assert res["best"] == 8  # 32 does not fit; 8 and 16 tie -> smaller chunk
    assert set(res["table"]) == {"4", "8", "16"}
    with pytest.raises(ValueError):
        autotune.choose(lambda c: 1.0, [4, 8], fits=lambda c: False)


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    key = autotune.cache_key("GB300", 40, 416, 1, 0)
    autotune.save_cache({key: {"best": 16, "table": {"16": 0.1}}}, p)
    assert autotune.load_cache(p)[key]["best"] == 16
    assert autotune.load_cache(str(tmp_path / "missing.json")) == {}
