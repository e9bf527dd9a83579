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


def test_coordinate_descent_tunes_one_parameter_at_a_time():
    """A separable cost: the chunk first (with the start values of the others), then the tile with
    the chosen chunk, then the panel; candidates outside the budget are skipped."""
    calls = []

    def cost(p):
        calls.append(dict(p))
        return {4: 3.0, 8: 2.0, 16: 1.5, 32: 1.0}[p["max_energies"]] + {0: 0.2, 16: 0.1, 32: 0.3}[p["gemm_tile"]] \
            + {0: 0.05, 8: 0.0}[p["inv_panel"]]

    res = autotune.coordinate_descent(cost, {"max_energies": (4, 8, 16, 32), "gemm_tile": (32, 16),
                                             "inv_panel": (0, 8)},
                                      {"max_energies": 4, "gemm_tile": 0, "inv_panel": 0},
                                      fits=lambda p: p["max_energies"] <= 16)
    assert res["best"] == {"max_energies": 16, "gemm_tile": 16, "inv_panel": 8}
    assert set(res["table"]["max_energies"]) == {"4", "8", "16"}
    assert len(calls) == 3 + 2 + 2
    assert all(c["gemm_tile"] == 0 for c in calls[:3]) and all(c["max_energies"] == 16 for c in calls[3:])
    with pytest.raises(ValueError):
        autotune.coordinate_descent(cost, {"max_energies": (32,)}, {"max_energies": 32, "gemm_tile": 0,
                                                                    "inv_panel": 0}, fits=lambda p: False)
