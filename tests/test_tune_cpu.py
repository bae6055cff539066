"""The launch-shape tuner's host side (no GPU): the committed table parses, names the knobs the
library exports, and survives a write / read round trip with changed values; the coordinate descent
finds the optimum of a synthetic cost, respects the gain threshold and scores each knob only on the
objectives it affects."""

import os

import pytest


def test_table_round_trip(tmp_path):
    from paper_1905_07311_gb300 import tune

    rows = tune.read_table()
    assert len(rows) >= 8
    names = [n for _, n, _ in rows]
    assert len(set(names)) == len(names)
    for key, name, value in rows:
        assert key.startswith("TUNE_") and 1 <= value <= 4096
    values = {n: (v % 7) + 1 for _, n, v in rows}
    out = os.path.join(tmp_path, "table.inc")
    tune.write_table(rows, values, out)
    back = tune.read_table(out)
    assert [(k, n) for k, n, _ in back] == [(k, n) for k, n, _ in rows]
    assert {n: v for _, n, v in back} == values


def test_table_names_match_the_library():
    from paper_1905_07311_gb300 import _lib, build, tune

    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    L = _lib.lib()
    lib_names = sorted(L.rh_tuning_name(i).decode() for i in range(L.rh_tuning_count()))
    assert lib_names == sorted(n for _, n, _ in tune.read_table())


def test_knob_scopes():
    from paper_1905_07311_gb300 import tune

    objs = ["batched_f32", "batched_f32_bf16x2", "dense_1024"]
    assert tune._affects("gram.min_tiles", objs) == objs
    assert tune._affects("small_tc_sketch.min_tiles", objs) == ["batched_f32", "batched_f32_bf16x2"]
    assert tune._candidates("ttm_small.ctas_per_sm") == tune.CANDIDATES["ctas_per_sm"]
    assert tune._candidates("ttm_small.min_tiles") == tune.CANDIDATES["min"]


def test_tuner_refuses_to_run_without_a_device():
    torch = pytest.importorskip("torch")
    from paper_1905_07311_gb300 import tune

    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present: the tuner would time kernels")
    with pytest.raises(SystemExit, match="needs a CUDA device"):
        tune.main(["--passes", "1"])


def _fake(rows, optimum, objectives):
    """A synthetic cost: every objective's time is 1 ms plus 0.01 ms times the squared number of
    octaves by which each knob it depends on lies away from that knob's optimum."""
    import math

    from paper_1905_07311_gb300 import tune

    state = {n: v for _, n, v in rows}
    calls = {"measure": 0}

    def measure(names):
        calls["measure"] += 1
        out = {}
        for o in names:
            t = 1.0
            for _, n, _ in rows:
                if o in tune._affects(n, objectives):
                    t += 0.01 * (math.log2(state[n]) - math.log2(optimum[n])) ** 2
            out[o] = t
        return out

    def apply(name, v):
        state[name] = v

    return state, calls, measure, apply


def test_coordinate_descent_finds_each_knobs_optimum():
    from paper_1905_07311_gb300 import tune

    rows = [("TUNE_A", "sketch_small.ctas_per_sm", 1), ("TUNE_B", "sketch_small.min_tiles", 1),
            ("TUNE_C", "gram.min_tiles", 256)]
    objectives = ["batched_f32", "batched_f32_bf16x2", "dense_1024"]
    optimum = {"sketch_small.ctas_per_sm": 4, "sketch_small.min_tiles": 32, "gram.min_tiles": 8}
    state, calls, measure, apply = _fake(rows, optimum, objectives)
    log = []
    got = tune.coordinate_descent(rows, {n: v for _, n, v in rows}, objectives, measure, apply, passes=3,
                                  min_gain=0.003, log=log.append)
    assert got == optimum
    assert state == optimum                      # the chosen values are the ones left applied
    # separable cost: the second pass moves nothing, so the descent stops after it
    chosen = [r for r in log if "chosen" in r]
    assert len(chosen) == 2 * len(rows)
    # every candidate of every knob was tried in each pass, except the current value
    tried = [r for r in log if "value" in r]
    per_pass = sum(len(tune._candidates(n)) - 1 for _, n, _ in rows)
    assert len(tried) == 2 * per_pass


def test_coordinate_descent_keeps_values_below_the_gain_threshold():
    from paper_1905_07311_gb300 import tune

    rows = [("TUNE_A", "ttm_small.ctas_per_sm", 2)]
    objectives = ["batched_f32"]
    # the optimum is one octave away: moving gains 0.01 ms of 1.01 ms (~1 %)
    state, _, measure, apply = _fake(rows, {"ttm_small.ctas_per_sm": 4}, objectives)
    kept = tune.coordinate_descent(rows, {"ttm_small.ctas_per_sm": 2}, objectives, measure, apply, passes=2,
                                   min_gain=0.05)
    assert kept == {"ttm_small.ctas_per_sm": 2} and state == kept
    moved = tune.coordinate_descent(rows, {"ttm_small.ctas_per_sm": 2}, objectives, measure, apply, passes=2,
                                    min_gain=0.003)
    assert moved == {"ttm_small.ctas_per_sm": 4} and state == moved


def test_coordinate_descent_scores_only_the_objectives_a_knob_affects():
    from paper_1905_07311_gb300 import tune

    rows = [("TUNE_A", "small_tc_ttm.min_tiles", 1)]
    objectives = ["batched_f32", "batched_f32_bf16x2", "dense_1024"]
    seen = set()
    _, _, measure, apply = _fake(rows, {"small_tc_ttm.min_tiles": 16}, objectives)

    def spy(names):
        seen.update(names)
        return measure(names)

    got = tune.coordinate_descent(rows, {"small_tc_ttm.min_tiles": 1}, objectives, spy, apply, passes=1,
                                  min_gain=0.003)
    assert got == {"small_tc_ttm.min_tiles": 16}
    assert seen == {"batched_f32", "batched_f32_bf16x2"}
