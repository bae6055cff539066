"""The launch-shape tuner's host side (no GPU): the committed table parses, names the knobs the
library exports, and survives a write / read round trip with changed values."""

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
    with pytest.raises(SystemExit):
        import torch

        if torch.cuda.is_available():
            raise SystemExit("skip")
        tune.main(["--passes", "1"])
