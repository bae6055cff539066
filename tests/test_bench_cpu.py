"""Host-side contracts of bench.py that need no GPU (CPU only).

* ``roofline.traffic`` comes from the committed ncu record only while the kernel's sources are the
  ones the counters were taken from: a changed source gives ``None``.
* The HBM roofline object carries achieved = algorithmic bytes / launch time and frac = achieved /
  peak.
"""

import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_traffic_record_follows_the_kernel_source(tmp_path, monkeypatch):
    import bench

    sketch, ttm = bench.traffic_for(0, tc=True), bench.traffic_for(1, tc=True)
    assert sketch is not None and ttm is not None and sketch > 4e9 and ttm > sketch
    # a copy of the tree with the mode product's source changed by one line: its record no longer
    # applies, the sketch's still does
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "traffic.txt"), tmp_path / "profiles" / "traffic.txt")
    csrc = tmp_path / "paper_1905_07311_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("sketch_tc.cu", "ttm_tc.cu", "tc.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_1905_07311_gb300", "csrc", f), csrc / f)
    with open(csrc / "ttm_tc.cu", "a") as fh:
        fh.write("\n// changed\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for(0, tc=True) == sketch
    assert bench.traffic_for(1, tc=True) is None
    # and a change of the shared header voids both
    with open(csrc / "tc.cuh", "a") as fh:
        fh.write("\n// changed\n")
    assert bench.traffic_for(0, tc=True) is None


def test_hbm_roofline_object():
    import bench

    peaks = {"hbm_gbs": 6800.0}
    r = bench._hbm_roof("k", 6.8e9, 2.0, peaks, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3400.0) and r["frac"] == pytest.approx(0.5)
    assert r["algorithmic_bytes"] == 6.8e9 and r["avg_launch_ms"] == 2.0 and r["traffic"] is None
