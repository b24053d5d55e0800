"""Host-side checks of bench.py's report (no GPU): the committed ncu summary of
each workload exists and carries a parsable traffic line, the source hash
covers files that exist, and the workload names and algorithmic bytes are the
ones the report states."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import sys

    sys.path.insert(0, ROOT)
    import bench as b

    return b


def test_profiles_exist_and_parse(bench):
    for w, (md, srcs, name) in bench.PROFILES.items():
        path = os.path.join(ROOT, "profiles", md)
        assert os.path.exists(path), md
        lines = [ln for ln in open(path) if ln.startswith("traffic:")]
        assert len(lines) == 1, md
        assert re.fullmatch(r"traffic: dram_bytes_per_launch=\d+ source_hash=[0-9a-f]{16}\n?", lines[0]), lines[0]
        for f in srcs:
            assert os.path.exists(os.path.join(ROOT, "paper_2001_03389_gb300", "csrc", f)), f
        t = bench.profiled_traffic(w)  # a float when the sources match the capture, else None
        assert t is None or t > 0


def test_workloads_and_algorithmic_bytes(bench):
    from paper_2001_03389_gb300 import synth

    assert set(bench.PROFILES) == {bench.ARTS, bench.FP32}
    assert bench.alg_bytes_per_sample("u8") == 2.125
    assert bench.alg_bytes_per_sample("f32") == 8.125
    arts = synth.WORKLOADS[bench.ARTS]
    assert (arts["B"], arts["C"], arts["T"], arts["dtype"]) == (12, 1536, 12500, "u8")
    cfg = bench.config_json(arts, 1)
    assert cfg["workload"] == "arts_12x1536x12500_u8_bct_tdsc_then_fdsc"
    assert cfg["parallelism"] == "single" and bench.config_json(arts, 4)["global_batch"] == 48
    f32 = synth.WORKLOADS[bench.FP32]
    assert (f32["B"], f32["C"], f32["T"], f32["dtype"]) == (32, 4096, 8192, "f32")
    assert (bench.F32_MARGIN, bench.F32_REL) == (1e-9, 1e-6)  # the float32 parity bar
