"""Host-side logic of bench.py's roofline report (no GPU): the committed DRAM
traffic of a kernel is reported only for the tile size it was captured at
and only while the kernel's source text is the one captured."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RASTER = os.path.join(ROOT, "paper_2605_30342_gb300", "csrc", "raster.cu")


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_keyed_by_kernel_tile_and_workload(bench):
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        entries = json.load(f)
    assert entries, "no committed traffic figures"
    for key, e in entries.items():
        kernel, tile = key.split("/tile")
        sha = bench.kernel_source_sha(os.path.join(ROOT, "paper_2605_30342_gb300", "csrc", e["source"]), kernel)
        got = bench.profile_for(kernel, int(tile), e["workload"])
        # reported exactly when the source still matches the capture
        assert (got["bytes_per_launch"] if got else None) == (e["bytes_per_launch"] if sha == e["kernel_sha"] else None), key
        # and only for the workload it was captured on
        for other in (1, 2, 3, 4):
            if other != e["workload"]:
                assert bench.profile_for(kernel, int(tile), other) is None, (key, other)
        # the full-launch figure is the capture scaled by the launch's units
        assert abs(e["bytes_per_launch"] - e["captured_bytes_per_launch"] * e["scale"]) <= 1e-4 * e["bytes_per_launch"]
    for tile in (8, 16, 32):   # a tile without a capture reports nothing
        if f"k_composite_vis/tile{tile}" not in entries:
            assert bench.profile_for("k_composite_vis", tile, 3) is None
    assert bench.profile_for("k_no_such_kernel", 16, 3) is None


def test_kernel_sha_follows_the_definition(bench, tmp_path):
    src = open(RASTER).read()
    base = bench.kernel_source_sha(RASTER, "k_composite_vis")
    assert base is not None and len(base) == 16
    # text outside the kernel does not change it; text inside does
    outside = tmp_path / "outside.cu"
    outside.write_text("// a comment before everything\n" + src + "\n// and after\n")
    assert bench.kernel_source_sha(str(outside), "k_composite_vis") == base
    i = src.index("k_composite_vis(CompositeArgs a)")
    j = src.index("{", i)
    inside = tmp_path / "inside.cu"
    inside.write_text(src[:j + 1] + "\n    // changed\n" + src[j + 1:])
    assert bench.kernel_source_sha(str(inside), "k_composite_vis") != base
    assert bench.kernel_source_sha(RASTER, "k_no_such_kernel") is None
