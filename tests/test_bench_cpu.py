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


def _work(**kw):
    w = dict(steps=5, workload=3, pairs_ua=2.8e9, pairs_vis=6.29e9, tile_sc=16, tile_vf=16, n_cand=256, n_train=200,
             W=640, H=480, vis_vf=37_450_361, vis_sc=59_298_525, sorted_vf=200_000_000, sorted_sc=0, n=1_000_000,
             K=16, Kc=16, b=2)
    w.update(kw)
    return w


def _stages(dom, ms=10.0):
    st = {k: (1.0, 5) for k in ("project", "scan", "emit", "sort", "ranges", "composite_ua", "composite_vis",
                                 "reduce", "vf_accum")}
    st[dom] = (ms, 5)
    return st


PEAKS = {"hbm_gbs": 6691.1, "sm_max_mhz": 2070.0}


def test_roofline_of_each_dominant_stage(bench):
    """Every stage the step can be dominated by gets a roofline whose
    fraction is its achieved rate over the peak, from the stated per-unit
    counts; the sort counts stage-B passes only for the sorted tile entries."""
    w = _work()
    fp32 = 2.0 * 152 * bench.FP32_LANES_PER_SM * 2070.0 * 1e6 / 1e12
    for dom, fpp, pairs in (("composite_vis", bench.FLOPS_PER_PAIR_VIS, w["pairs_vis"]),
                            ("composite_ua", bench.FLOPS_PER_PAIR_UA, w["pairs_ua"])):
        r = bench.stage_roofline(_stages(dom, 50.0), w, PEAKS, "measured", 152)
        assert r["kernel"] == "k_" + dom and r["bound"] == "alu" and r["peak"] == pytest.approx(fp32)
        assert r["achieved"] == pytest.approx(pairs * w["steps"] * fpp / 0.05 / 1e12)
        assert r["frac"] == pytest.approx(r["achieved"] / fp32)
    r = bench.stage_roofline(_stages("sort", 25.0), w, PEAKS, "measured", 152)
    tiles_sc = 256 * 40 * 30
    per_step = (w["vis_vf"] + w["vis_sc"]) * 64 + w["sorted_vf"] * 32 + tiles_sc * 16
    assert r["kernel"] == "sort" and r["algorithmic_bytes_per_step"] == pytest.approx(per_step)
    assert r["frac"] == pytest.approx(per_step * 5 / 0.025 / 1e9 / 6691.1)
    # counted tile lists add no stage-B sort bytes
    r2 = bench.stage_roofline(_stages("sort", 25.0), _work(sorted_vf=0), PEAKS, "measured", 152)
    assert r2["algorithmic_bytes_per_step"] == pytest.approx(per_step - w["sorted_vf"] * 32)
    r = bench.stage_roofline(_stages("project", 20.0), w, PEAKS, "measured", 152)
    coeff = (16 * 3 + 16) * 2
    per_step = (7 * 1e6 * 44 + 8 * 1e6 * (44 + coeff) + 456 * 1e6 / 8 + w["vis_vf"] * 44 + w["vis_sc"] * 76)
    assert r["kernel"] == "k_project" and r["bound"] == "hbm"
    assert r["algorithmic_bytes_per_step"] == pytest.approx(per_step)
    assert r["frac"] == pytest.approx(per_step * 5 / 0.020 / 1e9 / 6691.1)
    # a stage without a model reports its time and no fraction
    r = bench.stage_roofline(_stages("emit", 30.0), w, PEAKS, "measured", 152)
    assert r["kernel"] == "emit" and r["frac"] is None and r["avg_launch_ms"] == pytest.approx(6.0)
