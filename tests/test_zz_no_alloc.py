"""The allocation-free single-view scoring entry point.

Callers whose device memory is entirely owned by their own memory manager, or
that cannot take the device-wide synchronisation an allocation may imply,
score a candidate view with gavis_score_view_noalloc: same kernels as
gavis_score_views, scratch in a fixed array inside the library.  These tests
call it through the C ABI and compare it with gavis_score_views on the same
view, on two calls in a row.  The file sorts last so that a run stopping at
the first failure has already run every other test; it also passes alone.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from _util import GAP, TOL, compare_views, score_excess, sorted_gap

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gv():
    import __graft_entry__ as g
    g.build()
    import paper_2605_30342_gb300 as pkg
    lib = pkg.load()
    lib.gavis_score_view_noalloc.argtypes = [C.POINTER(pkg.gavis_gaussians), C.POINTER(pkg.gavis_vf),
                                             C.POINTER(pkg.gavis_camera), C.POINTER(pkg.gavis_params), C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_char_p, C.c_size_t, C.c_void_p]
    lib.gavis_score_view_noalloc.restype = C.c_int
    return pkg


def call_noalloc(gv, gs, vf, cam, prm):
    lib = gv.load()
    rgb = torch.full((3, cam.H, cam.W), float("nan"), device="cuda")
    unc = torch.full((cam.H, cam.W), float("nan"), device="cuda")
    score = torch.full((1,), float("nan"), device="cuda")
    err = C.create_string_buffer(256)
    rec = gv.camera_records([cam])
    vs = vf.struct()
    rc = lib.gavis_score_view_noalloc(C.byref(gs.struct), C.byref(vs), rec, C.byref(prm), C.c_void_p(rgb.data_ptr()),
                                      C.c_void_p(unc.data_ptr()), C.c_void_p(score.data_ptr()), err, 256,
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, err.value.decode(), rgb, unc, score


@pytest.mark.parametrize("k,kw", [(1, dict(n=2000, n_train=4, n_cand=3)),
                                  (2, dict(n=20000, n_train=4, n_cand=3, train_wh=(160, 120), cand_wh=(200, 136)))])
def test_noalloc_matches_score_views_twice(gv, k, kw):
    c = sg.config(k, **kw)
    gs = gv.Gaussians.from_numpy(c["scene"])
    ctx = gv.Context(0)
    L = c["vf_degree"]
    vf = ctx.vf_build(gs, c["train"], degree=L)
    prm = gv.Params(vf_degree=L)
    # two calls in a row on different views, then the first view again
    for v in (0, 1, 0):
        cam = c["cand"][v]
        ref = ctx.score_views(gs, vf, [cam], params=prm)
        rc, msg, rgb, unc, score = call_noalloc(gv, gs, vf, cam, prm)
        assert rc == 0, msg
        assert (unc - ref["unc"][0]).abs().max().item() <= TOL
        assert (rgb - ref["rgb"][0]).abs().max().item() <= TOL
        assert abs(score.item() - ref["score"][0].item()) <= TOL
    ctx.close()


def test_noalloc_matches_oracle(gv):
    """Against the oracle directly: the field comes from the oracle's VF CONST
    (rounded to f32), each view is scored by the allocation-free call, and
    per-pixel entropy, RGB and the view score agree with the oracle's
    VF QUERY + UA raster + entropy score within the parity tolerance."""
    c = sg.config(1, n=900, n_train=3, n_cand=3, train_wh=(100, 75), cand_wh=(100, 75))
    sc, cand, L = c["scene"], c["cand"], c["vf_degree"]
    g, _, _ = oracle.vf_build(c["train"], sc, L)
    g32 = g.astype(np.float32)
    gs = gv.Gaussians.from_numpy(sc)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), L, len(c["train"]), 1.0)
    ref = oracle.score_views(sc, g32.astype(np.float64), L, len(c["train"]), cand)
    prm = gv.Params(vf_degree=L)
    unc_all, rgb_all, score_all = [], [], []
    for cam in cand:
        rc, msg, rgb, unc, score = call_noalloc(gv, gs, vf, cam, prm)
        assert rc == 0, msg
        unc_all.append(unc.cpu().numpy())
        rgb_all.append(rgb.cpu().numpy())
        score_all.append(score.item())
    err, n_band = compare_views(np.stack(unc_all), np.stack(rgb_all), ref)
    assert err <= TOL, (err, n_band)
    score_all = np.asarray(score_all, dtype=np.float32)
    assert score_excess(score_all, ref).max() <= TOL
    if sorted_gap(ref["score"]) > GAP:
        assert int(np.argmax(score_all)) == ref["best"]


def test_noalloc_rejects_oversized_inputs(gv):
    c = sg.config(1, n=40000, n_train=1, n_cand=1)          # above the 32768-Gaussian maximum
    gs = gv.Gaussians.from_numpy(c["scene"])
    K = (c["vf_degree"] + 1) ** 2
    vf = gv.VisibilityField(torch.zeros((gs.n, K), device="cuda"), c["vf_degree"], 0, 1.0)
    rc, msg, _, _, _ = call_noalloc(gv, gs, vf, c["cand"][0], gv.Params())
    assert rc == gv.ERR_ARG and "maximum" in msg
    big = sg.config(1, n=100, n_train=1, n_cand=1, cand_wh=(2048, 2048))["cand"][0]   # 16384 tiles
    small = gv.Gaussians.from_numpy(sg.tiny_scene(100))
    vf2 = gv.VisibilityField(torch.zeros((100, K), device="cuda"), c["vf_degree"], 0, 1.0)
    rc, msg, _, _, _ = call_noalloc(gv, small, vf2, big, gv.Params())
    assert rc == gv.ERR_ARG and "tiles" in msg
