"""Scoring plans (the scoring chain captured as a CUDA graph): a replay must
give the same bits as gavis_score_views for the same poses, pick up new poses
and in-place scene updates, and flag an undersized tile-entry capacity."""
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
    return pkg


@pytest.fixture(scope="module")
def ctx(gv):
    c = gv.Context(0)
    yield c
    c.close()


def setup(gv, ctx, k=2, **kw):
    c = sg.config(k, **kw)
    gs = gv.Gaussians.from_numpy(c["scene"])
    vf = ctx.vf_build(gs, c["train"], degree=c["vf_degree"])
    return c, gs, vf


def needed(gv, ctx, gs, vf, cams, p):
    """(visible records, tile keys) gavis_score_views used for `cams`."""
    ctx.prof_enable(True)
    ctx.score_views(gs, vf, cams, params=p, want_rgb=False, want_unc=False)
    r = ctx.prof_read()
    ctx.prof_enable(False)
    return int(r["visible"]), int(r["keys"])


def assert_same(plan, ref):
    assert torch.equal(plan.score, ref["score"])
    assert int(plan.best_dev.item()) == ref["best"]
    if plan.rgb is not None:
        assert torch.equal(plan.rgb, ref["rgb"])
    if plan.unc is not None:
        assert torch.equal(plan.unc, ref["unc"])


@pytest.mark.parametrize("lists", [1, 2])   # tile lists by counting / by sorting in the captured chain
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_plan_equals_score_views(ctx, gv, tile, lists):
    c, gs, vf = setup(gv, ctx, n=20000, n_train=4, n_cand=6, train_wh=(160, 120), cand_wh=(200, 136))
    cand = c["cand"]
    p = gv.Params(tile=tile, vf_degree=c["vf_degree"], tile_lists=lists)
    rec, cap = needed(gv, ctx, gs, vf, cand, p)
    plan = ctx.plan(gs, vf, len(cand), cand[0].W, cand[0].H, cap, record_capacity=rec, params=p, want_rgb=True,
                    want_unc=True)
    assert plan.kernels > 10
    plan.launch(cand)
    torch.cuda.synchronize()
    assert plan.overflowed() == (False, rec, cap)
    assert_same(plan, ctx.score_views(gs, vf, cand, params=p))
    plan.close()


def test_plan_equals_score_views_sorted_tiles(ctx, gv):
    """Views of more than 2048 tiles (here 96 x 88 at tile 8) take the sorted
    tile lists in the captured chain too; replays equal gavis_score_views."""
    c, gs, vf = setup(gv, ctx, n=20000, n_train=4, n_cand=3, train_wh=(160, 120), cand_wh=(768, 704))
    cand = c["cand"]
    p = gv.Params(tile=8, vf_degree=c["vf_degree"])
    rec, cap = needed(gv, ctx, gs, vf, cand, p)
    plan = ctx.plan(gs, vf, len(cand), 768, 704, cap, record_capacity=rec, params=p, want_rgb=True, want_unc=True)
    plan.launch(cand)
    torch.cuda.synchronize()
    assert plan.overflowed() == (False, rec, cap)
    assert_same(plan, ctx.score_views(gs, vf, cand, params=p))
    plan.close()


def test_plan_matches_oracle(ctx, gv):
    c = sg.config(1, n=900, n_train=3, n_cand=5, train_wh=(100, 75), cand_wh=(100, 75))
    sc, cand, L = c["scene"], c["cand"], c["vf_degree"]
    g, _, _ = oracle.vf_build(c["train"], sc, L)
    g32 = g.astype(np.float32)
    gs = gv.Gaussians.from_numpy(sc)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), L, len(c["train"]), 1.0)
    p = gv.Params(tile=16, vf_degree=L)
    plan = ctx.plan(gs, vf, len(cand), cand[0].W, cand[0].H, 1 << 20, params=p, want_rgb=True, want_unc=True)
    plan.launch(cand)
    torch.cuda.synchronize()
    ref = oracle.score_views(sc, g32.astype(np.float64), L, len(c["train"]), cand)
    err, n_band = compare_views(plan.unc.cpu().numpy(), plan.rgb.cpu().numpy(), ref)
    assert err <= TOL, (err, n_band)
    assert score_excess(plan.score.cpu().numpy(), ref).max() <= TOL
    if sorted_gap(ref["score"]) > GAP:
        assert int(plan.best_dev.item()) == ref["best"]


def test_plan_relaunch_with_new_poses(ctx, gv):
    c, gs, vf = setup(gv, ctx, n=20000, n_train=4, n_cand=8, train_wh=(160, 120), cand_wh=(160, 120))
    a, b = c["cand"][:4], c["cand"][4:]
    p = gv.Params(tile=16, vf_degree=c["vf_degree"])
    cap = 2 * max(needed(gv, ctx, gs, vf, a, p)[1], needed(gv, ctx, gs, vf, b, p)[1])
    plan = ctx.plan(gs, vf, 4, 160, 120, cap, params=p, want_unc=True)
    for poses in (a, b, a, b):
        plan.launch(gv.camera_records(poses))
        assert_same(plan, ctx.score_views(gs, vf, poses, params=p, want_rgb=False))
    assert not plan.overflowed()[0]
    plan.close()


def test_plan_reads_scene_values_at_launch(ctx, gv):
    c, gs, vf = setup(gv, ctx, n=20000, n_train=4, n_cand=4, train_wh=(160, 120), cand_wh=(160, 120))
    cand = c["cand"]
    p = gv.Params(tile=16, vf_degree=c["vf_degree"])
    cap = 2 * needed(gv, ctx, gs, vf, cand, p)[1]
    plan = ctx.plan(gs, vf, len(cand), 160, 120, cap, params=p)
    plan.launch(cand)
    torch.cuda.synchronize()
    before = plan.score.clone()
    with torch.no_grad():
        gs.opac.mul_(0.5)          # in place: same addresses
        vf.coeffs.mul_(0.25)
    torch.cuda.synchronize()
    plan.launch(cand)
    ref = ctx.score_views(gs, vf, cand, params=p, want_rgb=False, want_unc=False)
    assert_same(plan, ref)
    assert not torch.equal(before, plan.score)
    plan.close()


@pytest.mark.parametrize("lists", [1, 2])
def test_plan_flags_overflow(ctx, gv, lists):
    c, gs, vf = setup(gv, ctx, n=20000, n_train=4, n_cand=4, train_wh=(160, 120), cand_wh=(160, 120))
    cand = c["cand"]
    p = gv.Params(tile=16, vf_degree=c["vf_degree"], tile_lists=lists)
    rec, need = needed(gv, ctx, gs, vf, cand, p)
    few_entries = ctx.plan(gs, vf, len(cand), 160, 120, need // 3, params=p)
    few_entries.launch(cand)
    assert few_entries.overflowed() == (True, rec, need)
    few_records = ctx.plan(gs, vf, len(cand), 160, 120, need, record_capacity=rec - 1, params=p)
    few_records.launch(cand)
    assert few_records.overflowed() == (True, rec, need)
    exact = ctx.plan(gs, vf, len(cand), 160, 120, need, record_capacity=rec, params=p)
    exact.launch(cand)
    assert exact.overflowed() == (False, rec, need)
    assert_same(exact, ctx.score_views(gs, vf, cand, params=p, want_rgb=False, want_unc=False))
    for pl in (few_entries, few_records, exact):
        pl.close()


def test_plan_rejects_bad_arguments(ctx, gv):
    c, gs, vf = setup(gv, ctx, k=1)
    cand = c["cand"]
    W, H = cand[0].W, cand[0].H
    with pytest.raises(ValueError):
        ctx.plan(gs, vf, len(cand), W, H, 1 << 16, params=gv.Params(tile=0, vf_degree=c["vf_degree"]))
    with pytest.raises(gv.GavisError):
        ctx.plan(gs, vf, len(cand), W, H, 0, params=gv.Params(tile=16, vf_degree=c["vf_degree"]))
    plan = ctx.plan(gs, vf, len(cand), W, H, 1 << 16, params=gv.Params(tile=16, vf_degree=c["vf_degree"]))
    with pytest.raises(ValueError):
        plan.launch(cand[:-1])
    other = sg.config(1, cand_wh=(W + 8, H))["cand"][:len(cand)]
    with pytest.raises(gv.GavisError):
        plan.launch(other)
    plan.close()


def test_plan_in_view_batches(ctx, gv):
    """views_per_batch: the views go through the captured chain in batches
    over the same buffers (here 4 + 4 + 2); results equal gavis_score_views',
    and the capacities apply per batch."""
    c, gs, vf = setup(gv, ctx, n=20000, n_train=4, n_cand=10, train_wh=(160, 120), cand_wh=(160, 120))
    cand = c["cand"]
    p = gv.Params(tile=16, vf_degree=c["vf_degree"], views_per_batch=4)
    rec, keys = needed(gv, ctx, gs, vf, cand, gv.Params(tile=16, vf_degree=c["vf_degree"]))
    plan = ctx.plan(gs, vf, len(cand), 160, 120, keys, record_capacity=rec, params=p, want_rgb=True, want_unc=True)
    plan.launch(cand)
    over, rec_b, keys_b = plan.overflowed()
    assert not over and 0 < rec_b < rec and 0 < keys_b < keys   # the largest batch needs less than all views
    assert_same(plan, ctx.score_views(gs, vf, cand, params=gv.Params(tile=16, vf_degree=c["vf_degree"])))
    tight = ctx.plan(gs, vf, len(cand), 160, 120, keys_b, record_capacity=rec_b, params=p)
    tight.launch(cand)
    assert tight.overflowed() == (False, rec_b, keys_b)
    assert torch.equal(tight.score, plan.score)
    plan.close()
    tight.close()


def test_plan_with_colour_variances(ctx, gv):
    """The captured chain also carries the per-Gaussian colour covariance
    (FisherRF variant): replays equal gavis_score_views with sh_var."""
    c = sg.config(2, n=20000, n_train=4, n_cand=5, train_wh=(160, 120), cand_wh=(160, 120))
    sc = c["scene"]
    var = np.random.default_rng(5).uniform(0.001, 0.05, sc.sh.shape).astype(np.float32)
    gs = gv.Gaussians(*(torch.as_tensor(x).cuda().contiguous() for x in (sc.means, sc.scales, sc.rots, sc.opac, sc.sh)),
                      sc.sh_degree, torch.as_tensor(var).cuda().contiguous())
    vf = ctx.vf_build(gs, c["train"], degree=c["vf_degree"])
    cand = c["cand"]
    p = gv.Params(tile=16, vf_degree=c["vf_degree"])
    plan = ctx.plan(gs, vf, len(cand), 160, 120, 1 << 22, params=p, want_unc=True)
    plan.launch(cand)
    assert_same(plan, ctx.score_views(gs, vf, cand, params=p, want_rgb=False))
    plan.close()
