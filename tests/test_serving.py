"""Continuous-batching server: every request's scores (and uncertainty maps)
are the same alone and in a mix of concurrent requests on several scenes and
resolutions, batches do mix requests, admission respects the HBM budget, and
errors come back as status codes."""
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
def scenes(gv):
    ctx = gv.Context(0)
    out = []
    for k, kw in ((1, dict(n=2000, n_train=4)), (2, dict(n=20000, n_train=4, train_wh=(160, 120)))):
        c = sg.config(k, **kw)
        gs = gv.Gaussians.from_numpy(c["scene"])
        vf = ctx.vf_build(gs, c["train"], degree=c["vf_degree"])
        out.append((c, gs, vf))
    torch.cuda.synchronize()
    yield ctx, out
    ctx.close()


def cams_for(c, n, wh, seed):
    if c["name"].startswith("tiny"):
        return sg.fibonacci_cameras(n, 3.0 + 0.1 * seed, wh[0], wh[1])
    return sg.se2_cameras(n, c["scene"], wh[0], wh[1], seed=seed)


def test_alone_equals_mix(gv, scenes):
    ctx, sc = scenes
    (c0, gs0, vf0), (c1, gs1, vf1) = sc
    reqs = [  # (scene, cams, params)
        (0, cams_for(c0, 12, (128, 128), 1), gv.Params(vf_degree=2)),
        (1, cams_for(c1, 5, (200, 136), 2), gv.Params(vf_degree=3)),
        (0, cams_for(c0, 9, (128, 128), 3), gv.Params(vf_degree=2)),
        (0, cams_for(c0, 6, (96, 64), 4), gv.Params(vf_degree=2)),
        (1, cams_for(c1, 7, (200, 136), 5), gv.Params(vf_degree=3)),
        (0, cams_for(c0, 20, (128, 128), 6), gv.Params(vf_degree=2)),
    ]
    # alone: direct library call per request
    alone = []
    for sid, cams, p in reqs:
        gs, vf = (gs0, vf0) if sid == 0 else (gs1, vf1)
        alone.append(ctx.score_views(gs, vf, cams, params=p))
    srv = gv.Server(0, n_workers=2, max_views_per_batch=32)
    ids = [srv.add_scene(gs0, vf0), srv.add_scene(gs1, vf1)]
    rids = [srv.submit(ids[sid], cams, params=p, want_unc=True) for sid, cams, p in reqs]   # all at once: a mix
    res = [srv.wait(r) for r in rids]
    for a, r in zip(alone, res):
        assert torch.equal(a["score"], r["score"])
        assert torch.equal(a["unc"], r["unc"])
        assert a["best"] == r["best"]
        assert r["latency_ms"] > 0
    st = srv.stats()
    assert st["views_scored"] == sum(len(c) for _, c, _ in reqs)
    assert st["max_requests_in_batch"] >= 2          # batches did mix requests
    # the same request again, now alone in the server
    rid = srv.submit(ids[0], reqs[0][1], params=reqs[0][2])
    again = srv.wait(rid)
    assert torch.equal(again["score"], alone[0]["score"])
    srv.close()


def test_server_matches_oracle(gv):
    """Through the server against the oracle directly: two requests at two
    resolutions on one scene whose field is the oracle's VF CONST, submitted
    together so that they share batches; each request's entropy maps and
    scores agree with the oracle's VF QUERY + UA raster + entropy score."""
    c = sg.config(1, n=900, n_train=3, n_cand=4, train_wh=(100, 75), cand_wh=(100, 75))
    sc, L = c["scene"], c["vf_degree"]
    g, _, _ = oracle.vf_build(c["train"], sc, L)
    g32 = g.astype(np.float32)
    gs = gv.Gaussians.from_numpy(sc)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), L, len(c["train"]), 1.0)
    reqs = [c["cand"], sg.fibonacci_cameras(3, 3.1, 64, 48)]
    srv = gv.Server(0, n_workers=1, max_views_per_batch=16)
    sid = srv.add_scene(gs, vf)
    rids = [srv.submit(sid, cams, params=gv.Params(vf_degree=L), want_unc=True) for cams in reqs]
    res = [srv.wait(r) for r in rids]
    srv.close()
    for cams, r in zip(reqs, res):
        ref = oracle.score_views(sc, g32.astype(np.float64), L, len(c["train"]), cams)
        err, n_band = compare_views(r["unc"].cpu().numpy(), None, ref)
        assert err <= TOL, (err, n_band)
        assert score_excess(r["score"].cpu().numpy(), ref).max() <= TOL
        if sorted_gap(ref["score"]) > GAP:
            assert r["best"] == ref["best"]


def test_admission_respects_budget(gv, scenes):
    ctx, sc = scenes
    c0, gs0, vf0 = sc[0]
    # the server's per-request workspace estimate (6 views, all in one batch
    # of at most 8); a budget between one and two requests' worth admits them
    # one at a time (and still holds one worker's workspace)
    one = 6 * (2000 * (32 + 32 + 16) + 2000 * 2 * 24 + 2000 // 4 * 4 * 16 + 128 * 128 * 4 + 64)
    srv = gv.Server(0, budget_bytes=int(1.5 * one), n_workers=1, max_views_per_batch=8)
    sid = srv.add_scene(gs0, vf0)
    rids = [srv.submit(sid, cams_for(c0, 6, (128, 128), s), params=gv.Params(vf_degree=2)) for s in range(5)]
    res = [srv.wait(r) for r in rids]
    st = srv.stats()
    assert st["views_scored"] == 30
    assert st["peak_reserved_bytes"] <= st["budget_bytes"]
    assert st["max_requests_in_batch"] == 1          # never two admitted at once
    for r in res:
        assert 0 <= r["best"] < 6
    srv.close()


def test_errors_are_status_codes(gv, scenes):
    ctx, sc = scenes
    c0, gs0, vf0 = sc[0]
    srv = gv.Server(0, n_workers=1)
    sid = srv.add_scene(gs0, vf0)
    with pytest.raises(gv.GavisError) as e:
        srv.submit(sid + 5, cams_for(c0, 2, (64, 64), 0))
    assert e.value.code == gv.ERR_ARG
    with pytest.raises(gv.GavisError) as e:
        srv.wait(12345, timeout_ms=0)
    assert e.value.code == gv.ERR_ARG
    # a request held behind paused workers cannot finish: a zero timeout
    # returns GAVIS_ERR_TIMEOUT, and after resuming the request completes
    srv.pause(True)
    rid = srv.submit(sid, cams_for(c0, 8, (128, 128), 1), params=gv.Params(vf_degree=2))
    with pytest.raises(gv.GavisError) as e:
        srv.wait(rid, timeout_ms=0)
    assert e.value.code == gv.ERR_TIMEOUT
    with pytest.raises(gv.GavisError) as e:
        srv.wait(rid, timeout_ms=50)
    assert e.value.code == gv.ERR_TIMEOUT
    assert srv.stats()["views_scored"] == 0
    srv.pause(False)
    r = srv.wait(rid)
    assert 0 <= r["best"] < 8 and srv.stats()["views_scored"] == 8
    srv.close()
