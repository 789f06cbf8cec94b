"""Parity of the CUDA library with the CPU oracle (element by element).

Tile bins and sort keys must match bit for bit; per-pixel uncertainty, colour,
visibility-field coefficients (as gamma/|P|), queried visibilities and view
scores within 1e-4 absolute; the selected view must match whenever the
oracle's top-2 gap exceeds 2e-4.  Where a transmittance test lands within
0.1% of eps_T in the float64 oracle, float32 rounding may stop the run one or
more entries earlier or later: there the oracle gives the range of values
every such stop produces, and the GPU value must lie in that range (within
the same 1e-4).  No pixel and no Gaussian is left out.
"""
import numpy as np
import pytest
import torch

import oracle
import scenegen as sg
from _util import GAP, TOL, compare_views, excess, score_excess, sorted_gap, visibility_check

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


def gpu_scene(gv, sc, sh_dtype=torch.float32):
    return gv.Gaussians.from_numpy(sc, sh_dtype=sh_dtype)


CASES = {
    "tiny": dict(k=1),                                                           # 2k Gaussians, 128x128
    "tiny_ragged": dict(k=1, n=900, n_train=3, n_cand=5, train_wh=(100, 75), cand_wh=(100, 75)),
    "room_small": dict(k=2, n=20000, n_train=4, n_cand=4, train_wh=(160, 120), cand_wh=(200, 136)),
}


def case(name):
    kw = dict(CASES[name])
    return sg.config(kw.pop("k"), **kw)


# --------------------------------------------------------------------------- bins / keys

@pytest.mark.parametrize("lists", [1, 2])   # tile lists by counting / by sorting
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tile", [16, 8])
def test_bins_bit_exact(ctx, gv, name, tile, lists):
    c = case(name)
    sc, cams = c["scene"], c["cand"]
    gs = gpu_scene(gv, sc)
    keys, vals, ranges = ctx.debug_bins(gs, cams, gv.Params(tile=tile, tile_lists=lists))
    rk, rv = oracle.bins(cams, sc, tile=tile)
    gk = keys.cpu().numpy().view(np.uint64)
    gvals = vals.cpu().numpy().view(np.uint32)
    assert len(gk) == len(rk) > 0
    assert np.array_equal(gk, rk)
    assert np.array_equal(gvals, rv)
    TT = ((cams[0].W + tile - 1) // tile) * ((cams[0].H + tile - 1) // tile)
    rr = oracle.ranges(rk, len(cams) * TT)
    assert np.array_equal(ranges.cpu().numpy().view(np.uint32), rr)


def test_bins_bit_exact_with_view_groups(ctx, gv):
    """600 views in one call: view bits + depth bits exceed 32 and view bits
    + tile bits exceed 16, so the depth sort runs per group of views (3
    groups) and the tile lists are counted over all 600 views at once; keys,
    values and ranges stay bit-exact, and scoring equals the
    one-view-per-batch path."""
    sc = sg.tiny_scene(2000, seed=3, sh_degree=1)
    cams = sg.fibonacci_cameras(600, 3.0, 128, 96, 60.0)
    TT = 16 * 12
    zbits = []
    for cam in cams:
        out, st = oracle.project(cam, sc, tile=8)
        zbits.append(out[st == 1, 0].astype(np.float32).view(np.uint32))
    zb = np.concatenate(zbits)
    vbits = (len(cams) - 1).bit_length()
    assert vbits + int(zb.max() - zb.min()).bit_length() > 32
    assert vbits + (TT - 1).bit_length() > 16
    gs = gpu_scene(gv, sc)
    rk, rv = oracle.bins(cams, sc, tile=8)
    for lists in (1, 2):
        keys, vals, ranges = ctx.debug_bins(gs, cams, gv.Params(tile=8, tile_lists=lists))
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), rk)
        assert np.array_equal(vals.cpu().numpy().view(np.uint32), rv)
        assert np.array_equal(ranges.cpu().numpy().view(np.uint32), oracle.ranges(rk, len(cams) * TT))
    vf = gv.VisibilityField(torch.zeros((sc.n, 9), device="cuda"), 2, 0, 1.0)
    a = ctx.score_views(gs, vf, cams, params=gv.Params(tile=8, views_per_batch=0))
    b = ctx.score_views(gs, vf, cams, params=gv.Params(tile=8, views_per_batch=1))
    for k in ("unc", "rgb", "score"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("lists", [0, 1, 2])
@pytest.mark.parametrize("W,H,tile,nv", [(640, 480, 16, 3),     # 1200 tiles a view
                                          (512, 256, 8, 3),      # 2048
                                          (328, 400, 8, 2),      # 2050
                                          (1280, 720, 16, 2)])   # 3600
def test_bins_bit_exact_tile_counts(ctx, gv, W, H, tile, nv, lists):
    """The tile lists are built by counting when a view's tile counters fit
    in shared memory (and asked for, or the batch is large) and by the
    segmented 16-bit sort otherwise (more than 2048 tiles a view, or
    tile_lists = 2); every choice gives the oracle's keys, values and ranges
    bit for bit, on either side of the tile-count switch."""
    sc = sg.tiny_scene(4000, seed=11, sh_degree=1)
    cams = sg.fibonacci_cameras(nv, 2.6, W, H, 70.0)
    gs = gpu_scene(gv, sc)
    keys, vals, ranges = ctx.debug_bins(gs, cams, gv.Params(tile=tile, tile_lists=lists))
    rk, rv = oracle.bins(cams, sc, tile=tile)
    TT = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    assert len(rk) > 0
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), rv)
    assert np.array_equal(ranges.cpu().numpy().view(np.uint32), oracle.ranges(rk, nv * TT))


@pytest.mark.parametrize("W,H,tile,fov", [(16, 2048, 8, 3.0),     # 2 x 256 tiles
                                          (4096, 16, 8, 90.0),    # 512 x 2
                                          (2000, 8, 16, 80.0),    # 125 x 1
                                          (24, 24, 16, 60.0)])    # 2 x 2, ragged
def test_bins_bit_exact_extreme_aspect(ctx, gv, W, H, tile, fov):
    """Tile grids one or two tiles wide or high: the counted lists' corner
    differences sit one tile column or row apart (or at the grid's far edge),
    and the lists still equal the oracle's; so do the sorted ones."""
    sc = sg.tiny_scene(4000, seed=11, sh_degree=1)
    cams = [sg.look_at_camera((0.1, 0.2, -3.0), (0, 0, 0), W, H, fov),
            sg.look_at_camera((2.5, 0.3, 1.0), (0, 0, 0), W, H, fov)]
    gs = gpu_scene(gv, sc)
    rk, rv = oracle.bins(cams, sc, tile=tile)
    TT = ((W + tile - 1) // tile) * ((H + tile - 1) // tile)
    assert len(rk) > 0
    for lists in (1, 2):
        keys, vals, ranges = ctx.debug_bins(gs, cams, gv.Params(tile=tile, tile_lists=lists))
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), rk), lists
        assert np.array_equal(vals.cpu().numpy().view(np.uint32), rv), lists
        assert np.array_equal(ranges.cpu().numpy().view(np.uint32), oracle.ranges(rk, len(cams) * TT)), lists


def _edge_scene(cams, n_per, seed):
    """Gaussians whose centres project near the image borders of each camera:
    up to 8 px inside to 40 px outside, at depths 0.25-8 and scales 1e-3-0.5,
    so that many footprints reach into the image by a little and many miss
    it by a little."""
    rng = np.random.default_rng(seed)
    means = []
    for cam in cams:
        side = rng.integers(0, 4, n_per)
        d = rng.uniform(-8.0, 40.0, n_per)
        along = rng.uniform(-20.0, max(cam.W, cam.H) + 20.0, n_per)
        u = np.select([side == 0, side == 1], [-d, cam.W + d], along)
        v = np.select([side == 2, side == 3], [-d, cam.H + d], along)
        z = np.exp(rng.uniform(np.log(0.25), np.log(8.0), n_per))
        xc = np.stack([(u - cam.cx) / cam.fx * z, (v - cam.cy) / cam.fy * z, z], 1)
        R = cam.R.astype(np.float64)
        means.append(np.linalg.solve(R, (xc - cam.t.astype(np.float64)).T).T)
    means = np.concatenate(means)
    n = len(means)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return sg.Scene(means=means.astype(np.float32),
                    scales=np.exp(rng.uniform(np.log(1e-3), np.log(0.5), (n, 3))).astype(np.float32),
                    rots=q.astype(np.float32), opac=rng.uniform(0.1, 1.0, n).astype(np.float32),
                    sh=rng.normal(0, 0.3, (n, 1, 3)).astype(np.float32), sh_degree=0)


@pytest.mark.parametrize("lists", [1, 2])
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_bins_bit_exact_screen_edges(ctx, gv, tile, lists):
    """Footprints that just reach into, or just miss, the tile grid at every
    border, for cameras with orthonormal, uniformly scaled and sheared
    rotation matrices and wide and narrow fields of view: the bins stay
    bit-exact (no Gaussian the exact projection keeps may be dropped early)."""
    base = [sg.look_at_camera((0, 0, 0), (1.0, 0.2, 0.1), 160, 120, 90.0),
            sg.look_at_camera((0.5, -1, 0.3), (0.0, 1.0, 0.0), 160, 120, 120.0),
            sg.look_at_camera((0, 0, 1), (0.3, 0.1, -1.0), 160, 120, 30.0)]
    cams = list(base)
    for k, M in enumerate([np.eye(3) * 1.25, np.array([[1.0, 0.15, 0.0], [0.0, 1.0, 0.0], [0.1, 0.0, 1.0]])]):
        c = sg.look_at_camera((0.2 * k, 0.1, 0.0), (-1.0, 0.4, 0.2), 160, 120, 75.0)
        R = (M @ c.R.astype(np.float64)).astype(np.float32)
        cams.append(sg.Camera(W=c.W, H=c.H, fx=c.fx, fy=c.fy, cx=c.cx, cy=c.cy, tan_half_fovx=c.tan_half_fovx,
                              tan_half_fovy=c.tan_half_fovy, R=R,
                              t=(-R.astype(np.float64) @ c.campos.astype(np.float64)).astype(np.float32),
                              campos=c.campos, znear=c.znear))
    sc = _edge_scene(cams, 3000, seed=11)
    reach = miss = 0
    for cam in cams:
        out, st = oracle.project(cam, sc, tile=tile)
        P = sc.means.astype(np.float64) @ cam.R.T.astype(np.float64) + cam.t
        u = cam.fx * P[:, 0] / P[:, 2] + cam.cx
        v = cam.fy * P[:, 1] / P[:, 2] + cam.cy
        outside = (P[:, 2] > cam.znear) & ((u < 0) | (u > cam.W) | (v < 0) | (v > cam.H))
        reach += int(np.sum(outside & (st == 1)))
        miss += int(np.sum(outside & (st != 1)))
    assert reach > 500 and miss > 500, (reach, miss)
    gs = gpu_scene(gv, sc)
    keys, vals, ranges = ctx.debug_bins(gs, cams, gv.Params(tile=tile, tile_lists=lists))
    rk, rv = oracle.bins(cams, sc, tile=tile)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), rv)
    TT = ((160 + tile - 1) // tile) * ((120 + tile - 1) // tile)
    assert np.array_equal(ranges.cpu().numpy().view(np.uint32), oracle.ranges(rk, len(cams) * TT))


# --------------------------------------------------------------------------- VF query

@pytest.mark.parametrize("L,P,dtype", [(2, 8, torch.float32), (3, 100, torch.float32), (3, 200, torch.float16),
                                       (1, 1, torch.float32), (0, 0, torch.float32), (4, 50, torch.float32),
                                       (5, 30, torch.float32), (5, 200, torch.float16)])
def test_vf_query_parity(ctx, gv, L, P, dtype):
    c = case("tiny")
    sc = c["scene"]
    rng = np.random.default_rng(L * 7 + P)
    K = (L + 1) ** 2
    gamma = rng.normal(0, 1, (sc.n, K)) * (P / 3.0 + 0.1)
    gamma[:, 0] = np.abs(gamma[:, 0]) * 3.0
    gamma[:50] = 0.0
    g_dev = torch.as_tensor(gamma).to("cuda", dtype)
    vf = gv.VisibilityField(g_dev.contiguous(), L, P, 1.0)
    gs = gpu_scene(gv, sc)
    V = ctx.vf_query(gs, vf, c["cand"][:4]).cpu().numpy()
    gq = g_dev.double().cpu().numpy()
    for v, cam in enumerate(c["cand"][:4]):
        Vr, _ = oracle.vf_query(gq, L, P, cam, sc.means)
        assert np.abs(V[v] - Vr).max() <= TOL
        assert np.all(V[v][:50] == 0.0)


def test_vf_query_more_views_than_one_launch(ctx, gv):
    """2,100 views: the query runs in launches of at most 1,024 cameras; the
    views of every launch (first, last, and either side of each boundary)
    match the oracle, and debug bins refuse more cameras than one launch."""
    sc = sg.tiny_scene(300, seed=5, sh_degree=0)
    cams = sg.fibonacci_cameras(2100, 3.0, 32, 32, 60.0)
    rng = np.random.default_rng(9)
    gamma = np.abs(rng.normal(0, 1, (sc.n, 4))) * 2.0
    g_dev = torch.as_tensor(gamma, dtype=torch.float32, device="cuda")
    vf = gv.VisibilityField(g_dev.contiguous(), 1, 5, 1.0)
    gs = gpu_scene(gv, sc)
    V = ctx.vf_query(gs, vf, cams).cpu().numpy()
    assert V.shape == (2100, sc.n)
    for v in (0, 1, 1023, 1024, 1025, 2047, 2048, 2099):
        Vr, _ = oracle.vf_query(gamma, 1, 5, cams[v], sc.means)
        assert np.abs(V[v] - Vr).max() <= TOL, v
    with pytest.raises(gv.GavisError, match="at most 1024 cameras"):
        ctx.debug_bins(gs, cams[:1025], gv.Params(tile=16))


def test_calls_on_two_streams_are_ordered(ctx, gv):
    """Two scoring calls on one context, issued on different streams back to
    back with no host synchronisation between them: they share the
    context's workspace, so the context orders the second after the first,
    and each equals the same call made alone."""
    c = sg.config(2, n=200000, n_train=4, n_cand=8, train_wh=(320, 240), cand_wh=(800, 600))
    gs = gpu_scene(gv, c["scene"])
    p = gv.Params(vf_degree=2)
    vf = ctx.vf_build(gs, c["train"], degree=2, params=p)
    cam_a, cam_b = c["cand"][:4], c["cand"][4:]
    ref_a = ctx.score_views(gs, vf, cam_a, params=p)
    ref_b = ctx.score_views(gs, vf, cam_b, params=p)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        a = ctx.score_views(gs, vf, cam_a, params=p, sync_best=False)
    with torch.cuda.stream(s2):
        b = ctx.score_views(gs, vf, cam_b, params=p, sync_best=False)
    torch.cuda.synchronize()
    for k in ("unc", "rgb", "score"):
        assert torch.equal(a[k], ref_a[k]), k
        assert torch.equal(b[k], ref_b[k]), k


# --------------------------------------------------------------------------- VF CONST

@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_single_view_visibility_parity(ctx, gv, name, tile):
    c = case(name)
    sc, cams = c["scene"], c["train"][:3]
    gs = gpu_scene(gv, sc)
    sumT, cnt = ctx.debug_visibility(gs, cams, gv.Params(tile=tile))
    sumT, cnt = sumT.cpu().numpy(), cnt.cpu().numpy()
    for v, cam in enumerate(cams):
        rs, rc, amb, _, b = oracle.visibility_view(cam, sc, want_bounds=True)
        bad, err, moved = visibility_check(sumT[v], cnt[v], b)
        n_band = int((b["cnt_late"] > b["cnt_early"]).sum())
        msg = f"view {v}: {n_band} Gaussians reachable by a band stop, GPU count off the early one for {moved}"
        assert bad == 0, msg                 # pixel counts are integers: inside [early, late] exactly
        assert err <= TOL, (err, msg)
        assert (cnt[v] > 0).sum() > 10


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("dtype", [torch.float32, torch.float16, torch.bfloat16])
def test_vf_build_parity(ctx, gv, name, dtype):
    c = case(name)
    sc, train = c["scene"], c["train"]
    gs = gpu_scene(gv, sc)
    L = c["vf_degree"]
    vf = ctx.vf_build(gs, train, degree=L, dtype=dtype)
    assert vf.n_train_views == len(train)
    g = vf.coeffs.double().cpu().numpy()
    ref, _, _, rad = oracle.vf_build(train, sc, L, want_rad=True)
    P = len(train)
    # half-precision storage rounds gamma to 2^-11 (f16) or 2^-8 (bf16) relative: state it and gate on it
    rel = {torch.float32: 0.0, torch.float16: 2.0 ** -11, torch.bfloat16: 2.0 ** -8}[dtype]
    # every coefficient of every Gaussian: within 1e-4 |P| of the oracle, plus
    # the radius that rounding-sensitive stops allow (0 for most Gaussians),
    # plus the storage rounding
    err = (np.abs(g - ref) - rad - rel * (np.abs(ref) + rad)) / P
    n_rad = int((rad.max(1) > 0).sum())
    assert err.max() <= TOL, (err.max(), f"{n_rad} of {sc.n} Gaussians have a nonzero radius")


@pytest.mark.parametrize("name", ["tiny", "room_small"])
@pytest.mark.parametrize("tile", [8, 32])
def test_vf_build_parity_other_tiles(ctx, gv, name, tile):
    """The field build at the tile edges other than the default (the
    visibility pass runs 1 or 16 warps per tile there)."""
    c = case(name)
    sc, train = c["scene"], c["train"]
    gs = gpu_scene(gv, sc)
    L = c["vf_degree"]
    vf = ctx.vf_build(gs, train, degree=L, dtype=torch.float32, params=gv.Params(tile=tile, vf_degree=L))
    g = vf.coeffs.double().cpu().numpy()
    ref, _, _, rad = oracle.vf_build(train, sc, L, want_rad=True)
    err = (np.abs(g - ref) - rad) / len(train)
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("L", [4, 5])
@pytest.mark.parametrize("kappa", [0.0, 0.3, 3.0, 10.0])
def test_vf_build_high_degree(ctx, gv, L, kappa):
    """Field degrees 4 and 5 over the concentrations of the paper's ablation
    (Tab. ablation: L in 1..5, kappa in 0, 0.1, 0.3, 3, 10): every
    coefficient within 1e-4 |P| of the oracle beyond its radius; then the
    queried V and the scores of candidate views from the oracle's field."""
    c = case("tiny")
    sc, train = c["scene"], c["train"]
    gs = gpu_scene(gv, sc)
    p = gv.Params(vf_degree=L, kappa=kappa)
    vf = ctx.vf_build(gs, train, degree=L, params=p)
    P = len(train)
    prm = oracle.params(kappa=kappa)
    ref, _, _, rad = oracle.vf_build(train, sc, L, prm, want_rad=True)
    err = ((np.abs(vf.coeffs.double().cpu().numpy() - ref) - rad) / P).max()
    assert err <= TOL, err
    g32 = ref.astype(np.float32)
    vfo = gv.VisibilityField(torch.as_tensor(g32).cuda(), L, P, kappa)
    cand = c["cand"][:4]
    V = ctx.vf_query(gs, vfo, cand, params=p).cpu().numpy()
    for v, cam in enumerate(cand):
        Vr, _ = oracle.vf_query(g32.astype(np.float64), L, P, cam, sc.means)
        assert np.abs(V[v] - Vr).max() <= TOL
    out = ctx.score_views(gs, vfo, cand, params=p)
    r = oracle.score_views(sc, g32.astype(np.float64), L, P, cand, prm)
    e, _ = compare_views(out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), r)
    assert e <= TOL
    assert score_excess(out["score"].cpu().numpy(), r).max() <= TOL


def test_vf_build_batched_equals_plain(ctx, gv):
    c = case("room_small")
    gs = gpu_scene(gv, c["scene"])
    a = ctx.vf_build(gs, c["train"], degree=3, params=gv.Params(views_per_batch=1, vf_degree=3)).coeffs
    b = ctx.vf_build(gs, c["train"], degree=3, params=gv.Params(views_per_batch=0, vf_degree=3)).coeffs
    assert torch.equal(a, b)   # integer visibility sums: batching changes nothing


def test_vf_accumulate_is_additive(ctx, gv):
    """eq:vis_gamma is a sum over views: building on P1 then adding P2 equals
    building on P1 u P2."""
    c = case("tiny")
    gs = gpu_scene(gv, c["scene"])
    full = ctx.vf_build(gs, c["train"], degree=2)
    part = ctx.vf_build(gs, c["train"][:5], degree=2)
    part = ctx.vf_build(gs, c["train"][5:], degree=2, out=part, accumulate=True)
    assert part.n_train_views == full.n_train_views == len(c["train"])
    assert torch.allclose(part.coeffs, full.coeffs, atol=1e-5)


# --------------------------------------------------------------------------- scoring

def oracle_gamma(c):
    g, _, _ = oracle.vf_build(c["train"], c["scene"], c["vf_degree"])
    return g.astype(np.float32)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_score_views_parity(ctx, gv, name, tile):
    c = case(name)
    sc, cand = c["scene"], c["cand"]
    L = c["vf_degree"]
    g32 = oracle_gamma(c)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), L, len(c["train"]), 1.0)
    gs = gpu_scene(gv, sc)
    out = ctx.score_views(gs, vf, cand, params=gv.Params(tile=tile, vf_degree=L))
    unc, rgb, score = out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), out["score"].cpu().numpy()
    ref = oracle.score_views(sc, g32.astype(np.float64), L, len(c["train"]), cand)
    err, n_band = compare_views(unc, rgb, ref)
    npix = len(cand) * cand[0].W * cand[0].H
    assert err <= TOL, (err, f"{n_band} of {npix} pixels have a stop inside the band")
    assert score_excess(score, ref).max() <= TOL
    if sorted_gap(ref["score"]) > GAP:
        assert out["best"] == ref["best"]


@pytest.mark.parametrize("name", ["tiny", "room_small"])
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_expected_depth_parity(ctx, gv, name, tile):
    """Expected depth (colour weights x camera depth, background 0) against the
    oracle; it grows with the depths (up to ~10 here), so the gate is 1e-4
    relative to max(1, |d|).  Asking for it leaves every other output bit for
    bit unchanged."""
    c = case(name)
    sc, cand = c["scene"], c["cand"]
    L = c["vf_degree"]
    g32 = oracle_gamma(c)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), L, len(c["train"]), 1.0)
    gs = gpu_scene(gv, sc)
    p = gv.Params(tile=tile, vf_degree=L)
    a = ctx.score_views(gs, vf, cand, params=p, want_depth=True)
    b = ctx.score_views(gs, vf, cand, params=p)
    for k in ("unc", "rgb", "score"):
        assert torch.equal(a[k], b[k]), k
    ref = oracle.score_views(sc, g32.astype(np.float64), L, len(c["train"]), cand, want_depth=True)
    d = a["depth"].cpu().numpy()
    for v in range(len(cand)):
        b = ref["bnd"][v]
        err = excess(d[v], b["depth_lo"], b["depth_hi"]) / np.maximum(1.0, np.abs(ref["depth"][v]))
        assert err.max() <= TOL, (v, err.max())
    assert np.abs(d).max() > 1.0   # the case exercises depths well above 1


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tile", [16, 8, 32])
def test_tile_list_builders_give_the_same_bits(ctx, gv, name, tile):
    """The field and the scores from tile lists built by counting and by
    sorting are the same bits (the lists are: test_bins_bit_exact pins both
    to the oracle)."""
    c = case(name)
    gs = gpu_scene(gv, c["scene"])
    L = c["vf_degree"]
    out = {}
    for lists in (1, 2):
        p = gv.Params(tile=tile, vf_degree=L, tile_lists=lists)
        vf = ctx.vf_build(gs, c["train"], degree=L, params=p)
        out[lists] = (vf.coeffs, ctx.score_views(gs, vf, c["cand"], params=p))
    assert torch.equal(out[1][0], out[2][0])
    for k in ("score", "unc", "rgb"):
        assert torch.equal(out[1][1][k], out[2][1][k]), k


def test_prof_counts_sorted_tile_entries(ctx, gv):
    """gavis_prof_read reports the tile entries whose lists were sorted: all
    of them with tile_lists = 2, none with tile_lists = 1 (views of at most
    2048 tiles), and the same total of entries and records either way."""
    c = case("room_small")
    gs = gpu_scene(gv, c["scene"])
    L = c["vf_degree"]
    vf = ctx.vf_build(gs, c["train"], degree=L)
    got = {}
    for lists in (1, 2):
        ctx.prof_enable(True)
        ctx.score_views(gs, vf, c["cand"], params=gv.Params(vf_degree=L, tile_lists=lists))
        got[lists] = ctx.prof_read()
        ctx.prof_enable(False)
    assert got[1]["keys"] == got[2]["keys"] > 0 and got[1]["visible"] == got[2]["visible"] > 0
    assert got[1]["sorted_keys"] == 0 and got[2]["sorted_keys"] == got[2]["keys"]


def test_score_batched_equals_plain(ctx, gv):
    c = case("room_small")
    g32 = oracle_gamma(c)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), 3, len(c["train"]), 1.0)
    gs = gpu_scene(gv, c["scene"])
    a = ctx.score_views(gs, vf, c["cand"], params=gv.Params(views_per_batch=1, vf_degree=3))
    b = ctx.score_views(gs, vf, c["cand"], params=gv.Params(views_per_batch=0, vf_degree=3))
    for k in ("unc", "rgb", "score"):
        assert torch.equal(a[k], b[k]), k
    assert a["best"] == b["best"]


def test_end_to_end_tiny(ctx, gv):
    """VF CONST on the GPU feeding scoring on the GPU, against the oracle run
    end to end on the same inputs: the field within its radius, every pixel
    and every view score within 1e-4 of the oracle's range.  (The ranges of
    the scoring pass cover its own rounding-sensitive stops; that the GPU's
    field build takes the oracle's stops on this case is part of what the
    test checks: a different stop moves a Gaussian's field by up to its
    radius, and the scores with it.)"""
    c = case("tiny")
    sc = c["scene"]
    gs = gpu_scene(gv, sc)
    vf = ctx.vf_build(gs, c["train"], degree=2)
    out = ctx.score_views(gs, vf, c["cand"])
    g, _, _, rad = oracle.vf_build(c["train"], sc, 2, want_rad=True)
    P = len(c["train"])
    gg = vf.coeffs.double().cpu().numpy()
    assert ((np.abs(gg - g) - rad) / P).max() <= TOL
    ref = oracle.score_views(sc, g, 2, P, c["cand"])
    err, n_band = compare_views(out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), ref)
    moved = int((np.abs(gg - g) / P > TOL).any(1).sum())
    assert err <= TOL, (err, f"{moved} Gaussians' fields moved by a band stop; {n_band} pixels in the band")
    assert score_excess(out["score"].cpu().numpy(), ref).max() <= TOL
    if sorted_gap(ref["score"]) > GAP:
        assert out["best"] == ref["best"]


# --------------------------------------------------------------------------- edge cases

def test_empty_scene(ctx, gv):
    c = case("tiny")
    sc = c["scene"].subset(np.arange(0))
    gs = gpu_scene(gv, sc)
    vf = ctx.vf_build(gs, c["train"], degree=2)
    out = ctx.score_views(gs, vf, c["cand"][:3], want_depth=True)
    assert torch.all(out["unc"] == 0) and torch.all(out["rgb"] == 0) and torch.all(out["score"] == 0)
    assert torch.all(out["depth"] == 0)
    assert out["best"] == 0


def test_no_candidates_and_no_training_views(ctx, gv):
    c = case("tiny")
    gs = gpu_scene(gv, c["scene"])
    vf = ctx.vf_build(gs, [], degree=2)
    assert vf.n_train_views == 0 and torch.all(vf.coeffs == 0)
    out = ctx.score_views(gs, vf, [])
    assert out["best"] == -1
    # |P| = 0: V = 0 everywhere, every Gaussian carries the prior (P8)
    out = ctx.score_views(gs, vf, c["cand"][:2])
    ref = oracle.score_views(c["scene"], np.zeros((c["scene"].n, 9)), 2, 0, c["cand"][:2])
    err, _ = compare_views(out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), ref)
    assert err <= TOL


def test_all_culled_view(ctx, gv):
    c = case("tiny")
    gs = gpu_scene(gv, c["scene"])
    away = sg.look_at_camera((0, 0, 3.0), (0, 0, 6.0), 64, 64)   # looks away from the cloud
    vf = ctx.vf_build(gs, [away], degree=2)
    assert torch.all(vf.coeffs == 0)
    out = ctx.score_views(gs, vf, [away])
    assert torch.all(out["unc"] == 0) and out["score"].item() == 0.0


def test_fp16_colour_and_field(ctx, gv):
    """Half-precision storage of colour and visibility coefficients, float32
    compositing: parity with the oracle run on the same rounded inputs, and the
    storage error against the float32 inputs stated."""
    c = case("room_small")
    sc = c["scene"]
    g32 = oracle_gamma(c)
    g16 = torch.as_tensor(g32).half()
    sh16 = torch.as_tensor(sc.sh).half()
    vf = gv.VisibilityField(g16.cuda(), 3, len(c["train"]), 1.0)
    gs = gpu_scene(gv, sc, sh_dtype=torch.float16)
    out = ctx.score_views(gs, vf, c["cand"])
    ref = oracle.score_views(sc, g16.double().numpy(), 3, len(c["train"]), c["cand"], sh=sh16.double().numpy())
    err, _ = compare_views(out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), ref)
    assert err <= TOL
    ref32 = oracle.score_views(sc, g32.astype(np.float64), 3, len(c["train"]), c["cand"])
    storage_err = np.abs(out["score"].cpu().numpy() - ref32["score"]).max()
    assert storage_err < 5e-3   # half-precision storage effect on the view score


def test_invalid_arguments_raise(ctx, gv):
    c = case("tiny")
    gs = gpu_scene(gv, c["scene"])
    cams = [c["cand"][0], sg.fibonacci_cameras(2, 3.0, 64, 64)[1]]
    vf = ctx.vf_build(gs, c["train"][:1], degree=2)
    with pytest.raises(gv.GavisError) as e:
        ctx.score_views(gs, vf, cams)      # mixed resolutions
    assert e.value.code == gv.ERR_ARG
    with pytest.raises(gv.GavisError):
        ctx.score_views(gs, vf, c["cand"][:1], params=gv.Params(tile=12))
    with pytest.raises(gv.GavisError) as e:
        ctx.score_views(gs, vf, c["cand"][:1], params=gv.Params(tile_lists=3))
    assert e.value.code == gv.ERR_ARG


# --------------------------------------------------------------------------- density control

@pytest.mark.parametrize("name", ["tiny", "room_small"])
def test_density_control_parity(ctx, gv, name):
    """Alg. Visibility Field Density Control against the oracle: multi-view
    visibility of every virtual particle within 1e-4 of the oracle's range,
    and the same keep decision wherever that range (widened by 1e-4) lies
    on one side of eps_v."""
    c = case(name)
    sc = c["scene"]
    lo, hi = sc.bbox_min.astype(np.float64), sc.bbox_max.astype(np.float64)
    rho = 2000.0 / float(np.prod(hi - lo))                    # ~2000 virtual particles
    nvirt = int(np.floor(rho * np.prod(hi - lo)))
    vm = np.random.default_rng(11).uniform(lo, hi, (nvirt, 3)).astype(np.float32)
    gs = gpu_scene(gv, sc)
    out = ctx.density_control(gs, torch.as_tensor(vm).cuda(), c["train"], rho=rho, eta=0.5, eps_v=0.95)
    vis_r, keep_r, _, vlo, vhi = oracle.density_control(c["train"], sc, vm, rho=rho, eta=0.5, eps_v=0.95,
                                                        want_bounds=True)
    vis_g = out["vis"].cpu().numpy()
    assert excess(vis_g, vlo, vhi).max() <= TOL
    clear = (vhi < 0.95 - TOL) | (vlo > 0.95 + TOL)
    assert clear.mean() > 0.98, clear.mean()
    assert np.array_equal(out["keep"].cpu().numpy()[clear], keep_r[clear])
    assert out["n_keep"] == int(out["keep"].sum().item())
    np.testing.assert_array_equal(out["kept_means"].cpu().numpy(), vm[out["keep"].cpu().numpy()])
    assert out["scale"] == pytest.approx(oracle.virtual_scale(rho, 0.5), rel=1e-6)
    assert 0 < out["n_keep"] < nvirt


def test_density_control_feeds_scoring(ctx, gv):
    """Kept virtual particles join scoring with V = 0 (zero field, zero
    opacity, zero colour): the scene augmented with the oracle's kept set,
    scored on the GPU, against the oracle run on the same augmented scene;
    and the GPU's own augmentation of its kept set holds exactly those
    records."""
    c = case("tiny")
    sc = c["scene"]
    vm = np.random.default_rng(12).uniform(-1.5, 1.5, (500, 3)).astype(np.float32)
    train = c["train"][:3]
    g, _, _ = oracle.vf_build(train, sc, 2)
    _, keep_r, _ = oracle.density_control(train, sc, vm, rho=100.0)
    k = int(keep_r.sum())
    assert k > 0
    s = np.float32(oracle.virtual_scale(100.0, 0.5))
    aug = sg.Scene(np.concatenate([sc.means, vm[keep_r]]),
                   np.concatenate([sc.scales, np.full((k, 3), s, np.float32)]),
                   np.concatenate([sc.rots, np.tile(np.array([[1, 0, 0, 0]], np.float32), (k, 1))]),
                   np.concatenate([sc.opac, np.zeros(k, np.float32)]),
                   np.concatenate([sc.sh, np.zeros((k,) + sc.sh.shape[1:], np.float32)]), sc.sh_degree)
    g_aug = np.concatenate([g, np.zeros((k, g.shape[1]))]).astype(np.float32)
    vf_aug = gv.VisibilityField(torch.as_tensor(g_aug).cuda(), 2, 3, 1.0)
    out = ctx.score_views(gpu_scene(gv, aug), vf_aug, c["cand"][:4])
    ref = oracle.score_views(aug, g_aug.astype(np.float64), 2, 3, c["cand"][:4])
    err, _ = compare_views(out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), ref)
    assert err <= TOL
    assert score_excess(out["score"].cpu().numpy(), ref).max() <= TOL
    # the GPU's augmentation of its own kept set: the scene's records, then
    # the kept particles as zero-opacity isotropic Gaussians with a zero field
    gs = gpu_scene(gv, sc)
    vf = ctx.vf_build(gs, train, degree=2)
    dc = ctx.density_control(gs, torch.as_tensor(vm).cuda(), train, rho=100.0)
    gs2, vf2 = ctx.augment(gs, vf, dc["kept_means"], dc["scale"])
    kg = dc["n_keep"]
    km = dc["kept_means"].cpu().numpy()
    assert torch.equal(gs2.means.cpu(), torch.as_tensor(np.concatenate([sc.means, km])))
    assert torch.equal(gs2.scales[sc.n:].cpu(), torch.full((kg, 3), dc["scale"], dtype=torch.float32))
    assert torch.equal(gs2.rots[sc.n:].cpu(), torch.tensor([[1.0, 0.0, 0.0, 0.0]]).repeat(kg, 1))
    assert torch.all(gs2.opac[sc.n:] == 0) and torch.all(gs2.sh[sc.n:] == 0)
    assert torch.equal(gs2.opac[:sc.n].cpu(), torch.as_tensor(sc.opac))
    assert torch.equal(vf2.coeffs[:sc.n], vf.coeffs) and torch.all(vf2.coeffs[sc.n:] == 0)
    assert vf2.n_train_views == vf.n_train_views


def test_autotune_picks_a_tile_and_caches(ctx, gv):
    c = case("room_small")
    gs = gpu_scene(gv, c["scene"])
    vf = ctx.vf_build(gs, c["train"], degree=3)
    p, ms = ctx.autotune(gs, c["cand"][:3], vf, gv.Params(vf_degree=3))
    assert p.tile in (8, 16, 32) and ms > 0
    p2, ms2 = ctx.autotune(gs, c["cand"][:3], vf, gv.Params(vf_degree=3))
    assert p2.tile == p.tile and ms2 == -1.0          # cached choice
    pv, msv = ctx.autotune(gs, c["train"][:2], None, gv.Params(vf_degree=3))
    assert pv.tile in (8, 16, 32)
    # the tuned parameters give the oracle's answer (scores within tolerance)
    out = ctx.score_views(gs, vf, c["cand"], params=p)
    ref = ctx.score_views(gs, vf, c["cand"], params=gv.Params(vf_degree=3, tile=16))
    assert (out["score"] - ref["score"]).abs().max().item() <= TOL


@pytest.mark.parametrize("tile", [16, 32])
def test_colour_variance_variant_parity(ctx, gv, tile):
    """Per-Gaussian colour covariance (FisherRF variant) against the oracle."""
    c = case("room_small")
    sc = c["scene"]
    var = np.random.default_rng(21).uniform(0.001, 0.05, sc.sh.shape).astype(np.float32)
    g32 = oracle_gamma(c)
    vf = gv.VisibilityField(torch.as_tensor(g32).cuda(), 3, len(c["train"]), 1.0)
    gs = gv.Gaussians(*(torch.as_tensor(x).cuda().contiguous() for x in (sc.means, sc.scales, sc.rots, sc.opac, sc.sh)),
                      sc.sh_degree, torch.as_tensor(var).cuda().contiguous())
    out = ctx.score_views(gs, vf, c["cand"], params=gv.Params(tile=tile, vf_degree=3))
    ref = oracle.score_views(sc, g32.astype(np.float64), 3, len(c["train"]), c["cand"], sh_var=var.astype(np.float64))
    err, _ = compare_views(out["unc"].cpu().numpy(), out["rgb"].cpu().numpy(), ref)
    assert err <= TOL
    # it differs from the constant-covariance render
    const = ctx.score_views(gpu_scene(gv, sc), vf, c["cand"], params=gv.Params(tile=tile, vf_degree=3))
    assert (const["score"] - out["score"]).abs().max().item() > 1e-2
