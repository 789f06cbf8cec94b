"""Pins of the CPU oracle against what the paper and mathematics fix.

Every test here checks the oracle against something other than itself: closed
forms (modified spherical Bessel functions, the Legendre expansion of the
exponential, the spherical-harmonic addition theorem, a single Gaussian seen
head-on), a library routine (scipy's complex spherical harmonics), invariants
(partition of unity, additivity of the coefficients over views, the AM-GM
inequality) and brute force on tiny inputs.  The paper prints no worked
numerical example, so there is no golden value taken from it.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen as sg

PRM = oracle.params()
KC = 1.5 * math.log(0.01) + 1.5 * math.log(2 * math.pi * math.e)   # 1/2 log|sigma_c^2 I_3| + 3/2 log(2 pi e)
K0 = 1.5 * math.log(2 * math.pi * math.e)                          # Q0 = I_3


def i_closed(l, x):
    """Closed forms of the modified spherical Bessel functions i_0..i_3."""
    s, c = math.sinh(x), math.cosh(x)
    if l == 0:
        return s / x
    if l == 1:
        return (x * c - s) / x ** 2
    if l == 2:
        return ((x * x + 3) * s - 3 * x * c) / x ** 3
    if l == 3:
        return ((x ** 3 + 15 * x) * c - (6 * x * x + 15) * s) / x ** 4
    raise ValueError


def phi(x):
    return -x * math.log(x) if x > 0 else 0.0


def rand_dirs(n, seed):
    r = np.random.default_rng(seed).standard_normal((n, 3))
    return r / np.linalg.norm(r, axis=1, keepdims=True)


# --------------------------------------------------------------------------- Bessel / vMF

@pytest.mark.parametrize("x", [0.1, 0.3, 1.0, 3.0, 10.0])
def test_bessel_closed_forms(x):
    sp = pytest.importorskip("scipy.special")
    for l in range(6):
        assert oracle.bessel_i(l, x) == pytest.approx(float(sp.spherical_in(l, x)), rel=1e-12)
    for l in range(4):
        if x >= 0.3 * l:   # the closed forms cancel badly for small x
            assert oracle.bessel_i(l, x) == pytest.approx(i_closed(l, x), rel=1e-9)


def test_bessel_recurrence_and_origin():
    for x in (0.5, 1.0, 4.0):
        for l in range(1, 8):
            lhs = oracle.bessel_i(l - 1, x) - oracle.bessel_i(l + 1, x)
            assert lhs == pytest.approx((2 * l + 1) / x * oracle.bessel_i(l, x), rel=1e-11)
    assert oracle.bessel_i(0, 0.0) == 1.0
    assert all(oracle.bessel_i(l, 0.0) == 0.0 for l in range(1, 5))


def test_vmf_coefficients_kappa1():
    # a_l = 4 pi e^-1 i_l(1), l = 0..3
    a = oracle.vmf_coeffs(3, 1.0)
    want = [4 * math.pi * math.exp(-1) * i_closed(l, 1.0) for l in range(4)]
    np.testing.assert_allclose(a, want, rtol=1e-12)
    np.testing.assert_allclose(a, [5.4328486440, 1.7006733264, 0.3308286650, 0.0465300016], atol=1e-9)


@pytest.mark.parametrize("kappa", [0.1, 1.0, 3.0])
def test_vmf_sh_expansion_converges_to_exponential(kappa):
    """zeta * exp(kappa d.dp) expanded with a_l Y_lm(d) Y_lm(dp) (eq:SH_vMF,
    eq:vmf_coeff) must reproduce exp(kappa (d.dp - 1)) once L is large."""
    L = 30
    a = oracle.vmf_coeffs(L, kappa)
    D = rand_dirs(12, 1)
    for k in range(0, 12, 2):
        d, dp = D[k], D[k + 1]
        Yd, Yp = oracle.sh_real(L, d), oracle.sh_real(L, dp)
        s = 0.0
        for l in range(L + 1):
            sl = slice(l * l, (l + 1) * (l + 1))
            s += a[l] * float(np.dot(Yd[sl], Yp[sl]))
        assert s == pytest.approx(math.exp(kappa * (float(d @ dp) - 1.0)), abs=1e-12)
    # nu(dp; dp) = 1
    dp = D[0]
    Yp = oracle.sh_real(L, dp)
    s = sum(a[l] * float(np.dot(Yp[l * l:(l + 1) ** 2], Yp[l * l:(l + 1) ** 2])) for l in range(L + 1))
    assert s == pytest.approx(1.0, abs=1e-12)


# --------------------------------------------------------------------------- spherical harmonics

def test_complex_sh_matches_scipy():
    sp = pytest.importorskip("scipy.special")
    D = rand_dirs(20, 2)
    for d in D:
        theta = math.acos(max(-1.0, min(1.0, d[2])))
        ph = math.atan2(d[1], d[0])
        for l in range(5):
            for m in range(-l, l + 1):
                if hasattr(sp, "sph_harm_y"):
                    ref = complex(sp.sph_harm_y(l, m, theta, ph))
                elif hasattr(sp, "sph_harm"):
                    ref = complex(sp.sph_harm(m, l, ph, theta))
                else:
                    pytest.skip("scipy without spherical harmonics")
                got = oracle.sh_complex(l, m, d)
                assert abs(got - ref) < 1e-12, (l, m)


def test_real_sh_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi is exact for the products."""
    L = 4
    x, w = np.polynomial.legendre.leggauss(2 * L + 2)
    nphi = 4 * L + 4
    G = np.zeros(((L + 1) ** 2, (L + 1) ** 2))
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            p = 2 * math.pi * k / nphi
            Y = oracle.sh_real(L, [st * math.cos(p), st * math.sin(p), ct])
            G += wt * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye((L + 1) ** 2), atol=1e-12)


def test_real_sh_addition_theorem():
    D = rand_dirs(10, 3)
    for k in range(0, 10, 2):
        a, b = D[k], D[k + 1]
        Ya, Yb = oracle.sh_real(6, a), oracle.sh_real(6, b)
        for l in range(7):
            sl = slice(l * l, (l + 1) ** 2)
            Pl = np.polynomial.legendre.legval(float(a @ b), [0] * l + [1])
            assert float(Ya[sl] @ Yb[sl]) == pytest.approx((2 * l + 1) / (4 * math.pi) * Pl, abs=1e-13)


def test_real_sh_low_order_shape():
    """Degree 0 is the constant 1/(2 sqrt(pi)); degree 1 spans (y, z, x) with
    the paper's sign rule (positive coefficient for each axis)."""
    c1 = math.sqrt(3 / (4 * math.pi))
    for d in rand_dirs(5, 4):
        Y = oracle.sh_real(1, d)
        assert Y[0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-15)
        np.testing.assert_allclose(Y[1:4], [c1 * d[1], c1 * d[2], c1 * d[0]], atol=1e-14)


# --------------------------------------------------------------------------- geometry / bins

def single_gaussian_scene(pos, scale=0.05, opac=0.8, sh=None, rot=(1, 0, 0, 0)):
    sh = np.zeros((1, 4, 3), np.float32) if sh is None else np.asarray(sh, np.float32).reshape(1, -1, 3)
    return sg.Scene(np.array([pos], np.float32), np.full((1, 3), scale, np.float32),
                    np.array([rot], np.float32), np.array([opac], np.float32), sh, int(round(math.sqrt(sh.shape[1]))) - 1)


def axis_camera(W=16, H=16, f=20.0, cx=7.5, cy=7.5):
    """Camera at the origin looking down +z (identity world->camera)."""
    return sg.Camera(W=W, H=H, fx=f, fy=f, cx=cx, cy=cy, tan_half_fovx=W / (2 * f), tan_half_fovy=H / (2 * f),
                     R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), campos=np.zeros(3, np.float32))


def test_projection_on_axis_closed_form():
    """Isotropic Gaussian on the optical axis: Sigma2D = (f s / z)^2 I + 0.3 I
    (EWA splatting with the 3DGS low-pass dilation), centre at (cx, cy)."""
    for z, s, f in [(2.0, 0.05, 20.0), (5.0, 0.3, 100.0), (1.0, 0.01, 300.0)]:
        cam = axis_camera(64, 48, f, 31.5, 23.5)
        out, st = oracle.project(cam, single_gaussian_scene((0, 0, z), s))
        assert st[0] == 1
        zz, u, v, A, B, Cc = out[0, :6]
        var = (f * s / z) ** 2 + 0.3
        assert zz == np.float32(z)
        assert (u, v) == (np.float32(31.5), np.float32(23.5))
        assert A == pytest.approx(1 / var, rel=1e-5) and Cc == pytest.approx(1 / var, rel=1e-5)
        assert abs(B) < 1e-7


def test_projection_centre_is_pinhole():
    sc = sg.tiny_scene(300, seed=5)
    cam = sg.fibonacci_cameras(3, 3.0, 96, 64)[1]
    out, st = oracle.project(cam, sc)
    X = sc.means.astype(np.float64) @ cam.R.T.astype(np.float64) + cam.t.astype(np.float64)
    ok = st > 0
    np.testing.assert_allclose(out[ok, 1], cam.fx * X[ok, 0] / X[ok, 2] + cam.cx, rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(out[ok, 2], cam.fy * X[ok, 1] / X[ok, 2] + cam.cy, rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(out[:, 0], X[:, 2], rtol=1e-6, atol=1e-6)
    assert np.all(st[X[:, 2] <= cam.znear] == 0)


def test_keys_layout_and_order():
    c = sg.config(1, n=400, n_cand=3, cand_wh=(80, 48))
    cams, sc = c["cand"], c["scene"]
    keys, vals = oracle.bins(cams, sc)
    TW, TH = 5, 3
    assert np.all(np.diff(keys.astype(np.float64)) >= 0) or np.all(keys[1:] >= keys[:-1])
    tile = keys >> np.uint64(32)
    assert tile.max() < 3 * TW * TH
    # low word = bit pattern of the camera-space depth of that Gaussian
    for v, cam in enumerate(cams):
        out, st = oracle.project(cam, sc)
        sel = (tile // np.uint64(TW * TH)) == v
        z = out[vals[sel], 0].view(np.uint32)
        assert np.array_equal((keys[sel] & np.uint64(0xffffffff)).astype(np.uint32), z)
        # each (view, Gaussian) appears once per tile of its rectangle
        n_tiles = ((out[:, 7] - out[:, 6] + 1) * (out[:, 9] - out[:, 8] + 1)).astype(np.int64)
        exp_count = np.where(st == 1, n_tiles, 0)
        np.testing.assert_array_equal(np.bincount(vals[sel], minlength=sc.n), exp_count)
    # ties on equal keys are in ascending index order
    same = keys[1:] == keys[:-1]
    assert np.all(vals[1:][same] > vals[:-1][same])
    r = oracle.ranges(keys, 3 * TW * TH)
    for t in range(3 * TW * TH):
        s, e = r[t]
        assert np.all(tile[s:e] == t)
    assert r[:, 1].max() == len(keys)


def test_pixel_lists_equal_brute_force():
    """P10: lists built by scattering each Gaussian over its ellipse box equal
    a full scan of every pixel for every Gaussian."""
    c = sg.config(1, n=300, n_cand=2, cand_wh=(48, 40))
    for cam in c["cand"]:
        s1, e1 = oracle.pixel_lists(cam, c["scene"])
        s2, e2 = oracle.pixel_lists(cam, c["scene"], brute=True)
        assert np.array_equal(s1, s2) and np.array_equal(e1, e2)
        assert len(e1) > 1000
        for p in range(len(s1) - 1):   # sorted by (depth, index) per pixel
            seg = e1[s1[p]:s1[p + 1]]
            assert np.all(seg[1:] > seg[:-1])


@pytest.mark.parametrize("k", [1, 2])
def test_tile_rect_is_conservative(k):
    """P11: every (pixel, Gaussian) with q <= q_cut lies in the Gaussian's tile
    rectangle, so a tiled rasterizer sees every pair the untiled one does."""
    c = sg.config(k, n=400 if k == 1 else 20000, n_cand=3, cand_wh=(96, 80))
    sc = c["scene"]
    for cam in c["cand"]:
        out, st = oracle.project(cam, sc)
        start, ent = oracle.pixel_lists(cam, sc)
        pix = np.repeat(np.arange(cam.W * cam.H), np.diff(start))
        g = (ent & np.uint64(0xffffffff)).astype(np.int64)
        tx, ty = (pix % cam.W) // 16, (pix // cam.W) // 16
        assert np.all(st[g] == 1)
        assert np.all((out[g, 6] <= tx) & (tx <= out[g, 7]) & (out[g, 8] <= ty) & (ty <= out[g, 9]))
        # at pixel granularity too: the pixel centre lies in the footprint box
        # [u - ex, u + ex] x [v - ey, v + ey] (what lets a warp skip an entry)
        px = (pix % cam.W).astype(np.float32) + np.float32(0.5)
        py = (pix // cam.W).astype(np.float32) + np.float32(0.5)
        assert np.all((out[g, 1] - out[g, 10] <= px) & (px <= out[g, 1] + out[g, 10]))
        assert np.all((out[g, 2] - out[g, 11] <= py) & (py <= out[g, 2] + out[g, 11]))


# --------------------------------------------------------------------------- compositing

def test_partition_of_unity_and_monotone_transmittance():
    """P9: sum_i w*_i + T_end = 1 for the compensated weights and likewise for
    the colour weights; 0 <= alpha* <= 1; T never increases."""
    rng = np.random.default_rng(7)
    for trial in range(50):
        n = rng.integers(1, 60)
        al = rng.uniform(0, 1, n) * (rng.uniform(size=n) < 0.9)
        V = rng.uniform(0, 1, n)
        col = rng.normal(size=(n, 3))
        r = oracle.composite(al, V, col)
        # both sums telescope regardless of where each accumulator stopped
        assert r["sum_w"] + r["T"] == pytest.approx(1.0, abs=1e-12)
        assert r["sum_wc"] + r["Tc"] == pytest.approx(1.0, abs=1e-12)
        Ts = [oracle.composite(al[:k], V[:k], col[:k])["T"] for k in range(n + 1)]
        assert all(Ts[k + 1] <= Ts[k] for k in range(n))
        a_star = (V + 0.5 * (1 - V)) * al + 0.15 * 0.5 * (1 - V)
        assert np.all((a_star >= 0) & (a_star <= 1))


def test_single_gaussian_pixel_closed_form():
    """P7: one Gaussian whose centre lands on a pixel centre (q = 0, alpha = o):
    alpha* from eq:alpha_comp, w1 = alpha* V, w0 = alpha* (1 - V),
    H = phi(w1) + w1 k_c + phi(w0) + w0 k_0 (eq:huber), rgb = o c(d)."""
    o, V = 0.8, 0.3
    th = np.zeros((4, 3))
    th[0] = [0.5, -0.2, 0.1]
    th[2] = [0.3, 0.4, -0.6]   # (l=1, m=0) coefficient -> z component
    sc = single_gaussian_scene((0, 0, 2.0), 0.05, o, th)
    cam = axis_camera()
    rgb, unc, amb, used = oracle.render_view(cam, sc, np.array([V]))
    a_s = (V + 0.5 * (1 - V)) * o + 0.15 * 0.5 * (1 - V)
    w1, w0 = a_s * V, a_s * (1 - V)
    H = phi(w1) + w1 * KC + phi(w0) + w0 * K0
    assert unc[7, 7] == pytest.approx(H, abs=1e-6)      # float32 alpha at q = 0 is exactly o
    c = th[0] * 0.5 / math.sqrt(math.pi) + th[2] * math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(rgb[:, 7, 7], np.float32(o) * c, atol=1e-6)
    # a pixel outside the footprint has an empty list: H = 0, rgb = 0
    assert unc[0, 0] == 0.0 and np.all(rgb[:, 0, 0] == 0.0) and used[0, 0] == 0


def test_unseen_gives_prior_mass_and_more_entropy():
    """P8: with V = 0 all weight goes to the prior component; for a single
    Gaussian pixel H(V=0) - H(V=1) >= 0.512 over alpha in [0, 1]."""
    gaps = []
    for a in np.linspace(0, 1, 1001):
        r0 = oracle.composite([a], [0.0], [[0, 0, 0]])
        r1 = oracle.composite([a], [1.0], [[0, 0, 0]])
        w0 = 0.5 * a + 0.075
        assert r0["w0"] == pytest.approx(w0, abs=1e-15)
        assert r0["H"] == pytest.approx(phi(w0) + w0 * K0, abs=1e-13)
        assert r1["H"] == pytest.approx(phi(a) + a * KC, abs=1e-13)
        gaps.append(r0["H"] - r1["H"])
    assert min(gaps) >= 0.512


def test_full_visibility_matches_plain_compositing():
    """P12: with V = 1, alpha* = alpha and the UQ weights are the colour
    weights w_i = alpha_i prod_{j<i}(1 - alpha_j); H = sum phi(w) + w k_c."""
    rng = np.random.default_rng(8)
    al = rng.uniform(0, 0.6, 40)
    col = rng.normal(size=(40, 3))
    r = oracle.composite(al, np.ones(40), col)
    T, H, C = 1.0, 0.0, np.zeros(3)
    for a, c in zip(al, col):
        w = a * T
        H += phi(w) + w * KC
        C += w * c
        T *= 1 - a
        if T < 1e-4:
            break
    assert r["H"] == pytest.approx(H, abs=1e-13)
    np.testing.assert_allclose(r["rgb"], C, atol=1e-13)
    assert r["T"] == pytest.approx(r["Tc"], abs=1e-15)


def test_termination_after_update():
    """The transmittance test follows the update (as printed): the Gaussian
    that drives T below eps_T still contributes, the next one does not."""
    r = oracle.composite([0.99999, 0.5], [1.0, 1.0], [[1, 0, 0], [0, 1, 0]])
    assert r["used"] == 1 and r["rgb"][1] == 0.0 and r["rgb"][0] == pytest.approx(0.99999)
    r = oracle.composite([0.9998, 0.5], [1.0, 1.0], [[1, 0, 0], [0, 1, 0]])   # T = 2e-4 stays on
    assert r["used"] == 2 and r["rgb"][1] == pytest.approx(0.5 * 2e-4)


# --------------------------------------------------------------------------- visibility field

def test_single_gaussian_single_view_field():
    """P3: a lone Gaussian seen by one camera has v = 1 (T = 1 at every
    footprint pixel).  Its field then is a_l Y_lm(d_p) and, by the addition
    theorem, V~(d) = zeta sum_l (2l+1) i_l(kappa) P_l(d . d_p)."""
    sc = single_gaussian_scene((0, 0, 2.0), 0.05, 0.8)
    cam = axis_camera()
    for L in (2, 3):
        gamma, amb, vis = oracle.vf_build([cam], sc, L, want_vis=True)
        assert vis[0, 0] == 1.0 and not amb.any()
        for dot in (1.0, -1.0, 0.0, 0.5):
            want = math.exp(-1) * sum((2 * l + 1) * i_closed(l, 1.0) *
                                      np.polynomial.legendre.legval(dot, [0] * l + [1]) for l in range(L + 1))
            # place a query camera so that normalize(x_g - campos) . (0,0,1) = dot
            s = math.sqrt(max(0.0, 1 - dot * dot))
            pos = np.array([0, 0, 2.0]) - 3.0 * np.array([s, 0, dot])
            qcam = sg.look_at_camera(pos, (0, 0, 2.0), 16, 16)
            V, vt = oracle.vf_query(gamma, L, 1, qcam, sc.means)
            assert vt[0] == pytest.approx(want, abs=2e-7)
            assert V[0] == pytest.approx(min(max(want, 0.0), 1.0), abs=2e-7)   # |P| = 1: V = clamp(V~)
    # the printed defaults L = 2, kappa = 1 seen head-on
    assert math.exp(-1) * sum((2 * l + 1) * i_closed(l, 1.0) for l in range(3)) == pytest.approx(0.9699708, abs=1e-7)


def test_occluded_and_transparent_occluder():
    """Alg. Single-view Particle Visibility: behind three opaque walls the rear
    Gaussian is never reached (v = 0, Phi T = 0); behind zero-opacity
    particles it is fully visible (v = 1)."""
    cam = axis_camera(32, 32, 30.0, 15.5, 15.5)
    for o_front, want in ((0.9999, 0.0), (0.0, 1.0)):
        sc = sg.Scene(np.array([[0, 0, 1.0], [0, 0, 1.1], [0, 0, 1.2], [0, 0, 3.0]], np.float32),
                      np.array([[20.0, 20.0, 0.01]] * 3 + [[0.05, 0.05, 0.05]], np.float32),
                      np.array([[1, 0, 0, 0]] * 4, np.float32),
                      np.array([o_front] * 3 + [0.9], np.float32), np.zeros((4, 1, 3), np.float32), 0)
        sumT, cnt, amb, _ = oracle.visibility_view(cam, sc)
        v = sumT[3] / cnt[3] if cnt[3] else 0.0
        assert v == pytest.approx(want, abs=1e-12)
        assert cnt[0] == 32 * 32
        assert (cnt[3] == 0) == (want == 0.0)


def field_case(kappa, n=400):
    c = sg.config(1, n=n, n_train=8, train_wh=(64, 64))
    return c["scene"], c["train"], oracle.params(kappa=kappa)


def test_isotropic_field_is_sum_of_views():
    """P4 (the isotropic ablation, kappa = 0): only l = 0 survives and
    V~(d) = sum_p v_p for every direction and any L."""
    sc, train, prm = field_case(0.0)
    for L in (0, 2, 3):
        gamma, amb, vis = oracle.vf_build(train, sc, L, prm, want_vis=True)
        assert L == 0 or np.abs(gamma[:, 1:]).max() == 0.0
        for cam in sg.fibonacci_cameras(3, 3.0, 16, 16):
            V, vt = oracle.vf_query(gamma, L, len(train), cam, sc.means)
            np.testing.assert_allclose(vt, vis.sum(0), atol=1e-12)


def test_field_additive_over_views():
    """P5: gamma(P1 u P2) = gamma(P1) + gamma(P2) (eq:vis_gamma is a sum)."""
    sc, train, prm = field_case(1.0)
    g_all, _, _ = oracle.vf_build(train, sc, 3, prm)
    g_a, _, _ = oracle.vf_build(train[:3], sc, 3, prm)
    g_b, _, _ = oracle.vf_build(train[3:], sc, 3, prm)
    np.testing.assert_allclose(g_all, g_a + g_b, atol=1e-12)
    assert np.abs(g_all).max() > 1.0


def test_am_gm_lower_bound():
    """P6: 1 - (1 - V~/|P|)^|P| <= 1 - prod_p (1 - V_p) (eq:vis_bound vs
    eq:vis_all), with equality when every V_p is equal."""
    sc, train, prm = field_case(0.0)
    gamma, _, vis = oracle.vf_build(train, sc, 0, prm, want_vis=True)
    dirs = np.stack([(sc.means - c.campos) / np.linalg.norm(sc.means - c.campos, axis=1, keepdims=True)
                     for c in train]).astype(np.float64)
    cam = sg.fibonacci_cameras(2, 3.0, 16, 16)[0]
    d = (sc.means - cam.campos).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Vb, _ = oracle.vf_query(gamma, 0, len(train), cam, sc.means)
    Ve = oracle.vf_exact(vis, dirs, 0.0, d)
    assert np.all(Vb <= Ve + 1e-12)
    assert np.max(Ve - Vb) > 1e-3   # strict somewhere: the bound is not an identity
    # equal per-view visibilities: the same camera three times
    g3, _, vis3 = oracle.vf_build([train[0]] * 3, sc, 0, prm, want_vis=True)
    Vb3, _ = oracle.vf_query(g3, 0, 3, cam, sc.means)
    Ve3 = oracle.vf_exact(vis3, np.stack([dirs[0]] * 3), 0.0, d)
    np.testing.assert_allclose(Vb3, Ve3, atol=1e-12)


def test_unseen_gaussians_have_zero_field():
    """Gaussians no training view sees get gamma = 0, hence V = 0 from every
    direction ('zero visibility, maximal uncertainty')."""
    sc = sg.tiny_scene(300, seed=3)
    cam = sg.look_at_camera((3.0, 0, 0), (0, 0, 0), 32, 32, 10.0)   # narrow: most fall outside
    gamma, _, vis = oracle.vf_build([cam], sc, 2, want_vis=True)
    unseen = vis[0] == 0
    assert unseen.sum() > 50
    assert np.all(gamma[unseen] == 0.0)
    V, _ = oracle.vf_query(gamma, 2, 1, sg.look_at_camera((-3.0, 0, 0), (0, 0, 0), 32, 32), sc.means)
    assert np.all(V[unseen] == 0.0)


def test_query_degenerate_counts():
    """|P| = 0 gives V = 0; V~ above |P| clamps to V = 1; V~ below 0 to V = 0."""
    means = np.array([[0, 0, 1.0]] * 3, np.float32)
    gamma = np.zeros((3, 1))
    gamma[:, 0] = np.array([0.0, 1e6, -5.0]) * 2 * math.sqrt(math.pi)   # V~ = gamma_00 Y_00
    cam = axis_camera()
    V, vt = oracle.vf_query(gamma, 0, 0, cam, means)
    assert np.all(V == 0)
    V, vt = oracle.vf_query(gamma, 0, 4, cam, means)
    np.testing.assert_allclose(vt, [0.0, 1e6, -5.0], rtol=1e-12)
    assert V[0] == 0.0 and V[1] == 1.0 and V[2] == 0.0


def test_score_is_mean_entropy_and_argmax():
    c = sg.config(1, n=300, n_cand=4, cand_wh=(32, 32))
    sc = c["scene"]
    gamma, _, _ = oracle.vf_build(c["train"][:2], sc, 2)
    out = oracle.score_views(sc, gamma, 2, 2, c["cand"])
    for v in range(4):
        assert out["score"][v] == pytest.approx(out["unc"][v].mean(), abs=1e-15)
    assert out["best"] == int(np.argmax(out["score"]))


# --------------------------------------------------------------------------- density control

def test_virtual_particle_scale():
    """(4/3) pi s^3 rho = 1 + eta; the defaults rho = 100, eta = 0.5."""
    for rho, eta in ((100.0, 0.5), (10.0, 0.5), (1000.0, 0.2)):
        s = oracle.virtual_scale(rho, eta)
        assert 4.0 / 3.0 * math.pi * s ** 3 * rho == pytest.approx(1.0 + eta, rel=1e-12)


def wall_scene(o):
    """Three large thin Gaussians at z = 1, 1.1, 1.2 covering the view."""
    return sg.Scene(np.array([[0, 0, 1.0], [0, 0, 1.1], [0, 0, 1.2]], np.float32),
                    np.array([[20.0, 20.0, 0.01]] * 3, np.float32), np.array([[1, 0, 0, 0]] * 3, np.float32),
                    np.array([o] * 3, np.float32), np.zeros((3, 1, 3), np.float32), 0)


def test_density_control_free_occluded_and_unseen():
    """A virtual particle in front of the camera with nothing before it is seen
    (visibility 1): free space, pruned.  Behind opaque walls, or outside the
    field of view, it is never reached (visibility 0): kept.  Virtual
    particles are transparent, so two on one ray are both seen."""
    cam = axis_camera(32, 32, 30.0, 15.5, 15.5)
    vm = np.array([[0, 0, 0.6], [0, 0, 0.8], [0, 0, 3.0], [5.0, 0, 1.0]], np.float32)
    vis, keep, amb = oracle.density_control([cam], wall_scene(0.9999), vm)
    np.testing.assert_allclose(vis, [1.0, 1.0, 0.0, 0.0], atol=1e-12)
    assert keep.tolist() == [False, False, True, True]
    # transparent walls: the far particle is seen too
    vis, keep, _ = oracle.density_control([cam], wall_scene(0.0), vm)
    np.testing.assert_allclose(vis[:3], [1.0, 1.0, 1.0], atol=1e-12)
    assert keep.tolist() == [False, False, False, True]


def test_density_control_product_over_views():
    """1 - prod_p (1 - v_p): one view that sees the particle fully is enough;
    the threshold eps_v decides with <=."""
    cam_a = axis_camera(32, 32, 30.0, 15.5, 15.5)
    cam_b = sg.Camera(W=32, H=32, fx=30.0, fy=30.0, cx=15.5, cy=15.5, tan_half_fovx=32 / 60, tan_half_fovy=32 / 60,
                      R=np.diag([1.0, -1.0, -1.0]).astype(np.float32), t=np.zeros(3, np.float32),
                      campos=np.zeros(3, np.float32))   # looks down -z: sees nothing of the particle
    vm = np.array([[0, 0, 0.6]], np.float32)
    empty = sg.tiny_scene(1, seed=1).subset(np.arange(0))
    vis, keep, _ = oracle.density_control([cam_b, cam_a], empty, vm)
    assert vis[0] == pytest.approx(1.0, abs=1e-12) and not keep[0]
    vis, keep, _ = oracle.density_control([cam_b], empty, vm)
    assert vis[0] == 0.0 and keep[0]
    vis, keep, _ = oracle.density_control([cam_a], empty, vm, eps_v=1.0)
    assert keep[0]   # visibility 1 <= eps_v = 1


# --------------------------------------------------------------------------- FisherRF colour covariance

def test_uniform_coefficient_variance_is_isotropic():
    """Q_c,k(d) = sum_j Y_j(d)^2 var_jk: with var_jk = s2 4 pi / (Lc+1)^2 the
    addition theorem gives Q_c = s2 I for every direction, so the render
    equals the constant-covariance one with sigma_c^2 = s2."""
    c = sg.config(1, n=300, n_cand=2, cand_wh=(40, 40))
    sc = c["scene"]
    gamma, _, _ = oracle.vf_build(c["train"][:3], sc, 2)
    s2 = 0.02
    var = np.full(sc.sh.shape, s2 * 4 * math.pi / 4.0)      # Lc = 1: 4 coefficients
    for cam in c["cand"]:
        V, _ = oracle.vf_query(gamma, 2, 3, cam, sc.means)
        _, u1, _, _ = oracle.render_view(cam, sc, V, oracle.params(sigma_c2=s2), sh_var=var)
        _, u2, _, _ = oracle.render_view(cam, sc, V, oracle.params(sigma_c2=s2))
        np.testing.assert_allclose(u1, u2, atol=1e-12)
        assert np.abs(u2).max() > 0.1


def test_coefficient_variance_single_gaussian_closed_form():
    """One Gaussian seen head-on, d = +z: Y_00 = 1/(2 sqrt(pi)), Y_10 = sqrt(3/(4 pi)),
    the other degree-1 terms vanish, so Q_k = Y_00^2 var_0k + Y_10^2 var_2k and
    the visible component carries 1/2 sum_k ln Q_k + 3/2 ln(2 pi e)."""
    o, V = 0.8, 0.6
    sc = single_gaussian_scene((0, 0, 2.0), 0.05, o)
    var = np.zeros((1, 4, 3))
    var[0, 0] = [0.01, 0.02, 0.05]
    var[0, 2] = [0.03, 0.001, 0.002]
    var[0, 1] = var[0, 3] = [7.0, 7.0, 7.0]                # multiplied by Y^2 = 0 here
    rgb, unc, _, _ = oracle.render_view(axis_camera(), sc, np.array([V]), sh_var=var)
    y00, y10 = 0.25 / math.pi, 3 / (4 * math.pi)
    Q = y00 * var[0, 0] + y10 * var[0, 2]
    kc = 0.5 * float(np.log(Q).sum()) + 1.5 * math.log(2 * math.pi * math.e)
    a_s = (V + 0.5 * (1 - V)) * o + 0.15 * 0.5 * (1 - V)
    w1, w0 = a_s * V, a_s * (1 - V)
    assert unc[7, 7] == pytest.approx(phi(w1) + w1 * kc + phi(w0) + w0 * K0, abs=1e-6)


def test_expected_depth_single_gaussian_and_occlusion():
    """Expected depth d of eq:id (colour weights alpha_i T_c,i, background 0):
    one Gaussian on the optical axis at z = 2 gives d = o * 2 at the centre
    pixel (alpha = o at q = 0) and 0 outside its footprint; a second Gaussian
    straight behind it at z = 3 adds (1 - o) o2 * 3."""
    o = 0.8
    sc = single_gaussian_scene((0, 0, 2.0), 0.05, o)
    cam = axis_camera()
    rgb, unc, amb, used, depth = oracle.render_view(cam, sc, np.array([0.5]), want_depth=True)
    assert depth[7, 7] == pytest.approx(np.float32(o) * 2.0, abs=1e-6)
    assert depth[0, 0] == 0.0
    o2 = 0.6
    two = sg.Scene(np.array([[0, 0, 2.0], [0, 0, 3.0]], np.float32), np.full((2, 3), 0.05, np.float32),
                   np.array([[1, 0, 0, 0], [1, 0, 0, 0]], np.float32), np.array([o, o2], np.float32),
                   np.zeros((2, 4, 3), np.float32), 1)
    _, _, _, _, d2 = oracle.render_view(cam, two, np.array([0.5, 0.5]), want_depth=True)
    assert d2[7, 7] == pytest.approx(np.float32(o) * 2.0 + (1 - np.float32(o)) * np.float32(o2) * 3.0, abs=1e-6)


def test_expected_depth_partition_of_unity():
    """With every Gaussian at the same depth z, d = z (1 - T_c,end): the colour
    weights sum to the opacity the pixel accumulated (P9 applied to d)."""
    rng = np.random.default_rng(11)
    for n in (1, 5, 40):
        al = rng.uniform(0.05, 0.9, n)
        r = oracle.composite(al, rng.uniform(0, 1, n), rng.normal(size=(n, 3)), z=np.full(n, 4.25))
        assert r["depth"] == pytest.approx(4.25 * (1.0 - r["Tc"]), rel=1e-12, abs=1e-12)
        assert r["depth"] == pytest.approx(4.25 * r["sum_wc"], rel=1e-12)


# --------------------------------------------------------------------------- bounds under rounding-sensitive stops

def _band_list(seed):
    """A list whose transmittance lingers inside the band around eps_T for
    several entries: a few opaque entries bring T near eps, then faint ones."""
    rng = np.random.default_rng(seed)
    eps = 1e-4
    a = list(rng.uniform(0.5, 0.9, 3))
    T = float(np.prod(1 - np.array(a)))
    a.append(1 - eps * 1.0004 / T)              # T lands at eps (1 + 4e-4)
    a += list(rng.uniform(1e-4, 4e-4, 6))       # T creeps down through the band
    a += list(rng.uniform(0.2, 0.6, 4))
    n = len(a)
    V = rng.uniform(0, 1, n)
    V[:10] = 1.0                                # alpha* = alpha there: both accumulators cross the band
    col = rng.normal(0, 1, (n, 3))
    z = rng.uniform(1, 5, n)
    return np.array(a), V, col, z


@pytest.mark.parametrize("seed", range(6))
def test_composite_bounds_are_runs_at_thresholds_in_the_band(seed):
    """[H_lo, H_hi] (and the rgb, depth ranges) equal the least and greatest
    outputs of plain runs (margin 0) whose threshold sweeps the band
    [eps (1 - m), eps (1 + m)]: every possible stop is some threshold's stop."""
    a, V, col, z = _band_list(seed)
    eps, m = 1e-4, 1e-3
    r = oracle.composite(a, V, col, oracle.params(eps_T=eps, margin=m), z=z)
    outs = []
    for thr in np.linspace(eps * (1 - m), eps * (1 + m), 801):
        outs.append(oracle.composite(a, V, col, oracle.params(eps_T=float(thr), margin=0.0), z=z))
    H = np.array([o["H"] for o in outs])
    rgb = np.array([o["rgb"] for o in outs])
    d = np.array([o["depth"] for o in outs])
    assert H.max() > H.min()        # the band holds more than one stop here
    assert r["H_lo"] == pytest.approx(H.min(), abs=1e-15) and r["H_hi"] == pytest.approx(H.max(), abs=1e-15)
    np.testing.assert_allclose(r["rgb_lo"], rgb.min(0), atol=1e-15)
    np.testing.assert_allclose(r["rgb_hi"], rgb.max(0), atol=1e-15)
    assert r["depth_lo"] == pytest.approx(d.min(), abs=1e-14) and r["depth_hi"] == pytest.approx(d.max(), abs=1e-14)
    assert r["H_lo"] <= r["H"] <= r["H_hi"]


def test_composite_bounds_collapse_away_from_the_band():
    rng = np.random.default_rng(3)
    a = rng.uniform(0.1, 0.5, 12)
    V = rng.uniform(0, 1, 12)
    col = rng.normal(0, 1, (12, 3))
    r = oracle.composite(a, V, col, oracle.params(eps_T=1e-4, margin=1e-3))
    assert not r["amb"]
    assert r["H_lo"] == r["H"] == r["H_hi"]
    assert np.array_equal(r["rgb_lo"], r["rgb"]) and np.array_equal(r["rgb_hi"], r["rgb"])


def test_visibility_bounds_are_runs_at_band_edges():
    """The early sums and counts are exactly the plain run stopping at
    eps (1 + m); the late counts the plain run stopping at eps (1 - m)."""
    c = sg.config(1, n=800, n_train=2, train_wh=(96, 80))
    sc = c["scene"]
    eps, m = 1e-4, 1e-2   # a wide band, so that small cases exercise it
    in_band = 0
    for cam in c["train"]:
        s, cn, _, _, b = oracle.visibility_view(cam, sc, oracle.params(eps_T=eps, margin=m), want_bounds=True)
        s_hi, c_hi, _, _ = oracle.visibility_view(cam, sc, oracle.params(eps_T=eps * (1 + m), margin=0.0))
        s_lo, c_lo, _, _ = oracle.visibility_view(cam, sc, oracle.params(eps_T=eps * (1 - m), margin=0.0))
        assert np.array_equal(b["cnt_early"], c_hi) and np.array_equal(b["cnt_late"], c_lo)
        np.testing.assert_allclose(b["sum_early"], s_hi, rtol=1e-12, atol=1e-15)
        assert np.all(b["cnt_early"] <= cn) and np.all(cn <= b["cnt_late"])
        in_band += int((b["cnt_late"] > b["cnt_early"]).sum())
    assert in_band > 0     # the case exercises the band


def test_field_radius_contains_builds_at_band_edges():
    """A field built with the thresholds at either edge of the band (two of
    the builds a rounding-sensitive pass could produce) lies within gamma +-
    the radius, coefficient by coefficient."""
    c = sg.config(1, n=800, n_train=3, train_wh=(96, 80))
    sc, L = c["scene"], 2
    eps, m = 1e-4, 1e-2   # a wide band, so that small cases exercise it
    g, _, _, rad = oracle.vf_build(c["train"], sc, L, oracle.params(eps_T=eps, margin=m), want_rad=True)
    assert rad.max() > 0
    for thr in (eps * (1 - m), eps * (1 + m)):
        g2, _, _ = oracle.vf_build(c["train"], sc, L, oracle.params(eps_T=thr, margin=0.0))
        assert np.all(np.abs(g2 - g) <= rad + 1e-12)
    # Gaussians untouched by the band have radius 0 and the same field
    g0, _, _, rad0 = oracle.vf_build(c["train"], sc, L, oracle.params(eps_T=eps, margin=0.0), want_rad=True)
    np.testing.assert_allclose(g0, g, rtol=1e-12, atol=1e-14)   # (sums over pixels run in parallel)
    assert np.all(rad0 <= 1e-12)


def test_density_control_range_contains_band_edges():
    c = sg.config(1, n=600, n_train=3, train_wh=(64, 64))
    sc = c["scene"]
    rng = np.random.default_rng(9)
    vm = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    eps, m = 1e-4, 1e-2   # a wide band, so that small cases exercise it
    vis, _, _, lo, hi = oracle.density_control(c["train"], sc, vm, prm=oracle.params(eps_T=eps, margin=m),
                                               want_bounds=True)
    assert np.all(lo <= vis + 1e-15) and np.all(vis <= hi + 1e-15)
    for thr in (eps * (1 - m), eps * (1 + m)):
        v2, _, _ = oracle.density_control(c["train"], sc, vm, prm=oracle.params(eps_T=thr, margin=0.0))
        assert np.all(lo - 1e-12 <= v2) and np.all(v2 <= hi + 1e-12)
