"""Closed-form pins of the oracle's projection (the EWA splatting of 3DGS that
the paper's visibility and uncertainty algorithms take as given).

Each pin compares the oracle's float32 projection with a float64 value worked
out by hand from the geometry, never with the oracle's own formula:

* rotation   -- a Gaussian on the optical axis seen by an identity camera has
               Sigma2D = (f/z)^2 [R diag(s^2) R^T]_{xy block} + 0.3 I.  For a
               rotation by theta about the camera z axis that block is
               [[c^2 s1^2 + s^2 s2^2, c s (s1^2 - s2^2)], [., s^2 s1^2 + c^2 s2^2]];
               about the x axis by 90 degrees, s3 lands on the image y axis;
               for random quaternions the matrix comes from scipy's Rotation;
* conic      -- q at one pixel along (1, 1) and (1, -1) from a 45-degree
               Gaussian, worked by hand (2.6/5.59 and 8.6/5.59);
* off axis   -- an isotropic Gaussian at (x, y, z) has
               Sigma2D = s^2 J J^T + 0.3 I with J = [[fx/z, 0, -fx x/z^2],
               [0, fy/z, -fy y/z^2]];
* clamp      -- past 1.3 tan(fov/2) the Jacobian's third column uses the
               clamped ratio, while the centre keeps the true one;
* camera     -- rotating the Gaussian and the camera together by the same
               world rotation leaves every projected quantity unchanged;
* footprint  -- a lone Gaussian's colour image is o exp(-q/2) per pixel with
               q = d^T Sigma2D^-1 d from the closed form above, and zero
               where q > q_cut.

`test_planted_mistakes_are_caught` compiles copies of the oracle with one
plausible mistake each (transposed rotation, S R instead of R S, a flipped
quaternion sign, the conic's off-diagonal sign, a dropped Jacobian column, no
clamp, fx and fy swapped, the camera rotation transposed, the cross term of q
halved, a missing dilation) and checks that some pin above fails for every
one of them.
"""
import math
import os
import subprocess

import numpy as np
import pytest

import oracle
import scenegen as sg

# float32 geometry evaluated once per operation: ~10 roundings on the way to
# Sigma2D; agreement with the float64 closed form measured below 1e-6 relative
RTOL = 2e-6


def identity_camera(W=64, H=48, fx=100.0, fy=None, cx=31.5, cy=23.5):
    fy = fx if fy is None else fy
    return sg.Camera(W=W, H=H, fx=fx, fy=fy, cx=cx, cy=cy, tan_half_fovx=W / (2 * fx),
                     tan_half_fovy=H / (2 * fy), R=np.eye(3, dtype=np.float32),
                     t=np.zeros(3, np.float32), campos=np.zeros(3, np.float32))


def one_gaussian(pos, scales, quat=(1.0, 0.0, 0.0, 0.0), opac=0.8, colour=None):
    sh = np.zeros((1, 1, 3), np.float32)
    if colour is not None:
        sh[0, 0, :] = np.asarray(colour, np.float64) * 2.0 * math.sqrt(math.pi)   # Y_0 = 1/(2 sqrt(pi))
    return sg.Scene(np.array([pos], np.float32), np.array([scales], np.float32),
                    np.array([quat], np.float32), np.array([opac], np.float32), sh, 0)


def sigma2d_from_oracle(cam, sc):
    """Sigma2D recovered in float64 from the oracle's conic (A, B, C):
    Sigma2D = [[C, -B], [-B, A]] / (A C - B^2)."""
    out, st = oracle.project(cam, sc)
    z, u, v, A, B, C = (float(x) for x in out[0, :6])
    det = A * C - B * B
    return np.array([[C / det, -B / det], [-B / det, A / det]]), (u, v, z), int(st[0])


def assert_sigma(S, a, b, c, rtol=RTOL):
    scale = max(abs(a), abs(c))
    assert S[0, 0] == pytest.approx(a, rel=rtol), (S, a, b, c)
    assert S[1, 1] == pytest.approx(c, rel=rtol), (S, a, b, c)
    assert abs(S[0, 1] - b) <= rtol * scale, (S, a, b, c)


def quat_about(axis, theta):
    h = 0.5 * theta
    w = math.cos(h)
    s = math.sin(h)
    ax = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    return (w, s * ax[0], s * ax[1], s * ax[2])


# --------------------------------------------------------------------------- pins

def pin_rotation_about_z():
    s1, s2, s3 = 0.04, 0.02, 0.01
    f, z = 100.0, 2.0
    k = (f / z) ** 2
    for deg in (90.0, 45.0, 30.0, 120.0, -60.0):
        th = math.radians(deg)
        c, s = math.cos(th), math.sin(th)
        S, (u, v, _), st = sigma2d_from_oracle(identity_camera(fx=f), one_gaussian((0, 0, z), (s1, s2, s3), quat_about((0, 0, 1), th)))
        assert st == 1
        assert_sigma(S, k * (c * c * s1 * s1 + s * s * s2 * s2) + 0.3,
                     k * c * s * (s1 * s1 - s2 * s2),
                     k * (s * s * s1 * s1 + c * c * s2 * s2) + 0.3)
        assert (u, v) == (31.5, 23.5)
    # 90 degrees swaps the image axes' variances exactly
    S, _, _ = sigma2d_from_oracle(identity_camera(fx=f), one_gaussian((0, 0, z), (s1, s2, s3), quat_about((0, 0, 1), math.pi / 2)))
    assert_sigma(S, k * s2 * s2 + 0.3, 0.0, k * s1 * s1 + 0.3)


def pin_rotation_about_x():
    """90 degrees about x maps the local z axis onto the camera's y axis."""
    s1, s2, s3 = 0.04, 0.02, 0.01
    f, z = 100.0, 2.0
    k = (f / z) ** 2
    S, _, st = sigma2d_from_oracle(identity_camera(fx=f), one_gaussian((0, 0, z), (s1, s2, s3), quat_about((1, 0, 0), math.pi / 2)))
    assert st == 1
    assert_sigma(S, k * s1 * s1 + 0.3, 0.0, k * s3 * s3 + 0.3)
    # and 90 degrees about y puts s3 on the image x axis
    S, _, _ = sigma2d_from_oracle(identity_camera(fx=f), one_gaussian((0, 0, z), (s1, s2, s3), quat_about((0, 1, 0), math.pi / 2)))
    assert_sigma(S, k * s3 * s3 + 0.3, 0.0, k * s2 * s2 + 0.3)


def pin_random_quaternions_against_scipy():
    """On the axis, Sigma2D = (f/z)^2 [G diag(s^2) G^T]_xy + 0.3 I with G the
    rotation matrix of the (unnormalised) quaternion, taken from scipy."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(7)
    f, z = 80.0, 3.0
    k = (f / z) ** 2
    for _ in range(20):
        q = rng.normal(size=4) * rng.uniform(0.3, 3.0)          # w, x, y, z; not unit length
        sc = np.exp(rng.normal(-3.0, 0.5, size=3))
        q32, s32 = q.astype(np.float32), sc.astype(np.float32)
        G = Rot.from_quat([q32[1], q32[2], q32[3], q32[0]]).as_matrix()   # scipy is scalar-last
        Sig = G @ np.diag(s32.astype(np.float64) ** 2) @ G.T
        S, _, st = sigma2d_from_oracle(identity_camera(fx=f), one_gaussian((0, 0, z), s32, q32))
        assert st == 1
        assert_sigma(S, k * Sig[0, 0] + 0.3, k * Sig[0, 1], k * Sig[1, 1] + 0.3, rtol=2e-5)


def pin_conic_worked_example():
    """45 degrees about z, s = (0.04, 0.02), f/z = 50: Sigma2D = [[2.8, 1.5],
    [1.5, 2.8]], det = 5.59, so q(1, 1) = (2.8 + 2.8 - 3.0)/5.59 and
    q(1, -1) = (2.8 + 2.8 + 3.0)/5.59.  The lone Gaussian's colour (set to 1)
    at a pixel is o exp(-q/2)."""
    o = 0.9
    cam = identity_camera(fx=100.0, cx=31.5, cy=23.5)
    sc = one_gaussian((0, 0, 2.0), (0.04, 0.02, 0.01), quat_about((0, 0, 1), math.pi / 4), opac=o, colour=(1, 1, 1))
    rgb, _, _, _ = oracle.render_view(cam, sc, np.zeros(1))
    img = rgb[0]
    assert img[23, 31] == pytest.approx(o, rel=1e-6)                      # centre pixel: q = 0
    assert img[24, 32] == pytest.approx(o * math.exp(-0.5 * 2.6 / 5.59), rel=1e-5)   # (+1, +1)
    assert img[22, 30] == pytest.approx(o * math.exp(-0.5 * 2.6 / 5.59), rel=1e-5)   # (-1, -1)
    assert img[22, 32] == pytest.approx(o * math.exp(-0.5 * 8.6 / 5.59), rel=1e-5)   # (+1, -1)
    assert img[24, 30] == pytest.approx(o * math.exp(-0.5 * 8.6 / 5.59), rel=1e-5)   # (-1, +1)
    assert img[23, 32] == pytest.approx(o * math.exp(-0.5 * 2.8 / 5.59), rel=1e-5)   # (+1, 0)


def pin_off_axis_jacobian():
    s = 0.03
    for (x, y, z), fx, fy in [((0.5, 0.0, 2.0), 100.0, 100.0), ((0.0, -0.4, 1.5), 100.0, 100.0),
                              ((0.6, -0.3, 2.5), 120.0, 70.0), ((-0.8, 0.5, 3.0), 90.0, 90.0)]:
        cam = identity_camera(W=96, H=64, fx=fx, fy=fy, cx=47.5, cy=31.5)
        S, (u, v, zz), st = sigma2d_from_oracle(cam, one_gaussian((x, y, z), (s, s, s)))
        assert st >= 1
        s2 = s * s
        assert_sigma(S, s2 * fx * fx * (1 / z ** 2 + x * x / z ** 4) + 0.3,
                     s2 * fx * fy * x * y / z ** 4,
                     s2 * fy * fy * (1 / z ** 2 + y * y / z ** 4) + 0.3)
        assert u == pytest.approx(fx * x / z + 47.5, rel=1e-6)
        assert v == pytest.approx(fy * y / z + 31.5, rel=1e-6)
        assert zz == pytest.approx(z, rel=1e-7)


def pin_jacobian_clamp():
    """x/z beyond 1.3 tan(fovx/2): the Jacobian's third column takes the
    clamped ratio lim = 1.3 tan(fovx/2), the centre keeps x/z."""
    s, z, f = 0.03, 2.0, 40.0
    cam = identity_camera(W=64, H=48, fx=f, cx=31.5, cy=23.5)      # tan(fovx/2) = 0.8, tan(fovy/2) = 0.6
    limx, limy = 1.3 * np.float32(0.8), 1.3 * np.float32(0.6)
    for x, y in [(3.0, 0.2), (-2.6, 0.0), (0.4, 2.2), (-3.5, -2.0)]:
        rx = max(-limx, min(limx, x / z))
        ry = max(-limy, min(limy, y / z))
        assert (rx != x / z) or (ry != y / z)
        S, (u, v, _), st = sigma2d_from_oracle(cam, one_gaussian((x, y, z), (s, s, s)))
        assert st >= 1
        s2 = s * s
        assert_sigma(S, s2 * f * f * (1 + rx * rx) / z ** 2 + 0.3,
                     s2 * f * f * rx * ry / z ** 2,
                     s2 * f * f * (1 + ry * ry) / z ** 2 + 0.3)
        assert u == pytest.approx(f * x / z + 31.5, rel=1e-6)
        assert v == pytest.approx(f * y / z + 23.5, rel=1e-6)


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return (w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2)


def pin_camera_rotation_equivariance():
    """A Gaussian given in camera coordinates (mean m, rotation q) and the same
    Gaussian moved to the world by a camera pose (Rc, tc) -- mean
    Rc^T (m - tc), rotation conj(q_Rc) q -- project to the same image
    quantities under that pose as under the identity pose."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(11)
    for _ in range(12):
        m = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.4, 0.4), rng.uniform(1.5, 3.0)])
        qg = rng.normal(size=4)
        qg /= np.linalg.norm(qg)
        sc = np.exp(rng.normal(-3.5, 0.4, size=3))
        cam0 = identity_camera(W=96, H=64, fx=70.0, fy=70.0, cx=47.5, cy=31.5)
        S0, (u0, v0, z0), st0 = sigma2d_from_oracle(cam0, one_gaussian(m, sc, qg))
        # camera pose: world -> camera rotation Rc, translation tc
        rc = Rot.random(random_state=int(rng.integers(1 << 30)))
        Rc = rc.as_matrix()
        tc = rng.normal(size=3)
        xq = rc.as_quat()                          # x, y, z, w of Rc
        q_rc = (xq[3], xq[0], xq[1], xq[2])
        q_w = _qmul((q_rc[0], -q_rc[1], -q_rc[2], -q_rc[3]), tuple(qg))   # Rc^T G
        m_w = Rc.T @ (m - tc)
        cam1 = identity_camera(W=96, H=64, fx=70.0, fy=70.0, cx=47.5, cy=31.5)
        cam1.R = Rc.astype(np.float32)
        cam1.t = tc.astype(np.float32)
        cam1.campos = (-Rc.T @ tc).astype(np.float32)
        S1, (u1, v1, z1), st1 = sigma2d_from_oracle(cam1, one_gaussian(m_w, sc, q_w))
        assert st0 == st1 == 1
        # float32 inputs of the world-frame case differ from the camera-frame
        # ones by one rounding of a rotated vector: relative ~1e-6 of |m|
        assert z1 == pytest.approx(z0, rel=2e-6, abs=2e-6)
        assert u1 == pytest.approx(u0, abs=5e-4) and v1 == pytest.approx(v0, abs=5e-4)
        assert_sigma(S1, S0[0, 0], S0[0, 1], S0[1, 1], rtol=3e-5)


def pin_footprint_image():
    """The lone Gaussian's colour image equals o exp(-q/2) with q from the
    closed-form Sigma2D of a 30-degree rotation about z, and 0 where q > 9."""
    s1, s2 = 0.05, 0.015
    f, z, o = 100.0, 2.0, 0.7
    th = math.radians(30.0)
    c, s = math.cos(th), math.sin(th)
    k = (f / z) ** 2
    Sig = np.array([[k * (c * c * s1 * s1 + s * s * s2 * s2) + 0.3, k * c * s * (s1 * s1 - s2 * s2)],
                    [k * c * s * (s1 * s1 - s2 * s2), k * (s * s * s1 * s1 + c * c * s2 * s2) + 0.3]])
    P = np.linalg.inv(Sig)
    cam = identity_camera(W=40, H=32, fx=f, cx=19.3, cy=15.8)
    sc = one_gaussian((0, 0, z), (s1, s2, 0.01), quat_about((0, 0, 1), th), opac=o, colour=(1, 1, 1))
    rgb, _, _, _ = oracle.render_view(cam, sc, np.zeros(1))
    jj, ii = np.mgrid[0:32, 0:40]
    dx = ii + 0.5 - 19.3
    dy = jj + 0.5 - 15.8
    q = P[0, 0] * dx * dx + 2 * P[0, 1] * dx * dy + P[1, 1] * dy * dy
    inside = q < 9.0 * (1 - 1e-4)
    outside = q > 9.0 * (1 + 1e-4)
    assert inside.sum() > 40 and outside.sum() > 100
    np.testing.assert_allclose(rgb[0][inside], o * np.exp(-0.5 * q[inside]), rtol=2e-5)
    assert np.all(rgb[0][outside] == 0.0)


PINS = [pin_rotation_about_z, pin_rotation_about_x, pin_random_quaternions_against_scipy,
        pin_conic_worked_example, pin_off_axis_jacobian, pin_jacobian_clamp,
        pin_camera_rotation_equivariance, pin_footprint_image]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_projection_pin(pin):
    pin()


# --------------------------------------------------------------------------- planted mistakes

# (name, exact source text in the oracle, replacement): each one a plausible
# slip in the projection or the footprint value
MUTANTS = [
    ("rotation transposed", "M[3 * i + j] = G[3 * i + j] * scale[j];", "M[3 * i + j] = G[3 * j + i] * scale[j];"),
    ("S R instead of R S", "M[3 * i + j] = G[3 * i + j] * scale[j];", "M[3 * i + j] = G[3 * i + j] * scale[i];"),
    ("sign of wz", "G[1] = 2.0f * (xy - wz);", "G[1] = 2.0f * (xy + wz);"),
    ("sign of wx", "G[7] = 2.0f * (yz + wx);", "G[7] = 2.0f * (yz - wx);"),
    ("conic off-diagonal sign", "o->B = -b / det;", "o->B = b / det;"),
    ("Jacobian J02 dropped", "J02 = -((fx * ctx) / tz2);", "J02 = 0.0f * ctx;"),
    ("Jacobian J12 dropped", "J12 = -((fy * cty) / tz2);", "J12 = 0.0f * cty;"),
    ("no 1.3 tan clamp", "float ctx = fminf(limx, fmaxf(-limx, txz)) * tz;", "float ctx = txz * tz;"),
    ("fx and fy swapped in J", "float J11 = fy / tz,", "float J11 = fx / tz,"),
    ("camera rotation transposed", "T01 = J00 * R[1] + J02 * R[7]", "T01 = J00 * R[3] + J02 * R[7]"),
    ("cross term of q halved", "float B2 = p->B + p->B;", "float B2 = p->B;"),
    ("dilation missing", "float c = ((U10 * T10 + U11 * T11) + U12 * T12) + 0.3f;",
     "float c = ((U10 * T10 + U11 * T11) + U12 * T12);"),
]


def _build_mutant(src, tmpdir, idx):
    path = os.path.join(tmpdir, f"mutant{idx}.c")
    with open(path, "w") as f:
        f.write(src)
    so = os.path.join(tmpdir, f"libmutant{idx}.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    path, "-o", so, "-lm"], check=True, capture_output=True)
    import ctypes
    L = ctypes.CDLL(so)
    oracle._declare(L)
    return L


def test_planted_mistakes_are_caught(tmp_path, monkeypatch):
    with open(oracle._SRC) as f:
        base = f.read()
    oracle.lib()
    caught = {}
    for idx, (name, old, new) in enumerate(MUTANTS):
        assert base.count(old) == 1, f"mutation site not unique or missing: {name}"
        L = _build_mutant(base.replace(old, new), str(tmp_path), idx)
        monkeypatch.setattr(oracle, "_lib", L)
        failed = []
        for pin in PINS:
            try:
                pin()
            except AssertionError:
                failed.append(pin.__name__)
        monkeypatch.undo()
        caught[name] = failed
    missed = [n for n, f in caught.items() if not f]
    assert not missed, f"planted mistakes no pin catches: {missed}; caught: {caught}"
