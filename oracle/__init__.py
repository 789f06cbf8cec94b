"""CPU oracle for the GAVIS hot path (arxiv 2605.30342).

TEST INFRASTRUCTURE ONLY: imported by the tests, by `__graft_entry__.smoke()`
and by the CPU-baseline leg of `bench.py`; the product library never loads it.

The arithmetic lives in `gavis_oracle.c` (plain C, float32 geometry with one
rounding per operation, float64 values).  This wrapper only marshals numpy
arrays through ctypes and compiles the C file with gcc on first use.

Paper anchors:
  vf_build     -- Alg. "Anisotropic Visibility Field Construction" with
                  Alg. "Single-view Particle Visibility" (eq:vis_gamma)
  vf_query     -- Alg. "Query Anisotropic Visibility Field" (eq:vis_sh,
                  eq:vis_bound)
  render_view  -- Alg. "3DGS Uncertainty Quantification with Visibility Field"
                  (eq:alpha_comp, eq:huber) and eq:orig_vr for colour
  score_views  -- eq:id with no correlation correction, argmax of eq:i_gain
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gavis_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

DEFAULTS = dict(kappa=1.0, eps_T=1e-4, q_cut=9.0, beta=0.5, o0=0.15,
                sigma_c2=0.01, logdet_Q0=0.0, tile=16, margin=1e-3)
_PKEYS = ["kappa", "eps_T", "q_cut", "beta", "o0", "sigma_c2", "logdet_Q0", "tile", "margin"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  Float contraction
    is off so that float32 geometry rounds once per operation."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _declare(L):
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
    L.oracle_bessel_i.argtypes = [i32, dbl]
    L.oracle_bessel_i.restype = dbl
    L.oracle_sh_complex.argtypes = [i32, i32, vp, vp, vp]
    L.oracle_sh_real.argtypes = [i32, vp, vp]
    L.oracle_vmf_coeffs.argtypes = [i32, dbl, vp]
    L.oracle_project.argtypes = [i64, vp, vp, vp, vp, dbl, i32, vp, vp]
    L.oracle_bins.argtypes = [i32, vp, i64, vp, vp, vp, dbl, i32, vp, vp, i64]
    L.oracle_bins.restype = i64
    L.oracle_ranges.argtypes = [i64, vp, i64, vp]
    L.oracle_pixel_lists.argtypes = [vp, i64, vp, vp, vp, dbl, i32, i32, vp, vp, i64]
    L.oracle_pixel_lists.restype = i64
    L.oracle_composite.argtypes = [i64, vp, vp, vp, vp, vp, vp, vp]
    L.oracle_vf_query.argtypes = [i64, vp, i32, i64, vp, vp, vp, vp]
    L.oracle_vf_exact.argtypes = [i64, i32, vp, vp, dbl, vp, vp]
    L.oracle_visibility_view.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.oracle_visibility_view.restype = i64
    L.oracle_vf_build.argtypes = [i32, vp, i64, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]
    L.oracle_render_view.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.oracle_density_control.argtypes = [i32, vp, i64, vp, vp, vp, vp, i64, vp, dbl, dbl, dbl, vp, vp, vp, vp, vp, vp]
    L.oracle_density_control.restype = i64


# ----------------------------------------------------------------------------
# marshalling
# ----------------------------------------------------------------------------

def params(**kw) -> np.ndarray:
    d = dict(DEFAULTS)
    d.update(kw)
    return np.array([float(d[k]) for k in _PKEYS], np.float64)


def cam_record(cam) -> np.ndarray:
    r = np.zeros(24, np.float32)
    r[0], r[1] = cam.W, cam.H
    r[2:8] = [cam.fx, cam.fy, cam.cx, cam.cy, cam.tan_half_fovx, cam.tan_half_fovy]
    r[8:17] = np.asarray(cam.R, np.float32).reshape(9)
    r[17:20] = cam.t
    r[20:23] = cam.campos
    r[23] = cam.znear
    return r


def cam_records(cams) -> np.ndarray:
    return np.ascontiguousarray(np.stack([cam_record(c) for c in cams]))


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


# ----------------------------------------------------------------------------
# special functions
# ----------------------------------------------------------------------------

def bessel_i(l: int, x: float) -> float:
    return lib().oracle_bessel_i(int(l), float(x))


def vmf_coeffs(L: int, kappa: float) -> np.ndarray:
    a = np.zeros(L + 1, np.float64)
    lib().oracle_vmf_coeffs(L, float(kappa), _p(a))
    return a


def sh_complex(l: int, m: int, d) -> complex:
    d = _f64(d)
    re, im = np.zeros(1), np.zeros(1)
    lib().oracle_sh_complex(l, m, _p(d), _p(re), _p(im))
    return complex(re[0], im[0])


def sh_real(L: int, d) -> np.ndarray:
    d = _f64(d)
    Y = np.zeros((L + 1) ** 2, np.float64)
    lib().oracle_sh_real(L, _p(d), _p(Y))
    return Y


# ----------------------------------------------------------------------------
# geometry and bins
# ----------------------------------------------------------------------------

def project(cam, scene, q_cut=9.0, tile=16):
    rec = cam_record(cam)
    n = scene.n
    out = np.zeros((n, 12), np.float32)
    st = np.zeros(n, np.int32)
    lib().oracle_project(n, _p(rec), _p(_f32(scene.means)), _p(_f32(scene.scales)),
                         _p(_f32(scene.rots)), float(q_cut), int(tile), _p(out), _p(st))
    return out, st


def bins(cams, scene, q_cut=9.0, tile=16):
    """Sorted (keys, vals) over all views, canonical order."""
    recs = cam_records(cams)
    args = (len(cams), _p(recs), scene.n, _p(_f32(scene.means)), _p(_f32(scene.scales)),
            _p(_f32(scene.rots)), float(q_cut), int(tile))
    M = lib().oracle_bins(*args, None, None, 0)
    keys = np.zeros(max(M, 1), np.uint64)
    vals = np.zeros(max(M, 1), np.uint32)
    lib().oracle_bins(*args, _p(keys), _p(vals), M)
    return keys[:M], vals[:M]


def ranges(keys, ntiles):
    keys = np.ascontiguousarray(keys, np.uint64)
    r = np.zeros(2 * ntiles, np.uint32)
    lib().oracle_ranges(len(keys), _p(keys), ntiles, _p(r))
    return r.reshape(ntiles, 2)


def pixel_lists(cam, scene, q_cut=9.0, tile=16, brute=False):
    rec = cam_record(cam)
    npix = cam.W * cam.H
    start = np.zeros(npix + 1, np.int64)
    args = [_p(rec), scene.n, _p(_f32(scene.means)), _p(_f32(scene.scales)), _p(_f32(scene.rots)),
            float(q_cut), int(tile), int(bool(brute)), _p(start)]
    tot = lib().oracle_pixel_lists(*args, None, 0)
    ent = np.zeros(max(tot, 1), np.uint64)
    lib().oracle_pixel_lists(*args[:-1], _p(start), _p(ent), tot)
    return start, ent[:tot]


# ----------------------------------------------------------------------------
# compositing, visibility field
# ----------------------------------------------------------------------------

def composite(alpha, V, col, prm=None, kc=None, z=None):
    """One pixel over an explicit list; returns dict of the outputs.  kc:
    optional per-entry 1/2 log((2 pi e)^3 |Q_c|); z: optional per-entry
    camera depths (for the expected depth)."""
    prm = params() if prm is None else prm
    alpha, V = _f64(alpha), _f64(V)
    col = _f64(np.asarray(col).reshape(-1, 3))
    kc = None if kc is None else _f64(kc)
    z = None if z is None else _f64(z)
    res = np.zeros(24)
    lib().oracle_composite(len(alpha), _p(alpha), _p(V), _p(col), _p(z) if z is not None else None, _p(prm),
                           _p(kc) if kc is not None else None, _p(res))
    return dict(H=res[0], rgb=res[1:4].copy(), T=res[4], Tc=res[5], sum_w=res[6], sum_wc=res[7],
                w0=res[8], used=int(res[9]), amb=bool(res[10]), depth=res[11],
                H_lo=res[12], H_hi=res[13], rgb_lo=res[14:17].copy(), rgb_hi=res[17:20].copy(),
                depth_lo=res[20], depth_hi=res[21])


def vf_query(gamma, L, P, cam, means):
    gamma = _f64(gamma)
    n = gamma.shape[0]
    V = np.zeros(n)
    vt = np.zeros(n)
    lib().oracle_vf_query(n, _p(gamma), int(L), int(P), _p(_f32(cam.campos)), _p(_f32(means)),
                          _p(V), _p(vt))
    return V, vt


def vf_exact(vis, dirs, kappa, d):
    """eq:vis_all from per-view visibilities vis (P,n), directions dirs (P,n,3)
    and query directions d (n,3)."""
    vis, dirs, d = _f64(vis), _f64(dirs), _f64(d)
    P, n = vis.shape
    V = np.zeros(n)
    lib().oracle_vf_exact(n, P, _p(vis), _p(dirs), float(kappa), _p(d), _p(V))
    return V


def visibility_view(cam, scene, prm=None, want_bounds=False):
    """Per-Gaussian sum of T and count of one view, the near-threshold mask and
    the number of pairs; with want_bounds also a dict of the early sums and
    the early and late counts (the run's range of possible stops)."""
    prm = params() if prm is None else prm
    n = scene.n
    sumT = np.zeros(n)
    cnt = np.zeros(n, np.int64)
    amb = np.zeros(n, np.uint8)
    se, ce, cl = np.zeros(n), np.zeros(n, np.int64), np.zeros(n, np.int64)
    bargs = [_p(se), _p(ce), _p(cl)] if want_bounds else [None, None, None]
    pairs = lib().oracle_visibility_view(_p(cam_record(cam)), n, _p(_f32(scene.means)), _p(_f32(scene.scales)),
                                         _p(_f32(scene.rots)), _p(_f32(scene.opac)), _p(prm),
                                         _p(sumT), _p(cnt), _p(amb), *bargs)
    if want_bounds:
        return sumT, cnt, amb.astype(bool), pairs, dict(sum_early=se, cnt_early=ce, cnt_late=cl)
    return sumT, cnt, amb.astype(bool), pairs


def vf_build(cams, scene, L, prm=None, want_vis=False, want_rad=False):
    """gamma (n,(L+1)^2) float64, ambiguous mask (n,), per-view vis (P,n) or
    None; with want_rad also the per-coefficient radius (n,(L+1)^2) within
    which a build with rounding-sensitive terminations stays."""
    prm = params() if prm is None else prm
    n = scene.n
    K = (L + 1) ** 2
    gamma = np.zeros((n, K))
    amb = np.zeros(n, np.uint8)
    vis = np.zeros((len(cams), n)) if want_vis else None
    rad = np.zeros((n, K)) if want_rad else None
    lib().oracle_vf_build(len(cams), _p(cam_records(cams)), n, _p(_f32(scene.means)), _p(_f32(scene.scales)),
                          _p(_f32(scene.rots)), _p(_f32(scene.opac)), int(L), _p(prm), _p(gamma),
                          _p(vis) if want_vis else None, _p(amb), _p(rad) if want_rad else None)
    if want_rad:
        return gamma, amb.astype(bool), vis, rad
    return gamma, amb.astype(bool), vis


def virtual_scale(rho, eta):
    """s with (4/3) pi s^3 rho = 1 + eta (Alg. Visibility Field Density Control)."""
    return (3.0 * (1.0 + eta) / (4.0 * np.pi * rho)) ** (1.0 / 3.0)


def density_control(cams, scene, vmeans, rho=100.0, eta=0.5, eps_v=0.95, prm=None, want_bounds=False):
    """Multi-view visibility of the virtual particles (float64), keep mask
    (visibility <= eps_v) and the rounding-ambiguity mask; with want_bounds
    also the range (lo, hi) of the visibility under rounding-sensitive
    terminations."""
    prm = params() if prm is None else prm
    vm = _f32(vmeans).reshape(-1, 3)
    nv = vm.shape[0]
    vis = np.zeros(nv)
    keep = np.zeros(nv, np.uint8)
    amb = np.zeros(nv, np.uint8)
    lo, hi = np.zeros(nv), np.zeros(nv)
    lib().oracle_density_control(len(cams), _p(cam_records(cams)), scene.n, _p(_f32(scene.means)),
                                 _p(_f32(scene.scales)), _p(_f32(scene.rots)), _p(_f32(scene.opac)), nv, _p(vm),
                                 float(rho), float(eta), float(eps_v), _p(prm), _p(vis), _p(keep), _p(amb),
                                 _p(lo), _p(hi))
    if want_bounds:
        return vis, keep.astype(bool), amb.astype(bool), lo, hi
    return vis, keep.astype(bool), amb.astype(bool)


def render_view(cam, scene, V, prm=None, sh=None, sh_var=None, want_depth=False, want_bounds=False):
    """rgb (3,H,W), unc (H,W), amb (H,W) bool, used (H,W) [, depth (H,W) if
    want_depth] [, bounds dict if want_bounds: the least and greatest value
    of unc, rgb and depth per pixel when the transmittance tests near eps_T
    go either way].  sh_var: optional per-coefficient colour variances
    (FisherRF variant of Q_c)."""
    prm = params() if prm is None else prm
    n = scene.n
    sh = _f64(scene.sh if sh is None else sh)
    var = None if sh_var is None else _f64(sh_var)
    Lc = int(round(np.sqrt(sh.shape[1]))) - 1
    rgb = np.zeros((3, cam.H, cam.W))
    unc = np.zeros((cam.H, cam.W))
    amb = np.zeros((cam.H, cam.W), np.uint8)
    used = np.zeros((cam.H, cam.W), np.int32)
    depth = np.zeros((cam.H, cam.W)) if want_depth else None
    bnd = np.zeros((10, cam.H, cam.W)) if want_bounds else None
    lib().oracle_render_view(_p(cam_record(cam)), n, _p(_f32(scene.means)), _p(_f32(scene.scales)),
                             _p(_f32(scene.rots)), _p(_f32(scene.opac)), _p(sh), _p(var) if var is not None else None,
                             Lc, _p(_f64(V)), _p(prm),
                             _p(rgb), _p(unc), _p(depth) if want_depth else None, _p(amb), _p(used),
                             _p(bnd) if want_bounds else None)
    out = [rgb, unc, amb.astype(bool), used]
    if want_depth:
        out.append(depth)
    if want_bounds:
        out.append(dict(unc_lo=bnd[0], unc_hi=bnd[1], rgb_lo=bnd[2:5], rgb_hi=bnd[5:8],
                        depth_lo=bnd[8], depth_hi=bnd[9]))
    return tuple(out)


def score_views(scene, gamma, L, P, cams, prm=None, sh=None, keep_images=True, sh_var=None, want_depth=False):
    """Per-view mean entropy score S_v (eq:id with f_corr = 0) and the argmax
    of eq:i_gain (ties to the lowest index).  Also the per-pixel bounds of
    render_view ("bnd") and the range of each score under rounding-sensitive
    terminations ("score_lo", "score_hi")."""
    prm = params() if prm is None else prm
    out = dict(rgb=[], unc=[], amb=[], used=[], depth=[], bnd=[], score=np.zeros(len(cams)),
               score_lo=np.zeros(len(cams)), score_hi=np.zeros(len(cams)))
    for v, cam in enumerate(cams):
        V, _ = vf_query(gamma, L, P, cam, scene.means)
        r = render_view(cam, scene, V, prm, sh, sh_var, want_depth=want_depth, want_bounds=True)
        rgb, unc, amb, used = r[:4]
        bnd = r[-1]
        if want_depth and keep_images:
            out["depth"].append(r[4])
        out["score"][v] = unc.mean()
        out["score_lo"][v] = bnd["unc_lo"].mean()
        out["score_hi"][v] = bnd["unc_hi"].mean()
        if keep_images:
            out["rgb"].append(rgb)
            out["unc"].append(unc)
            out["amb"].append(amb)
            out["used"].append(used)
            out["bnd"].append(bnd)
    out["best"] = int(np.argmax(out["score"])) if len(cams) else -1
    return out
