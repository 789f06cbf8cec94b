"""GB300-native GAVIS hot path: Python binding of the C ABI (include/gavis.h).

This module only marshals arguments: torch tensors become device pointers,
camera objects become `gavis_camera` records, and every step of the method
runs in the CUDA library `libgavis.so`.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.

    import paper_2605_30342_gb300 as gv
    ctx = gv.Context()
    gs = gv.Gaussians(means, scales, rots, opac, sh, sh_degree)      # cuda tensors
    vf = ctx.vf_build(gs, train_cams, degree=2)                      # eq:vis_gamma
    out = ctx.score_views(gs, vf, cand_cams)                         # Alg. UQ + argmax
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

__all__ = ["Context", "Gaussians", "VisibilityField", "Params", "GavisError", "Server", "load", "library_path",
           "F32", "F16", "BF16"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "libgavis.so")
_lock = threading.Lock()
_lib = None

F32, F16, BF16 = 0, 1, 2
_TORCH_DTYPE = {F32: torch.float32, F16: torch.float16, BF16: torch.bfloat16}
_DTYPE_CODE = {torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_BUDGET, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5


class GavisError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gavis error {code}: {msg}")
        self.code = code


class gavis_camera(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("tan_half_fovx", C.c_float), ("tan_half_fovy", C.c_float),
                ("R", C.c_float * 9), ("t", C.c_float * 3), ("campos", C.c_float * 3), ("znear", C.c_float)]


class gavis_gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("scales", C.c_void_p), ("rots", C.c_void_p),
                ("opac", C.c_void_p), ("sh", C.c_void_p), ("sh_degree", C.c_int32), ("sh_dtype", C.c_int32),
                ("sh_var", C.c_void_p)]


class gavis_vf(C.Structure):
    _fields_ = [("n", C.c_int64), ("coeffs", C.c_void_p), ("degree", C.c_int32), ("dtype", C.c_int32),
                ("n_train_views", C.c_int32), ("kappa", C.c_float)]


class gavis_params(C.Structure):
    _fields_ = [("kappa", C.c_float), ("vf_degree", C.c_int32), ("eps_T", C.c_float), ("q_cut", C.c_float),
                ("beta", C.c_float), ("o0", C.c_float), ("sigma_c2", C.c_float), ("logdet_Q0", C.c_float),
                ("tile", C.c_int32), ("views_per_batch", C.c_int32), ("tile_lists", C.c_int32)]


class gavis_views_out(C.Structure):
    _fields_ = [("rgb", C.c_void_p), ("unc", C.c_void_p), ("depth", C.c_void_p), ("score", C.c_void_p),
                ("best_dev", C.c_void_p), ("best_host", C.c_void_p)]


EXPORTS = ["gavis_ctx_create", "gavis_ctx_destroy", "gavis_last_error", "gavis_params_default",
           "gavis_vmf_coeffs", "gavis_vf_build", "gavis_score_views", "gavis_vf_query", "gavis_debug_bins",
           "gavis_debug_visibility", "gavis_prof_enable", "gavis_prof_read", "gavis_vf_density_control",
           "gavis_server_create", "gavis_server_destroy", "gavis_server_last_error", "gavis_server_add_scene",
           "gavis_server_submit", "gavis_server_wait", "gavis_server_stats", "gavis_autotune",
           "gavis_plan_create", "gavis_plan_launch", "gavis_plan_overflowed", "gavis_plan_kernels",
           "gavis_plan_destroy", "gavis_render_views", "gavis_augment", "gavis_server_pause"]

STAGES = ["project", "scan", "emit", "sort", "ranges", "composite_ua", "composite_vis", "reduce", "vf_accum"]


def library_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Load libgavis.so (built by `__graft_entry__.build()` or
    `python -m paper_2605_30342_gb300.build`).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libgavis.so not built ({p}); run __graft_entry__.build()")
        lib = C.CDLL(p)
        vp, i32, i64 = C.c_void_p, C.c_int, C.c_int64
        lib.gavis_ctx_create.argtypes = [C.POINTER(vp), i32, C.c_size_t]
        lib.gavis_ctx_destroy.argtypes = [vp]
        lib.gavis_ctx_destroy.restype = None
        lib.gavis_last_error.argtypes = [vp]
        lib.gavis_last_error.restype = C.c_char_p
        lib.gavis_params_default.argtypes = [C.POINTER(gavis_params)]
        lib.gavis_vmf_coeffs.argtypes = [i32, C.c_double, C.POINTER(C.c_double)]
        lib.gavis_vf_build.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_camera), i32,
                                       C.POINTER(gavis_params), C.POINTER(gavis_vf), i32, vp]
        lib.gavis_score_views.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf),
                                          C.POINTER(gavis_camera), i32, C.POINTER(gavis_params), vp, vp, vp, vp,
                                          C.POINTER(C.c_int32), vp]
        lib.gavis_vf_query.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf), C.POINTER(gavis_camera),
                                       i32, C.POINTER(gavis_params), vp, vp]
        lib.gavis_debug_bins.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_camera), i32,
                                         C.POINTER(gavis_params), vp, vp, i64, C.POINTER(C.c_int64), vp, vp]
        lib.gavis_debug_visibility.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_camera), i32,
                                               C.POINTER(gavis_params), vp, vp, vp]
        lib.gavis_vf_density_control.argtypes = [vp, C.POINTER(gavis_gaussians), vp, i64, C.POINTER(gavis_camera), i32,
                                                 C.POINTER(gavis_params), C.c_float, C.c_float, C.c_float, vp, vp, vp,
                                                 C.POINTER(C.c_int64), C.POINTER(C.c_float), vp]
        lib.gavis_augment.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf), vp, i64, C.c_float,
                                      vp, vp, vp, vp, vp, vp, vp, vp]
        lib.gavis_server_create.argtypes = [C.POINTER(vp), i32, C.c_size_t, i32, i32]
        lib.gavis_server_destroy.argtypes = [vp]
        lib.gavis_server_destroy.restype = None
        lib.gavis_server_last_error.argtypes = [vp]
        lib.gavis_server_last_error.restype = C.c_char_p
        lib.gavis_server_add_scene.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf), C.POINTER(C.c_int)]
        lib.gavis_server_submit.argtypes = [vp, i32, C.POINTER(gavis_camera), i32, C.POINTER(gavis_params), vp, vp,
                                            C.POINTER(C.c_int64)]
        lib.gavis_server_wait.argtypes = [vp, i64, i32, C.POINTER(C.c_int32), C.POINTER(C.c_double)]
        lib.gavis_server_pause.argtypes = [vp, i32]
        lib.gavis_server_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                           C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
        lib.gavis_autotune.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf), C.POINTER(gavis_camera), i32,
                                       i32, C.POINTER(gavis_params), C.POINTER(C.c_double), vp]
        lib.gavis_render_views.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf),
                                           C.POINTER(gavis_camera), i32, C.POINTER(gavis_params),
                                           C.POINTER(gavis_views_out), vp]
        lib.gavis_plan_create.argtypes = [vp, C.POINTER(gavis_gaussians), C.POINTER(gavis_vf), i32, i32, i32,
                                          C.POINTER(gavis_params), i64, i64, vp, vp, vp, vp, C.POINTER(vp)]
        lib.gavis_plan_launch.argtypes = [vp, C.POINTER(gavis_camera), vp]
        lib.gavis_plan_overflowed.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.gavis_plan_kernels.argtypes = [vp]
        lib.gavis_plan_kernels.restype = i64
        lib.gavis_plan_destroy.argtypes = [vp]
        lib.gavis_plan_destroy.restype = None
        lib.gavis_prof_enable.argtypes = [vp, i32]
        lib.gavis_prof_read.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_uint64)]
        _lib = lib
        return lib


# ----------------------------------------------------------------------------
# argument marshalling
# ----------------------------------------------------------------------------

def Params(**kw) -> gavis_params:
    """Paper defaults (gavis_params_default) with keyword overrides."""
    p = gavis_params()
    load().gavis_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def camera_records(cams) -> C.Array:
    """Any objects with W, H, fx, fy, cx, cy, tan_half_fovx, tan_half_fovy,
    R (3x3), t (3), campos (3) and znear attributes."""
    arr = (gavis_camera * max(len(cams), 1))()
    for i, c in enumerate(cams):
        r = arr[i]
        r.W, r.H = int(c.W), int(c.H)
        r.fx, r.fy, r.cx, r.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        r.tan_half_fovx, r.tan_half_fovy = float(c.tan_half_fovx), float(c.tan_half_fovy)
        R = [float(x) for row in c.R for x in row]
        for k in range(9):
            r.R[k] = R[k]
        for k in range(3):
            r.t[k] = float(c.t[k])
            r.campos[k] = float(c.campos[k])
        r.znear = float(getattr(c, "znear", 0.2))
    return arr


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dev(t: torch.Tensor, name: str, dtype=None) -> int:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


class Gaussians:
    """Structure-of-arrays Gaussian scene resident on the device."""

    def __init__(self, means, scales, rots, opac, sh=None, sh_degree=None, sh_var=None):
        """sh_var: optional variances of the colour coefficients (same shape and
        dtype as sh) for the per-Gaussian colour covariance."""
        self.means, self.scales, self.rots, self.opac, self.sh, self.sh_var = means, scales, rots, opac, sh, sh_var
        self.n = int(means.shape[0])
        if sh is not None and sh_degree is None:
            sh_degree = int(round(sh.shape[1] ** 0.5)) - 1
        self.sh_degree = int(sh_degree or 0)
        s = gavis_gaussians()
        s.n = self.n
        s.means = _dev(means, "means", torch.float32)
        s.scales = _dev(scales, "scales", torch.float32)
        s.rots = _dev(rots, "rots", torch.float32)
        s.opac = _dev(opac, "opac", torch.float32)
        s.sh = _dev(sh, "sh") if sh is not None else None
        s.sh_degree = self.sh_degree
        s.sh_dtype = _DTYPE_CODE[sh.dtype] if sh is not None else 0
        if sh_var is not None:
            if sh is None or sh_var.shape != sh.shape or sh_var.dtype != sh.dtype:
                raise ValueError("sh_var must match sh in shape and dtype")
            s.sh_var = _dev(sh_var, "sh_var")
        else:
            s.sh_var = None
        self.struct = s

    @classmethod
    def from_numpy(cls, scene, device="cuda", sh_dtype=torch.float32):
        t = lambda a, dt=torch.float32: torch.as_tensor(a).to(device=device, dtype=dt).contiguous()
        return cls(t(scene.means), t(scene.scales), t(scene.rots), t(scene.opac),
                   t(scene.sh, sh_dtype), scene.sh_degree)


class VisibilityField:
    """gamma [n, (L+1)^2] on the device plus |P| and kappa."""

    def __init__(self, coeffs: torch.Tensor, degree: int, n_train_views: int, kappa: float):
        self.coeffs, self.degree, self.n_train_views, self.kappa = coeffs, int(degree), int(n_train_views), float(kappa)

    def struct(self) -> gavis_vf:
        s = gavis_vf()
        s.n = int(self.coeffs.shape[0])
        s.coeffs = _dev(self.coeffs, "coeffs")
        s.degree = self.degree
        s.dtype = _DTYPE_CODE[self.coeffs.dtype]
        s.n_train_views = self.n_train_views
        s.kappa = self.kappa
        return s


class Context:
    """A device context with a bounded, grow-only workspace."""

    def __init__(self, device: int = 0, budget_bytes: int = 0):
        self._lib = load()
        self._h = C.c_void_p()
        rc = self._lib.gavis_ctx_create(C.byref(self._h), int(device), C.c_size_t(int(budget_bytes)))
        if rc != OK:
            raise GavisError(rc, f"gavis_ctx_create(device={device}) failed")
        self.device = device

    def close(self):
        if self._h:
            self._lib.gavis_ctx_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise GavisError(rc, self._lib.gavis_last_error(self._h).decode())

    @staticmethod
    def vmf_coeffs(L: int, kappa: float):
        a = (C.c_double * (L + 1))()
        rc = load().gavis_vmf_coeffs(int(L), float(kappa), a)
        if rc != OK:
            raise GavisError(rc, "gavis_vmf_coeffs")
        return list(a)

    # -------------------------------------------------------------- VF CONST
    def vf_build(self, gs: Gaussians, train_cams, degree: int = 2, dtype=torch.float32, params=None,
                 out: VisibilityField | None = None, accumulate: bool = False, stream=None) -> VisibilityField:
        p = params or Params(vf_degree=degree)
        if out is None:
            coeffs = torch.zeros((gs.n, (degree + 1) ** 2), dtype=dtype, device=gs.means.device)
            out = VisibilityField(coeffs, degree, 0, float(p.kappa))
        vs = out.struct()
        cams = camera_records(train_cams)
        self._check(self._lib.gavis_vf_build(self._h, C.byref(gs.struct), cams, len(train_cams), C.byref(p),
                                             C.byref(vs), int(bool(accumulate)), _stream_ptr(stream)))
        out.n_train_views, out.kappa = int(vs.n_train_views), float(vs.kappa)
        return out

    # -------------------------------------------------------------- scoring
    def score_views(self, gs: Gaussians, vf: VisibilityField, cand_cams, params=None, want_rgb=True,
                    want_unc=True, out=None, sync_best=True, stream=None, want_depth=False):
        """Returns dict(score [n], best (int or device tensor), rgb [n,3,H,W], unc [n,H,W],
        depth [n,H,W] (expected depth, when want_depth))."""
        p = params or Params(vf_degree=vf.degree)
        n = len(cand_cams)
        dev = gs.means.device
        W, H = (int(cand_cams[0].W), int(cand_cams[0].H)) if n else (0, 0)
        out = out or {}
        rgb = out.get("rgb") if "rgb" in out else (torch.empty((n, 3, H, W), device=dev) if want_rgb else None)
        unc = out.get("unc") if "unc" in out else (torch.empty((n, H, W), device=dev) if want_unc else None)
        score = out.get("score") if "score" in out else torch.empty(n, device=dev)
        best_dev = out.get("best_dev") if "best_dev" in out else torch.empty(1, dtype=torch.int32, device=dev)
        depth = out.get("depth") if "depth" in out else (torch.empty((n, H, W), device=dev) if want_depth else None)
        best_host = C.c_int32(-1)
        vs = vf.struct()
        cams = camera_records(cand_cams)
        o = gavis_views_out()
        o.rgb = rgb.data_ptr() if rgb is not None else None
        o.unc = unc.data_ptr() if unc is not None else None
        o.depth = depth.data_ptr() if depth is not None else None
        o.score = score.data_ptr()
        o.best_dev = best_dev.data_ptr()
        o.best_host = C.cast(C.pointer(best_host), C.c_void_p) if sync_best else None
        self._check(self._lib.gavis_render_views(self._h, C.byref(gs.struct), C.byref(vs), cams, n, C.byref(p),
                                                 C.byref(o), _stream_ptr(stream)))
        return dict(score=score, best=int(best_host.value) if sync_best else best_dev, rgb=rgb, unc=unc,
                    depth=depth, best_dev=best_dev)

    def plan(self, gs: Gaussians, vf: VisibilityField, n_cams: int, W: int, H: int, entry_capacity: int,
             record_capacity: int = 0, params=None, want_rgb=False, want_unc=False) -> "Plan":
        """Candidate scoring captured as a CUDA graph (gavis_plan_create)."""
        return Plan(self, gs, vf, n_cams, W, H, record_capacity, entry_capacity, params, want_rgb, want_unc)

    def vf_query(self, gs: Gaussians, vf: VisibilityField, cams, params=None, stream=None):
        p = params or Params(vf_degree=vf.degree)
        V = torch.empty((len(cams), gs.n), device=gs.means.device)
        vs = vf.struct()
        self._check(self._lib.gavis_vf_query(self._h, C.byref(gs.struct), C.byref(vs), camera_records(cams),
                                             len(cams), C.byref(p), C.c_void_p(V.data_ptr()), _stream_ptr(stream)))
        return V

    # -------------------------------------------------------------- autotuner
    def autotune(self, gs: Gaussians, sample_cams, vf: VisibilityField | None = None, params=None, stream=None):
        """Pick the tile edge for scoring (vf given) or field construction
        (vf None) on sample cameras; returns (params, best_ms)."""
        p = params or Params(vf_degree=vf.degree if vf is not None else 2)
        ms = C.c_double(0.0)
        vs = vf.struct() if vf is not None else None
        self._check(self._lib.gavis_autotune(self._h, C.byref(gs.struct), C.byref(vs) if vs is not None else None,
                                             camera_records(sample_cams), len(sample_cams), 0 if vf is not None else 1,
                                             C.byref(p), C.byref(ms), _stream_ptr(stream)))
        return p, float(ms.value)

    # -------------------------------------------------------------- density control
    def density_control(self, gs: Gaussians, virt_means: torch.Tensor, train_cams, rho: float = 100.0,
                        eta: float = 0.5, eps_v: float = 0.95, params=None, stream=None):
        """Alg. "Visibility Field Density Control": returns dict(vis [n_virt],
        keep [n_virt] bool, kept_means [n_keep, 3], n_keep, scale)."""
        p = params or Params()
        vm = virt_means.contiguous()
        nv = int(vm.shape[0])
        vis = torch.empty(nv, device=gs.means.device)
        keep = torch.empty(nv, dtype=torch.uint8, device=gs.means.device)
        kept = torch.empty((max(nv, 1), 3), device=gs.means.device)
        nk, scale = C.c_int64(0), C.c_float(0.0)
        self._check(self._lib.gavis_vf_density_control(
            self._h, C.byref(gs.struct), C.c_void_p(_dev(vm, "virt_means", torch.float32) if nv else None), nv,
            camera_records(train_cams), len(train_cams), C.byref(p), float(rho), float(eta), float(eps_v),
            C.c_void_p(vis.data_ptr() if nv else None), C.c_void_p(keep.data_ptr() if nv else None),
            C.c_void_p(kept.data_ptr()), C.byref(nk), C.byref(scale), _stream_ptr(stream)))
        n_keep = int(nk.value)
        return dict(vis=vis, keep=keep.bool(), kept_means=kept[:n_keep], n_keep=n_keep, scale=float(scale.value))

    def augment(self, gs: Gaussians, vf: VisibilityField, kept_means: torch.Tensor, scale: float, stream=None):
        """The scene used for uncertainty scoring after density control
        (gavis_augment): the trained Gaussians plus the kept virtual
        particles (identity rotation, isotropic `scale`, zero opacity, zero
        colour, gamma = 0 so V = 0).  Allocates the outputs only."""
        k = int(kept_means.shape[0])
        n = int(gs.means.shape[0])
        dev = gs.means.device
        km = kept_means.contiguous()
        means = torch.empty((n + k, 3), device=dev)
        scales = torch.empty((n + k, 3), device=dev)
        rots = torch.empty((n + k, 4), device=dev)
        opac = torch.empty(n + k, device=dev)
        sh = torch.empty((n + k,) + tuple(gs.sh.shape[1:]), dtype=gs.sh.dtype, device=dev)
        var = None if gs.sh_var is None else torch.empty_like(sh)
        coeffs = torch.empty((n + k, vf.coeffs.shape[1]), dtype=vf.coeffs.dtype, device=dev)
        self._check(self._lib.gavis_augment(
            self._h, C.byref(gs.struct), C.byref(vf.struct()),
            C.c_void_p(_dev(km, "kept_means", torch.float32) if k else None), k, float(scale),
            C.c_void_p(means.data_ptr()), C.c_void_p(scales.data_ptr()), C.c_void_p(rots.data_ptr()),
            C.c_void_p(opac.data_ptr()), C.c_void_p(sh.data_ptr()),
            C.c_void_p(var.data_ptr() if var is not None else None), C.c_void_p(coeffs.data_ptr()),
            _stream_ptr(stream)))
        return (Gaussians(means, scales, rots, opac, sh, gs.sh_degree, var),
                VisibilityField(coeffs, vf.degree, vf.n_train_views, vf.kappa))

    # -------------------------------------------------------------- instrumentation
    def prof_enable(self, on: bool = True, pairs: bool = False):
        """Stage timing on later calls; with pairs, also count the composited
        pixel-Gaussian pairs (device counters: slower)."""
        self._check(self._lib.gavis_prof_enable(self._h, (2 if pairs else 1) if on else 0))

    def prof_read(self):
        """dict(stage -> (ms, launches)), total kernel launches, pairs (ua, vis), tile entries (keys), visible
        records, and the tile entries whose lists were sorted (sorted_keys; the others were counted)."""
        ms = (C.c_double * len(STAGES))()
        la = (C.c_int64 * len(STAGES))()
        tot = C.c_int64(0)
        pairs = (C.c_uint64 * 5)()
        self._check(self._lib.gavis_prof_read(self._h, ms, la, C.byref(tot), pairs))
        return dict(stages={k: (ms[i], int(la[i])) for i, k in enumerate(STAGES)}, total_launches=int(tot.value),
                    pairs=(int(pairs[0]), int(pairs[1])), keys=int(pairs[2]), visible=int(pairs[3]),
                    sorted_keys=int(pairs[4]))

    # -------------------------------------------------------------- verification hooks
    def debug_bins(self, gs: Gaussians, cams, params=None, cap=None, stream=None):
        p = params or Params()
        TW = (int(cams[0].W) + p.tile - 1) // p.tile
        TH = (int(cams[0].H) + p.tile - 1) // p.tile
        ranges = torch.zeros((len(cams) * TW * TH, 2), dtype=torch.int32, device=gs.means.device)
        M = C.c_int64(0)
        recs = camera_records(cams)
        self._check(self._lib.gavis_debug_bins(self._h, C.byref(gs.struct), recs, len(cams), C.byref(p), None,
                                               None, 0, C.byref(M), C.c_void_p(ranges.data_ptr()),
                                               _stream_ptr(stream)))
        m = int(M.value)
        keys = torch.empty(max(m, 1), dtype=torch.int64, device=gs.means.device)
        vals = torch.empty(max(m, 1), dtype=torch.int32, device=gs.means.device)
        self._check(self._lib.gavis_debug_bins(self._h, C.byref(gs.struct), recs, len(cams), C.byref(p),
                                               C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()), m,
                                               C.byref(M), C.c_void_p(ranges.data_ptr()), _stream_ptr(stream)))
        return keys[:m], vals[:m], ranges

    def debug_visibility(self, gs: Gaussians, cams, params=None, stream=None):
        p = params or Params()
        sumT = torch.zeros((len(cams), gs.n), device=gs.means.device)
        cnt = torch.zeros((len(cams), gs.n), dtype=torch.int32, device=gs.means.device)
        self._check(self._lib.gavis_debug_visibility(self._h, C.byref(gs.struct), camera_records(cams), len(cams),
                                                     C.byref(p), C.c_void_p(sumT.data_ptr()),
                                                     C.c_void_p(cnt.data_ptr()), _stream_ptr(stream)))
        return sumT, cnt


class Plan:
    """A replayable scoring graph for n_cams candidate views of W x H pixels.
    Owns its output tensors (score [n], best_dev [1], optional rgb/unc) and
    keeps the scene, field and parameters it was built on alive."""

    def __init__(self, ctx: Context, gs: Gaussians, vf: VisibilityField, n_cams, W, H, record_capacity,
                 entry_capacity, params, want_rgb, want_unc):
        self._lib, self._ctx = ctx._lib, ctx
        self.gs, self.vf = gs, vf
        self.params = params or Params(vf_degree=vf.degree)
        if self.params.tile == 0:
            raise ValueError("a plan needs a fixed tile edge (8, 16 or 32)")
        dev = gs.means.device
        self.n_cams, self.W, self.H = int(n_cams), int(W), int(H)
        self.score = torch.empty(self.n_cams, device=dev)
        self.best_dev = torch.empty(1, dtype=torch.int32, device=dev)
        self.rgb = torch.empty((self.n_cams, 3, self.H, self.W), device=dev) if want_rgb else None
        self.unc = torch.empty((self.n_cams, self.H, self.W), device=dev) if want_unc else None
        self._vs = vf.struct()
        self._h = C.c_void_p()
        ctx._check(self._lib.gavis_plan_create(
            ctx._h, C.byref(gs.struct), C.byref(self._vs), self.n_cams, self.W, self.H, C.byref(self.params),
            int(record_capacity), int(entry_capacity), C.c_void_p(self.rgb.data_ptr() if self.rgb is not None else None),
            C.c_void_p(self.unc.data_ptr() if self.unc is not None else None), C.c_void_p(self.score.data_ptr()),
            C.c_void_p(self.best_dev.data_ptr()), C.byref(self._h)))
        self.kernels = int(self._lib.gavis_plan_kernels(self._h))

    def launch(self, cams, stream=None):
        """Score the poses `cams` (n_cams cameras of W x H, or their
        camera_records array) asynchronously."""
        if len(cams) != self.n_cams:
            raise ValueError(f"plan expects {self.n_cams} cameras, got {len(cams)}")
        recs = cams if isinstance(cams, C.Array) else camera_records(cams)
        rc = self._lib.gavis_plan_launch(self._h, recs, _stream_ptr(stream))
        if rc != OK:
            raise GavisError(rc, "gavis_plan_launch")

    def overflowed(self):
        """(overflowed, records_needed, entries_needed) of the last launch;
        waits for it."""
        o, r, m = C.c_int(0), C.c_int64(0), C.c_int64(0)
        rc = self._lib.gavis_plan_overflowed(self._h, C.byref(o), C.byref(r), C.byref(m))
        if rc != OK:
            raise GavisError(rc, "gavis_plan_overflowed")
        return bool(o.value), int(r.value), int(m.value)

    def close(self):
        if self._h:
            self._lib.gavis_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching scoring server over resident scenes (C ABI
    gavis_server_*).  Scenes and their fields must outlive the server; this
    wrapper keeps references to them and to each request's output tensors."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, n_workers: int = 2, max_views_per_batch: int = 64):
        self._lib = load()
        self._h = C.c_void_p()
        rc = self._lib.gavis_server_create(C.byref(self._h), int(device), C.c_size_t(int(budget_bytes)),
                                           int(n_workers), int(max_views_per_batch))
        if rc != OK:
            raise GavisError(rc, "gavis_server_create failed")
        self.device = device
        self._keep = {}
        self._scenes = []

    def _check(self, rc):
        if rc != OK:
            raise GavisError(rc, self._lib.gavis_server_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._lib.gavis_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_scene(self, gs: Gaussians, vf: VisibilityField) -> int:
        vs = vf.struct()
        sid = C.c_int(-1)
        self._check(self._lib.gavis_server_add_scene(self._h, C.byref(gs.struct), C.byref(vs), C.byref(sid)))
        self._scenes.append((gs, vf, vs))
        return int(sid.value)

    def submit(self, scene_id: int, cams, params=None, want_unc: bool = False) -> int:
        p = params or Params()
        dev = torch.device("cuda", self.device)
        score = torch.empty(len(cams), device=dev)
        unc = torch.empty((len(cams), int(cams[0].H), int(cams[0].W)), device=dev) if want_unc else None
        rid = C.c_int64(0)
        self._check(self._lib.gavis_server_submit(self._h, int(scene_id), camera_records(cams), len(cams), C.byref(p),
                                                  C.c_void_p(score.data_ptr()),
                                                  C.c_void_p(unc.data_ptr() if unc is not None else None),
                                                  C.byref(rid)))
        self._keep[int(rid.value)] = (score, unc)
        return int(rid.value)

    def pause(self, paused: bool = True):
        """Stop (or restart) the workers from taking new batches."""
        self._check(self._lib.gavis_server_pause(self._h, int(bool(paused))))

    def wait(self, request_id: int, timeout_ms: int = 600000):
        """dict(score, unc, best, latency_ms); raises GavisError (code
        ERR_TIMEOUT) if the request is not finished in time."""
        best, lat = C.c_int32(-1), C.c_double(0.0)
        self._check(self._lib.gavis_server_wait(self._h, int(request_id), int(timeout_ms), C.byref(best),
                                                C.byref(lat)))
        score, unc = self._keep.pop(int(request_id))
        return dict(score=score, unc=unc, best=int(best.value), latency_ms=float(lat.value))

    def stats(self):
        v, b, m = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        pk, bud = C.c_size_t(0), C.c_size_t(0)
        self._check(self._lib.gavis_server_stats(self._h, C.byref(v), C.byref(b), C.byref(m), C.byref(pk),
                                                 C.byref(bud)))
        return dict(views_scored=int(v.value), batches=int(b.value), max_requests_in_batch=int(m.value),
                    peak_reserved_bytes=int(pk.value), budget_bytes=int(bud.value))
