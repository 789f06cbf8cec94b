"""Seeded synthetic inputs for the GAVIS hot path.

This module only draws random numbers and lays out arrays: Gaussian scenes
(centres, scales, unit quaternions, opacities, colour SH coefficients) and
pinhole cameras.  It holds none of the method's arithmetic (no projection, no
spherical harmonics, no compositing), so both the CPU oracle and the CUDA
library can be fed from it without sharing any of the computation they are
compared on.

Scenes follow the paper's evaluation setting (Sec. "Environment Setup" and
"Active Mapping Setup"): indoor rooms seen from a camera at 1.5 m height with
SE(2) candidate poses and a 90 degree horizontal field of view, plus a small
object-centric scene for fast parity cases.  The paper's datasets (HM3D,
Gibson, NeRF Synthetic) are not reproduced; these shapes stand in for them.

Camera convention: world->camera rotation R (rows are the camera x/right,
y/down, z/forward axes in world coordinates), t = -R @ campos, pixel (i, j)
has its centre at (i + 0.5, j + 0.5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Scene", "Camera", "look_at_camera", "tiny_scene", "room_scene",
    "multi_room_scene", "ring_cameras", "fibonacci_cameras",
    "walk_cameras", "se2_cameras", "config",
]


@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    tan_half_fovx: float
    tan_half_fovy: float
    R: np.ndarray          # (3,3) float32, world -> camera
    t: np.ndarray          # (3,)  float32
    campos: np.ndarray     # (3,)  float32
    znear: float = 0.2


@dataclass
class Scene:
    means: np.ndarray      # (N,3) float32
    scales: np.ndarray     # (N,3) float32, activated (> 0)
    rots: np.ndarray       # (N,4) float32, unit quaternion (w,x,y,z)
    opac: np.ndarray       # (N,)  float32 in [0,1]
    sh: np.ndarray         # (N,(Lc+1)^2,3) float32, coefficient-major
    sh_degree: int
    bbox_min: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    bbox_max: np.ndarray = field(default_factory=lambda: np.ones(3, np.float32))
    obstacles: list = field(default_factory=list)   # [(lo(3), hi(3))]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx], self.scales[idx], self.rots[idx],
                     self.opac[idx], self.sh[idx], self.sh_degree,
                     self.bbox_min, self.bbox_max, self.obstacles)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def look_at_camera(pos, target, W, H, fovx_deg=90.0, up=(0.0, 0.0, 1.0),
                   znear=0.2) -> Camera:
    """Pinhole camera at `pos` looking at `target` (square pixels, principal
    point at the image centre).  Trigonometry is done in float64 and rounded
    once to float32."""
    pos = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - pos
    f /= np.linalg.norm(f)
    upv = np.asarray(up, np.float64)
    if abs(float(np.dot(f, upv))) > 0.999:
        upv = np.array([0.0, 1.0, 0.0]) if abs(f[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
    x = np.cross(f, upv)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ pos
    fx = W / (2.0 * math.tan(math.radians(fovx_deg) / 2.0))
    fy = fx
    return Camera(W=int(W), H=int(H), fx=float(np.float32(fx)), fy=float(np.float32(fy)),
                  cx=float(np.float32(W / 2.0)), cy=float(np.float32(H / 2.0)),
                  tan_half_fovx=float(np.float32(W / (2.0 * fx))),
                  tan_half_fovy=float(np.float32(H / (2.0 * fy))),
                  R=R.astype(np.float32), t=t.astype(np.float32),
                  campos=pos.astype(np.float32), znear=float(znear))


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def tiny_scene(n=2000, seed=0, sh_degree=1) -> Scene:
    """Object-centric cloud: centres U[-1,1]^3, log-scales N(-3,0.3), uniform
    unit quaternions, opacity sigmoid(N(0,1.5)), colour SH N(0,0.3)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    scales = np.exp(rng.normal(-3.0, 0.3, (n, 3)))
    rots = _unit_quats(rng, n)
    opac = _sigmoid(rng.normal(0.0, 1.5, n))
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, k, 3))
    return Scene(means.astype(np.float32), scales.astype(np.float32),
                 rots.astype(np.float32), opac.astype(np.float32),
                 sh.astype(np.float32), sh_degree,
                 np.full(3, -1.0, np.float32), np.full(3, 1.0, np.float32))


def _quat_from_frame(nrm, spin):
    """Unit quaternions (w,x,y,z) of rotations mapping local z to `nrm`, with
    an extra spin about the normal (vectorised; input float64)."""
    n = nrm.shape[0]
    # orthonormal tangent frame
    a = np.where(np.abs(nrm[:, 0:1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    t1 = np.cross(a, nrm)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(nrm, t1)
    c, s = np.cos(spin)[:, None], np.sin(spin)[:, None]
    u = c * t1 + s * t2
    v = np.cross(nrm, u)
    M = np.stack([u, v, nrm], axis=2)      # columns = rotated local axes
    # matrix -> quaternion (Shepperd), vectorised
    tr = M[:, 0, 0] + M[:, 1, 1] + M[:, 2, 2]
    q = np.zeros((n, 4))
    m0 = tr > 0
    sq = np.sqrt(np.maximum(tr[m0] + 1.0, 1e-300)) * 2
    q[m0, 0] = 0.25 * sq
    q[m0, 1] = (M[m0, 2, 1] - M[m0, 1, 2]) / sq
    q[m0, 2] = (M[m0, 0, 2] - M[m0, 2, 0]) / sq
    q[m0, 3] = (M[m0, 1, 0] - M[m0, 0, 1]) / sq
    m1 = (~m0) & (M[:, 0, 0] > M[:, 1, 1]) & (M[:, 0, 0] > M[:, 2, 2])
    sq = np.sqrt(np.maximum(1.0 + M[m1, 0, 0] - M[m1, 1, 1] - M[m1, 2, 2], 1e-300)) * 2
    q[m1, 0] = (M[m1, 2, 1] - M[m1, 1, 2]) / sq
    q[m1, 1] = 0.25 * sq
    q[m1, 2] = (M[m1, 0, 1] + M[m1, 1, 0]) / sq
    q[m1, 3] = (M[m1, 0, 2] + M[m1, 2, 0]) / sq
    m2 = (~m0) & (~m1) & (M[:, 1, 1] > M[:, 2, 2])
    sq = np.sqrt(np.maximum(1.0 + M[m2, 1, 1] - M[m2, 0, 0] - M[m2, 2, 2], 1e-300)) * 2
    q[m2, 0] = (M[m2, 0, 2] - M[m2, 2, 0]) / sq
    q[m2, 1] = (M[m2, 0, 1] + M[m2, 1, 0]) / sq
    q[m2, 2] = 0.25 * sq
    q[m2, 3] = (M[m2, 1, 2] + M[m2, 2, 1]) / sq
    m3 = (~m0) & (~m1) & (~m2)
    sq = np.sqrt(np.maximum(1.0 + M[m3, 2, 2] - M[m3, 0, 0] - M[m3, 1, 1], 1e-300)) * 2
    q[m3, 0] = (M[m3, 1, 0] - M[m3, 0, 1]) / sq
    q[m3, 1] = (M[m3, 0, 2] + M[m3, 2, 0]) / sq
    q[m3, 2] = (M[m3, 1, 2] + M[m3, 2, 1]) / sq
    q[m3, 3] = 0.25 * sq
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _layout_rooms(n_rooms_x, n_rooms_y, room=(6.0, 4.0, 3.0)):
    """Grid of rooms; returns list of (lo, hi) room boxes."""
    rx, ry, rz = room
    rooms = []
    for j in range(n_rooms_y):
        for i in range(n_rooms_x):
            rooms.append((np.array([i * rx, j * ry, 0.0]), np.array([(i + 1) * rx, (j + 1) * ry, rz])))
    return rooms


def _surface_patches(rooms, obstacles, door_w=1.0, door_h=2.1):
    """Planar rectangles (origin, edge u, edge v, normal, door-hole or None)."""
    patches = []
    if not rooms:
        return patches
    lo = np.min([r[0] for r in rooms], axis=0)
    hi = np.max([r[1] for r in rooms], axis=0)
    for (rlo, rhi) in rooms:
        sx, sy, sz = rhi - rlo
        # floor, ceiling
        patches.append((np.array([rlo[0], rlo[1], rlo[2]]), np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, 1.0]), None))
        patches.append((np.array([rlo[0], rlo[1], rhi[2]]), np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, -1.0]), None))
        # walls at x = rlo.x and x = rhi.x (shared walls only once: emit the low
        # side always, the high side only on the outer boundary)
        for xw, nx in ((rlo[0], 1.0), (rhi[0], -1.0)):
            if nx < 0 and xw < hi[0] - 1e-9:
                continue
            hole = None
            if 1e-9 < xw - lo[0] and xw < hi[0] - 1e-9:
                hole = (0.5 * sy - 0.5 * door_w, 0.5 * sy + 0.5 * door_w, 0.0, door_h)
            patches.append((np.array([xw, rlo[1], rlo[2]]), np.array([0, sy, 0]), np.array([0, 0, sz]), np.array([nx, 0, 0]), hole))
        for yw, ny in ((rlo[1], 1.0), (rhi[1], -1.0)):
            if ny < 0 and yw < hi[1] - 1e-9:
                continue
            hole = None
            if 1e-9 < yw - lo[1] and yw < hi[1] - 1e-9:
                hole = (0.5 * sx - 0.5 * door_w, 0.5 * sx + 0.5 * door_w, 0.0, door_h)
            patches.append((np.array([rlo[0], yw, rlo[2]]), np.array([sx, 0, 0]), np.array([0, 0, sz]), np.array([0, ny, 0]), hole))
    for (blo, bhi) in obstacles:
        sx, sy, sz = bhi - blo
        patches.append((np.array([blo[0], blo[1], bhi[2]]), np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, 1.0]), None))
        patches.append((np.array([blo[0], blo[1], blo[2]]), np.array([0, sy, 0]), np.array([0, 0, sz]), np.array([-1.0, 0, 0]), None))
        patches.append((np.array([bhi[0], blo[1], blo[2]]), np.array([0, sy, 0]), np.array([0, 0, sz]), np.array([1.0, 0, 0]), None))
        patches.append((np.array([blo[0], blo[1], blo[2]]), np.array([sx, 0, 0]), np.array([0, 0, sz]), np.array([0, -1.0, 0]), None))
        patches.append((np.array([blo[0], bhi[1], blo[2]]), np.array([sx, 0, 0]), np.array([0, 0, sz]), np.array([0, 1.0, 0]), None))
    return patches


def _random_obstacles(rng, rooms, per_room):
    obs = []
    for (rlo, rhi) in rooms:
        for _ in range(per_room):
            size = np.array([rng.uniform(0.3, 1.2), rng.uniform(0.3, 1.2), rng.uniform(0.4, 1.5)])
            x = rng.uniform(rlo[0] + 0.2, rhi[0] - 0.2 - size[0])
            y = rng.uniform(rlo[1] + 0.2, rhi[1] - 0.2 - size[1])
            blo = np.array([x, y, rlo[2]])
            obs.append((blo, blo + size))
    return obs


def multi_room_scene(n, n_rooms_x=1, n_rooms_y=1, seed=0, sh_degree=3,
                     obstacles_per_room=20, opac_mu=1.0, opac_sigma=1.0,
                     floater_frac=0.0) -> Scene:
    """Gaussians on the walls, floor and ceiling of a grid of 6x4x3 m rooms
    (door gaps between neighbours) and on the faces of random box obstacles.
    Tangent log-scales N(-4,0.5); the normal-axis scale is 0.1x; rotations map
    local z to the face normal with a random spin; opacity
    sigmoid(N(opac_mu, opac_sigma)); colour SH N(0,0.3).  An optional fraction
    of small floaters (log-scale N(-6,0.5)) is spread uniformly in the room
    volumes."""
    rng = np.random.default_rng(seed)
    rooms = _layout_rooms(n_rooms_x, n_rooms_y)
    obstacles = _random_obstacles(rng, rooms, obstacles_per_room)
    patches = _surface_patches(rooms, obstacles)
    n_float = int(round(n * floater_frac))
    n_surf = n - n_float
    areas = np.array([np.linalg.norm(p[1]) * np.linalg.norm(p[2]) for p in patches])
    counts = rng.multinomial(n_surf, areas / areas.sum())
    means, nrms = [], []
    for (o, eu, ev, nr, hole), c in zip(patches, counts):
        if c == 0:
            continue
        a = rng.uniform(0, 1, c)
        b = rng.uniform(0, 1, c)
        if hole is not None:
            lu, lv = np.linalg.norm(eu), np.linalg.norm(ev)
            inside = (a * lu > hole[0]) & (a * lu < hole[1]) & (b * lv > hole[2]) & (b * lv < hole[3])
            # resample points that fall into the door opening onto the rest of the wall
            for _ in range(20):
                k = int(inside.sum())
                if k == 0:
                    break
                a[inside] = rng.uniform(0, 1, k)
                b[inside] = rng.uniform(0, 1, k)
                inside = (a * lu > hole[0]) & (a * lu < hole[1]) & (b * lv > hole[2]) & (b * lv < hole[3])
        means.append(o[None, :] + a[:, None] * eu[None, :] + b[:, None] * ev[None, :])
        nrms.append(np.repeat(nr[None, :], c, axis=0))
    means = np.concatenate(means)
    nrms = np.concatenate(nrms)
    ls = rng.normal(-4.0, 0.5, (n_surf, 3))
    scales = np.exp(ls)
    scales[:, 2] *= 0.1
    rots = _quat_from_frame(nrms, rng.uniform(0, 2 * math.pi, n_surf))
    if n_float:
        lo = np.min([r[0] for r in rooms], axis=0)
        hi = np.max([r[1] for r in rooms], axis=0)
        fm = rng.uniform(lo, hi, (n_float, 3))
        fs = np.exp(rng.normal(-6.0, 0.5, (n_float, 3)))
        fr = _unit_quats(rng, n_float)
        means = np.concatenate([means, fm])
        scales = np.concatenate([scales, fs])
        rots = np.concatenate([rots, fr])
    perm = rng.permutation(n)
    means, scales, rots = means[perm], scales[perm], rots[perm]
    opac = _sigmoid(rng.normal(opac_mu, opac_sigma, n))
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.3, (n, k, 3))
    lo = np.min([r[0] for r in rooms], axis=0)
    hi = np.max([r[1] for r in rooms], axis=0)
    return Scene(means.astype(np.float32), scales.astype(np.float32), rots.astype(np.float32),
                 opac.astype(np.float32), sh.astype(np.float32), sh_degree,
                 lo.astype(np.float32), hi.astype(np.float32), obstacles)


def room_scene(n=200_000, seed=0, sh_degree=3) -> Scene:
    return multi_room_scene(n, 1, 1, seed=seed, sh_degree=sh_degree)


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def ring_cameras(n, radius=3.0, W=128, H=128, fovx_deg=60.0):
    """n cameras on a ring in the z=0 plane looking at the origin (up +z)."""
    cams = []
    for i in range(n):
        a = 2 * math.pi * i / n
        cams.append(look_at_camera((radius * math.cos(a), radius * math.sin(a), 0.0), (0, 0, 0), W, H, fovx_deg))
    return cams


def fibonacci_cameras(n, radius=3.0, W=128, H=128, fovx_deg=60.0):
    """n cameras on a Fibonacci sphere looking at the origin."""
    cams = []
    ga = math.pi * (3.0 - math.sqrt(5.0))
    for i in range(n):
        z = 1.0 - 2.0 * (i + 0.5) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        a = ga * i
        pos = (radius * r * math.cos(a), radius * r * math.sin(a), radius * z)
        cams.append(look_at_camera(pos, (0, 0, 0), W, H, fovx_deg))
    return cams


def _free(p, obstacles, margin=0.3):
    for (lo, hi) in obstacles:
        if np.all(p[:2] > lo[:2] - margin) and np.all(p[:2] < hi[:2] + margin):
            return False
    return True


def walk_cameras(n, scene: Scene, W, H, seed=1, x_frac=(0.0, 0.5), height=1.5, fovx_deg=90.0):
    """Training trajectory: a random walk at `height` confined to the slab
    x in [lo + x_frac[0]*size, lo + x_frac[1]*size], yaw drifting, slight pitch."""
    rng = np.random.default_rng(seed)
    lo, hi = scene.bbox_min.astype(np.float64), scene.bbox_max.astype(np.float64)
    xlo = lo[0] + x_frac[0] * (hi[0] - lo[0]) + 0.5
    xhi = lo[0] + x_frac[1] * (hi[0] - lo[0]) - 0.5
    ylo, yhi = lo[1] + 0.5, hi[1] - 0.5
    p = np.array([0.5 * (xlo + xhi), 0.5 * (ylo + yhi), height])
    for _ in range(100):
        if _free(p, scene.obstacles):
            break
        p[:2] = [rng.uniform(xlo, xhi), rng.uniform(ylo, yhi)]
    yaw = rng.uniform(0, 2 * math.pi)
    cams = []
    for _ in range(n):
        for _ in range(50):
            step = rng.normal(0, 0.25, 2)
            q = p.copy()
            q[0] = min(max(q[0] + step[0], xlo), xhi)
            q[1] = min(max(q[1] + step[1], ylo), yhi)
            if _free(q, scene.obstacles):
                p = q
                break
        yaw += rng.normal(0, 0.6)
        pitch = rng.normal(0, 0.15)
        fwd = np.array([math.cos(yaw) * math.cos(pitch), math.sin(yaw) * math.cos(pitch), math.sin(pitch)])
        cams.append(look_at_camera(p, p + fwd, W, H, fovx_deg))
    return cams


def se2_cameras(n, scene: Scene, W, H, seed=2, height=1.5, fovx_deg=90.0):
    """Candidate poses: uniform collision-free SE(2) poses at `height`."""
    rng = np.random.default_rng(seed)
    lo, hi = scene.bbox_min.astype(np.float64), scene.bbox_max.astype(np.float64)
    cams = []
    while len(cams) < n:
        p = np.array([rng.uniform(lo[0] + 0.4, hi[0] - 0.4), rng.uniform(lo[1] + 0.4, hi[1] - 0.4), height])
        if not _free(p, scene.obstacles):
            continue
        yaw = rng.uniform(0, 2 * math.pi)
        fwd = np.array([math.cos(yaw), math.sin(yaw), 0.0])
        cams.append(look_at_camera(p, p + fwd, W, H, fovx_deg))
    return cams


# ----------------------------------------------------------------------------
# the five workload shapes
# ----------------------------------------------------------------------------

def config(k: int, seed: int = 0, n=None, n_train=None, n_cand=None, train_wh=None, cand_wh=None):
    """Workload `k` (1..5) with optional size overrides for reduced parity
    cases.  Returns dict(scene, train, cand, vf_degree, coeff_dtype, name)."""
    if k == 1:
        sc = tiny_scene(n or 2000, seed=seed, sh_degree=1)
        tw, th = train_wh or (128, 128)
        cw, ch = cand_wh or (128, 128)
        return dict(name="tiny: 2k Gaussians, 8 train / 16 candidate views at 128x128",
                    scene=sc, train=ring_cameras(n_train or 8, 3.0, tw, th, 60.0),
                    cand=fibonacci_cameras(n_cand or 16, 3.0, cw, ch, 60.0),
                    vf_degree=2, coeff_dtype="f32")
    if k == 2:
        sc = multi_room_scene(n or 200_000, 1, 1, seed=seed, sh_degree=3)
        tw, th = train_wh or (800, 800)
        cw, ch = cand_wh or (800, 800)
        return dict(name="room: 200k Gaussians, 100 train / 64 candidate views at 800x800",
                    scene=sc, train=walk_cameras(n_train or 100, sc, tw, th, seed=seed + 1, x_frac=(0.0, 0.5)),
                    cand=se2_cameras(n_cand or 64, sc, cw, ch, seed=seed + 2),
                    vf_degree=3, coeff_dtype="f32")
    if k == 3:
        sc = multi_room_scene(n or 1_000_000, 3, 1, seed=seed, sh_degree=3)
        tw, th = train_wh or (1280, 720)
        cw, ch = cand_wh or (640, 480)
        return dict(name="batched: 1M Gaussians in 3 rooms, 200 train views at 1280x720, 256 candidates at 640x480",
                    scene=sc, train=walk_cameras(n_train or 200, sc, tw, th, seed=seed + 1, x_frac=(0.0, 0.45)),
                    cand=se2_cameras(n_cand or 256, sc, cw, ch, seed=seed + 2),
                    vf_degree=3, coeff_dtype="f16")
    if k == 4:
        sc = multi_room_scene(n or 3_000_000, 4, 2, seed=seed, sh_degree=3, opac_mu=0.0,
                              opac_sigma=2.0, floater_frac=0.2)
        tw, th = train_wh or (1280, 720)
        cw, ch = cand_wh or (320, 240)
        return dict(name="house: 3M Gaussians in 8 rooms, 300 train views at 1280x720, 1024 candidates at 320x240",
                    scene=sc, train=walk_cameras(n_train or 300, sc, tw, th, seed=seed + 1, x_frac=(0.0, 0.5)),
                    cand=se2_cameras(n_cand or 1024, sc, cw, ch, seed=seed + 2),
                    vf_degree=3, coeff_dtype="bf16")
    raise ValueError(f"unknown workload {k}")
