"""Seeded synthetic workloads for the surfel non-rigid solver.

This module only *makes inputs*: depth frames of deforming analytic surfaces,
a reference surfel model and the node positions that carry the warp field.  It
contains none of the method's arithmetic (no depth-map processing, no
dual-quaternion blending, no association, no solver): the ground-truth motions
are produced with plain linear blending of rigid node motions or with analytic
displacement fields, and depth images are rendered by per-pixel Newton ray
casting against the analytically deformed surface.

Both the CUDA path (through the C-ABI) and the FP64 oracle consume exactly the
float32 arrays returned here.

Workloads (the paper's recorded sequences are not available; these stand in):

* ``plain_tiny``  -- 160x120 wavy height field z = 1 + 0.05 sin(6x) cos(6y),
  19,200 surfels, 64 nodes on an 8x8 grid, per-node random rigid motions
  (rotation <= 5 deg, translation <= 2 cm) blended smoothly, 1 mm depth noise.
* ``plain_full``  -- 640x480 sphere (r = 0.3 m at 1.2 m), 300k surfels from a
  Fibonacci sampling of the whole sphere, 2048 nodes by voxel subsampling,
  a 100-frame bending sequence (sum of three low-frequency sinusoidal
  displacement fields, |d| <= 4 cm), 1.5 mm noise and 1 % outlier pixels.
* ``random_scene`` -- small seeded scenes for stage tests.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np

__all__ = [
    "Camera", "Scene", "plain_tiny", "plain_full", "random_scene",
    "batch_scenes", "random_rigid_dq_inputs",
]


@dataclass(frozen=True)
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float

    def rays(self):
        """Per-pixel normalised ray directions (a, b) with z = 1, float64."""
        u, v = np.meshgrid(np.arange(self.width, dtype=np.float64),
                           np.arange(self.height, dtype=np.float64))
        return (u - self.cx) / self.fx, (v - self.cy) / self.fy


@dataclass
class Scene:
    """A reference surfel model, its nodes and a source of depth frames.

    All arrays are float32/int32 and C-contiguous; they are the exact values
    handed to both implementations.
    """
    name: str
    cam: Camera
    surfel_v: np.ndarray          # (Ns, 3) float32 reference positions [m]
    surfel_n: np.ndarray          # (Ns, 3) float32 unit normals
    surfel_r: np.ndarray          # (Ns,)   float32 radii [m]
    surfel_c: np.ndarray          # (Ns,)   float32 confidences
    surfel_t: np.ndarray          # (Ns, 2) int32 (t_init, t_observed)
    node_p: np.ndarray            # (Nn, 3) float32 node positions
    node_sigma: np.ndarray        # (Nn,)   float32 node radius parameter
    n_frames: int
    gn_iters: int
    pcg_iters: int
    _frame_fn: Callable[[int], np.ndarray] = field(repr=False, default=None)
    _cache: dict = field(repr=False, default_factory=dict)
    truth: dict = field(repr=False, default_factory=dict)

    def frame(self, t: int) -> np.ndarray:
        """Depth image of frame ``t`` (H, W) float32 metres, 0 = invalid."""
        if t not in self._cache:
            d = self._frame_fn(t)
            self._cache[t] = np.ascontiguousarray(d, dtype=np.float32)
        return self._cache[t]


# ---------------------------------------------------------------------------
# small geometry helpers (generator-only)
# ---------------------------------------------------------------------------

def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _rot_axis_angle(axis, angle):
    """Rotation matrices from unit axes (n,3) and angles (n,) (Rodrigues)."""
    axis = np.asarray(axis, dtype=np.float64)
    k = np.zeros(axis.shape[:-1] + (3, 3))
    k[..., 0, 1], k[..., 0, 2] = -axis[..., 2], axis[..., 1]
    k[..., 1, 0], k[..., 1, 2] = axis[..., 2], -axis[..., 0]
    k[..., 2, 0], k[..., 2, 1] = -axis[..., 1], axis[..., 0]
    s = np.sin(angle)[..., None, None]
    c = np.cos(angle)[..., None, None]
    return np.eye(3) + s * k + (1 - c) * (k @ k)


def _random_dirs(rng, n):
    return _unit(rng.normal(size=(n, 3)))


def _newton2(fun, x0, iters=14, h=1e-7, tol=1e-12):
    """Vectorised 2-D Newton solve of fun(x) = 0, x of shape (n, 2).

    Returns (x, ok).  The Jacobian is taken by central differences.
    """
    x = x0.copy()
    for _ in range(iters):
        f = fun(x)
        jac = np.empty(x.shape[:-1] + (2, 2))
        for c in range(2):
            e = np.zeros(2)
            e[c] = h
            jac[..., :, c] = (fun(x + e) - fun(x - e)) / (2 * h)
        det = jac[..., 0, 0] * jac[..., 1, 1] - jac[..., 0, 1] * jac[..., 1, 0]
        det = np.where(np.abs(det) < 1e-30, 1e-30, det)
        dx0 = (jac[..., 1, 1] * f[..., 0] - jac[..., 0, 1] * f[..., 1]) / det
        dx1 = (-jac[..., 1, 0] * f[..., 0] + jac[..., 0, 0] * f[..., 1]) / det
        step = np.stack([dx0, dx1], axis=-1)
        step = np.clip(step, -0.05, 0.05)
        x = x - step
    f = fun(x)
    ok = np.all(np.isfinite(f), axis=-1) & (np.max(np.abs(f), axis=-1) < tol)
    return x, ok


def _voxel_nodes(points, target, lo=0.002, hi=0.2):
    """Voxel subsampling of ``points`` to exactly ``target`` nodes.

    The voxel edge is bisected to the smallest grid with at least ``target``
    occupied voxels; each voxel contributes the member point closest to the
    members' centroid.  Surplus voxels are dropped evenly spread over the
    lexicographic voxel-key order.  Returns (node positions, voxel edge).
    """
    def vkeys(s):
        k = np.floor(points / s).astype(np.int64) + (1 << 20)
        return (k[:, 0] << 42) | (k[:, 1] << 21) | k[:, 2]

    def occupied(s):
        return len(np.unique(vkeys(s)))

    if occupied(lo) < target:
        raise ValueError("cannot reach the requested node count")
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if occupied(mid) >= target:
            lo = mid
        else:
            hi = mid
    s = lo
    uniq, inv = np.unique(vkeys(s), return_inverse=True)
    inv = inv.reshape(-1)
    m = len(uniq)
    cnt = np.bincount(inv, minlength=m).astype(np.float64)
    cen = np.stack([np.bincount(inv, weights=points[:, c], minlength=m)
                    for c in range(3)], axis=1) / cnt[:, None]
    d2 = np.sum((points - cen[inv]) ** 2, axis=1)
    order = np.lexsort((np.arange(len(points)), d2, inv))
    first = np.ones(len(order), dtype=bool)
    first[1:] = inv[order[1:]] != inv[order[:-1]]
    pick = order[first]                      # one point per voxel, key order
    if m > target:
        drop = np.round(np.linspace(0, m - 1, m - target + 2)[1:-1]).astype(int)
        keep = np.ones(m, dtype=bool)
        keep[drop] = False
        pick = pick[keep]
    return points[pick], s


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


# ---------------------------------------------------------------------------
# plain_tiny: 160x120 wavy height field, 64 grid nodes, one frame pair
# ---------------------------------------------------------------------------

def _wavy(x, y):
    return 1.0 + 0.05 * np.sin(6 * x) * np.cos(6 * y)


def _wavy_grad(x, y):
    return (0.3 * np.cos(6 * x) * np.cos(6 * y),
            -0.3 * np.sin(6 * x) * np.sin(6 * y))


def _raycast_wavy(a, b):
    """Depth along rays (a, b, 1) to the undeformed height field (Newton)."""
    z = np.ones_like(a)
    for _ in range(30):
        x, y = z * a, z * b
        fx, fy = _wavy_grad(x, y)
        g = z - _wavy(x, y)
        dg = 1.0 - (fx * a + fy * b)
        z = z - g / dg
    return z


def plain_tiny(seed: int = 0, noise: float = 1e-3, rigid: bool = False) -> Scene:
    """160x120 wavy surface with a smooth non-rigid motion (one frame pair).

    Frame 0 is the undeformed surface, frame 1 the deformed one; both carry
    N(0, ``noise``) depth noise (frame noise is seeded per frame).  With
    ``rigid`` every node receives the same rigid motion.
    """
    cam = Camera(160, 120, 140.0, 140.0, 80.0, 60.0)
    rng = np.random.default_rng(seed)
    a, b = cam.rays()
    z = _raycast_wavy(a, b)
    v = np.stack([z * a, z * b, z], axis=-1).reshape(-1, 3)
    gx, gy = _wavy_grad(v[:, 0], v[:, 1])
    n = _unit(np.stack([gx, gy, -np.ones_like(gx)], axis=-1))
    ns = v.shape[0]
    radius = 1.5 * v[:, 2] / cam.fx

    # 8x8 node grid over the frustum at z ~ 1, lifted onto the surface
    xs = -0.57 + (np.arange(8) + 0.5) * (1.14 / 8)
    ys = -0.43 + (np.arange(8) + 0.5) * (0.86 / 8)
    gxx, gyy = np.meshgrid(xs, ys)
    node_p = np.stack([gxx.ravel(), gyy.ravel(),
                       _wavy(gxx.ravel(), gyy.ravel())], axis=-1)
    sigma = 0.5 * (1.14 / 8 + 0.86 / 8)
    nn = node_p.shape[0]

    # ground truth: node-local rigid motions, blended linearly with
    # normalised Gaussian weights over all nodes
    if rigid:
        axis = np.repeat(_random_dirs(rng, 1), nn, axis=0)
        ang = np.repeat(rng.uniform(0, np.deg2rad(5.0), 1), nn)
        tr = np.repeat(_random_dirs(rng, 1) * rng.uniform(0, 0.02, (1, 1)), nn, axis=0)
    else:
        axis = _random_dirs(rng, nn)
        ang = rng.uniform(0, np.deg2rad(5.0), nn)
        tr = _random_dirs(rng, nn) * rng.uniform(0, 0.02, (nn, 1))
    rot = _rot_axis_angle(axis, ang)
    if rigid:
        # one global rigid motion about the camera origin
        rot_g, tr_g = rot[0], tr[0]

        def warp(x):
            return x @ rot_g.T + tr_g
    else:
        offs = node_p + tr - np.einsum('kij,kj->ki', rot, node_p)
        rot9 = rot.reshape(nn, 9)

        def warp(x):
            d2 = (np.sum(x * x, axis=1)[:, None] - 2.0 * x @ node_p.T
                  + np.sum(node_p * node_p, axis=1)[None])
            wgt = np.exp(-d2 / (2 * sigma ** 2))
            wgt /= wgt.sum(axis=1, keepdims=True)
            m = (wgt @ rot9).reshape(-1, 3, 3)
            return np.einsum('nij,nj->ni', m, x) + wgt @ offs

    def render_deformed():
        aa, bb = a.ravel(), b.ravel()
        z0 = _raycast_wavy(aa, bb)

        def fun(p):
            s = np.stack([p[:, 0], p[:, 1], _wavy(p[:, 0], p[:, 1])], axis=-1)
            w = warp(s)
            return np.stack([w[:, 0] - aa * w[:, 2], w[:, 1] - bb * w[:, 2]], -1)

        p, ok = _newton2(fun, np.stack([z0 * aa, z0 * bb], axis=-1))
        s = np.stack([p[:, 0], p[:, 1], _wavy(p[:, 0], p[:, 1])], axis=-1)
        depth = warp(s)[:, 2]
        return np.where(ok, depth, 0.0).reshape(cam.height, cam.width)

    def frame(t):
        fr = np.random.default_rng([seed, 1000 + t])
        if t == 0:
            d = z.copy()
        elif t == 1:
            d = render_deformed()
        else:
            raise IndexError("plain_tiny has frames 0 and 1")
        valid = d > 0
        d = d + fr.normal(0.0, noise, d.shape) * valid if noise > 0 else d
        return np.where(valid, d, 0.0)

    t2 = np.zeros((ns, 2), dtype=np.int32)
    return Scene(
        name="plain_tiny_160x120", cam=cam,
        surfel_v=_f32(v), surfel_n=_f32(n), surfel_r=_f32(radius),
        surfel_c=np.ones(ns, dtype=np.float32), surfel_t=t2,
        node_p=_f32(node_p), node_sigma=np.full(nn, sigma, dtype=np.float32),
        n_frames=2, gn_iters=5, pcg_iters=10, _frame_fn=frame,
        truth={"rot": rot, "trans": tr, "warp": warp})


# ---------------------------------------------------------------------------
# plain_full: 640x480 bending sphere, 300k surfels, 2048 nodes, 100 frames
# ---------------------------------------------------------------------------

def _fibonacci_sphere(n):
    i = np.arange(n, dtype=np.float64)
    zc = 1.0 - 2.0 * (i + 0.5) / n
    rr = np.sqrt(np.maximum(0.0, 1.0 - zc * zc))
    phi = i * (np.pi * (3.0 - np.sqrt(5.0)))
    return np.stack([rr * np.cos(phi), rr * np.sin(phi), zc], axis=-1)


class _Bending:
    """Sum of three low-frequency sinusoidal displacement fields."""

    def __init__(self, rng, amplitude=0.04, k_range=(3.0, 8.0),
                 period_range=(40.0, 100.0)):
        self.e = _random_dirs(rng, 3)
        self.k = _random_dirs(rng, 3) * rng.uniform(*k_range, (3, 1))
        self.phase = rng.uniform(0, 2 * np.pi, 3)
        split = rng.dirichlet(np.ones(3))
        self.amp = amplitude * split
        self.period = rng.uniform(*period_range, 3)

    def __call__(self, x, t):
        out = x.copy()
        for m in range(3):
            a_t = self.amp[m] * np.sin(2 * np.pi * t / self.period[m])
            out = out + (a_t * np.sin(x @ self.k[m] + self.phase[m]))[..., None] * self.e[m]
        return out


def _render_sphere(cam, center, radius, deform, noise, outlier_frac, rng):
    """Depth of the deformed sphere by per-pixel Newton ray casting."""
    a, b = cam.rays()
    aa, bb = a.ravel(), b.ravel()
    ray = np.stack([aa, bb, np.ones_like(aa)], axis=-1)
    rn = ray / np.linalg.norm(ray, axis=1, keepdims=True)
    # front intersection with the undeformed sphere
    bq = rn @ center
    disc = bq * bq - (center @ center - radius * radius)
    hit = disc > (0.02 * radius) ** 2
    idx = np.nonzero(hit)[0]
    tt = bq[idx] - np.sqrt(disc[idx])
    d0 = _unit(rn[idx] * tt[:, None] - center)
    e1 = _unit(np.cross(d0, np.array([0.0, 1.0, 0.0])))
    e2 = np.cross(d0, e1)
    a_i, b_i = aa[idx], bb[idx]

    def surf(p):
        dirs = _unit(d0 + p[:, :1] * e1 + p[:, 1:] * e2)
        return deform(center + radius * dirs)

    def fun(p):
        w = surf(p)
        return np.stack([w[:, 0] - a_i * w[:, 2], w[:, 1] - b_i * w[:, 2]], -1)

    p, ok = _newton2(fun, np.zeros((len(idx), 2)))
    w = surf(p)
    h = 1e-6
    tu = surf(p + np.array([h, 0.0])) - surf(p - np.array([h, 0.0]))
    tv = surf(p + np.array([0.0, h])) - surf(p - np.array([0.0, h]))
    nrm = np.cross(tu, tv)
    out_dir = np.sum(nrm * d0, axis=1)       # orient with the undeformed normal
    nrm = nrm * np.sign(out_dir)[:, None]
    facing = np.sum(nrm * ray[idx], axis=1) < 0
    ok &= facing & (w[:, 2] > 0)
    depth = np.zeros(aa.shape)
    depth[idx[ok]] = w[ok, 2]
    valid = depth > 0
    depth = depth + rng.normal(0.0, noise, depth.shape) * valid
    if outlier_frac > 0:
        n_out = int(round(outlier_frac * depth.size))
        pos = rng.choice(depth.size, n_out, replace=False)
        depth[pos] = rng.uniform(0.5, 2.0, n_out)
    return depth.reshape(cam.height, cam.width)


def plain_full(seed: int = 0, n_surfels: int = 300_000, n_nodes: int = 2048,
               width: int = 640, height: int = 480, f: float = 570.0,
               noise: float = 1.5e-3, outliers: float = 0.01,
               n_frames: int = 100) -> Scene:
    """640x480 bending sphere sequence (radius 0.3 m at 1.2 m depth)."""
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0)
    rng = np.random.default_rng(seed)
    center = np.array([0.0, 0.0, 1.2])
    radius = 0.3
    dirs = _fibonacci_sphere(n_surfels)
    v = center + radius * dirs
    node_p, vox = _voxel_nodes(v, n_nodes)
    bend = _Bending(rng)
    spacing = 2.0 * radius / np.sqrt(n_surfels)
    t2 = np.zeros((n_surfels, 2), dtype=np.int32)

    def frame(t):
        fr = np.random.default_rng([seed, 2000 + t])
        return _render_sphere(cam, center, radius, lambda x: bend(x, t),
                              noise, outliers, fr)

    return Scene(
        name=f"sphere_{width}x{height}_{n_surfels}s_{n_nodes}n", cam=cam,
        surfel_v=_f32(v), surfel_n=_f32(dirs),
        surfel_r=np.full(n_surfels, spacing, dtype=np.float32),
        surfel_c=np.full(n_surfels, 15.0, dtype=np.float32), surfel_t=t2,
        node_p=_f32(node_p), node_sigma=np.full(len(node_p), vox, dtype=np.float32),
        n_frames=n_frames, gn_iters=10, pcg_iters=20, _frame_fn=frame,
        truth={"bend": bend, "center": center, "radius": radius})


# ---------------------------------------------------------------------------
# small scenes for stage tests
# ---------------------------------------------------------------------------

def random_scene(seed: int, n_surfels: int = 3000, n_nodes: int = 40,
                 width: int = 96, height: int = 72, f: float = 90.0,
                 noise: float = 1e-3, outliers: float = 0.0) -> Scene:
    """A small bending-sphere scene (fills a good part of the image)."""
    cam = Camera(width, height, f, f, width / 2.0 - 0.5, height / 2.0 - 0.25)
    rng = np.random.default_rng(seed)
    center = np.array([0.0, 0.0, 0.75])
    radius = 0.3
    dirs = _fibonacci_sphere(n_surfels)
    v = center + radius * dirs
    node_p, vox = _voxel_nodes(v, n_nodes, lo=0.01, hi=0.6)
    bend = _Bending(rng, amplitude=0.02, period_range=(8.0, 20.0))
    conf = rng.uniform(0.5, 20.0, n_surfels)
    t2 = np.stack([np.zeros(n_surfels), rng.integers(0, 3, n_surfels)], -1)

    def frame(t):
        fr = np.random.default_rng([seed, 3000 + t])
        return _render_sphere(cam, center, radius, lambda x: bend(x, t),
                              noise, outliers, fr)

    return Scene(
        name=f"random_{seed}", cam=cam,
        surfel_v=_f32(v), surfel_n=_f32(dirs),
        surfel_r=_f32(rng.uniform(0.5e-3, 3e-3, n_surfels)),
        surfel_c=_f32(conf), surfel_t=np.ascontiguousarray(t2, dtype=np.int32),
        node_p=_f32(node_p), node_sigma=np.full(len(node_p), vox, dtype=np.float32),
        n_frames=20, gn_iters=3, pcg_iters=8, _frame_fn=frame,
        truth={"bend": bend})


def random_rigid_dq_inputs(seed: int, n: int, max_angle_deg: float = 10.0,
                           max_trans: float = 0.05):
    """Seeded random rigid motions as (unit axis, angle, translation) arrays.

    Stage tests turn these into node transforms on each side; this module
    does not build dual quaternions itself.
    """
    rng = np.random.default_rng(seed)
    axis = _random_dirs(rng, n)
    ang = rng.uniform(0, np.deg2rad(max_angle_deg), n)
    tr = _random_dirs(rng, n) * rng.uniform(0, max_trans, (n, 1))
    return axis, ang, tr


def _render_param(cam, surf, u0, deform, noise, outlier_frac, rng):
    """Depth of a deformed parametric surface x = deform(surf(u)), u in R^2.

    The undeformed surface is sampled at ``u0`` (n, 2) and splatted into a
    per-pixel z-buffer to pick each pixel's starting parameter; Newton then
    puts the deformed point exactly on the pixel's ray.  Pixels whose
    surface faces away or whose solve does not converge stay invalid.
    """
    a, b = cam.rays()
    x0 = deform(surf(u0))
    z0 = x0[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        px = np.floor(cam.fx * x0[:, 0] / z0 + cam.cx + 0.5)
        py = np.floor(cam.fy * x0[:, 1] / z0 + cam.cy + 0.5)
    ok = (z0 > 0) & (px >= 0) & (px < cam.width) & (py >= 0) & (py < cam.height)
    lin = (py[ok] * cam.width + px[ok]).astype(np.int64)
    order = np.lexsort((z0[ok], lin))
    first = np.ones(len(order), dtype=bool)
    first[1:] = lin[order][1:] != lin[order][:-1]
    pix = lin[order][first]
    start = u0[ok][order][first]
    aa, bb = a.ravel()[pix], b.ravel()[pix]

    def fun(p):
        w = deform(surf(p))
        return np.stack([w[:, 0] - aa * w[:, 2], w[:, 1] - bb * w[:, 2]], -1)

    p, conv = _newton2(fun, start)
    w = deform(surf(p))
    h = 1e-6
    tu = deform(surf(p + np.array([h, 0.0]))) - deform(surf(p - np.array([h, 0.0])))
    tv = deform(surf(p + np.array([0.0, h]))) - deform(surf(p - np.array([0.0, h])))
    nrm = np.cross(tu, tv)
    ray = np.stack([aa, bb, np.ones_like(aa)], axis=-1)
    facing = np.abs(np.sum(nrm * ray, axis=1)) > 1e-3 * np.linalg.norm(nrm, axis=1) * np.linalg.norm(ray, axis=1)
    good = conv & facing & (w[:, 2] > 0)
    depth = np.zeros(cam.width * cam.height)
    depth[pix[good]] = w[good, 2]
    valid = depth > 0
    depth = depth + rng.normal(0.0, noise, depth.shape) * valid
    if outlier_frac > 0:
        n_out = int(round(outlier_frac * depth.size))
        pos = rng.choice(depth.size, n_out, replace=False)
        depth[pos] = rng.uniform(0.5, 2.0, n_out)
    return depth.reshape(cam.height, cam.width)


def _param_scene(name, cam, surf, u_model, u_render, seed, n_nodes, noise, outliers, n_frames,
                 conf=15.0):
    """Reference surfels at surf(u_model) with normals from the parameter
    derivatives (oriented towards the camera), voxel-subsampled nodes, and
    frames of the surface bent by three sinusoidal fields."""
    rng = np.random.default_rng(seed)
    v = surf(u_model)
    h = 1e-6
    tu = surf(u_model + np.array([h, 0.0])) - surf(u_model - np.array([h, 0.0]))
    tv = surf(u_model + np.array([0.0, h])) - surf(u_model - np.array([0.0, h]))
    n = _unit(np.cross(tu, tv))
    n = np.where((np.sum(n * v, axis=1) > 0)[:, None], -n, n)
    node_p, vox = _voxel_nodes(v, n_nodes)
    bend = _Bending(rng)
    spacing = np.sqrt(np.linalg.norm(np.cross(tu, tv), axis=1) / (4 * h * h)
                      * (np.ptp(u_model[:, 0]) * np.ptp(u_model[:, 1]) / len(u_model)))

    def frame(t):
        fr = np.random.default_rng([seed, 4000 + t])
        return _render_param(cam, surf, u_render, lambda x: bend(x, t), noise, outliers, fr)

    ns = len(v)
    return Scene(name=name, cam=cam, surfel_v=_f32(v), surfel_n=_f32(n),
                 surfel_r=_f32(np.maximum(spacing, 1e-4)), surfel_c=np.full(ns, conf, dtype=np.float32),
                 surfel_t=np.zeros((ns, 2), dtype=np.int32), node_p=_f32(node_p),
                 node_sigma=np.full(len(node_p), vox, dtype=np.float32), n_frames=n_frames,
                 gn_iters=10, pcg_iters=20, _frame_fn=frame, truth={"bend": bend})


def wavy_plane(seed: int = 0, n_surfels: int = 100_000, n_nodes: int = 1024, width: int = 640,
               height: int = 480, f: float = 570.0, noise: float = 1.5e-3, outliers: float = 0.01,
               n_frames: int = 100) -> Scene:
    """A bending wavy sheet z = 1.1 + 0.04 sin(7x) cos(5y) facing the camera."""
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0)
    hx, hy = 0.5 * width / f * 1.1, 0.5 * height / f * 1.1

    def surf(u):
        x, y = u[:, 0] * hx, u[:, 1] * hy
        return np.stack([x, y, 1.1 + 0.04 * np.sin(7 * x) * np.cos(5 * y)], axis=-1)

    m = int(np.sqrt(n_surfels * hx / hy))
    k = max(2, n_surfels // max(m, 1))
    gu, gv = np.meshgrid(np.linspace(-1, 1, m), np.linspace(-1, 1, k))
    u_model = np.stack([gu.ravel(), gv.ravel()], -1)[:n_surfels]
    ru, rv = np.meshgrid(np.linspace(-1, 1, 3 * width), np.linspace(-1, 1, 3 * height))
    return _param_scene(f"wavy_{width}x{height}_{len(u_model)}s_{n_nodes}n", cam, surf, u_model,
                        np.stack([ru.ravel(), rv.ravel()], -1), seed, n_nodes, noise, outliers, n_frames)


def torus(seed: int = 0, n_surfels: int = 200_000, n_nodes: int = 2048, width: int = 640, height: int = 480,
          f: float = 570.0, noise: float = 1.5e-3, outliers: float = 0.01, n_frames: int = 100) -> Scene:
    """A bending torus (R = 0.25 m, r = 0.08 m) at 1.2 m, tilted 40 degrees."""
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0)
    R, r = 0.25, 0.08
    tilt = _rot_axis_angle(np.array([[1.0, 0.0, 0.0]]), np.array([np.deg2rad(40.0)]))[0]
    center = np.array([0.0, 0.0, 1.2])

    def surf(u):
        a, b = np.pi * u[:, 0], np.pi * u[:, 1]
        p = np.stack([(R + r * np.cos(b)) * np.cos(a), (R + r * np.cos(b)) * np.sin(a), r * np.sin(b)], -1)
        return p @ tilt.T + center

    m = int(np.sqrt(n_surfels * R / r))
    k = max(2, n_surfels // max(m, 1))
    gu, gv = np.meshgrid(np.linspace(-1, 1, m, endpoint=False), np.linspace(-1, 1, k, endpoint=False))
    u_model = np.stack([gu.ravel(), gv.ravel()], -1)[:n_surfels]
    ru, rv = np.meshgrid(np.linspace(-1, 1, 2000, endpoint=False), np.linspace(-1, 1, 700, endpoint=False))
    return _param_scene(f"torus_{width}x{height}_{len(u_model)}s_{n_nodes}n", cam, surf, u_model,
                        np.stack([ru.ravel(), rv.ravel()], -1), seed, n_nodes, noise, outliers, n_frames)


def batch_member(k: int, seed: int = 0, scale: float = 1.0) -> Scene:
    """Member k of the uneven multi-stream workload: depth 320x240..640x480,
    surfels 40k..400k and nodes 256..4096 drawn log-uniformly (seeded by k),
    shapes cycling sphere, torus, wavy plane."""
    rng = np.random.default_rng([seed, k])
    w = int(rng.choice([320, 480, 640]))
    h = w * 3 // 4
    ns = int(np.exp(rng.uniform(np.log(40_000), np.log(400_000))) * scale)
    nn = int(np.exp(rng.uniform(np.log(256), np.log(4096))) * min(1.0, scale * 4))
    nn = max(nn, 16)
    ns = max(ns, 20 * nn)
    f = 570.0 * w / 640.0
    shape = k % 3
    if shape == 0:
        return plain_full(seed=100 + k, n_surfels=ns, n_nodes=nn, width=w, height=h, f=f)
    if shape == 1:
        return torus(seed=100 + k, n_surfels=ns, n_nodes=nn, width=w, height=h, f=f)
    return wavy_plane(seed=100 + k, n_surfels=ns, n_nodes=nn, width=w, height=h, f=f)


def batch_scenes(n_streams: int = 16, seed: int = 0, scale: float = 1.0):
    """The uneven multi-stream workload (see ``batch_member``)."""
    return [batch_member(k, seed, scale) for k in range(n_streams)]
