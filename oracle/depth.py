"""Depth image processing (Sec. 5, Eq. 4), FP64.

For every pixel u = (x, y) (pixel centres at integer coordinates):

* vertex      V(u) = D(u) K⁻¹ (x, y, 1)ᵀ = D ((x−cx)/fx, (y−cy)/fy, 1);
* normal      N(u) by central differences of V:
              normalize((V(x,y+1) − V(x,y−1)) × (V(x+1,y) − V(x−1,y))),
              which faces the camera (N·V < 0) on a fronto-parallel plane.
              Reading: N is invalid on the image border, where any of the
              four neighbours has D ≤ 0, or where the cross product is zero;
* confidence  c = exp(−γ² / (2 φ²)), φ = 0.6, γ = |u − (cx, cy)| / |(cx, cy)|
              (reading: radial distance from the principal point normalised
              by the principal point's distance to the image corner);
* radius      r = √2 d / (f |n_z|) (Eq. 4), f = (fx + fy) / 2, with |n_z|
              clamped below at cos 75° for grazing views (reading of the
              "clamp": clamp the angle, do not discard).

A pixel is usable (a depth surfel) when D > 0 and its normal is valid.
"""
import numpy as np

PHI = 0.6
GRAZING_DEG = 75.0


def depth_maps(depth, fx, fy, cx, cy):
    """Return dict(V (H,W,3), N (H,W,3), valid (H,W) bool, conf, radius)."""
    d = np.asarray(depth, dtype=np.float64)
    h, w = d.shape
    xs, ys = np.meshgrid(np.arange(w, dtype=np.float64), np.arange(h, dtype=np.float64))
    V = np.stack([d * (xs - cx) / fx, d * (ys - cy) / fy, d], axis=-1)
    V[d <= 0] = 0.0

    N = np.zeros_like(V)
    valid = np.zeros((h, w), dtype=bool)
    inner = (slice(1, h - 1), slice(1, w - 1))
    dy = V[2:, 1:-1] - V[:-2, 1:-1]          # V(x, y+1) − V(x, y−1)
    dx = V[1:-1, 2:] - V[1:-1, :-2]          # V(x+1, y) − V(x−1, y)
    cr = np.cross(dy, dx)
    nrm = np.linalg.norm(cr, axis=-1)
    ok = ((d[1:-1, 1:-1] > 0) & (d[2:, 1:-1] > 0) & (d[:-2, 1:-1] > 0)
          & (d[1:-1, 2:] > 0) & (d[1:-1, :-2] > 0) & (nrm > 0))
    N[inner] = np.where(ok[..., None], cr / np.where(nrm > 0, nrm, 1.0)[..., None], 0.0)
    valid[inner] = ok

    gamma = np.hypot(xs - cx, ys - cy) / np.hypot(cx, cy)
    conf = np.exp(-gamma ** 2 / (2.0 * PHI ** 2))
    f = 0.5 * (fx + fy)
    nz = np.maximum(np.abs(N[..., 2]), np.cos(np.deg2rad(GRAZING_DEG)))
    radius = np.where(valid, np.sqrt(2.0) * d / (f * nz), 0.0)
    conf = np.where(valid, conf, 0.0)
    return {"V": V, "N": N, "valid": valid, "conf": conf, "radius": radius}
