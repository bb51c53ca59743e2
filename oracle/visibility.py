"""Visibility prediction before the non-rigid solve (Sec. 7: the live surfels
are rendered as opaque disk-shaped splats spanned by their position, normal
and radius, into an index map at the depth image's resolution; only stable
or recently observed surfels are rendered).

TEST INFRASTRUCTURE ONLY: see the package docstring.

Readings of what the paper leaves open:

* rendered surfels: the ones the solver selects (stable, or observed within
  δ_recent frames), at their live positions under the warp the solve starts
  from; the radius is the surfel's own (a warp does not scale it);
* a pixel (x, y) -- centre at integer coordinates, ray q = ((x − cx)/fx,
  (y − cy)/fy, 1) as for the depth map -- is covered by a splat (v, n, r)
  when the ray meets the splat's plane at t = (n·v)/(n·q) > 0 inside the
  disk, ‖t q − v‖² ≤ r²; the pixel's depth for that splat is t;
* opaque rendering: each pixel keeps the splat with the smallest depth,
  equal depths going to the lower surfel id; no back-face culling;
* the pixels tried for a splat: those within h of the pixel of its centre
  (the association's pixel rule) in x and in y, h = min(16, ceil(r·f / (z −
  r)) + 1) with f = max(fx, fy) -- the projected radius of the disk's
  bounding sphere, a pixel of margin and a cap of 16 pixels -- clipped to the
  image; a splat whose bounding sphere reaches the camera plane (z − r ≤ 0)
  is not rendered;
* a surfel is visible when it keeps at least one pixel, and only visible
  surfels take part in the association of every Gauss-Newton iteration of
  the frame.

Every test above decides an integer and is evaluated in FP32 with a fixed
operation order (no fused multiply-add), the precision the CUDA kernel takes
it in.
"""
import numpy as np

from .solver import project_fp32

_F32 = np.float32
MAX_HALF = 16


def splat_half_width(v32, r32, fx, fy):
    """h per surfel (int), or −1 when the splat is not rendered."""
    den = v32[:, 2] - r32
    fm = _F32(max(fx, fy))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        h = np.ceil((r32 * fm) / den) + _F32(1)
        h = np.minimum(h, _F32(MAX_HALF))
    ok = (den > 0) & (v32[:, 2] > 0)
    return np.where(ok, h, -1).astype(np.int64)


def splat_cover(v32, n32, r32, xs, ys, cx, cy, fx, fy):
    """Covered flag and depth t of the splats at the given pixels (FP32, fixed order)."""
    qx = (xs.astype(_F32) - _F32(cx)) / _F32(fx)
    qy = (ys.astype(_F32) - _F32(cy)) / _F32(fy)
    nv = ((n32[:, 0] * v32[:, 0]) + (n32[:, 1] * v32[:, 1])) + (n32[:, 2] * v32[:, 2])
    nq = ((n32[:, 0] * qx) + (n32[:, 1] * qy)) + n32[:, 2]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        t = nv / nq
        dx = (t * qx) - v32[:, 0]
        dy = (t * qy) - v32[:, 1]
        dz = t - v32[:, 2]
        d2 = ((dx * dx) + (dy * dy)) + (dz * dz)
        cov = (t > 0) & (d2 <= r32 * r32)
    return cov, t


def visibility_map(v_live, n_live, radius, selected, cam, chunk=4096):
    """(H, W) int64 map of the nearest covering surfel per pixel (−1: none)."""
    fx, fy, cx, cy, width, height = cam
    v32 = np.asarray(v_live, dtype=_F32)
    n32 = np.asarray(n_live, dtype=_F32)
    r32 = np.asarray(radius, dtype=_F32)
    ids = np.nonzero(np.asarray(selected, dtype=bool))[0]
    h = splat_half_width(v32[ids], r32[ids], fx, fy)
    px, py = project_fp32(v32[ids], fx, fy, cx, cy)
    keep = h >= 0
    ids, h, px, py = ids[keep], h[keep], px[keep].astype(np.int64), py[keep].astype(np.int64)
    off = np.arange(-MAX_HALF, MAX_HALF + 1)
    oy, ox = np.meshgrid(off, off, indexing="ij")
    oy, ox = oy.reshape(-1), ox.reshape(-1)
    pix_all, key_t, key_id = [], [], []
    for s in range(0, len(ids), chunk):
        sl = slice(s, s + chunk)
        i_c, h_c = ids[sl], h[sl]
        xs = px[sl, None] + ox[None, :]
        ys = py[sl, None] + oy[None, :]
        m = (np.abs(ox)[None, :] <= h_c[:, None]) & (np.abs(oy)[None, :] <= h_c[:, None])
        m &= (xs >= 0) & (xs < width) & (ys >= 0) & (ys < height)
        si, k = np.nonzero(m)
        sid = i_c[si]
        xs, ys = xs[si, k], ys[si, k]
        cov, t = splat_cover(v32[sid], n32[sid], r32[sid], xs, ys, cx, cy, fx, fy)
        pix_all.append((ys * width + xs)[cov])
        key_t.append(t[cov])
        key_id.append(sid[cov])
    out = np.full(width * height, -1, dtype=np.int64)
    if pix_all:
        pix = np.concatenate(pix_all)
        tb = np.concatenate(key_t).astype(_F32).view(np.uint32)   # t > 0: bit order = value order
        sid = np.concatenate(key_id)
        order = np.lexsort((sid, tb, pix))
        pix, sid = pix[order], sid[order]
        first = np.ones(len(pix), dtype=bool)
        first[1:] = pix[1:] != pix[:-1]
        out[pix[first]] = sid[first]
    return out.reshape(height, width)


def visible_mask(vis_map, n):
    """Surfels that keep at least one pixel."""
    vis = np.zeros(n, dtype=bool)
    ids = vis_map.reshape(-1)
    vis[ids[ids >= 0]] = True
    return vis
