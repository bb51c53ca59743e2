"""Fusion at the live frame and the inverse warp (Sec. 6.1, Eq. 5-6; Sec. 4, Eq. 3).

* Index map (Sec. 6.1): every live surfel with z > 0 is projected as an
  unsized point into a 4x super-sampled map (4W x 4H): sub-pixel
  (floor(4 (u + ½)), floor(4 (v + ½))) with u = fx x / z + cx in FP32 (the
  same projection as association), so sub-pixel s lies in pixel floor(s/4).
  Each sub-pixel keeps the nearest surfel (smallest FP32 z); equal depths go
  to the lower surfel id.  A surfel lands in at most one sub-pixel.
* Window (Sec. 6.1): reading of the "4x4 window centred at u": exactly the
  16 sub-pixels of depth pixel u, so each surfel is a candidate of exactly one
  pixel and no surfel can be fused twice.
* Candidates: discard a surfel farther than δ_distance from the depth vertex
  (kept when ‖v − V(u)‖² ≤ δ_distance²) or with n · N(u) < δ_normal (kept when
  ≥); among the rest take the highest confidence, then the smallest distance,
  then (reading) the lowest surfel id.  All tests in FP32 with fixed order.
* Update (Eq. 5-6): c ← c + c_d; v, n, r ← confidence-weighted averages;
  t_observed ← t_now.  Reading: n is re-normalised after averaging.
* Inverse warp (Eq. 3) of every fused surfel with its own skinning and the
  final node transforms: v_ref = R⁻¹ (v_live − t), n_ref = R⁻¹ n_live.
"""
import numpy as np

from . import dq as DQ
from .solver import project_fp32, dist2_fp32, dot_fp32

_F32 = np.float32
SUPER = 4


def index_map(v_live, cam):
    """(4H, 4W) int64 map of surfel ids (−1 = empty)."""
    fx, fy, cx, cy, width, height = cam
    v32 = np.asarray(v_live, dtype=_F32)
    ok = v32[:, 2] > 0
    u, v = _subpixel(v32, fx, fy, cx, cy)
    with np.errstate(invalid="ignore"):
        ok &= (u >= 0) & (u < SUPER * width) & (v >= 0) & (v < SUPER * height)
    ids = np.nonzero(ok)[0]
    lin = v[ids].astype(np.int64) * (SUPER * width) + u[ids].astype(np.int64)
    zbits = v32[ids, 2].view(np.uint32)
    order = np.lexsort((ids, zbits, lin))
    lin_s, ids_s = lin[order], ids[order]
    first = np.ones(len(order), dtype=bool)
    first[1:] = lin_s[1:] != lin_s[:-1]
    out = np.full(SUPER * SUPER * width * height, -1, dtype=np.int64)
    out[lin_s[first]] = ids_s[first]
    return out.reshape(SUPER * height, SUPER * width)


def _subpixel(v32, fx, fy, cx, cy):
    """Sub-pixel coordinates floor(4 (u + ½)) in FP32 (4x is exact)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        u = ((_F32(fx) * v32[:, 0]) / v32[:, 2]) + _F32(cx)
        v = ((_F32(fy) * v32[:, 1]) / v32[:, 2]) + _F32(cy)
        return (np.floor(_F32(SUPER) * (u + _F32(0.5))),
                np.floor(_F32(SUPER) * (v + _F32(0.5))))


def select_fusion_targets(imap, v_live, n_live, conf, V32, N32, usable,
                          fuse_dist, fuse_normal):
    """For each usable depth pixel, the surfel it fuses into (−1 if none)."""
    hh, ww = usable.shape
    win = imap.reshape(hh, SUPER, ww, SUPER).transpose(0, 2, 1, 3).reshape(hh * ww, SUPER * SUPER)
    v32 = np.asarray(v_live, dtype=_F32)
    n32 = np.asarray(n_live, dtype=_F32)
    c32 = np.asarray(conf, dtype=_F32)
    Vf, Nf = V32.reshape(-1, 3), N32.reshape(-1, 3)
    ok_pix = usable.reshape(-1)
    fd = _F32(fuse_dist)
    fd2 = fd * fd
    best = np.full(hh * ww, -1, dtype=np.int64)
    best_c = np.full(hh * ww, -np.inf, dtype=_F32)
    best_d = np.full(hh * ww, np.inf, dtype=_F32)
    for k in range(SUPER * SUPER):
        sid = win[:, k]
        cand = (sid >= 0) & ok_pix
        pix = np.nonzero(cand)[0]
        s = sid[pix]
        d2 = dist2_fp32(v32[s], Vf[pix])
        dt = dot_fp32(n32[s], Nf[pix])
        keep = (d2 <= fd2) & (dt >= _F32(fuse_normal))
        pix, s, d2 = pix[keep], s[keep], d2[keep]
        c = c32[s]
        better = ((c > best_c[pix])
                  | ((c == best_c[pix]) & (d2 < best_d[pix]))
                  | ((c == best_c[pix]) & (d2 == best_d[pix]) & (s < best[pix])))
        pix, s, d2, c = pix[better], s[better], d2[better], c[better]
        best[pix], best_c[pix], best_d[pix] = s, c, d2
    return best


def fuse(v_live, n_live, radius, conf, t_obs, maps, target, t_now):
    """Eq. 5-6 for every pixel with a target surfel.  Returns updated copies
    (v_live, n_live, radius, conf, t_obs) and the fused-surfel mask."""
    v_live, n_live = v_live.copy(), n_live.copy()
    radius, conf, t_obs = radius.copy(), conf.copy(), t_obs.copy()
    pix = np.nonzero(target >= 0)[0]
    s = target[pix]
    cd = maps["conf"].reshape(-1)[pix]
    vd = maps["V"].reshape(-1, 3)[pix]
    nd = maps["N"].reshape(-1, 3)[pix]
    rd = maps["radius"].reshape(-1)[pix]
    c_old = conf[s]
    c_new = c_old + cd
    v_live[s] = (c_old[:, None] * v_live[s] + cd[:, None] * vd) / c_new[:, None]
    n_avg = (c_old[:, None] * n_live[s] + cd[:, None] * nd) / c_new[:, None]
    n_live[s] = n_avg / np.linalg.norm(n_avg, axis=1, keepdims=True)
    radius[s] = (c_old * radius[s] + cd * rd) / c_new
    conf[s] = c_new
    t_obs[s] = t_now
    fused = np.zeros(len(v_live), dtype=bool)
    fused[s] = True
    return v_live, n_live, radius, conf, t_obs, fused


def inverse_warp(b, v_live, n_live):
    """Eq. 3 with the surfel's own (unchanged) blend b."""
    return (DQ.dq_inverse_transform_point(b, v_live),
            DQ.dq_inverse_rotate_vector(b, n_live))
