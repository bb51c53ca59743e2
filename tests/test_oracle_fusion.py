"""Pins of the oracle's index map, fusion (Sec. 6.1, Eq. 5-6) and inverse warp
(Eq. 3) against brute force on tiny inputs and the paper's stated facts."""
import numpy as np

from oracle import dq as DQ
from oracle import depth as DEPTH
from oracle import fusion as FU
from oracle import solver as S

F32 = np.float32


def _brute_index_map(v, cam):
    fx, fy, cx, cy, w, h = cam
    best = {}
    for i, (x, y, z) in enumerate(np.asarray(v, dtype=F32)):
        if not z > 0:
            continue
        u = F32(F32(F32(F32(fx) * x) / z) + F32(cx))
        vv = F32(F32(F32(F32(fy) * y) / z) + F32(cy))
        su = int(np.floor(F32(4) * F32(u + F32(0.5))))
        sv = int(np.floor(F32(4) * F32(vv + F32(0.5))))
        if not (0 <= su < 4 * w and 0 <= sv < 4 * h):
            continue
        key = (F32(z), i)
        if (sv, su) not in best or key < best[(sv, su)]:
            best[(sv, su)] = key
    out = np.full((4 * h, 4 * w), -1)
    for (sv, su), (_, i) in best.items():
        out[sv, su] = i
    return out


def test_index_map_matches_brute_force_and_ties():
    rng = np.random.default_rng(0)
    cam = (20.0, 20.0, 4.5, 3.5, 10, 8)
    v = np.stack([rng.uniform(-0.3, 0.3, 400), rng.uniform(-0.2, 0.2, 400),
                  rng.uniform(0.8, 1.2, 400)], -1)
    v[3] = [0.01, 0.01, 0.5]           # in the image and nearer than every other surfel
    v[10] = v[3]                       # exact duplicates: the lower id wins
    v[50] = v[3]
    v[7, 2] = -1.0                     # behind the camera
    got = FU.index_map(v, cam)
    np.testing.assert_array_equal(got, _brute_index_map(v, cam))
    ids = got[got >= 0]
    assert len(np.unique(ids)) == len(ids)          # at most one sub-pixel per surfel
    assert 3 in ids and 10 not in ids and 50 not in ids and 7 not in ids


def test_window_search_brute_force_and_update():
    rng = np.random.default_rng(1)
    cam = (30.0, 30.0, 3.5, 2.5, 8, 6)
    d = np.full((6, 8), 1.0, dtype=F32)
    m = DEPTH.depth_maps(d, *cam[:4])
    V32, N32 = m["V"].astype(F32), m["N"].astype(F32)
    # surfels scattered around the usable pixels' vertices
    pix = np.nonzero(m["valid"].reshape(-1))[0]
    base = m["V"].reshape(-1, 3)[np.repeat(pix, 5)]
    v = base + rng.normal(0, 6e-4, base.shape)
    n = np.tile([0.0, 0.0, -1.0], (len(v), 1)) + rng.normal(0, 0.3, (len(v), 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    conf = rng.choice([1.0, 2.0, 3.0], len(v))
    imap = FU.index_map(v, cam)
    tgt = FU.select_fusion_targets(imap, v, n, conf, V32, N32, m["valid"], 1e-3, 0.85)
    # brute force per pixel
    h, w = 6, 8
    for y in range(h):
        for x in range(w):
            best = None
            if m["valid"][y, x]:
                for sid in imap[4 * y:4 * y + 4, 4 * x:4 * x + 4].ravel():
                    if sid < 0:
                        continue
                    dv = v[sid].astype(F32) - V32[y, x]
                    d2 = F32(F32(F32(dv[0] * dv[0]) + F32(dv[1] * dv[1])) + F32(dv[2] * dv[2]))
                    nn = n[sid].astype(F32)
                    dt = F32(F32(F32(nn[0] * N32[y, x, 0]) + F32(nn[1] * N32[y, x, 1]))
                             + F32(nn[2] * N32[y, x, 2]))
                    if d2 <= F32(F32(1e-3) * F32(1e-3)) and dt >= F32(0.85):
                        key = (-F32(conf[sid]), d2, sid)
                        best = key if best is None or key < best else best
            assert tgt[y * w + x] == (-1 if best is None else best[2])
    assert np.sum(tgt >= 0) > 5


def test_surfel_on_noise_free_depth_keeps_geometry():
    cam = (30.0, 30.0, 3.5, 2.5, 8, 6)
    d = np.full((6, 8), 1.0, dtype=F32)
    m = DEPTH.depth_maps(d, *cam[:4])
    y, x = 3, 4
    v = m["V"][y, x][None].copy()
    n = m["N"][y, x][None].copy()
    conf, rad, tob = np.array([2.0]), np.array([5e-3]), np.array([0])
    imap = FU.index_map(v, cam)
    tgt = FU.select_fusion_targets(imap, v, n, conf, m["V"].astype(F32), m["N"].astype(F32),
                                   m["valid"], 1e-3, 0.85)
    assert tgt[y * 8 + x] == 0
    v2, n2, r2, c2, t2, fused = FU.fuse(v, n, rad, conf, tob, m, tgt, 7)
    np.testing.assert_allclose(v2, v, atol=1e-16)
    np.testing.assert_allclose(n2, n, atol=1e-16)
    assert c2[0] == 2.0 + m["conf"][y, x] and t2[0] == 7 and fused[0]
    cd, rd = m["conf"][y, x], m["radius"][y, x]
    assert r2[0] == (2.0 * 5e-3 + cd * rd) / (2.0 + cd)


def test_inverse_warp_undoes_forward_warp():
    rng = np.random.default_rng(2)
    nodes = 5
    dq = DQ.dq_from_rt(DQ.rodrigues_quat(rng.normal(size=(nodes, 3)) * 0.1),
                       rng.normal(size=(nodes, 3)) * 0.02)
    knn = rng.integers(0, nodes, (50, 4))
    w = rng.uniform(0.1, 1, (50, 4))
    v = rng.normal(size=(50, 3))
    n = rng.normal(size=(50, 3))
    b, vl, nl = S.warp_surfels(v, n, knn, w, dq)
    vr, nr = FU.inverse_warp(b, vl, nl)
    np.testing.assert_allclose(vr, v, atol=1e-13)
    np.testing.assert_allclose(nr, n, atol=1e-13)
