"""Pins of the splat-visibility oracle (Sec. 7) against closed forms and a
float64 brute force of the ray-disk intersection over every pixel."""
import numpy as np

from oracle import visibility as VIS
from oracle import stream as OST

import synth

CAM = (100.0, 100.0, 31.5, 23.5, 64, 48)   # fx fy cx cy W H


def _brute(v, n, r, sel, cam):
    """Nearest covering splat per pixel in float64, every pixel of the image;
    also the margin of each decision (|d² − r²| and the depth gap), so that
    pixels on a rounding boundary can be left out of the comparison."""
    fx, fy, cx, cy, W, H = cam
    ys, xs = np.mgrid[0:H, 0:W]
    q = np.stack([(xs - cx) / fx, (ys - cy) / fy, np.ones_like(xs, dtype=float)], axis=-1)
    best = np.full((H, W), -1)
    bt = np.full((H, W), np.inf)
    margin = np.full((H, W), np.inf)
    for i in np.nonzero(sel)[0]:
        nq = q @ n[i]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (n[i] @ v[i]) / nq
            d2 = np.sum((t[..., None] * q - v[i]) ** 2, axis=-1)
        cov = (t > 0) & (d2 <= r[i] ** 2)
        near = np.abs(d2 - r[i] ** 2) / r[i] ** 2
        margin = np.minimum(margin, np.where(np.isfinite(near), near, np.inf))
        closer = cov & ((t < bt) | ((t == bt) & (i < best)))
        gap = np.abs(t - bt)
        margin = np.minimum(margin, np.where(cov & np.isfinite(bt), gap / np.maximum(t, 1e-9), np.inf))
        best = np.where(closer, i, best)
        bt = np.where(closer, t, bt)
    return best, margin


def test_fronto_parallel_disk_closed_form():
    """A disk facing the camera at depth z0 covers exactly the pixels whose ray
    passes within r of its centre: ((x−cx)/fx − a)² + ((y−cy)/fy − b)² ≤ (r/z0)²."""
    z0, r = 1.0, 0.05
    a, b = 0.013, -0.021
    v = np.array([[a * z0, b * z0, z0]])
    n = np.array([[0.0, 0.0, -1.0]])
    vm = VIS.visibility_map(v, n, np.array([r]), np.array([True]), CAM)
    fx, fy, cx, cy, W, H = CAM
    ys, xs = np.mgrid[0:H, 0:W]
    lhs = ((xs - cx) / fx - a) ** 2 + ((ys - cy) / fy - b) ** 2
    rhs = (r / z0) ** 2
    clear = np.abs(lhs - rhs) > 1e-5
    assert np.array_equal((vm >= 0)[clear], (lhs <= rhs)[clear])
    assert (vm >= 0).sum() > 60            # π (r f / z0)² ≈ 79 pixels


def test_random_splats_match_float64_brute_force():
    """Tilted overlapping splats at several depths: the nearest covering splat
    per pixel equals a float64 brute force away from rounding boundaries,
    and unselected surfels are never drawn."""
    rng = np.random.default_rng(4)
    k = 60
    z = rng.uniform(0.8, 1.5, k)
    v = np.stack([rng.uniform(-0.3, 0.3, k) * z, rng.uniform(-0.22, 0.22, k) * z, z], axis=1)
    n = rng.normal(size=(k, 3))
    n[:, 2] = -np.abs(n[:, 2]) - 0.3
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r = rng.uniform(0.01, 0.06, k)
    sel = rng.random(k) < 0.85
    v32, n32, r32 = v.astype(np.float32), n.astype(np.float32), r.astype(np.float32)
    vm = VIS.visibility_map(v32, n32, r32, sel, CAM)
    want, margin = _brute(v32.astype(float), n32.astype(float), r32.astype(float), sel, CAM)
    # pixels the 16-pixel cap leaves out of a splat's square are not compared
    fx = CAM[0]
    big = r32 * fx / (v32[:, 2] - r32) + 1 > VIS.MAX_HALF
    assert not big[sel].any()
    ok = margin > 1e-5
    assert np.array_equal(vm[ok], want[ok])
    assert ok.mean() > 0.9 and (want >= 0).sum() > 500
    drawn = np.unique(vm[vm >= 0])
    assert sel[drawn].all()
    vis = VIS.visible_mask(vm, k)
    assert vis.sum() < sel.sum()          # some selected splats are hidden
    assert np.array_equal(vis, np.isin(np.arange(k), drawn))


def test_equal_depths_go_to_the_lower_id_and_hidden_splats_are_invisible():
    v = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0], [0.0, 0.0, 1.2]])
    n = np.array([[0.0, 0.0, -1.0]] * 3)
    r = np.array([0.04, 0.04, 0.02])
    vm = VIS.visibility_map(v, n, r, np.array([True, True, True]), CAM)
    assert set(np.unique(vm)) == {-1, 0}
    assert list(VIS.visible_mask(vm, 3)) == [True, False, False]
    # surfel 2 alone is drawn
    vm2 = VIS.visibility_map(v, n, r, np.array([False, False, True]), CAM)
    assert (vm2 == 2).sum() > 0


def test_half_width_rule():
    v = np.array([[0, 0, 1.0], [0, 0, 0.03], [0, 0, 0.5], [0, 0, -1.0]], np.float32)
    r = np.array([0.02, 0.05, 0.2, 0.01], np.float32)
    h = VIS.splat_half_width(v, r, 100.0, 120.0)
    # ceil(0.02·120 / 0.98) + 1 = 4; z − r ≤ 0: not drawn; capped at 16; behind the camera
    assert list(h) == [4, -1, 16, -1]


def test_stream_visibility_hides_the_back_of_a_sphere():
    """On a closed surface sampled at least once per pixel, whose surfels
    carry the radius a depth pixel gives them (Sec. 5: r = √2 z / (f
    max(|n_z|, cos 75°))), the splats close over the front half: every depth
    pixel of the sphere is drawn, and no surfel facing away from the camera
    is visible (beyond grazing ones at the silhouette, whose clamped radius
    reaches past the rim)."""
    import dataclasses
    sc = synth.random_scene(seed=3, n_surfels=40000, n_nodes=48)
    c = sc.cam
    v, n = sc.surfel_v.astype(float), sc.surfel_n.astype(float)
    view = v / np.linalg.norm(v, axis=1, keepdims=True)
    cosv = np.abs(np.einsum('ij,ij->i', n, view))
    r = np.sqrt(2.0) * v[:, 2] / (c.fx * np.maximum(cosv, np.cos(np.deg2rad(75.0))))
    sc = dataclasses.replace(sc, surfel_r=r.astype(np.float32), surfel_c=np.full(len(v), 20.0, np.float32))
    st = OST.OracleStream(OST.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy, visibility=True))
    st.set_model(sc.surfel_v, sc.surfel_n, sc.surfel_r, sc.surfel_c, sc.surfel_t, sc.node_p, sc.node_sigma)
    st.upload_depth(sc.frame(0), 0)
    vis = st.predict_visibility()
    cos_view = np.einsum('ij,ij->i', n, view)   # > 0: facing away
    assert vis.sum() > 1000
    assert cos_view[vis].max() < 0.15 and np.sum(cos_view > 0.15) > 10000
    assert vis.sum() > 0.5 * (st.vis_map >= 0).sum()
    drawn = st.vis_map >= 0
    valid = st.maps["valid"]
    assert (drawn & valid).sum() >= 0.98 * valid.sum()
