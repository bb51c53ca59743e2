"""Appending and removal on the GPU (Sec. 6.2-6.4, Eq. 7-8) against the oracle.

The record test hands both sides identical FP32 inputs (depth maps, live
surfels, node transforms), so the integer decisions -- candidate pixels, the
live k-NN, the Eq. 7 node mask, the appended set and the new caller order --
must agree exactly; the weight-sum and strain tests are FP64 on both sides and
may differ only within 1e-9 of their thresholds.  The end-to-end test runs
the normal calls (solve, fusion, appending, the next solve on the grown
model) and compares within the solve's tolerances."""
import dataclasses

import numpy as np
import pytest

import synth
import oracle
import paper_1904_13073_gb300 as sw
from oracle import append as AP
from oracle import fusion as OFU
from oracle import skinning as OSK
from oracle import solver as OS

from gpu_helpers import ensure_built, rigid_dq8_from, rotation_angle_between

pytestmark = pytest.mark.gpu
F32 = np.float32
# the library's parameters are FP32: the oracle takes the same values
EPS = float(F32(0.2))
DNN = float(F32(0.3))
FDH = float(F32(1e-3))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _cut(scene, frac=0.3, unstable=7):
    """The scene with the surfels of its largest-x fraction removed (a hole
    that new depth fills) and `unstable` low-confidence surfels made old."""
    keep = scene.surfel_v[:, 0] < np.quantile(scene.surfel_v[:, 0], 1.0 - frac)
    c = scene.surfel_c[keep].copy()
    t = scene.surfel_t[keep].copy()
    c[:unstable] = 5.0
    t[:unstable, 0] = -40
    c[unstable:2 * unstable] = 5.0     # low confidence but young: they stay
    t[unstable:2 * unstable, 0] = -10
    return dataclasses.replace(scene, surfel_v=scene.surfel_v[keep], surfel_n=scene.surfel_n[keep],
                               surfel_r=scene.surfel_r[keep], surfel_c=c, surfel_t=t)


class Both:
    def __init__(self, scene, max_surfels, precision=sw.SW_PRECISION_MIXED, max_nodes=None):
        c = scene.cam
        self.scene = scene
        v4, n4, t2, node4 = sw.model_arrays(scene)
        self.h = sw.sw_create_stream(sw.params_for(c, max_surfels, max_nodes or len(node4), precision=precision))
        sw.sw_set_model(self.h, v4, n4, t2, node4)
        self.o = oracle.OracleStream(oracle.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy))
        self.o.set_model(scene.surfel_v, scene.surfel_n, scene.surfel_r, scene.surfel_c, scene.surfel_t,
                         scene.node_p, scene.node_sigma)
        self.max_surfels = max_surfels

    def close(self):
        sw.sw_destroy_stream(self.h)

    def set_maps(self, far_frac=0.0, seed=0):
        """Identical FP32 maps on both sides; a fraction of the vertices pushed
        0.5 m back (far from every node: the weight-sum test rejects them)."""
        m = self.o.maps
        if far_frac:
            rng = np.random.default_rng(seed)
            far = (rng.random(m["valid"].shape) < far_frac) & m["valid"]
            m["V"] = m["V"].copy()
            m["V"][far] *= (m["V"][far][:, 2:3] + 0.5) / m["V"][far][:, 2:3]
        V4 = np.zeros(m["V"].shape[:2] + (4,), F32)
        N4 = np.zeros_like(V4)
        V4[..., :3] = m["V"]
        V4[..., 3] = np.where(m["valid"], m["conf"], 0.0)
        N4[..., :3] = m["N"]
        N4[..., 3] = m["radius"]
        sw.sw_debug_set_maps(self.h, V4, N4)
        m["V"] = V4[..., :3].astype(np.float64)
        m["N"] = N4[..., :3].astype(np.float64)
        m["conf"] = V4[..., 3].astype(np.float64)
        m["radius"] = N4[..., 3].astype(np.float64)
        self.o.V32 = V4[..., :3].copy()
        self.o.N32 = N4[..., :3].copy()


def _warp(scene, seed, angle, trans, alpha=0.19):
    """Node transforms: small random rigid motions, then, for the nodes in the
    upper half (y below the median), a contraction by `alpha` towards the
    nodes' centroid.  Live node distances there shrink by 1 − alpha (inside
    Eq. 7's band for alpha < ε) while the inverse warp expands by about
    1 / (1 − alpha), past Eq. 8's bound 1 + ε; across the border of the
    region Eq. 7 drops nodes."""
    axis, ang, tr = synth.random_rigid_dq_inputs(seed, len(scene.node_p), angle, trans)
    q = rigid_dq8_from(axis, ang, tr).astype(np.float64)
    p = scene.node_p.astype(np.float64)
    t = -np.where(p[:, 1] < np.median(p[:, 1]), alpha, 0.0)[:, None] * (p - p.mean(axis=0))
    # (1, 0; 0, t/2) ⊗ q: the contraction's translation applied after q
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    tx, ty, tz = 0.5 * t[:, 0], 0.5 * t[:, 1], 0.5 * t[:, 2]
    out = q.copy()
    out[:, 4] += -tx * x - ty * y - tz * z
    out[:, 5] += tx * w + ty * z - tz * y
    out[:, 6] += -tx * z + ty * w + tz * x
    out[:, 7] += tx * y - ty * x + tz * w
    return out.astype(F32)


SCENES = {
    "tiny": lambda: _cut(synth.plain_tiny(seed=0)),
    "small": lambda: _cut(synth.random_scene(seed=5, n_surfels=5000, n_nodes=60, outliers=0.01)),
}


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_MIXED, sw.SW_PRECISION_FP64])
@pytest.mark.parametrize("which", ["tiny", "small"])
def test_append_records_and_model_match_oracle(which, precision):
    scene = SCENES[which]()
    c = scene.cam
    b = Both(scene, len(scene.surfel_v) + c.width * c.height, precision)
    try:
        d = scene.frame(1)
        sw.sw_upload_depth(b.h, d, 1)
        b.o.upload_depth(d, 1)
        b.set_maps(far_frac=0.03)
        dq8 = _warp(scene, 21, 1.0, 0.005)
        odq = dq8.astype(np.float64)
        sw.sw_set_node_dq(b.h, dq8)
        _, vl, nl = OS.warp_surfels(b.o.v_ref, b.o.n_ref, b.o.knn, b.o.w, odq)
        vl32, nl32 = vl.astype(F32), nl.astype(F32)
        sw.sw_debug_set_live(b.h, vl32, nl32)
        sw.sw_debug_fusion_targets(b.h, c.height, c.width)
        st = sw.sw_append_frame(b.h)
        rec = sw.sw_debug_read_append(b.h)

        m = b.o.maps
        pix = AP.empty_window_pixels(OFU.index_map(vl32, b.o.p.cam), m["valid"])
        res = AP.append_candidates(pix, m, odq, b.o.node_p, b.o.node_sigma, EPS, DNN, FDH)
        np.testing.assert_array_equal(rec["pix"], pix)
        np.testing.assert_array_equal(rec["knn"], res["knn"])
        keep_bits = sum((res["keep"][:, k].astype(np.int32) << k) for k in range(4))
        np.testing.assert_array_equal(rec["flags"] & 15, keep_bits)
        ok = res["wsum"] > 1e-6   # a blend of all-but-vanishing weights is not compared
        np.testing.assert_allclose(rec["wsum"], res["wsum"], rtol=1e-12, atol=1e-300)
        np.testing.assert_allclose(rec["strain"][ok], res["strain"][ok], atol=1e-8)
        np.testing.assert_allclose(rec["v4"][ok, :3], res["v_ref"][ok], atol=2e-6)
        np.testing.assert_allclose(rec["n4"][ok, :3], res["n_ref"][ok], atol=2e-6)
        low = (rec["flags"] & 32) != 0
        comp = (rec["flags"] & 64) != 0
        near_nn = np.abs(res["wsum"] - DNN) < 1e-9
        near_s = np.abs(res["strain_norm"] - (1 + EPS)) < 1e-9
        assert np.all((low == (res["wsum"] < DNN)) | near_nn)
        assert np.all((comp == (res["strain_norm"] > 1 + EPS)) | near_s | ~ok)
        acc = (rec["flags"] & 16) != 0
        assert np.all((acc == res["accept"]) | near_nn | near_s)
        # every test did something on this input (the sphere's wide node
        # support smooths the contraction below Eq. 8's bound)
        assert low.sum() > 0 and acc.sum() > 0 and (keep_bits != 15).sum() > 0
        assert comp.sum() > 0 or which == "small"
        assert st["candidates"] == len(pix) and st["appended"] == int(acc.sum())
        assert st["rejected_nn"] == int(low.sum()) and st["rejected_strain"] == int(comp.sum())

        # the new model: survivors in caller order, then the appended ones
        stay = ~AP.unstable(b.o.conf, b.o.t_init, 1, b.o.p.stable_conf)
        assert st["removed"] == int((~stay).sum()) == 7
        ns = int(stay.sum())
        v, n, t2 = sw.sw_read_surfels(b.h)
        knn, w = sw.sw_read_skinning(b.h)
        assert len(v) == st["n_surfels"] == ns + st["appended"]
        np.testing.assert_array_equal(v[:ns, :3], b.o.v_ref[stay].astype(F32))
        np.testing.assert_array_equal(t2[:ns, 0], b.o.t_init[stay])
        np.testing.assert_array_equal(knn[:ns], b.o.knn[stay])
        ia = np.nonzero(acc)[0]
        np.testing.assert_allclose(v[ns:, :3], res["v_ref"][ia], atol=2e-6)
        np.testing.assert_allclose(n[ns:, :3], res["n_ref"][ia], atol=2e-6)
        np.testing.assert_array_equal(v[ns:, 3], m["radius"].reshape(-1)[pix[ia]].astype(F32))
        np.testing.assert_array_equal(n[ns:, 3], m["conf"].reshape(-1)[pix[ia]].astype(F32))
        assert np.all(t2[ns:] == 1)
        # reference skinning of the appended surfels by the initialisation rule
        oknn = OSK.knn_fp32(res["v_ref"][ia].astype(F32), b.o.node_p.astype(F32), 4)
        np.testing.assert_array_equal(knn[ns:], oknn)
        ow = OSK.skin_weights(res["v_ref"][ia], b.o.node_p, b.o.node_sigma, oknn)
        np.testing.assert_allclose(w[ns:], ow, rtol=2e-6, atol=1e-30)
        # the node transforms are untouched
        np.testing.assert_array_equal(sw.sw_read_nodes(b.h)[1], dq8)
    finally:
        b.close()


def test_append_capacity_cuts_from_the_end():
    scene = SCENES["tiny"]()
    c = scene.cam
    ns0 = len(scene.surfel_v)
    b = Both(scene, ns0 + c.width * c.height)
    cap = ns0 - 7 + 25   # room for 25 after the removals
    b2 = Both(scene, cap)
    try:
        outs = []
        dq8 = _warp(scene, 3, 0.5, 0.002, alpha=0.0)
        for x in (b, b2):   # the same fixed warp (the solve's FP32 atomics are not bitwise repeatable)
            sw.sw_upload_depth(x.h, scene.frame(1), 1)
            sw.sw_set_node_dq(x.h, dq8)
            sw.sw_fuse_frame(x.h)
            outs.append(sw.sw_append_frame(x.h))
        full, cut = outs
        assert full["appended"] > 25 and cut["appended"] == 25 and cut["n_surfels"] == cap
        v_full = sw.sw_read_surfels(b.h)[0]
        v_cut = sw.sw_read_surfels(b2.h)[0]
        np.testing.assert_array_equal(v_cut, v_full[:cap])
        # a second call without a new fusion is refused (no GPU work)
        with pytest.raises(sw.SwError) as e:
            sw.sw_append_frame(b.h)
        assert e.value.status == 3
    finally:
        b.close()
        b2.close()


def test_append_end_to_end_then_solve_on_the_grown_model():
    """Normal calls on both sides: solve + fusion + appending on frame 1, then
    the same depth as frame 2 solved with the grown model (the new surfels
    are recent, so they take part in the association of frame 2)."""
    scene = SCENES["tiny"]()
    c = scene.cam
    b = Both(scene, len(scene.surfel_v) + c.width * c.height)
    try:
        d = scene.frame(1)
        sw.sw_upload_depth(b.h, d, 1)
        b.o.upload_depth(d, 1)
        sw.sw_solve_frame(b.h, 3, 8)
        b.o.solve_frame(3, 8)
        sw.sw_fuse_frame(b.h)
        b.o.fuse_frame()
        st = sw.sw_append_frame(b.h)
        n_cand, n_app, n_rem = b.o.append_frame(b.max_surfels, EPS, DNN, FDH)
        assert st["removed"] == n_rem == 7
        # 1-ulp differences of the warps may move a few surfels across sub-pixel borders
        assert abs(st["candidates"] - n_cand) <= max(3, n_cand // 200)
        assert abs(st["appended"] - n_app) <= max(3, n_app // 200)
        assert n_app > 500
        v, n, t2 = sw.sw_read_surfels(b.h)
        ns = len(v) - st["appended"]
        rec = sw.sw_debug_read_append(b.h)
        gpix = rec["pix"][(rec["flags"] & 16) != 0]
        opix = b.o.last_append["pix"][b.o.last_append["appended"]]
        common, gi, oi = np.intersect1d(gpix, opix, return_indices=True)
        assert len(common) >= 0.99 * len(opix)
        np.testing.assert_allclose(v[ns + gi, :3], b.o.v_ref[len(b.o.v_ref) - n_app + oi], atol=5e-5)
        # frame 2 on the grown model
        sw.sw_upload_depth(b.h, d, 2)
        b.o.upload_depth(d, 2)
        st2 = sw.sw_solve_frame(b.h, 3, 8)
        ost2 = b.o.solve_frame(3, 8)
        assert abs(st2["n_corr"][0] - ost2[0].n_corr) <= max(5, ost2[0].n_corr // 500)
        _, dq = sw.sw_read_nodes(b.h)
        dq = dq.astype(np.float64)
        assert rotation_angle_between(dq, b.o.node_dq).max() < 1e-4
        got = OS.node_transform(dq, b.o.node_p)
        assert np.linalg.norm(got - b.o.warped_nodes(), axis=1).max() < 2e-5
    finally:
        b.close()


def _cut_nodes(scene, frac=0.3):
    """The scene with its largest-x surfels and the nodes in that region removed,
    so that the appended surfels there are farther than every node's radius."""
    x_cut = np.quantile(scene.surfel_v[:, 0], 1.0 - frac)
    sc = _cut(scene, frac)
    keep_n = scene.node_p[:, 0] < x_cut - 0.05
    return dataclasses.replace(sc, node_p=scene.node_p[keep_n], node_sigma=scene.node_sigma[keep_n])


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_MIXED, sw.SW_PRECISION_FP64])
def test_node_extension_matches_oracle(precision):
    """Identical FP32 inputs on both sides (maps, node transforms, live
    surfels); appending with node-graph extension: the new nodes, their
    transforms, the graph and every surfel's skinning agree, and the next
    solve runs on the extended graph."""
    scene = _cut_nodes(synth.plain_tiny(seed=2))
    c = scene.cam
    n_old = len(scene.node_p)
    b = Both(scene, len(scene.surfel_v) + c.width * c.height, precision, max_nodes=n_old + 64)
    try:
        d = scene.frame(1)
        sw.sw_upload_depth(b.h, d, 1)
        b.o.upload_depth(d, 1)
        b.set_maps()
        dq8 = _warp(scene, 5, 0.5, 0.002, alpha=0.0)
        sw.sw_set_node_dq(b.h, dq8)
        b.o.node_dq = dq8.astype(np.float64)
        _, vl, nl = OS.warp_surfels(b.o.v_ref, b.o.n_ref, b.o.knn, b.o.w, b.o.node_dq)
        vl32, nl32 = vl.astype(F32), nl.astype(F32)
        sw.sw_debug_set_live(b.h, vl32, nl32)
        sw.sw_debug_fusion_targets(b.h, c.height, c.width)
        st = sw.sw_append_frame(b.h)
        b.o.last_index_map = OFU.index_map(vl32, b.o.p.cam)
        _, n_app, n_rem = b.o.append_frame(b.max_surfels, EPS, DNN, FDH, extend_nodes=True, max_nodes=n_old + 64)
        assert st["appended"] == n_app and st["removed"] == n_rem
        assert st["new_nodes"] == b.o.new_nodes > 0
        pos, dq = sw.sw_read_nodes(b.h)
        assert len(pos) == len(b.o.node_p) == n_old + st["new_nodes"]
        np.testing.assert_allclose(pos[:, :3], b.o.node_p, atol=2e-6)
        np.testing.assert_array_equal(pos[:, 3], b.o.node_sigma.astype(F32))
        np.testing.assert_array_equal(dq[:n_old], dq8)
        assert np.max(rotation_angle_between(dq[n_old:].astype(np.float64), b.o.node_dq[n_old:])) < 1e-6
        np.testing.assert_allclose(OS.node_transform(dq[n_old:].astype(np.float64), b.o.node_p[n_old:]),
                                   OS.node_transform(b.o.node_dq[n_old:], b.o.node_p[n_old:]), atol=2e-6)
        np.testing.assert_array_equal(sw.sw_read_graph(b.h), b.o.graph)
        knn, w = sw.sw_read_skinning(b.h)
        np.testing.assert_array_equal(knn, b.o.knn)
        np.testing.assert_allclose(w, b.o.w, rtol=2e-6, atol=1e-30)
        # the next frame solves on the extended graph
        sw.sw_upload_depth(b.h, d, 2)
        b.o.upload_depth(d, 2)
        b.set_maps()
        st2 = sw.sw_solve_frame(b.h, 2, 8)
        ost2 = b.o.solve_frame(2, 8)
        assert abs(st2["n_corr"][0] - ost2[0].n_corr) <= 3
        _, dq2 = sw.sw_read_nodes(b.h)
        dq2 = dq2.astype(np.float64)
        assert rotation_angle_between(dq2, b.o.node_dq).max() < 1e-4
        assert np.linalg.norm(OS.node_transform(dq2, b.o.node_p) - b.o.warped_nodes(), axis=1).max() < 2e-5
    finally:
        b.close()


def test_fast_update_on_a_growing_model_matches_oracle():
    """Four appending frames on identical inputs, on a model with 5% of its
    surfels cut away, under growing warps.  Worked out on the oracle's model:
    frame 1 appends 892 surfels, most in known node sets, 4 new sets whose
    node pairs are all blocks of the pattern already (fast update: new sets
    added, pattern kept); frame 2 forms 2 new sets with a pair the pattern
    lacks (pattern rebuilt from the set table, no re-sort; a solve follows on
    this model); frame 3's 365 surfels would bring the surfels placed after
    the sorted ones past 1/16 of the model (re-sort); frame 4 again needs a
    new block (pattern rebuilt).  The model, its skinning and the solves
    agree with the oracle."""
    scene = _cut(synth.plain_tiny(seed=0), frac=0.05, unstable=0)
    c = scene.cam
    b = Both(scene, len(scene.surfel_v) + c.width * c.height)
    try:
        d = scene.frame(1)
        resorted = []
        for t, (seed, amp, tr) in enumerate([(5, 0.5, 0.002), (6, 0.6, 0.003), (7, 0.7, 0.004), (8, 0.8, 0.005)], 1):
            sw.sw_upload_depth(b.h, d, t)
            b.o.upload_depth(d, t)
            b.set_maps()
            dq8 = _warp(scene, seed, amp, tr, alpha=0.0)
            sw.sw_set_node_dq(b.h, dq8)
            b.o.node_dq = dq8.astype(np.float64)
            _, vl, nl = OS.warp_surfels(b.o.v_ref, b.o.n_ref, b.o.knn, b.o.w, b.o.node_dq)
            vl32, nl32 = vl.astype(F32), nl.astype(F32)
            sw.sw_debug_set_live(b.h, vl32, nl32)
            sw.sw_debug_fusion_targets(b.h, c.height, c.width)
            st = sw.sw_append_frame(b.h)
            b.o.last_index_map = OFU.index_map(vl32, b.o.p.cam)
            _, n_app, _ = b.o.append_frame(b.max_surfels, EPS, DNN, FDH)
            assert st["appended"] == n_app and st["n_surfels"] == len(b.o.v_ref), (t, st, n_app)
            resorted.append(st["resorted"])
            if t == 2:   # a solve on the model with appended surfels after the sorted ones
                st3 = sw.sw_solve_frame(b.h, 2, 8)
                ost3 = b.o.solve_frame(2, 8)
                assert abs(st3["n_corr"][0] - ost3[0].n_corr) <= 3
                _, dq3 = sw.sw_read_nodes(b.h)
                dq3 = dq3.astype(np.float64)
                assert rotation_angle_between(dq3, b.o.node_dq).max() < 1e-4
                assert np.linalg.norm(OS.node_transform(dq3, b.o.node_p) - b.o.warped_nodes(), axis=1).max() < 2e-5
        assert resorted == [0, 2, 1, 2]
        v, n, t2 = sw.sw_read_surfels(b.h)
        np.testing.assert_allclose(v[:, :3], b.o.v_ref, atol=2e-6)
        np.testing.assert_allclose(n[:, :3], b.o.n_ref, atol=2e-6)
        np.testing.assert_array_equal(t2[:, 0], b.o.t_init)
        knn, w = sw.sw_read_skinning(b.h)
        np.testing.assert_array_equal(knn, b.o.knn)
        np.testing.assert_allclose(w, b.o.w, rtol=2e-6, atol=1e-30)
        # and a solve on the model with the rebuilt pattern
        sw.sw_upload_depth(b.h, d, 4)
        b.o.upload_depth(d, 4)
        b.set_maps()
        st4 = sw.sw_solve_frame(b.h, 2, 8)
        ost4 = b.o.solve_frame(2, 8)
        assert abs(st4["n_corr"][0] - ost4[0].n_corr) <= 3
        _, dq = sw.sw_read_nodes(b.h)
        dq = dq.astype(np.float64)
        assert rotation_angle_between(dq, b.o.node_dq).max() < 1e-4
        assert np.linalg.norm(OS.node_transform(dq, b.o.node_p) - b.o.warped_nodes(), axis=1).max() < 2e-5
    finally:
        b.close()
