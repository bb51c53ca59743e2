"""Edge cases of appending and visibility on the GPU: an empty model grown
from its first depth frame, a stream already at capacity, and visibility on
an image whose size is not a multiple of the kernels' tiles."""
import dataclasses

import numpy as np
import pytest

import synth
import oracle
import paper_1904_13073_gb300 as sw
from oracle import solver as OS
from oracle import visibility as OV

from gpu_helpers import Pair, ensure_built, rigid_dq8_from
from test_gpu_append import Both, _cut, EPS, DNN, FDH
from test_gpu_visibility import _depth_radii

pytestmark = pytest.mark.gpu
F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def test_empty_model_grows_from_its_first_frame():
    """No surfels, identity warp: fusion finds every usable pixel's window
    empty, so every usable depth surfel is a candidate and (identity warp:
    strain 1, weights of the nodes around it) is appended in pixel order."""
    sc = synth.plain_tiny(seed=0)
    c = sc.cam
    empty = dataclasses.replace(sc, surfel_v=np.zeros((0, 3), F32), surfel_n=np.zeros((0, 3), F32),
                                surfel_r=np.zeros(0, F32), surfel_c=np.zeros(0, F32),
                                surfel_t=np.zeros((0, 2), np.int32))
    b = Both(empty, c.width * c.height)
    try:
        d = sc.frame(0)
        sw.sw_upload_depth(b.h, d, 0)
        b.o.upload_depth(d, 0)
        b.set_maps()
        sw.sw_fuse_frame(b.h)
        b.o.fuse_frame()
        st = sw.sw_append_frame(b.h)
        n_cand, n_app, n_rem = b.o.append_frame(b.max_surfels, EPS, DNN, FDH)
        usable = int(b.o.maps["valid"].sum())
        assert st["candidates"] == n_cand == usable
        assert st["appended"] == n_app and st["removed"] == n_rem == 0 and n_app > 0.99 * usable
        v, n, t2 = sw.sw_read_surfels(b.h)
        np.testing.assert_allclose(v[:, :3], b.o.v_ref, atol=2e-6)
        np.testing.assert_allclose(n[:, :3], b.o.n_ref, atol=2e-6)
        assert np.all(t2 == 0)
        knn, w = sw.sw_read_skinning(b.h)
        np.testing.assert_array_equal(knn, b.o.knn)
        np.testing.assert_allclose(w, b.o.w, rtol=2e-6, atol=1e-30)
        # the grown model solves the next frame
        sw.sw_upload_depth(b.h, sc.frame(1), 1)
        st2 = sw.sw_solve_frame(b.h, 2, 8)
        assert st2["n_corr"][0] > 0.5 * n_app
    finally:
        b.close()


def test_stream_at_capacity_appends_nothing():
    sc = _cut(synth.plain_tiny(seed=0), unstable=0)
    c = sc.cam
    b = Both(sc, len(sc.surfel_v))
    try:
        sw.sw_upload_depth(b.h, sc.frame(1), 1)
        sw.sw_solve_frame(b.h, 2, 8)
        sw.sw_fuse_frame(b.h)
        before = sw.sw_read_surfels(b.h)[0]
        st = sw.sw_append_frame(b.h)
        assert st["candidates"] > 1000 and st["appended"] == 0 and st["removed"] == 0
        assert st["n_surfels"] == len(sc.surfel_v) and st["rebuild_ms"] == 0.0
        np.testing.assert_array_equal(sw.sw_read_surfels(b.h)[0], before)
    finally:
        b.close()


def test_visibility_on_a_ragged_image():
    """97 x 71 pixels: neither a multiple of the 32 x 8 pixel tiles nor of 4."""
    scene = _depth_radii(synth.random_scene(seed=8, n_surfels=20000, n_nodes=40, width=97, height=71))
    c = scene.cam
    p = Pair(scene)
    try:
        p.upload(1)
        axis, ang, tr = synth.random_rigid_dq_inputs(9, len(scene.node_p), 2.0, 0.01)
        dq8 = rigid_dq8_from(axis, ang, tr)
        _, vl, nl = OS.warp_surfels(p.o.v_ref, p.o.n_ref, p.o.knn, p.o.w, dq8.astype(np.float64))
        vl32, nl32 = vl.astype(F32), nl.astype(F32)
        sw.sw_debug_set_live(p.h, vl32, nl32)
        vm, vis = sw.sw_debug_visibility(p.h, c.height, c.width)
        sel = OS.select_surfels(p.o.conf, p.o.t_obs, 1, p.o.p.stable_conf, p.o.p.recent_frames)
        ovm = OV.visibility_map(vl32, nl32, scene.surfel_r, sel, p.o.p.cam)
        np.testing.assert_array_equal(vm, ovm)
        np.testing.assert_array_equal(vis, OV.visible_mask(ovm, len(vl32)))
        assert (vm[:, -1] >= 0).any() or (vm[-1, :] >= 0).any() or vis.sum() > 100
    finally:
        p.close()
