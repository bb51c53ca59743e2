"""Batched execution: several streams of uneven size advanced by one launch per
stage must give each stream the result it gets alone (up to floating-point
summation order), leave inactive members untouched, and report stage timing."""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import solver as OS

from gpu_helpers import ensure_built, rotation_angle_between

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _scenes():
    return [synth.random_scene(seed=20, n_surfels=3000, n_nodes=30),
            synth.random_scene(seed=21, n_surfels=9000, n_nodes=90, width=128, height=96, f=120.0),
            synth.random_scene(seed=22, n_surfels=5000, n_nodes=55, outliers=0.01)]


def _make(scene):
    v4, n4, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(scene.cam, len(v4), len(node4)))
    sw.sw_set_model(h, v4, n4, t2, node4)
    return h


def _warped(h, node_p):
    _, dq = sw.sw_read_nodes(h)
    dq = dq.astype(np.float64)
    return dq, OS.node_transform(dq, node_p.astype(np.float64))


def test_batch_matches_streams_alone():
    scenes = _scenes()
    alone = [_make(s) for s in scenes]
    mixed = [_make(s) for s in scenes]
    b = sw.sw_batch_create(mixed)
    try:
        for t in (1, 2):
            for h, s in zip(alone, scenes):
                sw.sw_upload_depth(h, s.frame(t), t)
                sw.sw_solve_frame(h, 3, 8)
                sw.sw_fuse_frame(h)
            sw.sw_batch_upload_depth(b, [s.frame(t) for s in scenes], [t] * 3)
            stats = sw.sw_batch_solve(b, 3, 8)
            sw.sw_batch_fuse(b)
            for k, (ha, hm, s) in enumerate(zip(alone, mixed, scenes)):
                qa, pa = _warped(ha, s.node_p)
                qm, pm = _warped(hm, s.node_p)
                assert np.max(rotation_angle_between(qa, qm)) < 1e-5, (t, k)
                assert np.max(np.abs(pa - pm)) < 2e-6, (t, k)
                assert stats[k]["n_corr"][0] > 0
                va, _, ta = sw.sw_read_surfels(ha)
                vm, _, tm = sw.sw_read_surfels(hm)
                assert np.sum(ta[:, 1] != tm[:, 1]) <= 3
                same = ta[:, 1] == tm[:, 1]
                assert np.max(np.abs(va[same, :3] - vm[same, :3])) < 1e-5
    finally:
        sw.sw_batch_destroy(b)
        for h in alone + mixed:
            sw.sw_destroy_stream(h)


def test_inactive_members_are_untouched_and_profile_counts_stages():
    scenes = _scenes()
    hs = [_make(s) for s in scenes]
    b = sw.sw_batch_create(hs)
    try:
        sw.sw_batch_upload_depth(b, [s.frame(1) for s in scenes], [1] * 3)
        sw.sw_batch_set_active(b, [1, 0, 1])
        before_q = sw.sw_read_nodes(hs[1])[1].copy()
        before_v = sw.sw_read_surfels(hs[1])[0].copy()
        sw.sw_batch_set_profiling(b, True)
        stats = sw.sw_batch_solve(b, 2, 5)
        sw.sw_batch_fuse(b)
        prof = sw.sw_batch_read_profile(b)
        assert stats[1]["gn_iters"] == 0
        np.testing.assert_array_equal(sw.sw_read_nodes(hs[1])[1], before_q)
        np.testing.assert_array_equal(sw.sw_read_surfels(hs[1])[0], before_v)
        assert stats[0]["n_corr"][0] > 0 and stats[2]["n_corr"][0] > 0
        # FP32 modes: one assembly launch of both terms, timed as the data stage
        assert prof["reg_assembly"] == (0.0, 0)
        assert prof["data_assembly"][1] == 2 and prof["pcg"][1] == 2
        assert prof["fusion"][1] == 1
        assert all(prof[k][0] > 0 for k in ("data_assembly", "pcg", "fusion"))
        # a member's model is replaced: the batch rebuilds its tables at its
        # next call and keeps the active flags
        v4, n4, t2, node4 = sw.model_arrays(scenes[0])
        sw.sw_set_model(hs[0], v4, n4, t2, node4)
        stats = sw.sw_batch_solve(b, 1, 1)
        assert stats[0]["gn_iters"] == 1 and stats[1]["gn_iters"] == 0 and stats[0]["n_corr"][0] > 0
        np.testing.assert_array_equal(sw.sw_read_nodes(hs[1])[1], before_q)
    finally:
        sw.sw_batch_destroy(b)
        for h in hs:
            sw.sw_destroy_stream(h)


def test_stream_profile_reports_each_stage():
    s = synth.random_scene(seed=23, n_surfels=3000, n_nodes=30)
    h = _make(s)
    try:
        sw.sw_set_profiling(h, True)
        sw.sw_upload_depth(h, s.frame(1), 1)
        sw.sw_solve_frame(h, 3, 6)
        sw.sw_fuse_frame(h)
        prof = sw.sw_read_profile(h)
        assert prof["depth"][1] == 1 and prof["fusion"][1] == 1
        assert prof["reg_assembly"] == (0.0, 0)   # with the data term in one launch
        assert prof["data_assembly"][1] == 3 and prof["pcg"][1] == 3
        assert prof["visibility"] == (0.0, 0)   # visibility prediction is off by default
        assert all(v[0] > 0 for k, v in prof.items() if k not in ("visibility", "reg_assembly"))
    finally:
        sw.sw_destroy_stream(h)


def test_batch_autotune_then_matches_alone():
    scenes = _scenes()
    alone = [_make(s) for s in scenes]
    mixed = [_make(s) for s in scenes]
    b = sw.sw_batch_create(mixed)
    try:
        sw.sw_batch_upload_depth(b, [s.frame(1) for s in scenes], [1] * 3)
        rows, us = sw.sw_batch_autotune(b, 8)
        assert rows in (16, 24, 32, 48, 64, 96) and us > 0
        sw.sw_batch_solve(b, 3, 8)
        sw.sw_batch_fuse(b)
        for h, s in zip(alone, scenes):
            sw.sw_upload_depth(h, s.frame(1), 1)
            sw.sw_solve_frame(h, 3, 8)
            sw.sw_fuse_frame(h)
        for ha, hm, s in zip(alone, mixed, scenes):
            qa, pa = _warped(ha, s.node_p)
            qm, pm = _warped(hm, s.node_p)
            assert np.max(rotation_angle_between(qa, qm)) < 1e-5
            assert np.max(np.abs(pa - pm)) < 2e-6
    finally:
        sw.sw_batch_destroy(b)
        for h in alone + mixed:
            sw.sw_destroy_stream(h)


def test_batch_refreshes_after_a_member_appends():
    """A member's model grows by appending between batch calls: the batch
    rebuilds its tables at its next call, keeps the active flags (an inactive
    member stays untouched) and gives the grown member the result it gets
    alone through the same calls."""
    from test_gpu_append import _cut
    scenes = [_cut(synth.plain_tiny(seed=3)), synth.random_scene(seed=24, n_surfels=4000, n_nodes=40)]

    def make(scene):
        v4, n4, t2, node4 = sw.model_arrays(scene)
        c = scene.cam
        h = sw.sw_create_stream(sw.params_for(c, len(v4) + c.width * c.height, len(node4)))
        sw.sw_set_model(h, v4, n4, t2, node4)
        return h
    alone = make(scenes[0])
    mixed = [make(s) for s in scenes]
    b = sw.sw_batch_create(mixed)
    try:
        sw.sw_upload_depth(alone, scenes[0].frame(1), 1)
        sw.sw_solve_frame(alone, 3, 8)
        sw.sw_fuse_frame(alone)
        st_alone = sw.sw_append_frame(alone)
        sw.sw_batch_upload_depth(b, [s.frame(1) for s in scenes], [1, 1])
        sw.sw_batch_solve(b, 3, 8)
        sw.sw_batch_fuse(b)
        sw.sw_batch_set_active(b, [1, 0])
        st = sw.sw_append_frame(mixed[0])
        assert st["appended"] > 500 and abs(st["appended"] - st_alone["appended"]) <= max(3, st["appended"] // 200)
        _, dq1_before = sw.sw_read_nodes(mixed[1])
        # frame 2 through the batch (member 1 inactive) and alone
        sw.sw_batch_upload_depth(b, [scenes[0].frame(1), None], [2, 0])
        sw.sw_batch_solve(b, 3, 8)
        sw.sw_upload_depth(alone, scenes[0].frame(1), 2)
        sw.sw_solve_frame(alone, 3, 8)
        np.testing.assert_array_equal(sw.sw_read_nodes(mixed[1])[1], dq1_before)
        qa, pa = _warped(alone, scenes[0].node_p)
        qm, pm = _warped(mixed[0], scenes[0].node_p)
        assert np.max(rotation_angle_between(qa, qm)) < 1e-4
        assert np.max(np.abs(pa - pm)) < 2e-5
    finally:
        sw.sw_batch_destroy(b)
        for h in mixed + [alone]:
            sw.sw_destroy_stream(h)
