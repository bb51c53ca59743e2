"""Serving: streams that arrive and leave while others are on the GPU,
continuous batching over whatever frames are queued, admission against a
memory budget.  Each stream's result must be the one it gets alone (up to
floating-point summation order, the tolerance of the batched tests)."""
import threading
import time

import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import solver as OS

from gpu_helpers import ensure_built, rotation_angle_between

pytestmark = pytest.mark.gpu
GN, PCG = 3, 8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    yield
    sw.sw_set_memory_budget(0)


def _scenes():
    return [synth.random_scene(seed=30, n_surfels=3000, n_nodes=30),
            synth.random_scene(seed=31, n_surfels=9000, n_nodes=90, width=128, height=96, f=120.0),
            synth.random_scene(seed=32, n_surfels=5000, n_nodes=55, outliers=0.01),
            synth.random_scene(seed=33, n_surfels=4000, n_nodes=40)]


def _alone(scene, frames):
    """The stream by itself, outside any server: solve + fuse per frame."""
    v4, n4, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(scene.cam, len(v4), len(node4)))
    try:
        sw.sw_set_model(h, v4, n4, t2, node4)
        for t in frames:
            sw.sw_upload_depth(h, scene.frame(t), t)
            sw.sw_solve_frame(h, GN, PCG)
            sw.sw_fuse_frame(h)
        _, dq = sw.sw_read_nodes(h)
    finally:
        sw.sw_destroy_stream(h)
    return dq.astype(np.float64)


def _open(srv, scene):
    v4, n4, t2, node4 = sw.model_arrays(scene)
    return sw.sw_server_open(srv, sw.params_for(scene.cam, len(v4), len(node4)), v4, n4, t2, node4)


def _wait_admitted(srv, sid, timeout=30.0):
    t0 = time.time()
    while not sw.sw_server_is_admitted(srv, sid):
        assert time.time() - t0 < timeout, "stream was not admitted"
        time.sleep(0.002)


def _submit(srv, sid, depth, t):
    while True:
        st = sw.sw_server_submit(srv, sid, depth, t)
        if st == 0:
            return
        assert st in (2, 3), st   # queue full or not admitted yet: try again
        time.sleep(0.001)


def _compare(scene, dq_got, dq_ref):
    p = scene.node_p.astype(np.float64)
    assert np.max(rotation_angle_between(dq_got, dq_ref)) < 1e-5
    assert np.max(np.abs(OS.node_transform(dq_got, p) - OS.node_transform(dq_ref, p))) < 2e-6


@pytest.mark.parametrize("adaptive", [False, True])
def test_served_streams_match_their_results_alone(adaptive):
    """Four streams of different sizes submit frames from their own threads
    with random gaps; one joins late and one leaves early.  Each stream's
    warp field equals the one it gets alone, whether every step is one batch
    or the adaptive policy runs some steps stream by stream."""
    scenes = _scenes()
    frames = {0: [1, 2, 3], 1: [1, 2, 3], 2: [1, 2], 3: [1, 2, 3]}
    refs = {k: _alone(s, frames[k]) for k, s in enumerate(scenes)}
    srv = sw.sw_server_create(0, GN, PCG, queue_depth=2)
    try:
        sw.sw_server_set_batch_window(srv, 20.0)
        sw.sw_server_set_adaptive(srv, adaptive)
        ids = {}
        for k in (0, 1, 2):
            ids[k] = _open(srv, scenes[k])
        for k in (0, 1, 2):
            _wait_admitted(srv, ids[k])
        got = {}
        depth = {k: [scenes[k].frame(t) for t in frames[k]] for k in range(4)}
        start = threading.Barrier(3)

        def client(k):
            if k == 3:   # joins while the others are being served
                time.sleep(0.03)
                ids[k] = _open(srv, scenes[k])
                _wait_admitted(srv, ids[k])
            else:
                start.wait()
            rng = np.random.default_rng(k)
            for t, d in zip(frames[k], depth[k]):
                _submit(srv, ids[k], d, t)
                time.sleep(float(rng.uniform(0.0, 0.01)))
        threads = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert sw.sw_server_wait(srv, 60000)
        results = sw.sw_server_poll(srv)
        for k, sid in ids.items():
            got[k] = sw.sw_server_read_nodes(srv, sid, len(scenes[k].node_p))[1].astype(np.float64)
        sw.sw_server_close(srv, ids[2])
        assert len(results) == sum(len(v) for v in frames.values())
        for r in results:
            assert r["status"] == 0
            assert r["submit_ms"] <= r["start_ms"] <= r["done_ms"]
            assert 1 <= r["batch_size"] <= 4
        # frames of one stream complete in order
        for k, sid in ids.items():
            seq = [r["frame_id"] for r in results if r["stream"] == sid]
            assert seq == frames[k]
        if not adaptive:
            assert max(r["batch_size"] for r in results) >= 2   # batches formed while frames overlapped
        for k in range(4):
            _compare(scenes[k], got[k], refs[k])
        st = sw.sw_server_read_stats(srv)
        assert st["frames"] == len(results) and st["steps"] >= 1
        assert adaptive or st["steps_alone"] == 0
    finally:
        sw.sw_server_destroy(srv)


def test_admission_waits_for_memory():
    """With a budget that holds one stream, a second one waits until the
    first leaves, then is admitted and served."""
    scene = synth.random_scene(seed=34, n_surfels=6000, n_nodes=50)
    srv = sw.sw_server_create(0, GN, PCG)
    try:
        a = _open(srv, scene)
        _wait_admitted(srv, a)
        one = sw.sw_server_read_stats(srv)["memory_in_use"]
    finally:
        sw.sw_server_destroy(srv)
    assert one > 0
    srv = sw.sw_server_create(int(one * 1.5), GN, PCG)
    try:
        a = _open(srv, scene)
        _wait_admitted(srv, a)
        b = _open(srv, scene)
        time.sleep(0.2)
        assert not sw.sw_server_is_admitted(srv, b)
        assert sw.sw_server_submit(srv, b, scene.frame(1), 1) == 3   # waits for admission
        st = sw.sw_server_read_stats(srv)
        assert st["admitted"] == 1 and st["waiting"] == 1
        _submit(srv, a, scene.frame(1), 1)
        assert sw.sw_server_wait(srv, 30000)
        sw.sw_server_close(srv, a)
        _wait_admitted(srv, b)
        _submit(srv, b, scene.frame(1), 1)
        assert sw.sw_server_wait(srv, 30000)
        res = sw.sw_server_poll(srv)
        assert [r["stream"] for r in res] == [a, b] and all(r["status"] == 0 for r in res)
        assert sw.sw_server_read_stats(srv)["memory_in_use"] <= int(one * 1.5)
    finally:
        sw.sw_server_destroy(srv)
        sw.sw_set_memory_budget(0)


def test_served_streams_append():
    """Appending on: every served frame is followed by sw_append_frame on its
    stream.  Two streams with a hole cut in their models grow at frame 1, the
    results report it, and each stream's warp field after frame 2 is the one
    it gets alone through solve + fusion + appending (within the appending
    tests' end-to-end tolerance: fusion and appending decisions may flip on
    the batch's summation order)."""
    from test_gpu_append import _cut
    scenes = [_cut(synth.plain_tiny(seed=4)), _cut(synth.random_scene(seed=35, n_surfels=6000, n_nodes=50))]

    def params(sc):
        v4, n4, t2, node4 = sw.model_arrays(sc)
        return (sw.params_for(sc.cam, len(v4) + sc.cam.width * sc.cam.height, len(node4)), v4, n4, t2, node4)
    refs = []
    for sc in scenes:
        p, v4, n4, t2, node4 = params(sc)
        h = sw.sw_create_stream(p)
        try:
            sw.sw_set_model(h, v4, n4, t2, node4)
            grown = []
            for t in (1, 2):
                sw.sw_upload_depth(h, sc.frame(1), t)
                sw.sw_solve_frame(h, GN, PCG)
                sw.sw_fuse_frame(h)
                grown.append(sw.sw_append_frame(h)["n_surfels"])
            refs.append((sw.sw_read_nodes(h)[1].astype(np.float64), grown))
        finally:
            sw.sw_destroy_stream(h)
    srv = sw.sw_server_create(0, GN, PCG, queue_depth=2)
    try:
        sw.sw_server_set_appending(srv, True)
        ids = []
        for sc in scenes:
            p, v4, n4, t2, node4 = params(sc)
            ids.append(sw.sw_server_open(srv, p, v4, n4, t2, node4))
        for sid in ids:
            _wait_admitted(srv, sid)
        for t in (1, 2):
            for sid, sc in zip(ids, scenes):
                _submit(srv, sid, sc.frame(1), t)
            assert sw.sw_server_wait(srv, 60000)
        res = sw.sw_server_poll(srv)
        assert len(res) == 4 and all(r["status"] == 0 for r in res)
        for k, (sid, sc) in enumerate(zip(ids, scenes)):
            mine = [r for r in res if r["stream"] == sid]
            assert mine[0]["appended"] > 100 and mine[0]["n_surfels"] > len(sc.surfel_v)
            for r, want in zip(mine, refs[k][1]):
                assert abs(r["n_surfels"] - want) <= max(3, want // 200)
            got = sw.sw_server_read_nodes(srv, sid, len(sc.node_p))[1].astype(np.float64)
            assert np.max(rotation_angle_between(got, refs[k][0])) < 1e-4
            p_ = sc.node_p.astype(np.float64)
            assert np.max(np.abs(OS.node_transform(got, p_) - OS.node_transform(refs[k][0], p_))) < 2e-5
    finally:
        sw.sw_server_destroy(srv)
