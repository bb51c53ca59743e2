"""Failure detection of the product's own bounded device waits.

The persistent PCG (Sec. 7) waits in two places: for the other CTAs' shares
of each reduction, and for the neighbours' vector words its SpMV reads.  The
depth stage (Sec. 5) waits on an mbarrier for each tile's TMA copy.  Each
test makes one of those waits run out without any fault on the GPU: a
debug hook has a kernel withhold what the wait expects (a CTA does not
publish its partial or its rows' vector; the TMA copies are not issued),
with a small poll limit.  The host must then see SW_ERR_TIMEOUT, the node
transforms must be left as they were, and the context must stay usable:
with the hook off, the same stream solves again and matches the FP64
oracle."""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import solver as OS

from gpu_helpers import Pair, ensure_built, rotation_angle_between

pytestmark = pytest.mark.gpu
SW_ERR_TIMEOUT = 5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    # the waits live in the cooperative PCG; the cluster PCG (which streams
    # that fit it take by default) synchronises with hardware barriers only
    sw.sw_debug_set_pcg_mode(2)
    yield
    sw.sw_debug_inject_wait_fault(sw.SW_FAULT_NONE)
    sw.sw_debug_set_pcg_mode(3)


def _matches_oracle(p, gn, pcg):
    st = sw.sw_solve_frame(p.h, gn, pcg)
    p.o.solve_frame(gn, pcg)
    _, dq = sw.sw_read_nodes(p.h)
    dq = dq.astype(np.float64)
    rot = rotation_angle_between(dq, p.o.node_dq).max()
    trans = np.linalg.norm(OS.node_transform(dq, p.o.node_p) - p.o.warped_nodes(), axis=1).max()
    assert rot <= 1e-4 and trans <= 1e-5, (rot, trans)
    return st


@pytest.mark.parametrize("kind", [sw.SW_FAULT_PCG_PARTIAL, sw.SW_FAULT_PCG_VECTOR])
@pytest.mark.parametrize("precision", [sw.SW_PRECISION_MIXED, sw.SW_PRECISION_FP64])
def test_pcg_wait_runs_out_reports_timeout_and_leaves_nodes(kind, precision):
    if precision == sw.SW_PRECISION_FP64 and kind == sw.SW_FAULT_PCG_VECTOR:
        pytest.skip("the FP64 solver reads its neighbours' vectors after a fenced reduction, with no wait of its own")
    scene = synth.plain_tiny(seed=0)       # 64 nodes: two PCG CTAs at 32 rows each
    p = Pair(scene, precision=precision)
    try:
        p.upload(1)
        _, before = sw.sw_read_nodes(p.h)
        sw.sw_debug_inject_wait_fault(kind, 2000)
        try:
            with pytest.raises(sw.SwError) as e:
                sw.sw_solve_frame(p.h, 2, 6)
        finally:
            sw.sw_debug_inject_wait_fault(sw.SW_FAULT_NONE)
        assert e.value.status == SW_ERR_TIMEOUT, e.value
        assert "PCG" in str(e.value)
        _, after = sw.sw_read_nodes(p.h)
        np.testing.assert_array_equal(after, before)
        # the context is usable and the stream solves as before
        _matches_oracle(p, scene.gn_iters, scene.pcg_iters)
    finally:
        p.close()


def test_pcg_wait_runs_out_in_a_batch_for_its_stream_only():
    """In a batch the hook hits the first member's CTA 1; that member reports
    the timeout and keeps its transforms, and the other member, whose CTAs
    never wait on the first member's, solves as it does alone."""
    a = synth.plain_tiny(seed=0)
    b_scene = synth.random_scene(seed=21, n_surfels=5000, n_nodes=60)
    hs = []
    for s in (a, b_scene):
        v4, n4, t2, node4 = sw.model_arrays(s)
        h = sw.sw_create_stream(sw.params_for(s.cam, len(v4), len(node4)))
        sw.sw_set_model(h, v4, n4, t2, node4)
        hs.append(h)
    v4, n4, t2, node4 = sw.model_arrays(b_scene)
    alone = sw.sw_create_stream(sw.params_for(b_scene.cam, len(v4), len(node4)))
    sw.sw_set_model(alone, v4, n4, t2, node4)
    bt = sw.sw_batch_create(hs)
    try:
        sw.sw_batch_upload_depth(bt, [a.frame(1), b_scene.frame(1)], [1, 1])
        _, before = sw.sw_read_nodes(hs[0])
        sw.sw_debug_inject_wait_fault(sw.SW_FAULT_PCG_PARTIAL, 2000)
        try:
            with pytest.raises(sw.SwError) as e:
                sw.sw_batch_solve(bt, 2, 6)
        finally:
            sw.sw_debug_inject_wait_fault(sw.SW_FAULT_NONE)
        assert e.value.status == SW_ERR_TIMEOUT
        np.testing.assert_array_equal(sw.sw_read_nodes(hs[0])[1], before)
        sw.sw_upload_depth(alone, b_scene.frame(1), 1)
        sw.sw_solve_frame(alone, 2, 6)
        qa = sw.sw_read_nodes(alone)[1].astype(np.float64)
        qm = sw.sw_read_nodes(hs[1])[1].astype(np.float64)
        assert np.max(rotation_angle_between(qa, qm)) < 1e-5
        # and the batch runs normally afterwards
        st = sw.sw_batch_solve(bt, 2, 6)
        assert st[0]["n_corr"][0] > 0 and st[1]["n_corr"][0] > 0
    finally:
        sw.sw_batch_destroy(bt)
        for h in hs + [alone]:
            sw.sw_destroy_stream(h)


def test_depth_tma_wait_runs_out_falls_back_and_reports():
    """The depth tiles' TMA copies are withheld: every CTA's bounded mbarrier
    wait runs out, the tile is read with plain loads (the maps are exactly
    those of the normal path), and the solve that follows reports the wait."""
    scene = synth.plain_tiny(seed=0)       # width 160: rows 16-byte aligned, so the TMA path is taken
    p = Pair(scene)
    try:
        c = scene.cam
        p.upload(1)
        V0, N0 = sw.sw_read_maps(p.h, c.height, c.width)
        sw.sw_debug_inject_wait_fault(sw.SW_FAULT_DEPTH_TMA)
        try:
            sw.sw_upload_depth(p.h, scene.frame(1), 1)
            V1, N1 = sw.sw_read_maps(p.h, c.height, c.width)
        finally:
            sw.sw_debug_inject_wait_fault(sw.SW_FAULT_NONE)
        np.testing.assert_array_equal(V1, V0)
        np.testing.assert_array_equal(N1, N0)
        with pytest.raises(sw.SwError) as e:
            sw.sw_solve_frame(p.h, 1, 4)
        assert e.value.status == SW_ERR_TIMEOUT and "depth" in str(e.value)
        # the next upload clears the report; the stream matches the oracle
        # from its first frame again
        sw.sw_set_model(p.h, *sw.model_arrays(scene))
        p.upload(1)
        _matches_oracle(p, scene.gn_iters, scene.pcg_iters)
    finally:
        p.close()
