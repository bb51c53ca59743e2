"""The checked build (-DSW_BOUNDS_CHECK, loaded with SW_BOUNDS_CHECK=1):
kernels range-check the indices they read or derive on the device and
report a bad one as SW_ERR_BOUNDS instead of accessing out of range.

The planted index (a skinning node id in [n_nodes, max_nodes)) lies inside
the node arrays' allocation, so the access it leads to stays in bounds in
either build; only the checked build notices it.  The test runs in the
checked build only."""
import numpy as np
import pytest
import torch

import synth
import paper_1904_13073_gb300 as sw

from gpu_helpers import ensure_built

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not sw.CHECKED_BUILD, reason="needs the checked build (SW_BOUNDS_CHECK=1)")]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def test_planted_node_id_is_reported_and_cleared_by_set_model():
    scene = synth.random_scene(seed=2, n_surfels=3000, n_nodes=40)
    v4, n4, t2, node4 = sw.model_arrays(scene)
    n_n = len(node4)
    h = sw.sw_create_stream(sw.params_for(scene.cam, len(v4), n_n + 16))
    try:
        sw.sw_set_model(h, v4, n4, t2, node4)
        depth = torch.from_numpy(scene.frame(1)).cuda()
        sw.sw_upload_depth(h, depth, 1)
        sw.sw_solve_frame(h, 2, 8)        # valid indices: no report
        sw.sw_fuse_frame(h)
        sw.sw_upload_depth(h, depth, 2)
        sw.sw_debug_set_skin_node(h, 5, 2, n_n + 3)
        with pytest.raises(sw.SwError) as e:
            sw.sw_solve_frame(h, 2, 8)
        assert e.value.status == 7, e.value    # SW_ERR_BOUNDS
        with pytest.raises(sw.SwError) as e:     # sticky until the model is set again
            sw.sw_read_nodes(h)
        assert e.value.status == 7
        sw.sw_set_model(h, v4, n4, t2, node4)
        sw.sw_upload_depth(h, depth, 3)
        sw.sw_solve_frame(h, 2, 8)
        pos, dq = sw.sw_read_nodes(h)
        assert np.all(np.isfinite(dq))
    finally:
        sw.sw_destroy_stream(h)


def test_hook_rejects_ids_outside_the_allocation():
    scene = synth.random_scene(seed=2, n_surfels=500, n_nodes=20)
    v4, n4, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(scene.cam, len(v4), len(node4) + 4))
    try:
        sw.sw_set_model(h, v4, n4, t2, node4)
        for args in [(0, 0, len(node4) + 4), (0, 4, 0), (len(v4), 0, 0), (0, 0, -1)]:
            with pytest.raises(sw.SwError):
                sw.sw_debug_set_skin_node(h, *args)
    finally:
        sw.sw_destroy_stream(h)
