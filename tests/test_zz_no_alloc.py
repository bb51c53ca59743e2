"""sw_fusion_targets_static: fusion targets for callers that may not allocate.

Some callers cannot call cudaMalloc -- code running while another component
captures its stream into a CUDA graph, real-time loops where an allocation
would stall the whole device, frameworks that own all device memory through
their own pool.  This entry point serves them: the caller passes device
inputs and the output buffer, and the only scratch (the index map) is an array
compiled into the library.  This test calls it twice in a row, on different
inputs, through the C ABI and checks each result against the allocating
stream path (sw_debug_fusion_targets) on the same inputs, bit for bit, which
also shows that the second call does not see the first call's index map.
Then it captures a call into a CUDA graph in PyTorch's global capture mode,
where any device allocation (or other unsafe call) in the capturing thread
fails the capture, replays the graph and compares again; and a call with no
surfels must leave every pixel without a target.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw

pytestmark = pytest.mark.gpu


def _live_inputs(scene, V, seed):
    """Live surfels near the depth vertices, some exactly on them (so that
    fusion finds targets), with exact duplicates (id ties)."""
    rng = np.random.default_rng(seed)
    n = len(scene.surfel_v)
    v = scene.surfel_v.astype(np.float32) + rng.normal(0, 4e-4, (n, 3)).astype(np.float32)
    usable = np.nonzero(V[..., 3].reshape(-1) > 0)[0]
    pick = rng.choice(usable, min(len(usable), n // 3), replace=False)
    k = len(pick)
    v[:k] = V.reshape(-1, 4)[pick, :3]
    v[k:k + k // 4] = v[:k // 4]
    nrm = scene.surfel_n.astype(np.float32)
    conf = rng.choice(np.array([1.0, 2.0, 12.0], np.float32), n)
    v4 = np.concatenate([v, scene.surfel_r[:, None]], axis=1).astype(np.float32)
    n4 = np.concatenate([nrm, conf[:, None]], axis=1).astype(np.float32)
    return v4, n4


def test_static_fusion_targets_match_stream_path_twice():
    import torch
    from paper_1904_13073_gb300 import build as B
    B.build()
    scene = synth.plain_tiny(seed=2)
    c = scene.cam
    assert c.width * c.height <= 76800
    v4m, n4m, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(c, len(v4m), len(node4)))
    try:
        sw.sw_set_model(h, v4m, n4m, t2, node4)
        results = []
        for call, (frame, seed) in enumerate([(0, 10), (1, 11)]):
            sw.sw_upload_depth(h, scene.frame(frame), frame)
            V, N = sw.sw_read_maps(h, c.height, c.width)
            v4, n4 = _live_inputs(scene, V, seed)
            # the allocating path: the stream's own index map
            sw.sw_set_model(h, v4m, np.concatenate([n4m[:, :3], n4[:, 3:]], axis=1), t2, node4)
            sw.sw_debug_set_maps(h, V, N)
            sw.sw_debug_set_live(h, v4[:, :3], n4[:, :3])
            want, _ = sw.sw_debug_fusion_targets(h, c.height, c.width)
            # the no-allocation path on the same inputs, caller-owned device memory
            dv, dn = torch.from_numpy(v4).cuda(), torch.from_numpy(n4).cuda()
            dV, dN = torch.from_numpy(V).cuda(), torch.from_numpy(N).cuda()
            out = torch.full((c.height * c.width,), -7, dtype=torch.int32, device="cuda")
            stream = torch.cuda.current_stream()
            sw.sw_fusion_targets_static(dv, dn, dV, dN, c.width, c.height, c.fx, c.fy, c.cx, c.cy,
                                        1e-3, 0.85, out, stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            np.testing.assert_array_equal(got, want)
            assert (want >= 0).sum() > 100, call
            results.append(got)
        assert not np.array_equal(results[0], results[1])
        # the last inputs again, captured into a graph: nothing may allocate
        out.fill_(-7)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, capture_error_mode="global"):
            sw.sw_fusion_targets_static(dv, dn, dV, dN, c.width, c.height, c.fx, c.fy, c.cx, c.cy,
                                        1e-3, 0.85, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.all(out.cpu().numpy() == -7)   # captured, not run
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        # no surfels: the index map stays empty and no pixel has a target
        sw.sw_fusion_targets_static(None, None, dV, dN, c.width, c.height, c.fx, c.fy, c.cx, c.cy,
                                    1e-3, 0.85, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.all(out.cpu().numpy() == -1)
    finally:
        sw.sw_destroy_stream(h)


def test_static_fusion_targets_rejects_oversized_images():
    import torch
    from paper_1904_13073_gb300 import build as B
    B.build()
    t = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(sw.SwError) as e:
        sw.sw_fusion_targets_static(None, None, t, t, 640, 480, 500.0, 500.0, 320.0, 240.0, 1e-3, 0.85, out)
    assert e.value.status == 1 and "SW_STATIC_MAX_PIXELS" in str(e.value)
