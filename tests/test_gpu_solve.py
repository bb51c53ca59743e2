"""End-to-end parity of the CUDA solve and fusion with the FP64 oracle, plus
edge cases, error paths and checkpoint / resume.

Tolerances for the solved warp field: node rotations within 1e-4 rad and
node translations within 1e-5 m of the oracle's.  Translation is measured at
the node (T_j p_j), where it is a physical displacement; the translation part
of T_j alone mixes in rotation error times the node's distance from the
camera origin."""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import solver as OS

from gpu_helpers import (Pair, ensure_built, handing_over, load_gpu_state_into_oracle, oracle_for,
                         rotation_angle_between)

pytestmark = pytest.mark.gpu
ROT_TOL = 1e-4
TRANS_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


def _compare_nodes(p):
    _, dq = sw.sw_read_nodes(p.h)
    dq = dq.astype(np.float64)
    rot = rotation_angle_between(dq, p.o.node_dq)
    got = OS.node_transform(dq, p.o.node_p)
    trans = np.linalg.norm(got - p.o.warped_nodes(), axis=1)
    return float(rot.max()), float(trans.max())


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_MIXED, sw.SW_PRECISION_MIXED_F64DOTS, sw.SW_PRECISION_FP64])
def test_plain_tiny_solve_matches_oracle(precision):
    """160x120 wavy surface, 64 nodes, 5 GN x 10 PCG, in each solve precision."""
    scene = synth.plain_tiny(seed=0)
    p = Pair(scene, precision=precision)
    try:
        p.upload(1)
        st = sw.sw_solve_frame(p.h, scene.gn_iters, scene.pcg_iters)
        ost = p.o.solve_frame(scene.gn_iters, scene.pcg_iters)
        for k in range(scene.gn_iters):
            assert abs(st["n_corr"][k] - ost[k].n_corr) <= 2
            assert st["e_depth"][k] == pytest.approx(ost[k].e_depth, rel=1e-3)
            assert st["e_reg"][k] == pytest.approx(ost[k].e_reg, rel=1e-3, abs=1e-9)
        rot, trans = _compare_nodes(p)
        assert rot <= ROT_TOL and trans <= TRANS_TOL, (rot, trans)
        # the solve reduced the data energy to the noise floor (1 mm noise)
        assert st["e_depth"][-1] < 0.25 * st["e_depth"][0]
    finally:
        p.close()


def test_fp64_variant_matches_oracle_closely():
    """The all-FP64 solve against the FP64 oracle on identical FP32 depth
    maps: what remains is the FP32 storage of the surfels, the skinning
    weights and the maps, so the agreement is far inside the FP32 modes'
    1e-4 rad / 1e-5 m."""
    scene = synth.plain_tiny(seed=0)
    errs = {}
    for prec in (sw.SW_PRECISION_MIXED, sw.SW_PRECISION_FP64):
        p = Pair(scene, precision=prec)
        try:
            p.upload(1)
            p.set_maps_from_oracle()
            st = sw.sw_solve_frame(p.h, scene.gn_iters, scene.pcg_iters)
            ost = p.o.solve_frame(scene.gn_iters, scene.pcg_iters)
            assert [st["n_corr"][k] for k in range(scene.gn_iters)] == [o.n_corr for o in ost]
            errs[prec] = _compare_nodes(p)
        finally:
            p.close()
    rot64, trans64 = errs[sw.SW_PRECISION_FP64]
    assert rot64 <= 1e-6 and trans64 <= 1e-7, errs
    rot32, trans32 = errs[sw.SW_PRECISION_MIXED]
    assert rot64 <= rot32 and trans64 <= trans32, errs


def _report(name, data):
    """Write a JSON report to $SW_REPORT_DIR when that is set."""
    import json
    import os
    out = os.environ.get("SW_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, name), "w") as f:
            json.dump(data, f, indent=1)


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_MIXED, sw.SW_PRECISION_MIXED_F64DOTS, sw.SW_PRECISION_FP64])
def test_sequence_frames_match_oracle_on_identical_inputs(precision):
    """Bending sphere with outliers over three frames of solve + fusion.

    Every frame is compared on identical inputs: both sides take the same
    FP32 depth maps, and before each solve the oracle takes the library's
    own model (its fused surfels, skinning and node transforms, FP32 values;
    load_gpu_state_into_oracle) -- after that model was compared with the
    oracle's own fusion of the previous frame.  Within the solve, the
    library records each Gauss-Newton iteration's association; a decision
    that differs from the oracle's must lie at a rounding boundary, and there
    the oracle takes the library's (handing_over).  Each frame's warp field
    must then agree to the configuration's 1e-4 rad / 1e-5 m (the FP64
    variant to 1e-6 rad / 1e-7 m).  A second oracle stream runs the whole sequence on
    its own inputs; its distance from the library after each frame (the
    multi-frame drift, where an FP32 fusion decision that flips changes the
    next frame's model) is reported, not asserted."""
    scene = synth.random_scene(seed=3, n_surfels=6000, n_nodes=48, outliers=0.01)
    p = Pair(scene, precision=precision)
    free = oracle_for(scene)    # runs the sequence on its own inputs
    tol = (1e-6, 1e-7) if precision == sw.SW_PRECISION_FP64 else (ROT_TOL, TRANS_TOL)
    report = {"frames": []}
    try:
        sw.sw_debug_record_correspondence(p.h, True)
        for t in (1, 2, 3):
            p.upload(t)
            p.set_maps_from_oracle()   # identical FP32 depth maps on both sides
            load_gpu_state_into_oracle(p)
            st = sw.sw_solve_frame(p.h, 3, 10)
            boundary = handing_over(p.o, [sw.sw_read_correspondence_iter(p.h, k) for k in range(3)])
            ost = p.o.solve_frame(3, 10)
            del p.o.associate
            rot, trans = _compare_nodes(p)
            flips = [int(st["n_corr"][k] - ost[k].n_corr) for k in range(3)]
            assert flips == [0, 0, 0], flips
            free.upload_depth(scene.frame(t), t)
            free.solve_frame(3, 10)
            _, dq = sw.sw_read_nodes(p.h)
            dq = dq.astype(np.float64)
            drift_rot = float(rotation_angle_between(dq, free.node_dq).max())
            drift_trans = float(np.linalg.norm(OS.node_transform(dq, free.node_p) - free.warped_nodes(),
                                               axis=1).max())
            report["frames"].append({"frame": t, "rot_err_rad": rot, "trans_err_m": trans,
                                     "corr_count_diff": flips, "boundary_decisions": boundary,
                                     "drift_rot_rad": drift_rot,
                                     "drift_trans_m": drift_trans})
            assert rot <= tol[0] and trans <= tol[1], (t, rot, trans)
            sw.sw_fuse_frame(p.h)
            n_fused = p.o.fuse_frame()
            free.fuse_frame()
            v, n, tt = sw.sw_read_surfels(p.h)
            fused_gpu = tt[:, 1] == t
            fused_ora = p.o.t_obs == t
            # a fusion decision may flip on a 1-ulp difference of the two warps
            assert np.sum(fused_gpu != fused_ora) <= max(3, n_fused // 200)
            both = fused_gpu & fused_ora
            assert np.max(np.abs(v[both, :3] - p.o.v_ref[both])) < 2e-5
            assert np.max(np.abs(n[both, 3] - p.o.conf[both])) < 1e-4
    finally:
        p.close()
        _report(f"sequence_identical_inputs_prec{precision}.json", report)
        print(report)


def test_identity_zero_residual_gives_identity_update():
    """Live depth equals the reference depth, surfels back-projected from it,
    identity warp: every term has a zero residual, so the nodes stay put."""
    scene = synth.plain_tiny(seed=0, noise=0.0)
    c = scene.cam
    d = scene.frame(0)
    p = sw.params_for(c, c.width * c.height, len(scene.node_p))
    h = sw.sw_create_stream(p)
    try:
        # surfels = the GPU's own depth surfels of this frame
        tmp = sw.sw_create_stream(sw.params_for(c, 1, len(scene.node_p)))
        sw.sw_set_model(tmp, np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32), None,
                        sw.model_arrays(scene)[3])
        sw.sw_upload_depth(tmp, d, 0)
        V, N = sw.sw_read_maps(tmp, c.height, c.width)
        sw.sw_destroy_stream(tmp)
        ok = V[..., 3].reshape(-1) > 0
        v4 = V.reshape(-1, 4)[ok].copy()
        n4 = N.reshape(-1, 4)[ok].copy()
        n4[:, 3] = 1.0
        sw.sw_set_model(h, v4, n4, None, sw.model_arrays(scene)[3])
        sw.sw_upload_depth(h, d, 1)
        st = sw.sw_solve_frame(h, 2, 10)
        assert st["n_corr"][0] == ok.sum()
        assert st["e_depth"][0] == 0.0 and st["e_reg"][0] == 0.0
        _, dq = sw.sw_read_nodes(h)
        np.testing.assert_array_equal(dq, np.tile(np.array([1, 0, 0, 0, 0, 0, 0, 0], np.float32), (len(dq), 1)))
    finally:
        sw.sw_destroy_stream(h)


def test_edge_cases_and_errors():
    scene = synth.random_scene(seed=4, n_surfels=500, n_nodes=9)
    c = scene.cam
    v4, n4, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4)))
    try:
        with pytest.raises(sw.SwError) as e:
            sw.sw_solve_frame(h, 1, 1)
        assert e.value.status == 3                       # no model yet
        # minimum node count, ragged surfel count
        sw.sw_set_model(h, v4[:333], n4[:333], t2[:333], node4)
        sw.sw_upload_depth(h, scene.frame(1), 1)
        st = sw.sw_solve_frame(h, 1, 1)
        assert st["gn_iters"] == 1
        with pytest.raises(sw.SwError) as e:
            sw.sw_solve_frame(h, 0, 5)
        assert e.value.status == 1
        with pytest.raises(sw.SwError) as e:
            sw.sw_solve_frame(h, 17, 5)
        assert e.value.status == 1
        with pytest.raises(sw.SwError) as e:
            sw.sw_set_model(h, v4, n4, t2, node4[:8])   # fewer than 9 nodes
        assert e.value.status == 1
        # an empty depth frame: no correspondences, regulariser only
        sw.sw_set_model(h, v4, n4, t2, node4)
        sw.sw_upload_depth(h, np.zeros((c.height, c.width), np.float32), 2)
        st = sw.sw_solve_frame(h, 2, 4)
        assert st["n_corr"] == [0, 0] and st["e_depth"] == [0.0, 0.0]
        sw.sw_fuse_frame(h)
        # no surfels at all
        sw.sw_set_model(h, np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32), None, node4)
        sw.sw_upload_depth(h, scene.frame(1), 1)
        st = sw.sw_solve_frame(h, 1, 3)
        assert st["n_corr"] == [0]
        sw.sw_fuse_frame(h)
    finally:
        sw.sw_destroy_stream(h)


def test_memory_budget_refuses_a_stream():
    scene = synth.random_scene(seed=4, n_surfels=500, n_nodes=12)
    base = sw.sw_memory_in_use()
    try:
        sw.sw_set_memory_budget(base + (1 << 20))
        with pytest.raises(sw.SwError) as e:
            sw.sw_create_stream(sw.params_for(scene.cam, 10_000_000, 4096))
        assert e.value.status == 2
        assert sw.sw_memory_in_use() == base
    finally:
        sw.sw_set_memory_budget(0)


def test_checkpoint_resume_gives_identical_next_frame():
    scene = synth.random_scene(seed=6, n_surfels=4000, n_nodes=40)
    c = scene.cam
    v4, n4, t2, node4 = sw.model_arrays(scene)
    a = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4)))
    b = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4)))
    try:
        sw.sw_set_model(a, v4, n4, t2, node4)
        sw.sw_upload_depth(a, scene.frame(1), 1)
        sw.sw_solve_frame(a, 3, 8)
        sw.sw_fuse_frame(a)
        state = sw.sw_export_state(a)
        sw.sw_import_state(b, state)
        for h in (a, b):
            sw.sw_upload_depth(h, scene.frame(2), 2)
            sw.sw_solve_frame(h, 3, 8)
            sw.sw_fuse_frame(h)
        va, na, ta = sw.sw_read_surfels(a)
        vb, nb, tb = sw.sw_read_surfels(b)
        _, qa = sw.sw_read_nodes(a)
        _, qb = sw.sw_read_nodes(b)
        np.testing.assert_allclose(qa, qb, atol=2e-6)
        np.testing.assert_allclose(va, vb, atol=2e-6)
        assert np.sum(ta != tb) <= 2
    finally:
        sw.sw_destroy_stream(a)
        sw.sw_destroy_stream(b)


def test_precision_report():
    """The precision configuration: the 160x120 frame solved in each mode
    against the FP64 oracle (max node rotation / translation error, and the
    point-to-plane RMS at the last Gauss-Newton linearisation).  Writes
    precision_report.json to $SW_REPORT_DIR when that is set."""
    import json
    import os
    scene = synth.plain_tiny(seed=0)
    names = {sw.SW_PRECISION_MIXED: "fp32_assembly_doublefloat_dots",
             sw.SW_PRECISION_MIXED_F64DOTS: "fp32_assembly_fp64_dots",
             sw.SW_PRECISION_FP64: "fp64"}
    report, oracle_rms = {}, None
    for prec, name in names.items():
        p = Pair(scene, precision=prec)
        try:
            p.upload(1)
            st = sw.sw_solve_frame(p.h, scene.gn_iters, scene.pcg_iters)
            if oracle_rms is None:
                ost = p.o.solve_frame(scene.gn_iters, scene.pcg_iters)
                oracle_rms = float(np.sqrt(ost[-1].e_depth / ost[-1].n_corr))
                ora_dq = p.o.node_dq.copy()
            else:
                p.o.node_dq = ora_dq.copy()
            rot, trans = _compare_nodes(p)
            last = scene.gn_iters - 1
            report[name] = {"max_rot_err_rad": rot, "max_trans_err_m": trans,
                            "rms_last_gn_m": float(np.sqrt(st["e_depth"][last] / st["n_corr"][last]))}
            assert rot <= ROT_TOL and trans <= TRANS_TOL, (name, rot, trans)
        finally:
            p.close()
    report["oracle_rms_last_gn_m"] = oracle_rms
    out = os.environ.get("SW_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, "precision_report.json"), "w") as f:
            json.dump(report, f, indent=1)
    assert report["fp64"]["max_rot_err_rad"] <= report["fp32_assembly_doublefloat_dots"]["max_rot_err_rad"]


def test_autotune_keeps_state_and_parity():
    """The PCG autotuner times candidate granularities on the current system:
    it leaves the node transforms as they were, and the solve that follows
    still matches the oracle."""
    scene = synth.plain_tiny(seed=0)
    p = Pair(scene)
    try:
        p.upload(1)
        _, before = sw.sw_read_nodes(p.h)
        rows, us = sw.sw_autotune(p.h, scene.pcg_iters)
        assert rows in (16, 24, 32, 48, 64, 96) and us > 0
        _, after = sw.sw_read_nodes(p.h)
        np.testing.assert_array_equal(before, after)
        sw.sw_solve_frame(p.h, scene.gn_iters, scene.pcg_iters)
        p.o.solve_frame(scene.gn_iters, scene.pcg_iters)
        rot, trans = _compare_nodes(p)
        assert rot <= ROT_TOL and trans <= TRANS_TOL, (rows, rot, trans)
    finally:
        p.close()
