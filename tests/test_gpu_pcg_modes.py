"""The PCG's modes (Sec. 7's linear solve) against the FP64 oracle.

Mode 3 is the cluster PCG: a stream whose JᵀJ fits one thread-block
cluster's shared memory (FP32 modes) solves in one cluster of CTAs that
read each other's vectors through distributed shared memory.  Otherwise
the cooperative PCG keeps what fits of each CTA's share of JᵀJ in shared
memory: the rows' 6x6 blocks and the per-entry products (mode 2), only the
products with the blocks read from global memory every iteration (mode 1),
or nothing, a warp per block row (mode 0).  The library takes the highest
mode that fits; large batch members fall back to 1 or 0.  Here each mode is
forced (sw_debug_set_pcg_mode) on the 160x120 frame and on a small uneven
batch, and must match the oracle at 1e-4 rad / 1e-5 m and the other modes
to FP32 summation order."""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import solver as OS

from gpu_helpers import Pair, ensure_built, oracle_for, rotation_angle_between, set_maps_from_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()
    yield
    sw.sw_debug_set_pcg_mode(3)


def _errors(dq, o):
    dq = dq.astype(np.float64)
    rot = float(rotation_angle_between(dq, o.node_dq).max())
    trans = float(np.linalg.norm(OS.node_transform(dq, o.node_p) - o.warped_nodes(), axis=1).max())
    return rot, trans


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_MIXED, sw.SW_PRECISION_FP64])
def test_each_spmv_mode_matches_oracle(precision):
    scene = synth.plain_tiny(seed=0)
    got = {}
    oracle_dq = None
    modes = (3, 2, 1, 0) if precision != sw.SW_PRECISION_FP64 else (2, 1, 0)
    for mode in modes:
        sw.sw_debug_set_pcg_mode(mode)
        try:
            p = Pair(scene, precision=precision)
        finally:
            sw.sw_debug_set_pcg_mode(3)
        try:
            assert sw.sw_debug_pcg_mode(p.h) == mode
            p.upload(1)
            p.set_maps_from_oracle()
            sw.sw_solve_frame(p.h, scene.gn_iters, scene.pcg_iters)
            if oracle_dq is None:
                p.o.solve_frame(scene.gn_iters, scene.pcg_iters)
                oracle_dq = p.o.node_dq.copy()
            p.o.node_dq = oracle_dq
            _, dq = sw.sw_read_nodes(p.h)
            rot, trans = _errors(dq, p.o)
            assert rot <= 1e-4 and trans <= 1e-5, (mode, rot, trans)
            got[mode] = dq.astype(np.float64)
        finally:
            p.close()
    # the modes differ only in where the SpMV reads the blocks from and in
    # the order of its FP32 sums
    for mode in modes[1:]:
        assert np.max(np.abs(got[mode] - got[modes[0]])) < 2e-6, mode


def test_each_spmv_mode_in_an_uneven_batch_matches_oracle():
    scenes = [synth.random_scene(seed=20, n_surfels=3000, n_nodes=30),
              synth.random_scene(seed=21, n_surfels=9000, n_nodes=90, width=128, height=96, f=120.0),
              synth.plain_tiny(seed=2)]
    oracles = []
    for s in scenes:
        o = oracle_for(s)
        o.upload_depth(s.frame(1), 1)
        oracles.append(o)
    solved = False
    for mode in (3, 2, 1, 0):
        hs = []
        for s in scenes:
            v4, n4, t2, node4 = sw.model_arrays(s)
            h = sw.sw_create_stream(sw.params_for(s.cam, len(v4), len(node4)))
            sw.sw_set_model(h, v4, n4, t2, node4)
            hs.append(h)
        sw.sw_debug_set_pcg_mode(mode)
        try:
            b = sw.sw_batch_create(hs)
        finally:
            sw.sw_debug_set_pcg_mode(3)
        try:
            assert sw.sw_batch_debug_pcg_mode(b) == mode
            sw.sw_batch_upload_depth(b, [s.frame(1) for s in scenes], [1] * len(scenes))
            for h, o in zip(hs, oracles):
                set_maps_from_oracle(h, o)   # the oracle's maps rounded to FP32, on both sides
            if not solved:
                for o in oracles:
                    o.solve_frame(3, 10)
                solved = True
            sw.sw_batch_solve(b, 3, 10)
            for k, (h, o) in enumerate(zip(hs, oracles)):
                rot, trans = _errors(sw.sw_read_nodes(h)[1], o)
                assert rot <= 1e-4 and trans <= 1e-5, (mode, k, rot, trans)
        finally:
            sw.sw_batch_destroy(b)
            for h in hs:
                sw.sw_destroy_stream(h)
