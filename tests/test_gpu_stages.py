"""Stage-by-stage parity of the CUDA path (through the C ABI) with the FP64
oracle on identical seeded inputs.

Integer results (k-NN ids, node graph, association pixels, index map, fusion
targets, usable-pixel masks) must match bit-exactly: both sides take those
decisions in FP32 with the same operation order on the same FP32 inputs.
Floating-point results are compared against tolerances derived from FP32
arithmetic (see each test)."""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import depth as ODEPTH
from oracle import skinning as OSKIN
from oracle import solver as OS
from oracle import fusion as OFU

from gpu_helpers import Pair, ensure_built, rigid_dq8_from, oracle_dq_from

pytestmark = pytest.mark.gpu
F32 = np.float32


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.fixture(scope="module")
def tiny():
    return synth.plain_tiny(seed=0)


@pytest.fixture(scope="module")
def small():
    return synth.random_scene(seed=5, n_surfels=5000, n_nodes=60, outliers=0.01)


# ---------------------------------------------------------------- K1 depth maps

@pytest.mark.parametrize("which", ["tiny", "small"])
def test_depth_maps(which, tiny, small):
    scene = tiny if which == "tiny" else small
    c = scene.cam
    p = Pair(scene)
    try:
        d = scene.frame(1).copy()
        d[5:9, 7:30] = 0.0                       # a hole: ragged validity
        sw.sw_upload_depth(p.h, d, 1)
        V, N = sw.sw_read_maps(p.h, c.height, c.width)
        m = ODEPTH.depth_maps(d, c.fx, c.fy, c.cx, c.cy)
        usable = V[..., 3] > 0
        np.testing.assert_array_equal(usable, m["valid"])
        ok = m["valid"]
        # FP32: a few ulps of |V| (~1 m) and of unit normals
        np.testing.assert_allclose(V[..., :3][ok], m["V"][ok], rtol=0, atol=4e-7)
        np.testing.assert_allclose(N[..., :3][ok], m["N"][ok], rtol=0, atol=2e-5)
        np.testing.assert_allclose(V[..., 3][ok], m["conf"][ok], rtol=2e-6, atol=0)
        np.testing.assert_allclose(N[..., 3][ok], m["radius"][ok], rtol=2e-5, atol=0)
    finally:
        p.close()


def test_depth_maps_without_tensor_map_path():
    """A width that is not a multiple of 4 (rows not 16-byte aligned) takes the
    plain-load staging instead of the TMA copy; same maps."""
    scene = synth.random_scene(seed=11, n_surfels=2000, n_nodes=30, width=162, height=98, f=130.0)
    c = scene.cam
    p = Pair(scene)
    try:
        d = scene.frame(1).copy()
        d[:, 40] = 0.0
        sw.sw_upload_depth(p.h, d, 1)
        V, N = sw.sw_read_maps(p.h, c.height, c.width)
        m = ODEPTH.depth_maps(d, c.fx, c.fy, c.cx, c.cy)
        np.testing.assert_array_equal(V[..., 3] > 0, m["valid"])
        ok = m["valid"]
        np.testing.assert_allclose(V[..., :3][ok], m["V"][ok], rtol=0, atol=4e-7)
        np.testing.assert_allclose(N[..., :3][ok], m["N"][ok], rtol=0, atol=2e-5)
    finally:
        p.close()


# ---------------------------------------------------------------- K2/K3 skinning, graph

@pytest.mark.parametrize("which", ["tiny", "small"])
def test_skinning_and_graph_bit_exact(which, tiny, small):
    scene = tiny if which == "tiny" else small
    p = Pair(scene)
    try:
        knn, w = sw.sw_read_skinning(p.h)
        np.testing.assert_array_equal(knn, p.o.knn)
        np.testing.assert_allclose(w, p.o.w, rtol=3e-6, atol=1e-30)
        np.testing.assert_array_equal(sw.sw_read_graph(p.h), p.o.graph)
    finally:
        p.close()


def test_skinning_full_size_sampled():
    """Full-size sphere (300k surfels, 2048 nodes): sampled surfels' 4-NN
    computed one by one by the oracle."""
    scene = synth.plain_full(seed=0)
    v4, n4, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(scene.cam, len(v4), len(node4)))
    try:
        sw.sw_set_model(h, v4, n4, t2, node4)
        knn, w = sw.sw_read_skinning(h)
        rng = np.random.default_rng(0)
        idx = np.sort(rng.choice(len(v4), 4000, replace=False))
        ref = OSKIN.knn_fp32(scene.surfel_v[idx], scene.node_p, 4)
        np.testing.assert_array_equal(knn[idx], ref)
        wr = OSKIN.skin_weights(scene.surfel_v[idx], scene.node_p, scene.node_sigma, ref)
        np.testing.assert_allclose(w[idx], wr, rtol=3e-6)
        np.testing.assert_array_equal(sw.sw_read_graph(h), OSKIN.node_graph(scene.node_p))
    finally:
        sw.sw_destroy_stream(h)


# ---------------------------------------------------------------- association

def _random_warp(scene, seed, angle=3.0, trans=0.01):
    axis, ang, tr = synth.random_rigid_dq_inputs(seed, len(scene.node_p), angle, trans)
    return rigid_dq8_from(axis, ang, tr), oracle_dq_from(axis, ang, tr)


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_association_bit_exact_on_given_live_surfels(which, tiny, small):
    scene = tiny if which == "tiny" else small
    p = Pair(scene)
    try:
        p.upload(1)
        p.set_maps_from_oracle()
        _, odq = _random_warp(scene, 11)
        _, vl, nl = OS.warp_surfels(p.o.v_ref, p.o.n_ref, p.o.knn, p.o.w, odq)
        vl32, nl32 = vl.astype(F32), nl.astype(F32)
        sw.sw_debug_set_live(p.h, vl32, nl32)
        sw.sw_debug_associate(p.h)
        got = sw.sw_read_correspondence(p.h)
        sel = OS.select_surfels(p.o.conf, p.o.t_obs, 1, 10.0, 2)
        ok, pix = OS.associate(vl32, nl32, sel, p.o.V32, p.o.N32, p.o.maps["valid"], p.o.p.cam,
                               p.o.p.corr_dist, p.o.p.corr_normal)
        np.testing.assert_array_equal(got, np.where(ok, pix, -1))
        assert ok.sum() > 0.3 * len(ok) if which == "tiny" else ok.sum() > 100
    finally:
        p.close()


# ---------------------------------------------------------------- index map and fusion targets

@pytest.mark.parametrize("which", ["tiny", "small"])
def test_fusion_targets_bit_exact_on_given_live_surfels(which, tiny, small):
    scene = tiny if which == "tiny" else small
    c = scene.cam
    p = Pair(scene)
    try:
        p.upload(1)
        p.set_maps_from_oracle()
        _, odq = _random_warp(scene, 12, angle=1.0, trans=0.003)
        _, vl, nl = OS.warp_surfels(p.o.v_ref, p.o.n_ref, p.o.knn, p.o.w, odq)
        vl32, nl32 = vl.astype(F32), nl.astype(F32)
        # put some surfels exactly on depth vertices so that fusion finds them
        V = p.o.V32.reshape(-1, 3)
        usable = p.o.maps["valid"].reshape(-1)
        pix = np.nonzero(usable)[0][::7]
        k = min(len(pix), len(vl32) // 3)
        vl32[:k] = V[pix[:k]]
        vl32[k:2 * k] = vl32[:k]                     # exact duplicates: id ties
        sw.sw_debug_set_live(p.h, vl32, nl32)
        target, imap = sw.sw_debug_fusion_targets(p.h, c.height, c.width)
        oim = OFU.index_map(vl32, p.o.p.cam)
        np.testing.assert_array_equal(imap, oim)
        otg = OFU.select_fusion_targets(oim, vl32, nl32, p.o.conf, p.o.V32, p.o.N32, p.o.maps["valid"],
                                        p.o.p.fuse_dist, p.o.p.fuse_normal)
        np.testing.assert_array_equal(target, otg)
        assert (otg >= 0).sum() > 0
    finally:
        p.close()


# ---------------------------------------------------------------- K4-K6 JᵀJ assembly

def _oracle_system(p, odq, absolute=True):
    o = p.o
    b, vl, nl = OS.warp_surfels(o.v_ref, o.n_ref, o.knn, o.w, odq)
    mask, tv, tn = o.associate(vl, nl)
    mask &= ~OS.unskinned(OS.DQ.blend(odq, o.knn, o.w))
    idx = np.nonzero(mask)[0]
    r, J = OS.data_terms(o.v_ref[idx], o.knn[idx], o.w[idx], odq, tv[idx], tn[idx])
    reg = OS.reg_terms(o.node_p, odq, o.graph, o.p.lam)
    A, g, S, gS = OS.assemble(o.pattern, len(o.node_p), o.knn[idx], J, r, reg, absolute=True)
    return mask, A, g, S, gS


@pytest.mark.parametrize("which", ["tiny", "small"])
def test_jtj_assembly_matches_oracle(which, tiny, small):
    """JᵀJ and Jᵀe of one linearisation: |gpu − oracle| <= 1e-4 · (|J|ᵀ|J|)
    entry-wise (FP32 sums of products are accurate relative to the sum of
    the absolute products, whatever their order)."""
    scene = tiny if which == "tiny" else small
    p = Pair(scene)
    try:
        p.upload(1)
        p.set_maps_from_oracle()
        dq8, odq = _random_warp(scene, 13, angle=2.0, trans=0.005)
        sw.sw_set_node_dq(p.h, dq8)
        nnzb, n_corr = sw.sw_debug_assemble(p.h)
        corr = sw.sw_read_correspondence(p.h)
        mask, A, g, S, gS = _oracle_system(p, odq)
        np.testing.assert_array_equal(corr >= 0, mask)      # the FP32 warps agree on every decision here
        assert n_corr == mask.sum()
        rows, cols, vals, gg = sw.sw_debug_read_jtj(p.h, nnzb, len(scene.node_p))
        assert np.all(rows <= cols)
        want = A.vals[A.index(rows, cols)]
        scale = S.vals[A.index(rows, cols)]
        err = np.abs(vals - want)
        assert np.all(err <= 1e-4 * scale + 1e-12), float(np.max(err / (scale + 1e-30)))
        # every upper block of the oracle's pattern is present on the GPU
        orows, ocols = A.rows_cols()
        assert nnzb == int(np.sum(orows <= ocols))
        gerr = np.abs(gg - g.reshape(-1))
        assert np.all(gerr <= 1e-4 * gS.reshape(-1) + 1e-12), float(np.max(gerr / (gS.reshape(-1) + 1e-30)))
    finally:
        p.close()
