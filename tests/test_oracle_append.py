"""Pins of the appending oracle (Sec. 6.2-6.4, Eq. 7-8) against closed forms,
hand-worked cases and brute force; nothing here re-calls the function under
test to make its own expected value."""
import json
import math
import os

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import append as AP
from oracle import dq as DQ
from oracle import stream as OST

import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))


def _maps(points, normals, conf=None, radius=None):
    """A one-row 'depth map' holding the given vertices (only what the append step reads)."""
    n = len(points)
    return {"V": np.asarray(points, dtype=np.float64).reshape(1, n, 3),
            "N": np.asarray(normals, dtype=np.float64).reshape(1, n, 3),
            "conf": np.ones((1, n)) if conf is None else np.asarray(conf).reshape(1, n),
            "radius": np.full((1, n), 0.002) if radius is None else np.asarray(radius).reshape(1, n),
            "valid": np.ones((1, n), dtype=bool)}


def _dq_translation_only(t):
    """Dual quaternions of pure translations (identity rotation): (1, 0; 0, t/2)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros((len(t), 8))
    out[:, 0] = 1.0
    out[:, 5:8] = 0.5 * t
    return out


def test_table1_values_are_the_defaults():
    assert AP.EPS == GOLDEN["epsilon"]
    assert AP.T_LOW_CONFID == GOLDEN["t_low_confid"]


def test_rigid_warp_field_inverts_exactly():
    """All nodes move by one rigid motion (R, t): every node stays (ratios 1),
    v_ref = Rᵀ(x − t), n_ref = Rᵀ n, and the strain is Rᵀ (singular values 1)."""
    rng = np.random.default_rng(1)
    node_p = rng.uniform(-0.1, 0.1, size=(12, 3)) + np.array([0, 0, 0.8])
    sigma = np.full(12, 0.025)
    rot = Rotation.from_rotvec([0.2, -0.1, 0.3])
    R = rot.as_matrix()
    t = np.array([0.01, -0.02, 0.015])
    q = rot.as_quat()                    # x y z w
    q0 = np.array([q[3], q[0], q[1], q[2]])
    dq = np.tile(DQ.dq_from_rt(q0[None], t[None])[0], (12, 1))
    live_nodes = node_p @ R.T + t
    x = live_nodes[:5] + rng.normal(scale=0.01, size=(5, 3))
    n = rng.normal(size=(5, 3))
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    res = AP.append_candidates(np.arange(5), _maps(x, n), dq, node_p, sigma)
    assert res["keep"].all()
    np.testing.assert_allclose(res["v_ref"], (x.astype(np.float32) - t) @ R, atol=1e-12)
    np.testing.assert_allclose(res["n_ref"], n.astype(np.float32) @ R, atol=1e-12)
    for J in res["strain"]:
        np.testing.assert_allclose(J, R.T, atol=1e-9)
    np.testing.assert_allclose(res["strain_norm"], 1.0, atol=1e-9)


def test_eq7_ratio_test_by_hand():
    """Node 0 at the origin, three nodes 5 cm away; their live distances to
    node 0 scale by 1.1, 1.3 and 0.7: node 1 stays, nodes 2 and 3 go."""
    node_p = np.array([[0, 0, 1.0], [0.05, 0, 1.0], [0, 0.05, 1.0], [0, 0, 1.05]])
    live = np.array([[0, 0, 1.0], [0.055, 0, 1.0], [0, 0.065, 1.0], [0, 0, 1.035]])
    dq = _dq_translation_only(live - node_p)
    x = np.array([[0.001, 0.001, 1.0]])
    res = AP.append_candidates(np.arange(1), _maps(x, [[0, 0, -1.0]]), dq, node_p, np.full(4, 0.025))
    # live d² from x: node 3 (0.035²+2e-6), node 1 (0.054²+1e-6), node 2 (0.064²+1e-6)
    assert list(res["knn"][0]) == [0, 3, 1, 2]      # nearest live node first
    assert list(res["keep"][0]) == [True, False, True, False]
    assert res["w"][0, 1] == 0.0 and res["w"][0, 3] == 0.0 and res["w"][0, 2] > 0.0


def test_eq7_coincident_reference_nodes_fail():
    node_p = np.array([[0, 0, 1.0], [0, 0, 1.0], [0.05, 0, 1.0], [0, 0.05, 1.0]])
    dq = _dq_translation_only(np.zeros((4, 3)))
    res = AP.append_candidates(np.arange(1), _maps([[0, 0, 1.0]], [[0, 0, -1.0]]), dq, node_p, np.full(4, 0.025))
    # slot 0 and slot 1 are the two coincident nodes (ids 0 then 1)
    assert list(res["knn"][0][:2]) == [0, 1]
    assert list(res["keep"][0]) == [True, False, True, True]


def test_delta_nn_weight_sum_closed_form():
    """Identity warp; the weight sum is Σ exp(−d²/2σ²) by hand.  A point near
    the nodes passes δ_nn, one 3σ from all of them fails."""
    s = 0.025
    node_p = np.array([[0, 0, 1.0], [0.03, 0, 1.0], [0, 0.03, 1.0], [0.03, 0.03, 1.0]])
    dq = _dq_translation_only(np.zeros((4, 3)))
    near = np.array([0.01, 0.01, 1.0])
    far = np.array([0.015, 0.015, 1.0 + 3 * s])
    res = AP.append_candidates(np.arange(2), _maps([near, far], [[0, 0, -1.0]] * 2), dq, node_p, np.full(4, s))
    for k, x in enumerate((near.astype(np.float32), far.astype(np.float32))):
        # the live nodes enter rounded to FP32 (the precision of the k-NN decision)
        want = sum(math.exp(-float(np.sum((x.astype(np.float64) - p.astype(np.float32)) ** 2)) / (2 * s * s))
                   for p in node_p)
        assert abs(res["wsum"][k] - want) < 1e-12
    assert res["wsum"][0] > AP.DELTA_NN and res["accept"][0]
    assert res["wsum"][1] < AP.DELTA_NN and not res["accept"][1]


def _analytic_strain(x, live_nodes, t, sigma):
    """J = I − Σ_i t_i ∇ŵ_iᵀ for pure translations (x_ref = x − Σ ŵ_i t_i)."""
    d = x[None, :] - live_nodes
    w = np.exp(-np.sum(d * d, axis=1) / (2 * sigma ** 2))
    gw = -(w / sigma ** 2)[:, None] * d
    W, G = w.sum(), gw.sum(axis=0)
    ghat = (gw * W - w[:, None] * G[None, :]) / W ** 2
    return np.eye(3) - t.T @ ghat


def test_strain_matches_analytic_jacobian_and_flags_compression():
    """Pure translations: the finite-difference strain equals the analytic one,
    and the Eq. 8 decision follows its largest singular value."""
    s = 0.015
    node_p = np.array([[0, 0, 1.0], [0.05, 0, 1.0], [0, 0.05, 1.0], [0.05, 0.05, 1.0]])
    sigma = np.full(4, s)
    # largest singular values of the analytic strain: about 1.10 and 1.37
    for amp, compressive in ((0.001, False), (0.004, True)):
        t = np.array([[amp, 0, 0], [-amp, 0, 0], [amp, 0, 0], [-amp, 0, 0]])
        dq = _dq_translation_only(t)
        live = (node_p + t).astype(np.float32).astype(np.float64)
        x = np.array([[0.025, 0.01, 1.0]])
        res = AP.append_candidates(np.arange(1), _maps(x, [[0, 0, -1.0]]), dq, node_p, sigma)
        assert res["keep"].all()
        J = _analytic_strain(x[0].astype(np.float32).astype(np.float64), live, t, s)
        fine = AP.strain(x.astype(np.float32).astype(np.float64), dq, res["knn"], res["keep"],
                         live.astype(np.float32), sigma, h=1e-5)[0]
        order = res["knn"][0]
        assert np.abs(fine - J).max() < 1e-6, (fine, J)   # O(h²) with h = 1e-5, σ = 1.5 cm
        assert np.abs(res["strain"][0] - J).max() < 5e-3
        smax = np.linalg.svd(J, compute_uv=False)[0]
        assert (smax > 1.0 + AP.EPS) == compressive, smax
        assert bool(res["accept"][0]) == (not compressive)
        assert list(order) == sorted(order, key=lambda j: (np.sum((x[0] - live[j]) ** 2), j))


def test_unstable_removal_boundaries():
    conf = np.array([9.9, 10.0, 9.9, 9.9, 3.0, 50.0])
    t_init = np.array([0, 0, 1, 2, 40, 0])
    t_now = 31
    # c < 10 and t_now − t_init >= 30
    assert list(AP.unstable(conf, t_init, t_now, 10.0)) == [True, False, True, False, False, False]


def test_empty_window_candidates_brute_force():
    rng = np.random.default_rng(3)
    hh, ww = 5, 7
    imap = rng.integers(-1, 3, size=(4 * hh, 4 * ww))
    imap[rng.random(imap.shape) < 0.8] = -1
    imap[0:4, 0:4] = -1
    usable = rng.random((hh, ww)) < 0.8
    usable[0, 0] = True
    want = []
    for y in range(hh):
        for x in range(ww):
            if not usable[y, x]:
                continue
            if all(imap[4 * y + a, 4 * x + b] < 0 for a in range(4) for b in range(4)):
                want.append(y * ww + x)
    got = AP.empty_window_pixels(imap, usable)
    assert list(got) == want and 0 in want


def test_append_frame_compaction_and_round_trip():
    """A tiny stream after one solve + fusion, with a hole cut in its model so
    that new surfels appear: survivors keep their order, appended surfels
    follow in pixel order, their live skinning warps v_ref back onto the depth
    vertex, and the capacity cuts from the end."""
    sc = synth.plain_tiny(seed=2)
    keep = sc.surfel_v[:, 0] < np.quantile(sc.surfel_v[:, 0], 0.7)   # cut away 30%
    c = sc.cam
    p = OST.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy)
    st = OST.OracleStream(p)
    t2 = np.zeros((int(keep.sum()), 2), dtype=np.int64)
    conf = np.full(int(keep.sum()), 5.0)
    t2[:7, 0] = -40          # seven old unstable surfels
    st.set_model(sc.surfel_v[keep], sc.surfel_n[keep], np.full(len(conf), 0.002), conf, t2, sc.node_p,
                 sc.node_sigma)
    st.upload_depth(sc.frame(1), 1)
    st.solve_frame(3, 8)
    st.fuse_frame()
    old_v = st.v_ref.copy()
    old_conf = st.conf.copy()
    dq = st.node_dq.copy()
    n_cand, n_app, n_rem = st.append_frame(max_surfels=10 ** 9)
    rec = st.last_append
    assert n_rem == 7 and n_app > 10 and n_cand >= n_app
    stay = ~AP.unstable(old_conf, t2[:, 0], 1, p.stable_conf)
    np.testing.assert_array_equal(st.v_ref[:int(stay.sum())], old_v[stay])
    pix = rec["pix"][rec["appended"]]
    assert np.all(np.diff(pix) > 0)
    # forward warp of v_ref with the live skinning lands on the depth vertex
    b = DQ.blend(dq, rec["knn"][rec["appended"]], rec["w"][rec["appended"]])
    x = st.maps["V"].reshape(-1, 3)[pix].astype(np.float32)
    np.testing.assert_allclose(DQ.dq_transform_point(b, st.v_ref[int(stay.sum()):]), x, atol=1e-12)
    assert np.all(st.t_init[int(stay.sum()):] == 1) and np.all(st.t_obs[int(stay.sum()):] == 1)
    # capacity
    st2 = OST.OracleStream(p)
    st2.set_model(sc.surfel_v[keep], sc.surfel_n[keep], np.full(len(conf), 0.002), conf, t2, sc.node_p,
                  sc.node_sigma)
    st2.upload_depth(sc.frame(1), 1)
    st2.solve_frame(3, 8)
    st2.fuse_frame()
    cap = int(stay.sum()) + 5
    _, n_app2, _ = st2.append_frame(max_surfels=cap)
    assert n_app2 == 5 and len(st2.v_ref) == cap
    np.testing.assert_array_equal(st2.v_ref[-5:], st.v_ref[int(stay.sum()):int(stay.sum()) + 5])


# ---------------------------------------------------------------- node-graph extension

def test_coverage_and_greedy_subsampling_by_hand():
    node_p = np.array([[0.0, 0.0, 1.0], [10.0, 0.0, 1.0]])
    sig = np.array([1.0, 1.0])
    pts = np.array([[0.5, 0.0, 1.0], [0.0, 0.99, 1.0], [0.0, 1.01, 1.0], [9.5, 0.5, 1.0], [5.0, 0.0, 1.0]])
    assert list(AP.covered(pts, node_p, sig)) == [True, True, False, True, False]
    # uncovered points on a line far from both nodes: 0, 0.3, 0.6, 1.0, 1.5, 2.2 (σ = 1)
    line = np.array([[4.0 + x, 5.0, 1.0] for x in (0.0, 0.3, 0.6, 1.0, 1.5, 2.2)])
    p, s = AP.subsample_nodes(line, node_p, sig, max_new=10)
    np.testing.assert_allclose(p[:, 0], [4.0, 5.0, 6.2], atol=1e-6)
    assert list(s) == [1.0, 1.0, 1.0]
    p2, _ = AP.subsample_nodes(line, node_p, sig, max_new=2)
    assert len(p2) == 2
    # a point within σ of an old node is never taken
    p3, _ = AP.subsample_nodes(np.array([[0.5, 0.0, 1.0]]), node_p, sig, max_new=10)
    assert len(p3) == 0


def test_new_node_takes_the_rigid_warp():
    """Every old node moves by one rigid motion: a new node's transform is it."""
    rot = Rotation.from_rotvec([0.1, 0.2, -0.05])
    q = rot.as_quat()
    q0 = np.array([q[3], q[0], q[1], q[2]])
    t = np.array([0.02, 0.01, -0.03])
    rng = np.random.default_rng(2)
    node_p = rng.uniform(-0.1, 0.1, (12, 3)) + [0, 0, 1.0]
    dq = np.tile(DQ.dq_from_rt(q0[None], t[None])[0], (12, 1))
    new = AP.new_node_transforms(np.array([[0.01, 0.02, 1.01], [0.05, -0.05, 0.95]], np.float32), node_p,
                                 np.full(12, 0.05), dq)
    for d in new:
        s = np.sign(d[0] * dq[0, 0])
        np.testing.assert_allclose(s * d, dq[0], atol=1e-12)


def _cut_nodes_scene():
    """plain_tiny with 30% of its surfels and every node in that region removed."""
    sc = synth.plain_tiny(seed=2)
    x_cut = np.quantile(sc.surfel_v[:, 0], 0.7)
    keep = sc.surfel_v[:, 0] < x_cut
    keep_n = sc.node_p[:, 0] < x_cut - 0.05
    return sc, keep, keep_n


def test_extend_nodes_on_a_stream_matches_the_definitions():
    from scipy.spatial import cKDTree
    sc, keep, keep_n = _cut_nodes_scene()
    c = sc.cam
    st = OST.OracleStream(OST.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy))
    n = int(keep.sum())
    st.set_model(sc.surfel_v[keep], sc.surfel_n[keep], np.full(n, 0.002), np.full(n, 15.0),
                 np.zeros((n, 2), np.int64), sc.node_p[keep_n], sc.node_sigma[keep_n])
    n_old = len(st.node_p)
    st.upload_depth(sc.frame(1), 1)
    st.solve_frame(2, 8)
    st.fuse_frame()
    dq_old = st.node_dq.copy()
    st.append_frame(10 ** 9, extend_nodes=True, max_nodes=n_old + 100)
    k = st.new_nodes
    assert k > 0 and len(st.node_p) == n_old + k
    np.testing.assert_array_equal(st.node_dq[:n_old], dq_old)
    new_p = st.node_p[n_old:]
    sig = st.node_sigma[n_old:]
    # new nodes are appended surfels, uncovered by the old nodes, at least σ apart
    app = st.v_ref[-len(st.last_append["appended"]):].astype(np.float32)
    assert all(np.any(np.all(app == p.astype(np.float32), axis=1)) for p in new_p)
    d_old = cKDTree(st.node_p[:n_old]).query(new_p)[0]
    assert np.all(d_old >= sig - 1e-6)
    if k > 1:
        dd = cKDTree(new_p).query(new_p, k=2)[0][:, 1]
        assert np.all(dd >= sig - 1e-6)
    # graph and skinning over all nodes (k-d tree, no ties expected on this data)
    _, g = cKDTree(st.node_p).query(st.node_p, k=9)
    np.testing.assert_array_equal(np.sort(st.graph, axis=1), np.sort(g[:, 1:], axis=1))
    # where a surfel's old set is still its 4-NN over the old nodes at its
    # current position (fusion may have moved it), the merged set is its
    # 4-NN over all nodes
    _, nn_old = cKDTree(st.node_p[:n_old]).query(st.v_ref, k=4)
    _, nn = cKDTree(st.node_p).query(st.v_ref, k=4)
    knn_before = st.knn_pre_extension
    fresh = np.all(np.sort(knn_before, axis=1) == np.sort(nn_old, axis=1), axis=1)
    assert fresh.mean() > 0.95
    np.testing.assert_array_equal(np.sort(st.knn[fresh], axis=1), np.sort(nn[fresh], axis=1))
    assert st.reskinned.sum() > 0 and np.all(st.knn[~st.reskinned] == knn_before[~st.reskinned])
    # a second stream with no room for new nodes keeps its graph
    st2 = OST.OracleStream(OST.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy))
    st2.set_model(sc.surfel_v[keep], sc.surfel_n[keep], np.full(n, 0.002), np.full(n, 15.0),
                  np.zeros((n, 2), np.int64), sc.node_p[keep_n], sc.node_sigma[keep_n])
    st2.upload_depth(sc.frame(1), 1)
    st2.solve_frame(2, 8)
    st2.fuse_frame()
    st2.append_frame(10 ** 9, extend_nodes=True, max_nodes=n_old)
    assert st2.new_nodes == 0 and len(st2.node_p) == n_old
