"""Pins of the oracle's skinning, association, residuals, Jacobians, JtJ, PCG and
Gauss-Newton (Sec. 6.5, Sec. 7, Eq. 9-11, Sec. 8) against brute force, closed
forms, finite differences and invariants."""
import numpy as np
import pytest
from scipy.linalg import cho_factor, cho_solve
from scipy.spatial import cKDTree

import synth
from oracle import dq as DQ
from oracle import depth as DEPTH
from oracle import skinning as SKIN
from oracle import solver as S
from oracle import stream as STREAM

F32 = np.float32


# ---------------------------------------------------------------- skinning

def test_knn_matches_kdtree():
    rng = np.random.default_rng(0)
    nodes = rng.uniform(-1, 1, (64, 3)).astype(F32)
    pts = rng.uniform(-1, 1, (500, 3)).astype(F32)
    got = SKIN.knn_fp32(pts, nodes, 4)
    _, ref = cKDTree(nodes.astype(np.float64)).query(pts.astype(np.float64), k=4)
    np.testing.assert_array_equal(got, ref)


def test_knn_brute_force_fp32_with_ties():
    # nodes on a unit grid: exact ties, decided by the lower id
    g = np.stack(np.meshgrid(np.arange(3.0), np.arange(3.0), [0.0]), -1).reshape(-1, 3).astype(F32)
    q = np.array([[0.5, 0.5, 0.0], [1.0, 1.0, 0.0], [0.25, 1.75, 0.5]], dtype=F32)
    got = SKIN.knn_fp32(q, g, 4)
    for qi, row in zip(q, got):
        d2 = []
        for j, p in enumerate(g):
            dx, dy, dz = F32(qi[0] - p[0]), F32(qi[1] - p[1]), F32(qi[2] - p[2])
            d2.append((F32(F32(F32(dx * dx) + F32(dy * dy)) + F32(dz * dz)), j))
        want = [j for _, j in sorted(d2)[:4]]
        assert list(row) == want
    assert list(got[0]) == [0, 1, 3, 4]


def test_graph_excludes_self_and_weights_closed_form():
    rng = np.random.default_rng(1)
    nodes = rng.uniform(-1, 1, (30, 3)).astype(F32)
    gr = SKIN.node_graph(nodes)
    assert gr.shape == (30, 8)
    assert not np.any(gr == np.arange(30)[:, None])
    _, ref = cKDTree(nodes.astype(np.float64)).query(nodes.astype(np.float64), k=9)
    np.testing.assert_array_equal(gr, ref[:, 1:])
    pts = rng.uniform(-1, 1, (5, 3)).astype(F32)
    sig = np.full(30, 0.3, dtype=F32)
    knn, w = SKIN.skin(pts, nodes, sig)
    d = np.linalg.norm(pts[:, None].astype(np.float64) - nodes[knn].astype(np.float64), axis=2)
    np.testing.assert_allclose(w, np.exp(-d ** 2 / (2 * np.float64(F32(0.3)) ** 2)), rtol=1e-14)


# ---------------------------------------------------------------- association

def test_association_brute_force_tiny():
    cam = (100.0, 100.0, 3.5, 2.5, 8, 6)
    V = np.zeros((6, 8, 3), dtype=F32)
    N = np.zeros((6, 8, 3), dtype=F32)
    usable = np.zeros((6, 8), dtype=bool)
    V[2, 5] = [0.015, -0.005, 1.0]
    N[2, 5] = [0.0, 0.0, -1.0]
    usable[2, 5] = True
    # u = 100*x/z + 3.5 -> floor(u + 0.5) = 5 needs x/z in [0.01, 0.02)
    v = np.array([[0.015, -0.005, 1.0],      # hits pixel (5, 2), exact vertex
                  [0.015, -0.005, 1.049],    # same pixel, 4.9 cm behind: kept
                  [0.015, -0.005, 1.06],     # projects to (5,2)? x/z=0.01415: yes; 6 cm: rejected
                  [0.0251, -0.005, 1.0],     # pixel (6, 2): not usable
                  [0.015, -0.005, -1.0],     # behind the camera
                  [0.015, -0.005, 1.0]])     # normal too far off
    n = np.array([[0, 0, -1.0], [0, 0, -1.0], [0, 0, -1.0], [0, 0, -1.0], [0, 0, -1.0],
                  [0.0, 0.75, -np.sqrt(1 - 0.75 ** 2)]])
    sel = np.array([True] * 6)
    ok, pix = S.associate(v, n, sel, V, N, usable, cam, 0.05, 0.7)
    assert list(ok) == [True, True, False, False, False, False]
    assert list(pix[:2]) == [2 * 8 + 5] * 2
    sel[0] = False
    ok, _ = S.associate(v, n, sel, V, N, usable, cam, 0.05, 0.7)
    assert not ok[0]


def test_projection_fp32_is_roundtrip_exact_on_pixel_centres():
    fx, fy, cx, cy = 140.0, 140.0, 80.0, 60.0
    xs, ys = np.meshgrid(np.arange(160.0), np.arange(120.0))
    d = np.full(xs.shape, 1.0)
    V = DEPTH.depth_maps(d, fx, fy, cx, cy)["V"].reshape(-1, 3).astype(F32)
    px, py = S.project_fp32(V, fx, fy, cx, cy)
    np.testing.assert_array_equal(px, xs.ravel())
    np.testing.assert_array_equal(py, ys.ravel())


def test_selection_rule():
    sel = S.select_surfels(np.array([10.0, 10.5, 1.0, 1.0]), np.array([0, 0, 3, 2]), 5, 10.0, 2)
    assert list(sel) == [False, True, True, False]


# ---------------------------------------------------------------- residuals / Jacobians

def _random_state(rng, n_nodes=6, n_pts=40, ang=0.3, tr=0.1):
    node_p = rng.normal(size=(n_nodes, 3))
    axis = rng.normal(size=(n_nodes, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    om = axis * rng.uniform(0, ang, (n_nodes, 1))
    node_dq = DQ.dq_from_rt(DQ.rodrigues_quat(om), rng.normal(size=(n_nodes, 3)) * tr)
    knn = np.stack([rng.permutation(n_nodes)[:4] for _ in range(n_pts)])
    w = rng.uniform(0.05, 1.0, (n_pts, 4))
    v = rng.normal(size=(n_pts, 3))
    tv = rng.normal(size=(n_pts, 3))
    tn = rng.normal(size=(n_pts, 3))
    tn /= np.linalg.norm(tn, axis=1, keepdims=True)
    return node_p, node_dq, knn, w, v, tv, tn


def test_data_jacobian_matches_finite_differences():
    rng = np.random.default_rng(3)
    node_p, node_dq, knn, w, v, tv, tn = _random_state(rng)
    r0, J = S.data_terms(v, knn, w, node_dq, tv, tn)
    h = 1e-6
    for node in range(len(node_p)):
        for c in range(6):
            xi = np.zeros((len(node_p), 6))
            xi[node, c] = h
            rp, _ = S.data_terms(v, knn, w, DQ.dq_mul(DQ.increment_dq(xi), node_dq), tv, tn)
            rm, _ = S.data_terms(v, knn, w, DQ.dq_mul(DQ.increment_dq(-xi), node_dq), tv, tn)
            fd = (rp - rm) / (2 * h)
            an = np.sum(np.where(knn == node, J[:, :, c], 0.0), axis=1)
            assert np.max(np.abs(fd - an)) <= 1e-6


def test_reg_jacobian_matches_finite_differences_and_rigid_zero():
    rng = np.random.default_rng(4)
    node_p, node_dq, *_ = _random_state(rng, n_nodes=12)
    graph = SKIN.node_graph(node_p.astype(F32))
    j, i, r, Jj, Ji = S.reg_terms(node_p, node_dq, graph, 5.0)
    h = 1e-6
    for node in range(12):
        for c in range(6):
            xi = np.zeros((12, 6))
            xi[node, c] = h
            rp = S.reg_terms(node_p, DQ.dq_mul(DQ.increment_dq(xi), node_dq), graph, 5.0)[2]
            rm = S.reg_terms(node_p, DQ.dq_mul(DQ.increment_dq(-xi), node_dq), graph, 5.0)[2]
            fd = (rp - rm) / (2 * h)
            an = (np.where((j == node)[:, None], Jj[:, :, c], 0.0)
                  + np.where((i == node)[:, None], Ji[:, :, c], 0.0))
            assert np.max(np.abs(fd - an)) <= 1e-6
    # one common rigid motion: zero regulariser residual
    rig = np.repeat(node_dq[:1], 12, axis=0)
    assert np.max(np.abs(S.reg_terms(node_p, rig, graph, 5.0)[2])) < 1e-14


def test_zero_residual_identity_update(tiny_scene):
    s = tiny_scene
    c = s.cam
    d = s.frame(0).astype(np.float64)
    d = np.where(d > 0, 1.0 + 0.0 * d, 0.0) + 0.05 * np.sin(np.arange(d.size).reshape(d.shape) * 0.001)
    d = d.astype(F32)
    m = DEPTH.depth_maps(d, c.fx, c.fy, c.cx, c.cy)
    ok = m["valid"].reshape(-1)
    V = m["V"].reshape(-1, 3)[ok]
    Nn = m["N"].reshape(-1, 3)[ok]
    p = STREAM.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy)
    st = STREAM.OracleStream(p)
    n = len(V)
    st.set_model(V, Nn, np.full(n, 1e-3), np.ones(n), np.zeros((n, 2), np.int64),
                 s.node_p, s.node_sigma)
    # surfels back-projected from this very depth image in FP64
    st.v_ref, st.n_ref = V.copy(), Nn.copy()
    st.upload_depth(d, 1)
    dq0 = st.node_dq.copy()
    stats = st.solve_frame(2, 10, keep_masks=True)
    assert stats[0].n_corr == n
    assert stats[0].e_depth == 0.0 and stats[0].e_reg == 0.0
    np.testing.assert_array_equal(st.node_dq, dq0)


def test_jtj_is_symmetric_psd_and_pcg_matches_cholesky(tiny_scene):
    s = tiny_scene
    c = s.cam
    p = STREAM.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy)
    st = STREAM.OracleStream(p)
    st.set_model(s.surfel_v, s.surfel_n, s.surfel_r, s.surfel_c, s.surfel_t, s.node_p, s.node_sigma)
    st.upload_depth(s.frame(1), 1)
    _, v_live, n_live = S.warp_surfels(st.v_ref, st.n_ref, st.knn, st.w, st.node_dq)
    mask, tv, tn = st.associate(v_live, n_live)
    idx = np.nonzero(mask)[0]
    r, J = S.data_terms(st.v_ref[idx], st.knn[idx], st.w[idx], st.node_dq, tv[idx], tn[idx])
    reg = S.reg_terms(st.node_p, st.node_dq, st.graph, p.lam)
    A, g = S.assemble(st.pattern, len(st.node_p), st.knn[idx], J, r, reg)
    Ad = A.dense()
    np.testing.assert_allclose(Ad, Ad.T, atol=1e-12 * np.abs(Ad).max())
    ev = np.linalg.eigvalsh(Ad)
    assert ev.min() > -1e-10 * ev.max()
    # dense definition: A = Jᵀ J over all terms
    n6 = 6 * len(st.node_p)
    Jd = np.zeros((len(idx) + 3 * len(reg[0]), n6))
    for t in range(len(idx)):
        for k in range(4):
            Jd[t, 6 * st.knn[idx[t], k]:6 * st.knn[idx[t], k] + 6] += J[t, k]
    base = len(idx)
    for e in range(len(reg[0])):
        Jd[base + 3 * e:base + 3 * e + 3, 6 * reg[0][e]:6 * reg[0][e] + 6] += reg[3][e]
        Jd[base + 3 * e:base + 3 * e + 3, 6 * reg[1][e]:6 * reg[1][e] + 6] += reg[4][e]
    e = np.concatenate([r, reg[2].reshape(-1)])
    np.testing.assert_allclose(Ad, Jd.T @ Jd, atol=1e-10 * np.abs(Ad).max())
    np.testing.assert_allclose(g.reshape(-1), Jd.T @ e, atol=1e-10 * np.abs(g).max())
    # PCG after 6N iterations equals the dense Cholesky solve
    Minv = S.block_jacobi_inverse(A)
    x, _, _ = S.pcg(A, -g.reshape(-1), Minv, n6)
    ref = cho_solve(cho_factor(Ad), -g.reshape(-1))
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)


def test_pcg_stops_on_zero_residual_and_detects_breakdown():
    A = S.BlockMatrix(2, np.array([0, 3]))
    A.vals[0] = np.eye(6) * 2
    A.vals[1] = np.eye(6) * 4
    Minv = S.block_jacobi_inverse(A)
    x, rz, done = S.pcg(A, np.zeros(12), Minv, 5)
    assert done == 0 and rz == 0.0 and not np.any(x)
    A.vals[1][2, 2] = -1.0
    with pytest.raises(S.SolverBreakdown):
        S.block_jacobi_inverse(A)


def test_exact_rigid_recovery_identity_association(tiny_scene):
    """All nodes share one rigid motion; targets are the rigidly moved surfels
    and normals at their own pixels: GN recovers T for every node."""
    s = tiny_scene
    rng = np.random.default_rng(9)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    om = axis * np.deg2rad(4.0)
    tr = np.array([0.012, -0.008, 0.015])
    T = DQ.dq_from_rt(DQ.rodrigues_quat(om[None]), tr[None])
    v = s.surfel_v.astype(np.float64)
    n = s.surfel_n.astype(np.float64)
    tv = DQ.dq_transform_point(np.repeat(T, len(v), 0), v)
    tn = DQ.dq_rotate_vector(np.repeat(T, len(v), 0), n)
    knn, w = SKIN.skin(s.surfel_v, s.node_p, s.node_sigma)
    graph = SKIN.node_graph(s.node_p)
    patt = S.BlockMatrix.pattern(len(s.node_p), knn, graph).keys
    node_p = s.node_p.astype(np.float64)
    dq, stats = S.gauss_newton(v, n, knn, w, node_p, DQ.dq_identity(len(node_p)), graph, patt,
                               5.0, 6, 6 * len(node_p),
                               fixed_targets=(np.ones(len(v), bool), tv, tn))
    got = S.node_transform(dq, node_p)
    want = DQ.dq_transform_point(np.repeat(T, len(node_p), 0), node_p)
    assert np.max(np.abs(got - want)) < 1e-9
    assert np.max(np.abs(DQ.qmatrix(dq[:, :4]) - DQ.qmatrix(T[:, :4]))) < 1e-9
    assert stats[-1].e_depth < 1e-20


def test_rigid_recovery_from_rendered_depth():
    """Depth rendered from the rigidly moved surface: recovery limited only by
    the discretisation of the depth image (~1e-4)."""
    s = synth.plain_tiny(seed=3, noise=0.0, rigid=True)
    c = s.cam
    p = STREAM.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy)
    st = STREAM.OracleStream(p)
    st.set_model(s.surfel_v, s.surfel_n, s.surfel_r, s.surfel_c, s.surfel_t, s.node_p, s.node_sigma)
    st.upload_depth(s.frame(1), 1)
    st.solve_frame(6, 60)
    want = s.truth["warp"](st.node_p)
    assert np.max(np.abs(st.warped_nodes() - want)) < 3e-4


def test_pcg_iterate_is_krylov_minimiser(tiny_scene):
    """k PCG steps minimise the A-norm error over x0 + K_k(M⁻¹A, M⁻¹b):
    compared with that minimiser built directly (QR basis, projected solve)."""
    s = tiny_scene
    c = s.cam
    p = STREAM.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy)
    st = STREAM.OracleStream(p)
    st.set_model(s.surfel_v, s.surfel_n, s.surfel_r, s.surfel_c, s.surfel_t, s.node_p, s.node_sigma)
    st.upload_depth(s.frame(1), 1)
    _, v_live, n_live = S.warp_surfels(st.v_ref, st.n_ref, st.knn, st.w, st.node_dq)
    mask, tv, tn = st.associate(v_live, n_live)
    idx = np.nonzero(mask)[0]
    r, J = S.data_terms(st.v_ref[idx], st.knn[idx], st.w[idx], st.node_dq, tv[idx], tn[idx])
    reg = S.reg_terms(st.node_p, st.node_dq, st.graph, p.lam)
    A, g = S.assemble(st.pattern, len(st.node_p), st.knn[idx], J, r, reg)
    Ad = A.dense()
    Minv = S.block_jacobi_inverse(A)
    Md = np.zeros_like(Ad)
    for j in range(A.n):
        Md[6 * j:6 * j + 6, 6 * j:6 * j + 6] = Minv[j]
    b = -g.reshape(-1)
    for k in range(1, 7):
        x, _, _ = S.pcg(A, b, Minv, k)
        K = [Md @ b]
        for _ in range(k - 1):
            K.append(Md @ (Ad @ K[-1]))
        Q, _ = np.linalg.qr(np.stack(K, axis=1))
        want = Q @ np.linalg.solve(Q.T @ Ad @ Q, Q.T @ b)
        assert np.linalg.norm(x - want) <= 1e-8 * np.linalg.norm(want)
