"""Pins of the rigid pre-alignment oracle (Sec. 7: rigid alignment in the
manner of KinectFusion before the non-rigid solve): the analytic Jacobian
against finite differences, exactness at zero motion, exact recovery of a
known rigid motion with fixed correspondences, the composition into the node
transforms, and recovery from rendered depth."""
import numpy as np

import synth
from oracle import dq as DQ
from oracle import rigid as R
from oracle import skinning as SKIN
from oracle import solver as S
from oracle import stream as STREAM


def _motion(seed, deg=4.0):
    rng = np.random.default_rng(seed)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    om = axis * np.deg2rad(deg)
    tr = rng.normal(size=3) * 0.01
    return DQ.dq_from_rt(DQ.rodrigues_quat(om[None]), tr[None])[0]


def _tiny_model():
    s = synth.plain_tiny(seed=0)
    knn, w = SKIN.skin(s.surfel_v, s.node_p, s.node_sigma)
    return s, s.surfel_v.astype(np.float64), s.surfel_n.astype(np.float64), knn, w


def test_rigid_jacobian_matches_finite_differences():
    rng = np.random.default_rng(1)
    y = rng.normal(size=(50, 3)) + np.array([0.0, 0.0, 1.0])
    n_d = rng.normal(size=(50, 3))
    n_d /= np.linalg.norm(n_d, axis=1, keepdims=True)
    v_d = y + 0.01 * rng.normal(size=(50, 3))
    r0, J = R.rigid_terms(y, n_d, v_d)
    h = 1e-6
    for k in range(6):
        xi = np.zeros(6)
        xi[k] = h
        Dp = DQ.increment_dq(xi[None])[0]
        Dm = DQ.increment_dq(-xi[None])[0]
        yp, _ = R.apply_rigid(Dp, y, n_d)
        ym, _ = R.apply_rigid(Dm, y, n_d)
        fd = (R.rigid_terms(yp, n_d, v_d)[0] - R.rigid_terms(ym, n_d, v_d)[0]) / (2 * h)
        assert np.max(np.abs(fd - J[:, k])) < 1e-7


def test_zero_motion_is_exact_identity():
    s, v, n, knn, w = _tiny_model()
    dq0 = DQ.dq_identity(len(s.node_p))
    fixed = (np.ones(len(v), bool), v.copy(), n.copy())
    dq, T, stats = R.rigid_align(v, n, knn, w, dq0, lambda y, ny: fixed, 3)
    assert np.array_equal(T, DQ.dq_identity(1)[0])
    assert np.array_equal(dq, dq0)
    assert all(e == 0.0 for _, e in stats)


def test_exact_recovery_of_a_rigid_motion_with_fixed_targets():
    """Targets are the model's points and normals moved by a known rigid M:
    Gauss-Newton on the point-to-plane energy converges to M."""
    s, v, n, knn, w = _tiny_model()
    M = _motion(2)
    tv, tn = R.apply_rigid(M, v, n)
    fixed = (np.ones(len(v), bool), tv, tn)
    _, T, stats = R.rigid_align(v, n, knn, w, DQ.dq_identity(len(s.node_p)), lambda y, ny: fixed, 6)
    assert np.max(np.abs(DQ.qmatrix(T[None, :4])[0] - DQ.qmatrix(M[None, :4])[0])) < 1e-10
    p = np.array([[0.1, -0.2, 1.0], [0.0, 0.0, 0.5]])
    assert np.max(np.abs(R.apply_rigid(T, p, p)[0] - R.apply_rigid(M, p, p)[0])) < 1e-10
    assert stats[-1][1] < 1e-20 and stats[0][1] > 1e-6


def test_result_is_composed_into_every_node():
    s, v, n, knn, w = _tiny_model()
    rng = np.random.default_rng(4)
    dq0 = DQ.dq_normalize(DQ.dq_mul(np.repeat(_motion(5, 2.0)[None], len(s.node_p), 0),
                                    DQ.dq_identity(len(s.node_p))))
    M = _motion(6)
    b, vl, nl = S.warp_surfels(v, n, knn, w, dq0)
    tv, tn = R.apply_rigid(M, vl, nl)
    fixed = (np.ones(len(v), bool), tv, tn)
    dq, T, _ = R.rigid_align(v, n, knn, w, dq0, lambda y, ny: fixed, 6)
    p = s.node_p.astype(np.float64)
    want = R.apply_rigid(T, S.node_transform(dq0, p), p)[0]
    assert np.max(np.abs(S.node_transform(dq, p) - want)) < 1e-12
    del rng


def test_rigid_align_from_rendered_depth():
    """A rigidly moved surface rendered to depth: the pre-alignment alone
    brings the nodes to the true motion up to the depth image's
    discretisation, and lowers the data energy of the frame."""
    s = synth.plain_tiny(seed=3, noise=0.0, rigid=True)
    c = s.cam
    st = STREAM.OracleStream(STREAM.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy))
    st.set_model(s.surfel_v, s.surfel_n, s.surfel_r, s.surfel_c, s.surfel_t, s.node_p, s.node_sigma)
    st.upload_depth(s.frame(1), 1)
    stats = st.rigid_align(6)
    assert stats[-1][1] < 0.05 * stats[0][1]
    want = s.truth["warp"](st.node_p)
    assert np.max(np.abs(st.warped_nodes() - want)) < 3e-4
