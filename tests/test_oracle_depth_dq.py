"""Pins of the oracle's depth processing (Sec. 5, Eq. 4) and dual-quaternion
algebra (Sec. 3-4, Eq. 1-3) against closed forms and independent libraries."""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import dq as DQ
from oracle import depth as DEPTH
from oracle import stream as STREAM

HERE = os.path.dirname(__file__)


def test_params_match_table1():
    g = json.load(open(os.path.join(HERE, "golden", "table1.json")))
    p = STREAM.Params(10, 10, 1, 1, 5, 5)
    assert p.lam == g["lambda"]
    assert p.fuse_dist == g["delta_distance_m"]
    assert p.fuse_normal == g["delta_normal"]
    assert p.stable_conf == g["delta_stable"]
    assert p.recent_frames == g["delta_recent"]
    assert DEPTH.PHI == g["phi"]
    assert DEPTH.GRAZING_DEG == g["grazing_clamp_deg"]


# ---------------------------------------------------------------- depth (Sec. 5)

def test_plane_normals_radius_confidence():
    z0, f = 1.25, 140.0
    d = np.full((21, 31), z0, dtype=np.float32)
    m = DEPTH.depth_maps(d, f, f, 15.0, 10.0)
    inner = m["valid"][1:-1, 1:-1]
    assert inner.all()
    assert not m["valid"][0].any() and not m["valid"][-1].any()
    assert not m["valid"][:, 0].any() and not m["valid"][:, -1].any()
    n = m["N"][1:-1, 1:-1]
    np.testing.assert_array_equal(n, np.broadcast_to([0.0, 0.0, -1.0], n.shape))
    np.testing.assert_allclose(m["radius"][1:-1, 1:-1], np.sqrt(2.0) * z0 / f, rtol=1e-15)
    assert m["conf"][10, 15] == 1.0                         # principal point
    # γ at (x, y) = |(x−cx, y−cy)| / |(cx, cy)|
    x, y = 20, 3
    gam = np.hypot(x - 15.0, y - 10.0) / np.hypot(15.0, 10.0)
    assert m["conf"][y, x] == pytest.approx(np.exp(-gam ** 2 / (2 * 0.36)), rel=1e-15)
    # vertex map: D K^-1 (u, 1)
    assert m["V"][y, x] == pytest.approx([z0 * (x - 15.0) / f, z0 * (y - 10.0) / f, z0])


def test_tilted_plane_normal_is_exact_and_faces_camera():
    # plane n·X = h seen by a pinhole camera: depth along ray (a, b, 1) is h / n·(a, b, 1)
    nrm = np.array([0.3, -0.2, -1.0])
    nrm /= np.linalg.norm(nrm)
    h = -1.0
    fx, fy, cx, cy = 100.0, 110.0, 12.0, 9.0
    xs, ys = np.meshgrid(np.arange(25.0), np.arange(19.0))
    ray = np.stack([(xs - cx) / fx, (ys - cy) / fy, np.ones_like(xs)], -1)
    depth = h / (ray @ nrm)
    m = DEPTH.depth_maps(depth, fx, fy, cx, cy)
    n = m["N"][m["valid"]]
    np.testing.assert_allclose(n, np.broadcast_to(nrm, n.shape), atol=1e-12)
    assert np.all(np.sum(n * m["V"][m["valid"]], axis=1) < 0)


def test_invalid_neighbour_and_grazing_clamp():
    d = np.full((9, 9), 1.0)
    d[4, 5] = 0.0
    m = DEPTH.depth_maps(d, 50.0, 50.0, 4.0, 4.0)
    assert not m["valid"][4, 4] and not m["valid"][4, 6] and not m["valid"][3, 5]
    assert not m["valid"][4, 5] and m["valid"][2, 2]
    # steep plane: |n_z| < cos 75° -> radius uses cos 75°
    xs, ys = np.meshgrid(np.arange(15.0), np.arange(15.0))
    nrm = np.array([0.99, 0.0, -np.sqrt(1 - 0.99 ** 2)])
    ray = np.stack([(xs - 7) / 60.0, (ys - 7) / 60.0, np.ones_like(xs)], -1)
    depth = -1.0 / (ray @ nrm)
    m = DEPTH.depth_maps(depth, 60.0, 60.0, 7.0, 7.0)
    ok = m["valid"]
    expect = np.sqrt(2) * depth[ok] / (60.0 * np.cos(np.deg2rad(75)))
    np.testing.assert_allclose(m["radius"][ok], expect, rtol=1e-9)


# ---------------------------------------------------------------- dual quaternions

def _rand_rt(rng, n):
    rot = Rotation.random(n, random_state=rng)
    qs = rot.as_quat()                                   # scipy is scalar-last
    q = np.concatenate([qs[:, 3:], qs[:, :3]], axis=1)
    t = rng.normal(size=(n, 3))
    return rot, q, t


def test_quaternion_rotation_matches_scipy():
    rng = np.random.default_rng(1)
    rot, q, _ = _rand_rt(rng, 50)
    p = rng.normal(size=(50, 3))
    np.testing.assert_allclose(DQ.qrotate(q, p), rot.apply(p), atol=1e-13)
    np.testing.assert_allclose(DQ.qmatrix(q), rot.as_matrix(), atol=1e-13)
    rot2, q2, _ = _rand_rt(rng, 50)
    np.testing.assert_allclose(DQ.qmatrix(DQ.qmul(q, q2)), (rot * rot2).as_matrix(), atol=1e-13)


def test_rodrigues_matches_scipy():
    rng = np.random.default_rng(2)
    om = rng.normal(size=(40, 3)) * 0.3
    om[0] = 0.0
    got = DQ.rodrigues_quat(om)
    ref = Rotation.from_rotvec(om).as_matrix()
    np.testing.assert_allclose(DQ.qmatrix(got), ref, atol=1e-14)


def test_dq_rigid_transform_and_composition_match_matrices():
    rng = np.random.default_rng(3)
    rot, q, t = _rand_rt(rng, 30)
    rot2, q2, t2 = _rand_rt(rng, 30)
    p = rng.normal(size=(30, 3))
    d1 = DQ.dq_from_rt(q, t)
    np.testing.assert_allclose(DQ.dq_transform_point(d1, p), rot.apply(p) + t, atol=1e-12)
    d2 = DQ.dq_from_rt(q2, t2)
    # left factor applied last: d1 ⊗ d2 is x -> R1 (R2 x + t2) + t1
    want = rot.apply(rot2.apply(p) + t2) + t
    np.testing.assert_allclose(DQ.dq_transform_point(DQ.dq_mul(d1, d2), p), want, atol=1e-12)
    np.testing.assert_allclose(DQ.dq_inverse_transform_point(d1, rot.apply(p) + t), p, atol=1e-12)


def test_blend_of_identical_transforms_is_that_transform():
    rng = np.random.default_rng(4)
    rot, q, t = _rand_rt(rng, 1)
    node_dq = np.repeat(DQ.dq_from_rt(q, t), 6, axis=0)
    knn = rng.integers(0, 6, (200, 4))
    w = rng.uniform(0.01, 3.0, (200, 4))
    p = rng.normal(size=(200, 3))
    b = DQ.blend(node_dq, knn, w)
    np.testing.assert_allclose(DQ.dq_transform_point(b, p), rot.apply(p) + t, atol=1e-12)
    n = rng.normal(size=(200, 3))
    np.testing.assert_allclose(DQ.dq_rotate_vector(b, n), rot.apply(n), atol=1e-12)


def test_single_node_weight_one_and_sign_flip_invariance():
    rng = np.random.default_rng(5)
    rot, q, t = _rand_rt(rng, 4)
    node_dq = DQ.dq_from_rt(q, t)
    knn = np.array([[2, 0, 1, 3]])
    p = rng.normal(size=(1, 3))
    b = DQ.blend(node_dq, knn, np.array([[1.0, 0.0, 0.0, 0.0]]))
    np.testing.assert_allclose(DQ.dq_transform_point(b, p), rot[2].apply(p) + t[2], atol=1e-12)
    w = np.array([[0.7, 0.4, 0.2, 0.1]])
    base = DQ.dq_transform_point(DQ.blend(node_dq, knn, w), p)
    flipped = node_dq.copy()
    flipped[1] *= -1.0
    flipped[3] *= -1.0
    np.testing.assert_allclose(DQ.dq_transform_point(DQ.blend(flipped, knn, w), p), base, atol=1e-13)
    # the blend is scale invariant in the weights
    np.testing.assert_allclose(DQ.dq_transform_point(DQ.blend(node_dq, knn, 7.5 * w), p), base, atol=1e-13)


def test_inverse_after_forward_is_identity():
    rng = np.random.default_rng(6)
    _, q, t = _rand_rt(rng, 8)
    node_dq = DQ.dq_from_rt(q, t * 0.1)
    knn = rng.integers(0, 8, (100, 4))
    w = rng.uniform(0.05, 1.0, (100, 4))
    p = rng.normal(size=(100, 3))
    n = rng.normal(size=(100, 3))
    b = DQ.blend(node_dq, knn, w)
    np.testing.assert_allclose(DQ.dq_inverse_transform_point(b, DQ.dq_transform_point(b, p)), p, atol=1e-12)
    np.testing.assert_allclose(DQ.dq_inverse_rotate_vector(b, DQ.dq_rotate_vector(b, n)), n, atol=1e-12)


def test_normalize_gives_rigid_motion():
    rng = np.random.default_rng(7)
    d = rng.normal(size=(20, 8))
    u = DQ.dq_normalize(d)
    np.testing.assert_allclose(np.linalg.norm(u[:, :4], axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(np.sum(u[:, :4] * u[:, 4:], axis=1), 0.0, atol=1e-15)


def test_increment_is_rotation_then_translation():
    rng = np.random.default_rng(8)
    xi = rng.normal(size=(10, 6)) * 0.2
    p = rng.normal(size=(10, 3))
    want = Rotation.from_rotvec(xi[:, :3]).apply(p) + xi[:, 3:]
    np.testing.assert_allclose(DQ.dq_transform_point(DQ.increment_dq(xi), p), want, atol=1e-13)
