"""Shared set-up for the GPU parity tests: one library stream and one oracle
stream built from the same seeded synthetic scene."""
import numpy as np

import oracle
import paper_1904_13073_gb300 as sw
from oracle import dq as ODQ

F32 = np.float32


def ensure_built():
    from paper_1904_13073_gb300 import build as B
    B.build()


class Pair:
    """A library stream and an oracle stream over one scene."""

    def __init__(self, scene, precision=None, **params):
        self.scene = scene
        c = scene.cam
        self.cam = c
        self.params = params
        v4, n4, t2, node4 = sw.model_arrays(scene)
        lib_params = dict(params)
        if precision is not None:
            lib_params["precision"] = precision
        self.h = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4), **lib_params))
        sw.sw_set_model(self.h, v4, n4, t2, node4)
        op = oracle.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy,
                           **{k: v for k, v in params.items()})
        self.o = oracle.OracleStream(op)
        self.o.set_model(scene.surfel_v, scene.surfel_n, scene.surfel_r, scene.surfel_c, scene.surfel_t,
                         scene.node_p, scene.node_sigma)

    def close(self):
        if self.h:
            sw.sw_destroy_stream(self.h)
            self.h = None

    def upload(self, t):
        d = self.scene.frame(t)
        sw.sw_upload_depth(self.h, d, t)
        self.o.upload_depth(d, t)

    def set_maps_from_oracle(self):
        """Give both sides the same FP32 depth-surfel maps (the oracle's,
        rounded to FP32); the oracle then works on exactly those values."""
        m = self.o.maps
        V4 = np.zeros(m["V"].shape[:2] + (4,), F32)
        N4 = np.zeros_like(V4)
        V4[..., :3] = m["V"]
        V4[..., 3] = np.where(m["valid"], m["conf"], 0.0)
        N4[..., :3] = m["N"]
        N4[..., 3] = m["radius"]
        sw.sw_debug_set_maps(self.h, V4, N4)
        m["V"] = V4[..., :3].astype(np.float64)
        m["N"] = N4[..., :3].astype(np.float64)
        m["conf"] = V4[..., 3].astype(np.float64)
        m["radius"] = N4[..., 3].astype(np.float64)
        self.o.V32 = V4[..., :3].copy()
        self.o.N32 = N4[..., :3].copy()


def rigid_dq8_from(axis, angle, trans):
    """Dual quaternions [n, 8] float32 of x -> R x + t, R = rotation by
    ``angle`` about ``axis``; written out independently of the oracle."""
    h = 0.5 * angle
    q = np.concatenate([np.cos(h)[:, None], np.sin(h)[:, None] * axis], axis=1)
    w, x, y, z = q.T
    tx, ty, tz = trans.T
    # ½ (0, t) ⊗ q
    dw = -0.5 * (tx * x + ty * y + tz * z)
    dx = 0.5 * (tx * w + ty * z - tz * y)
    dy = 0.5 * (-tx * z + ty * w + tz * x)
    dz = 0.5 * (tx * y - ty * x + tz * w)
    return np.stack([w, x, y, z, dw, dx, dy, dz], axis=1).astype(F32)


def oracle_dq_from(axis, angle, trans):
    return ODQ.dq_from_rt(ODQ.rodrigues_quat(axis * angle[:, None]), trans)


def rotation_angle_between(dq_a, dq_b):
    """Angle (rad) of R_a R_bᵀ for unit real parts."""
    qa = dq_a[:, :4] / np.linalg.norm(dq_a[:, :4], axis=1, keepdims=True)
    qb = dq_b[:, :4] / np.linalg.norm(dq_b[:, :4], axis=1, keepdims=True)
    rel = ODQ.qmul(ODQ.qconj(qb), qa)
    return 2.0 * np.arctan2(np.linalg.norm(rel[:, 1:], axis=1), np.abs(rel[:, 0]))
