"""Shared set-up for the GPU parity tests: one library stream and one oracle
stream built from the same seeded synthetic scene."""
import numpy as np

import oracle
import paper_1904_13073_gb300 as sw
from oracle import dq as ODQ
from oracle import solver as OS

F32 = np.float32


def ensure_built():
    from paper_1904_13073_gb300 import build as B
    B.build()


def oracle_for(scene, **params):
    """An oracle stream with the scene's model (params: oracle.Params fields)."""
    c = scene.cam
    o = oracle.OracleStream(oracle.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy, **params))
    o.set_model(scene.surfel_v, scene.surfel_n, scene.surfel_r, scene.surfel_c, scene.surfel_t,
                scene.node_p, scene.node_sigma)
    return o


def set_maps_from_oracle(h, o):
    """Give both sides the same FP32 depth-surfel maps (the oracle's,
    rounded to FP32); the oracle then works on exactly those values."""
    m = o.maps
    V4 = np.zeros(m["V"].shape[:2] + (4,), F32)
    N4 = np.zeros_like(V4)
    V4[..., :3] = m["V"]
    V4[..., 3] = np.where(m["valid"], m["conf"], 0.0)
    N4[..., :3] = m["N"]
    N4[..., 3] = m["radius"]
    sw.sw_debug_set_maps(h, V4, N4)
    m["V"] = V4[..., :3].astype(np.float64)
    m["N"] = N4[..., :3].astype(np.float64)
    m["conf"] = V4[..., 3].astype(np.float64)
    m["radius"] = N4[..., 3].astype(np.float64)
    o.V32 = V4[..., :3].copy()
    o.N32 = N4[..., :3].copy()


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
        self.o = oracle_for(scene, **params)

    def close(self):
        if self.h:
            sw.sw_destroy_stream(self.h)
            self.h = None

    def upload(self, t):
        d = self.scene.frame(t)
        sw.sw_upload_depth(self.h, d, t)
        self.o.upload_depth(d, t)

    def set_maps_from_oracle(self):
        set_maps_from_oracle(self.h, self.o)


def load_gpu_state_into_oracle(p):
    """Give the oracle the library stream's own model before a frame: its
    fused surfels (positions, normals, radii, confidences, time stamps), its
    skinning and its node transforms (FP32 values, exactly).  In the FP64
    mode the library's FP64 transforms are set to those FP32 values too, so
    both sides start the frame from identical inputs."""
    v, n, tt = sw.sw_read_surfels(p.h)
    knn, w = sw.sw_read_skinning(p.h)
    _, dq = sw.sw_read_nodes(p.h)
    sw.sw_set_node_dq(p.h, dq)
    p.o.load_state(v, n, tt, knn, w, dq.astype(np.float64))


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


def association_flips(o, v_live, n_live, pix_gpu, visible=None):
    """Surfels whose association differs between the library (pix_gpu:
    pixel or -1) and the oracle's FP32 decision on its FP64 warp, each with
    whether the oracle's FP64 quantities lie at a decision boundary (a
    pixel edge within 1e-4 px, the distance or normal test within 1e-5
    relative): there the two valid roundings of one warp may decide either
    way.  Returns (flipped indices, boolean array: that flip is at a
    boundary, the oracle's pixel per surfel)."""
    sel = OS.select_surfels(o.conf, o.t_obs, o.t_now, o.p.stable_conf, o.p.recent_frames)
    if visible is not None:
        sel = sel & visible
    ok, pix_o = OS.associate(v_live, n_live, sel, o.V32, o.N32, o.maps["valid"], o.p.cam,
                             o.p.corr_dist, o.p.corr_normal)
    flipped = np.nonzero(np.where(ok, pix_o, -1) != pix_gpu)[0]
    fx, fy, cx, cy, width, height = o.p.cam
    v = np.asarray(v_live, dtype=np.float64)[flipped]
    n = np.asarray(n_live, dtype=np.float64)[flipped]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * v[:, 0] / v[:, 2] + cx + 0.5
        w = fy * v[:, 1] / v[:, 2] + cy + 0.5
    edge = (np.abs(u - np.round(u)) < 1e-4) | (np.abs(w - np.round(w)) < 1e-4)
    V = o.maps["V"].reshape(-1, 3)
    N = o.maps["N"].reshape(-1, 3)
    near = np.zeros(len(flipped), bool)
    for k, i in enumerate(flipped):
        for px in (pix_o[i], pix_gpu[i]):
            if px < 0:
                continue
            d2 = float(np.sum((v[k] - V[px]) ** 2))
            dt = float(np.dot(n[k], N[px]))
            if abs(d2 - o.p.corr_dist ** 2) < 1e-5 * o.p.corr_dist ** 2 or abs(dt - o.p.corr_normal) < 1e-5:
                near[k] = True
    return flipped, edge | near, pix_o


def handing_over(o, recorded):
    """Make oracle stream o's association take the library's decisions where
    the two differ at a rounding boundary: its k-th association (k-th
    Gauss-Newton iteration of the solves that follow) compares its own
    decisions with recorded[k] (the library's, sw_read_correspondence_iter);
    every difference must lie at a decision boundary (association_flips),
    and there the library's decision is taken.  Returns the list that
    receives each iteration's number of such surfels; undo with
    `del o.associate`."""
    flips = []

    def associate(v_live, n_live, visibility=True):
        k = len(flips)
        vis = o.visible if (o.p.visibility and visibility) else None
        flipped, at_boundary, pix_o = association_flips(o, v_live, n_live, recorded[k], visible=vis)
        # surfels without skinning take no term on either side (the library
        # does not associate them; the oracle drops them after associating)
        real = ~OS.unskinned(OS.DQ.blend(o.node_dq, o.knn, o.w))[flipped]
        assert np.all(at_boundary[real]), (k, flipped[real & ~at_boundary])
        sel = OS.select_surfels(o.conf, o.t_obs, o.t_now, o.p.stable_conf, o.p.recent_frames)
        if vis is not None:
            sel = sel & vis
        ok, pix = OS.associate(v_live, n_live, sel, o.V32, o.N32, o.maps["valid"], o.p.cam,
                               o.p.corr_dist, o.p.corr_normal)
        dec = np.where(ok, pix, -1)
        dec[flipped] = recorded[k][flipped]
        flips.append(int(real.sum()))
        mask = dec >= 0
        tv = np.zeros_like(v_live)
        tn = np.zeros_like(v_live)
        tv[mask] = o.maps["V"].reshape(-1, 3)[dec[mask]]
        tn[mask] = o.maps["N"].reshape(-1, 3)[dec[mask]]
        return mask, tv, tn

    o.associate = associate
    return flips


def set_maps_like(dst, src):
    """Give oracle stream dst the FP32 depth-surfel maps of src (same frame)."""
    dst.t_now = src.t_now
    dst.depth = src.depth
    dst.maps = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in src.maps.items()}
    dst.V32 = src.V32.copy()
    dst.N32 = src.N32.copy()


def pcg_fp32_spmv(A, b, Minv, iters):
    """The oracle's PCG (standard recurrences, FP64 vectors and inner
    products) with one change: every product A p is evaluated in FP32 (A and
    p rounded to FP32, FP32 products and sums).  The distance of its result
    from the FP64 PCG's measures how much the configured precision's FP32
    SpMV alone moves a solve."""
    import scipy.sparse as sp
    n = A.n
    As32 = A.to_scipy().astype(np.float32)

    def precond(v):
        return np.einsum('nij,nj->ni', Minv, v.reshape(n, 6)).reshape(-1)

    x = np.zeros(6 * n)
    r = b.astype(np.float64).copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    done = 0
    for _ in range(iters):
        if rz == 0.0:
            break
        q = (As32 @ p.astype(np.float32)).astype(np.float64)
        pq = float(p @ q)
        if not pq > 0.0:
            raise OS.SolverBreakdown("pᵀAp <= 0 in PCG")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = precond(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        done += 1
    return x, rz, done


def solve_with_fp32_spmv(o, gn, pcg, visible=None):
    """The oracle stream's Gauss-Newton solve with pcg_fp32_spmv as its linear solve."""
    return o.solve_frame(gn, pcg, linear_solver=pcg_fp32_spmv, visible=visible)


def solve_with_fp32_system(o, gn, pcg, visible=None):
    """The oracle stream's Gauss-Newton solve with its linear system formed
    as the configured precision forms it: the data and regulariser terms
    evaluated in FP32 arithmetic from FP32 inputs, JᵀJ and Jᵀe summed in FP32
    (term order), the block inverses in FP64 of the FP32 blocks, and the PCG
    with an FP32 SpMV (pcg_fp32_spmv).  Warp, association (the oracle's, with
    `visible` when given) and update are the oracle's.  Its distance from the
    oracle's own solve measures the error that FP32 terms, sums and products
    alone cause on a given system, the yardstick for the FP32 modes."""
    f = np.float32
    if o.p.visibility:
        if visible is None:
            o.predict_visibility()
        else:
            o.visible = np.asarray(visible, dtype=bool).copy()
    n = len(o.node_p)
    for _ in range(gn):
        _, v_live, n_live = OS.warp_surfels(o.v_ref, o.n_ref, o.knn, o.w, o.node_dq)
        mask, tv, tn = o.associate(v_live, n_live)
        mask = mask & ~OS.unskinned(OS.DQ.blend(o.node_dq, o.knn, o.w))
        idx = np.nonzero(mask)[0]
        r, J = OS.data_terms(o.v_ref[idx].astype(f), o.knn[idx], o.w[idx].astype(f), o.node_dq.astype(f),
                             tv[idx].astype(f), tn[idx].astype(f))
        j, i, rr, Jj, Ji = OS.reg_terms(o.node_p.astype(f), o.node_dq.astype(f), o.graph, f(o.p.lam))
        A = OS.BlockMatrix(n, o.pattern, np.zeros((len(o.pattern), 6, 6), f))
        g = np.zeros((n, 6), f)
        knn = o.knn[idx]
        for a_ in range(knn.shape[1]):
            np.add.at(g, knn[:, a_], (J[:, a_] * r[:, None]).astype(f))
            for b_ in range(knn.shape[1]):
                A.add(knn[:, a_], knn[:, b_], (J[:, a_, :, None] * J[:, b_, None, :]).astype(f))
        for (ra, Ja), (rb, Jb) in (((j, Jj), (j, Jj)), ((j, Jj), (i, Ji)), ((i, Ji), (j, Jj)), ((i, Ji), (i, Ji))):
            A.add(ra, rb, np.einsum('eri,erj->eij', Ja, Jb).astype(f))
        np.add.at(g, j, np.einsum('eri,er->ei', Jj, rr).astype(f))
        np.add.at(g, i, np.einsum('eri,er->ei', Ji, rr).astype(f))
        A64 = OS.BlockMatrix(n, o.pattern, A.vals.astype(np.float64))
        Minv = OS.block_jacobi_inverse(A64)
        x, _, _ = pcg_fp32_spmv(A64, -g.astype(np.float64).reshape(-1), Minv, pcg)
        o.node_dq = OS.apply_increment(o.node_dq, x)
