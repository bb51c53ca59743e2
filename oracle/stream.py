"""The five per-stream calls over host memory, in FP64 (the CUDA library's
``sw_create_stream`` / ``sw_set_model`` / ``sw_upload_depth`` /
``sw_solve_frame`` / ``sw_fuse_frame`` / ``sw_read_nodes`` counterparts).

Per frame (Sec. 4): the warp field starts from the previous frame's, is
re-estimated against the new depth image (Sec. 7), then the depth surfels are
fused into the live surfels (Sec. 6.1) and the fused surfels are warped back to
the reference frame (Eq. 3).
"""
from dataclasses import dataclass

import numpy as np

from . import dq as DQ
from . import depth as DEPTH
from . import skinning as SKIN
from . import solver as SOLVER
from . import fusion as FUSION
from . import rigid as RIGID
from . import append as APPEND
from . import visibility as VIS


@dataclass
class Params:
    """Table 1 values, plus the readings for what the paper leaves open."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    lam: float = 5.0               # λ, Table 1
    fuse_dist: float = 1e-3        # δ_distance, Table 1
    fuse_normal: float = 0.85      # δ_normal, Table 1
    corr_dist: float = 0.05        # association distance (reading)
    corr_normal: float = 0.7       # association normal dot (reading)
    stable_conf: float = 10.0      # δ_stable, Table 1
    recent_frames: int = 2         # δ_recent, Table 1
    visibility: bool = False       # splat visibility before the solve (see visibility.py)

    @property
    def cam(self):
        return (self.fx, self.fy, self.cx, self.cy, self.width, self.height)


class OracleStream:
    def __init__(self, params: Params):
        self.p = params
        self.maps = None
        self.t_now = 0

    # -- model ---------------------------------------------------------------
    def set_model(self, v, n, r, c, t, node_p, node_sigma):
        """Reference surfels and nodes; node transforms start at identity;
        skinning (4-NN) and the 8-NN node graph are computed (Sec. 6.5)."""
        self.v_ref = np.asarray(v, dtype=np.float64).copy()
        self.n_ref = np.asarray(n, dtype=np.float64).copy()
        self.radius = np.asarray(r, dtype=np.float64).copy()
        self.conf = np.asarray(c, dtype=np.float64).copy()
        t = np.asarray(t)
        self.t_init = t[:, 0].astype(np.int64).copy()
        self.t_obs = t[:, 1].astype(np.int64).copy()
        self.node_p = np.asarray(node_p, dtype=np.float64).copy()
        self.node_sigma = np.asarray(node_sigma, dtype=np.float64).copy()
        self.knn = SKIN.knn_fp32(np.asarray(v, dtype=np.float32),
                                 np.asarray(node_p, dtype=np.float32), SKIN.K_SKIN)
        self.w = SKIN.skin_weights(v, node_p, node_sigma, self.knn)
        self.graph = SKIN.node_graph(np.asarray(node_p, dtype=np.float32))
        self.node_dq = DQ.dq_identity(len(node_p))
        self.pattern = SOLVER.BlockMatrix.pattern(len(node_p), self.knn, self.graph).keys

    # -- per frame -----------------------------------------------------------
    def upload_depth(self, depth, frame_id):
        p = self.p
        self.depth = np.asarray(depth, dtype=np.float32)
        self.maps = DEPTH.depth_maps(self.depth, p.fx, p.fy, p.cx, p.cy)
        self.V32 = self.maps["V"].astype(np.float32)
        self.N32 = self.maps["N"].astype(np.float32)
        self.t_now = frame_id

    def predict_visibility(self):
        """Sec. 7: the selected live surfels under the current warp rendered as
        opaque splats at the depth resolution; the surfels that keep a pixel."""
        p = self.p
        _, v_live, n_live = SOLVER.warp_surfels(self.v_ref, self.n_ref, self.knn, self.w, self.node_dq)
        sel = SOLVER.select_surfels(self.conf, self.t_obs, self.t_now, p.stable_conf, p.recent_frames)
        self.vis_map = VIS.visibility_map(v_live, n_live, self.radius, sel, p.cam)
        self.visible = VIS.visible_mask(self.vis_map, len(self.v_ref))
        return self.visible

    def associate(self, v_live, n_live, visibility=True):
        p = self.p
        sel = SOLVER.select_surfels(self.conf, self.t_obs, self.t_now,
                                    p.stable_conf, p.recent_frames)
        if p.visibility and visibility:
            sel = sel & self.visible
        ok, pix = SOLVER.associate(v_live, n_live, sel, self.V32, self.N32,
                                   self.maps["valid"], p.cam, p.corr_dist, p.corr_normal)
        tv = np.zeros_like(v_live)
        tn = np.zeros_like(v_live)
        tv[ok] = self.maps["V"].reshape(-1, 3)[pix[ok]]
        tn[ok] = self.maps["N"].reshape(-1, 3)[pix[ok]]
        return ok, tv, tn

    def solve_frame(self, gn_iters, pcg_iters, keep_masks=False, visible=None, linear_solver=None):
        """Sec. 7: the frame's Gauss-Newton solve.  With visibility on, the
        visible surfels are predicted first, unless ``visible`` gives them
        (a mask over the surfels, for comparisons on identical inputs).
        ``linear_solver`` replaces the PCG (see solver.gauss_newton)."""
        if self.p.visibility:
            if visible is None:
                self.predict_visibility()
            else:
                self.visible = np.asarray(visible, dtype=bool).copy()
        self.node_dq, stats = SOLVER.gauss_newton(
            self.v_ref, self.n_ref, self.knn, self.w, self.node_p, self.node_dq,
            self.graph, self.pattern, self.p.lam, gn_iters, pcg_iters,
            associate_fn=self.associate, keep_masks=keep_masks, linear_solver=linear_solver)
        return stats

    def rigid_align(self, iters):
        """Rigid pre-alignment of the current frame (see rigid.py); returns
        [(correspondences, Σ r²)] per iteration."""
        self.node_dq, T, stats = RIGID.rigid_align(self.v_ref, self.n_ref, self.knn, self.w, self.node_dq,
                                                  lambda y, ny: self.associate(y, ny, visibility=False), iters)
        self.last_rigid = T
        return stats

    def fuse_frame(self):
        p = self.p
        b, v_live, n_live = SOLVER.warp_surfels(self.v_ref, self.n_ref, self.knn,
                                                self.w, self.node_dq)
        imap = FUSION.index_map(v_live, p.cam)
        target = FUSION.select_fusion_targets(imap, v_live, n_live, self.conf,
                                              self.V32, self.N32, self.maps["valid"],
                                              p.fuse_dist, p.fuse_normal)
        v_live, n_live, self.radius, self.conf, self.t_obs, fused = FUSION.fuse(
            v_live, n_live, self.radius, self.conf, self.t_obs, self.maps, target, self.t_now)
        vr, nr = FUSION.inverse_warp(b[fused], v_live[fused], n_live[fused])
        self.v_ref[fused] = vr
        self.n_ref[fused] = nr
        self.last_target = target
        self.last_index_map = imap
        return int(fused.sum())

    def append_frame(self, max_surfels, eps=APPEND.EPS, delta_nn=APPEND.DELTA_NN, h=APPEND.FD_STEP,
                     t_low=APPEND.T_LOW_CONFID, extend_nodes=False, max_nodes=0):
        """Appending and removal after fuse_frame (see append.py).  Returns
        (candidates, appended, removed); the per-candidate record is kept in
        ``last_append``."""
        p = self.p
        pix = APPEND.empty_window_pixels(self.last_index_map, self.maps["valid"])
        res = APPEND.append_candidates(pix, self.maps, self.node_dq, self.node_p, self.node_sigma,
                                       eps, delta_nn, h)
        stay = ~APPEND.unstable(self.conf, self.t_init, self.t_now, p.stable_conf, t_low)
        acc = np.nonzero(res["accept"])[0]
        acc = acc[:max(0, max_surfels - int(stay.sum()))]
        res["pix"] = pix
        res["appended"] = acc
        self.last_append = res
        new_pix = pix[acc]
        new_v = res["v_ref"][acc]
        new_n = res["n_ref"][acc]
        new_knn = SKIN.knn_fp32(new_v.astype(np.float32), self.node_p.astype(np.float32), SKIN.K_SKIN)
        new_w = SKIN.skin_weights(new_v, self.node_p, self.node_sigma, new_knn)
        t_new = np.full(len(acc), self.t_now, dtype=np.int64)
        self.v_ref = np.concatenate([self.v_ref[stay], new_v])
        self.n_ref = np.concatenate([self.n_ref[stay], new_n])
        self.radius = np.concatenate([self.radius[stay], self.maps["radius"].reshape(-1)[new_pix]])
        self.conf = np.concatenate([self.conf[stay], self.maps["conf"].reshape(-1)[new_pix]])
        self.t_init = np.concatenate([self.t_init[stay], t_new])
        self.t_obs = np.concatenate([self.t_obs[stay], t_new])
        self.knn = np.concatenate([self.knn[stay], new_knn])
        self.w = np.concatenate([self.w[stay], new_w])
        self.new_nodes = 0
        if extend_nodes and len(acc):
            self.extend_nodes(new_v, max_nodes)
        self.pattern = SOLVER.BlockMatrix.pattern(len(self.node_p), self.knn, self.graph).keys
        return len(pix), len(acc), int((~stay).sum())

    def extend_nodes(self, v_app, max_nodes):
        """Node-graph extension over the appended reference surfels (see
        append.py): new nodes, their transforms, the graph and every surfel's
        skinning over all nodes."""
        unc = ~APPEND.covered(v_app, self.node_p, self.node_sigma)
        new_p, new_s = APPEND.subsample_nodes(np.asarray(v_app)[unc], self.node_p, self.node_sigma,
                                              min(APPEND.MAX_NEW_NODES, max(0, max_nodes - len(self.node_p))))
        self.new_nodes = len(new_p)
        if not len(new_p):
            return
        new_dq = APPEND.new_node_transforms(new_p, self.node_p, self.node_sigma, self.node_dq)
        self.node_p = np.concatenate([self.node_p, new_p.astype(np.float64)])
        self.node_sigma = np.concatenate([self.node_sigma, new_s.astype(np.float64)])
        self.node_dq = np.concatenate([self.node_dq, new_dq])
        self.graph = SKIN.node_graph(self.node_p.astype(np.float32))
        self.knn_pre_extension = self.knn.copy()
        self.knn, self.w, self.reskinned = APPEND.merge_skinning(self.v_ref, self.knn, self.w, self.node_p,
                                                                 self.node_sigma, len(self.node_p) - len(new_p))

    def load_state(self, v4, n4, t2, knn, w, node_dq):
        """Replace the surfel model, its skinning and the node transforms by
        given values (v4: x y z radius, n4: nx ny nz confidence, t2: t_init,
        t_observed; knn / w in distance order), keeping the nodes and the
        graph: a frame can then be compared on identical inputs."""
        v4, n4 = np.asarray(v4, dtype=np.float64), np.asarray(n4, dtype=np.float64)
        self.v_ref, self.radius = v4[:, :3].copy(), v4[:, 3].copy()
        self.n_ref, self.conf = n4[:, :3].copy(), n4[:, 3].copy()
        t2 = np.asarray(t2)
        self.t_init = t2[:, 0].astype(np.int64).copy()
        self.t_obs = t2[:, 1].astype(np.int64).copy()
        self.knn = np.asarray(knn).astype(np.int64).copy()
        self.w = np.asarray(w, dtype=np.float64).copy()
        self.node_dq = np.asarray(node_dq, dtype=np.float64).copy()
        self.pattern = SOLVER.BlockMatrix.pattern(len(self.node_p), self.knn, self.graph).keys

    # -- read-back -----------------------------------------------------------
    def read_nodes(self):
        """(node positions (Nn,3), node dual quaternions (Nn,8))."""
        return self.node_p.copy(), self.node_dq.copy()

    def warped_nodes(self):
        """T_j p_j: where every node's own transform takes it."""
        return SOLVER.node_transform(self.node_dq, self.node_p)
