"""Surfel appending after fusion (Sec. 6.2 live skinning with the Eq. 7
consistency test, Sec. 6.3 compressive warp field, Eq. 8; Sec. 6.4 appending
and removal; Sec. 6.6 GPU selection that compacts the surfel array).

TEST INFRASTRUCTURE ONLY: see the package docstring.

Steps, in the paper's order, for one frame after fusion (all readings of
what the paper leaves open are marked):

1. Candidates (Sec. 6.2: a depth surfel with no corresponding live surfel).
   Reading: a usable depth pixel whose own 16 index-map sub-pixels (the
   fusion window) hold no live surfel at all.  A pixel whose window holds a
   surfel that failed the fusion tests is an inconsistent observation of
   geometry that already exists, not new geometry, and is not appended.
2. Live skinning (Sec. 6.2): the warped nodes p̂_j = T_j p_j; the 4 nearest
   of them to the depth vertex x = V(u), by FP32 squared distance with ties
   to the lower node id (the rule of the reference-frame skinning); slot 0
   is node_0.  p̂_j is evaluated in FP64 and rounded to FP32, the precision
   the decision is taken in.
3. Eq. 7: node i (slot ≥ 1) stays when 1 − ε < |p̂_i − p̂_0| / |p_i − p_0| <
   1 + ε.  Reading: the test is taken on squares in FP32,
   (1−ε)² d_ref² < d_live² < (1+ε)² d_ref², with (1±ε)² rounded to FP32 once;
   coincident reference nodes (d_ref² = 0) fail it.  Node 0 always stays.
4. Weights at the live frame (Eq. 1 with the warped nodes): w_i =
   exp(−‖x − p̂_i‖² / (2 σ_i²)) for the nodes that stay, 0 for the others, in
   FP64.
5. δ_nn test (Sec. 6.4): the candidate is discarded when Σ w_i < δ_nn.
   δ_nn is not in Table 1; reading: 0.3 (a point 2σ from all four nodes sums
   to 4 e⁻² ≈ 0.54 and passes, one 3σ away sums to 0.04 and fails).
6. Inverse warp (Eq. 3) with that skinning: b = Σ w_i s_i q̂_i (signs against
   node 0, Eq. 1), v_ref = b⁻¹ x, n_ref = rotation(b)⁻¹ N(u).
7. Eq. 8: the 3x3 strain ∂x_ref/∂x_live by central finite differences with
   step h (reading: 1 mm), the node set and signs of step 3 held fixed and
   the weights re-evaluated at x ± h e_a.  Reading of |·| in 3D: the largest
   singular value; the candidate is discarded when it exceeds 1 + ε.
8. Appended surfel: v_ref, n_ref of step 6; radius and confidence of the
   depth surfel; t_init = t_observed = t_now; its skinning is recomputed in
   the reference frame at v_ref by the initialisation rule (4-NN over the
   reference nodes, Eq. 1 weights), the frame every later warp blends in.
9. Removal (Sec. 6.4): an existing surfel is removed when c < δ_stable and
   t_now − t_init ≥ t_low_confid (Table 1: 10 and 30).  Reading: the second
   criterion (similar to its neighbours on the index map) is defined only in
   a cited work and is not applied.
10. Compaction (Sec. 6.6): the surviving surfels in their order, then the
    appended ones in pixel order (row-major); appended surfels past the
    capacity are dropped from the end.
"""
import numpy as np

from . import dq as DQ
from . import skinning as SKIN
from .fusion import SUPER

_F32 = np.float32

EPS = 0.2            # ε, Table 1
DELTA_NN = 0.3       # δ_nn (reading)
FD_STEP = 1e-3       # finite-difference step of Eq. 8, metres (reading)
T_LOW_CONFID = 30    # t_low_confid, Table 1
MAX_NEW_NODES = 2048  # node-graph extension: most new nodes per call (reading)


def empty_window_pixels(imap, usable):
    """Step 1: flat indices of usable pixels whose 4x4 window holds no surfel."""
    hh, ww = usable.shape
    win = imap.reshape(hh, SUPER, ww, SUPER).transpose(0, 2, 1, 3).reshape(hh * ww, SUPER * SUPER)
    empty = np.all(win < 0, axis=1)
    return np.nonzero(empty & usable.reshape(-1))[0]


def warped_nodes_fp32(node_dq, node_p):
    """Step 2: p̂_j = T_j p_j in FP64, rounded to FP32."""
    p = np.asarray(node_p, dtype=np.float64)
    return DQ.dq_transform_point(np.asarray(node_dq, dtype=np.float64), p).astype(_F32)


def d2_fp32(a, b):
    """FP32 squared distance ((dx·dx) + (dy·dy)) + (dz·dz), row by row."""
    a = np.asarray(a, dtype=_F32)
    b = np.asarray(b, dtype=_F32)
    d = a - b
    return ((d[..., 0] * d[..., 0]) + (d[..., 1] * d[..., 1])) + (d[..., 2] * d[..., 2])


def consistent(knn, p_live32, p_ref32, eps=EPS):
    """Step 3, Eq. 7 on squares in FP32: (n, 4) mask of the nodes that stay."""
    lo = _F32((1.0 - eps) ** 2)
    hi = _F32((1.0 + eps) ** 2)
    keep = np.ones(knn.shape, dtype=bool)
    for i in range(1, knn.shape[1]):
        dl = d2_fp32(p_live32[knn[:, i]], p_live32[knn[:, 0]])
        dr = d2_fp32(p_ref32[knn[:, i]], p_ref32[knn[:, 0]])
        keep[:, i] = (dl > lo * dr) & (dl < hi * dr)
    return keep


def live_weights(x, p_live32, sigma, knn, keep):
    """Step 4: Eq. 1 weights at the live frame, zero for removed nodes (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    p = p_live32.astype(np.float64)[knn]
    s = np.asarray(sigma, dtype=np.float64)[knn]
    d2 = np.sum((x[:, None, :] - p) ** 2, axis=-1)
    return np.where(keep, np.exp(-d2 / (2.0 * s * s)), 0.0)


def inverse_warp_live(x, n, node_dq, knn, w):
    """Step 6: (v_ref, n_ref) of live points with their live skinning (Eq. 1, 3)."""
    b = DQ.blend(node_dq, knn, w)
    return DQ.dq_inverse_transform_point(b, x), DQ.dq_inverse_rotate_vector(b, n)


def strain(x, node_dq, knn, keep, p_live32, sigma, h=FD_STEP):
    """Step 7: (n, 3, 3) central differences of x_ref with respect to x_live;
    column a is (x_ref(x + h e_a) − x_ref(x − h e_a)) / 2h."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty(x.shape + (3,))
    zero = np.zeros_like(x)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        xp, xm = x + e, x - e
        rp, _ = inverse_warp_live(xp, zero, node_dq, knn, live_weights(xp, p_live32, sigma, knn, keep))
        rm, _ = inverse_warp_live(xm, zero, node_dq, knn, live_weights(xm, p_live32, sigma, knn, keep))
        out[:, :, a] = (rp - rm) / (2.0 * h)
    return out


def strain_norm(J):
    """Largest singular value of each 3x3 strain (the 3D reading of |dx_ref/dx_live|)."""
    return np.linalg.norm(J, ord=2, axis=(1, 2)) if len(J) else np.zeros(0)


def unstable(conf, t_init, t_now, stable_conf, t_low=T_LOW_CONFID):
    """Step 9: surfels still below δ_stable t_low_confid frames after t_init."""
    return (np.asarray(conf) < stable_conf) & (t_now - np.asarray(t_init) >= t_low)


def append_candidates(pix, maps, node_dq, node_p, node_sigma, eps=EPS, delta_nn=DELTA_NN, h=FD_STEP):
    """Steps 2-7 for the candidate pixels `pix`.  Returns a dict with, per
    candidate: knn (live, distance order), keep (Eq. 7), w, wsum, v_ref, n_ref,
    strain norm, and `accept` (δ_nn and Eq. 8 both passed)."""
    Vf = maps["V"].reshape(-1, 3)
    Nf = maps["N"].reshape(-1, 3)
    x32 = Vf[pix].astype(_F32)
    x = x32.astype(np.float64)
    p_live32 = warped_nodes_fp32(node_dq, node_p)
    p_ref32 = np.asarray(node_p, dtype=_F32)
    knn = SKIN.knn_fp32(x32, p_live32, SKIN.K_SKIN)
    keep = consistent(knn, p_live32, p_ref32, eps)
    w = live_weights(x, p_live32, node_sigma, knn, keep)
    wsum = w.sum(axis=1)
    v_ref, n_ref = inverse_warp_live(x, Nf[pix].astype(_F32).astype(np.float64), node_dq, knn, w)
    J = strain(x, node_dq, knn, keep, p_live32, node_sigma, h)
    snorm = strain_norm(J)
    accept = (wsum >= delta_nn) & ~(snorm > 1.0 + eps)
    return dict(knn=knn, keep=keep, w=w, wsum=wsum, v_ref=v_ref, n_ref=n_ref, strain=J,
                strain_norm=snorm, accept=accept)


# ---------------------------------------------------------------------------
# node-graph extension (Sec. 6.4, last paragraph; the paper defers the details
# to DynamicFusion's Sec. 3.4, which is summarised there: the coverage of the
# appended reference geometry by the node graph is computed, the uncovered
# vertices are sub-sampled into new nodes, and the edges are recomputed; the
# surfels' nearest-neighbour sets are then compared with the new nodes)
#
# Readings:
# * an appended surfel at v is covered when some node j has ‖v − p_j‖² < σ_j²
#   (inside the node's radius parameter), decided in FP32 with the k-NN's
#   fixed operation order;
# * sub-sampling: the uncovered surfels are visited in their (caller) order;
#   one becomes a node when it is at least σ away from every node, old or
#   accepted before it (‖v − p‖² ≥ σ², FP32), σ being the radius parameter of
#   its nearest old node (the local sampling distance); the new node takes
#   that σ;
# * a new node's transform starts as the current warp at its position: the
#   normalised blend (Eq. 1) of its 4 nearest old nodes with their weights;
# * the graph is recomputed over all nodes (the 8-NN rule);
# * every surfel's set is compared with the new nodes: the 4 smallest
#   (FP32 distance, id) among its old set and the new nodes, all measured at
#   its current reference position; a surfel whose set changed gets that set
#   in distance order and its Eq. 1 weights at its current position, the
#   others keep their set and weights (fusion may have moved them a little
#   since they were skinned);
# * new nodes past the stream's node capacity, or past 2048 in one call, are
#   not added.
# ---------------------------------------------------------------------------

def covered(v_app, node_p, node_sigma):
    """Step 1: (n,) mask of appended surfels inside some node's radius."""
    v32 = np.asarray(v_app, dtype=_F32)
    p32 = np.asarray(node_p, dtype=_F32)
    s32 = np.asarray(node_sigma, dtype=_F32)
    out = np.zeros(len(v32), dtype=bool)
    for j in range(len(p32)):
        out |= d2_fp32(v32, p32[j][None, :]) < s32[j] * s32[j]
    return out


def subsample_nodes(v_unc, node_p, node_sigma, max_new):
    """Step 2: greedy sub-sampling of the uncovered surfels (in order);
    returns (positions (k, 3) float32, σ (k,) float32)."""
    v32 = np.asarray(v_unc, dtype=_F32)
    p32 = np.asarray(node_p, dtype=_F32)
    s32 = np.asarray(node_sigma, dtype=_F32)
    new_p, new_s = [], []
    for v in v32:
        if len(new_p) >= max_new:
            break
        d_old = d2_fp32(p32, v[None, :])
        j0 = int(np.lexsort((np.arange(len(p32)), d_old.view(np.uint32)))[0])   # nearest old node, ties to the lower id
        sig = s32[j0]
        s2 = sig * sig
        if np.any(d_old < s2):
            continue
        if new_p and np.any(d2_fp32(np.asarray(new_p, dtype=_F32), v[None, :]) < s2):
            continue
        new_p.append(v)
        new_s.append(sig)
    return np.asarray(new_p, dtype=_F32).reshape(-1, 3), np.asarray(new_s, dtype=_F32)


def new_node_transforms(new_p, node_p, node_sigma, node_dq):
    """Step 3: the current warp at each new node, as a unit dual quaternion."""
    if len(new_p) == 0:
        return np.zeros((0, 8))
    knn = SKIN.knn_fp32(np.asarray(new_p, dtype=_F32), np.asarray(node_p, dtype=_F32), SKIN.K_SKIN)
    w = SKIN.skin_weights(new_p, node_p, node_sigma, knn)
    return DQ.dq_normalize(DQ.blend(node_dq, knn, w))


def merge_skinning(v_ref, knn, w, node_p, node_sigma, first_new):
    """Step 5: each surfel's set compared with the nodes from `first_new` on."""
    v32 = np.asarray(v_ref, dtype=_F32)
    p32 = np.asarray(node_p, dtype=_F32)
    new_ids = np.arange(first_new, len(p32))
    cand = np.concatenate([knn, np.broadcast_to(new_ids, (len(knn), len(new_ids)))], axis=1)
    d2 = d2_fp32(v32[:, None, :], p32[cand])
    key = (d2.view(np.uint32).astype(np.uint64) << np.uint64(32)) | cand.astype(np.uint64)
    best = np.sort(key, axis=1)[:, :SKIN.K_SKIN]
    ids = (best & np.uint64(0xFFFFFFFF)).astype(np.int64)
    changed = np.any(np.sort(ids, axis=1) != np.sort(knn, axis=1), axis=1)
    knn_out, w_out = knn.copy(), w.copy()
    knn_out[changed] = ids[changed]
    w_out[changed] = SKIN.skin_weights(np.asarray(v_ref, dtype=np.float64)[changed], node_p, node_sigma,
                                       ids[changed])
    return knn_out, w_out, changed
