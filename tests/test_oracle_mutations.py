"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in the oracle (on the CPU, through monkeypatch)
-- a flipped sign, a dropped term, a transposed operand, a wrong tie order --
and checks that at least one pin then fails.
"""
import numpy as np
import pytest

from oracle import dq as DQ
from oracle import depth as DEPTH
from oracle import skinning as SKIN
from oracle import solver as S
from oracle import fusion as FU

import test_oracle_depth_dq as T_DQ
import test_oracle_skin_solver as T_SOLVE
import test_oracle_fusion as T_FU


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_flipped_sign_in_dq_translation(monkeypatch):
    def bad(c0, ce):
        w0, a0 = c0[..., :1], c0[..., 1:]
        we, ae = ce[..., :1], ce[..., 1:]
        return 2.0 * (w0 * ae + we * a0 + np.cross(a0, ae))
    monkeypatch.setattr(DQ, "dq_translation", bad)
    _fails(T_DQ.test_dq_rigid_transform_and_composition_match_matrices)


def test_dropped_normalisation_term_in_jacobian(monkeypatch):
    orig = S.transform_jacobian

    def bad(b, p):
        out = orig(b, p)
        W, A = b[:, 0], b[:, 1:4]
        We, Ae = b[:, 4], b[:, 5:8]
        n2 = W * W + np.sum(A * A, axis=1)
        Axp = np.cross(A, p)
        h = np.cross(A, Axp) + W[:, None] * Axp + W[:, None] * Ae - We[:, None] * A + np.cross(A, Ae)
        out[:, :, 0:4] += (4.0 / n2 ** 2)[:, None, None] * h[:, :, None] * b[:, None, 0:4]
        return out
    monkeypatch.setattr(S, "transform_jacobian", bad)
    _fails(T_SOLVE.test_data_jacobian_matches_finite_differences)


def test_transposed_operand_in_increment_jacobian(monkeypatch):
    def bad(q):
        L0 = DQ.left_mult_matrix(q[..., :4])
        Le = DQ.left_mult_matrix(q[..., 4:])
        out = np.zeros(q.shape[:-1] + (8, 6))
        out[..., 0:4, 0:3] = 0.5 * L0
        out[..., 4:8, 0:3] = 0.5 * L0          # should be Le
        out[..., 4:8, 3:6] = 0.5 * Le          # should be L0
        return out
    monkeypatch.setattr(S, "node_increment_jacobian", bad)
    _fails(T_SOLVE.test_data_jacobian_matches_finite_differences)


def test_swapped_cross_product_in_normals(monkeypatch):
    orig = np.cross

    def swapped(a, b, *args, **kw):
        return orig(b, a, *args, **kw)
    monkeypatch.setattr(DEPTH.np, "cross", swapped)
    try:
        _fails(T_DQ.test_plane_normals_radius_confidence)
    finally:
        monkeypatch.undo()


def test_wrong_reg_jacobian_sign(monkeypatch):
    orig = S.reg_terms

    def bad(node_p, node_dq, graph, lam):
        j, i, r, Jj, Ji = orig(node_p, node_dq, graph, lam)
        return j, i, r, Jj, -Ji
    monkeypatch.setattr(S, "reg_terms", bad)
    _fails(T_SOLVE.test_reg_jacobian_matches_finite_differences_and_rigid_zero)


def test_wrong_beta_in_pcg(monkeypatch, tiny_scene):
    def bad_pcg(A, b, Minv, iters):
        n = A.n
        As = A.to_scipy()

        def pre(v):
            return np.einsum('nij,nj->ni', Minv, v.reshape(n, 6)).reshape(-1)
        x = np.zeros(6 * n)
        r = b.copy()
        z = pre(r)
        p = z.copy()
        rz = r @ z
        for _ in range(iters):
            q = As @ p
            pq = p @ q
            alpha = rz / pq
            x += alpha * p
            r -= alpha * q
            z = pre(r)
            rz_new = r @ z
            p = z + (rz_new / pq) * p      # wrong denominator
            rz = rz_new
        return x, rz, iters
    monkeypatch.setattr(S, "pcg", bad_pcg)
    _fails(T_SOLVE.test_pcg_iterate_is_krylov_minimiser, tiny_scene)


def test_wrong_knn_tie_order(monkeypatch):
    orig = SKIN.knn_fp32

    def bad(q, nodes, k, exclude_self=False, chunk=4096):
        nn = len(nodes)
        rev = orig(q, np.asarray(nodes)[::-1], k, exclude_self, chunk)
        return nn - 1 - rev                 # ties now go to the higher id
    monkeypatch.setattr(SKIN, "knn_fp32", bad)
    _fails(T_SOLVE.test_knn_brute_force_fp32_with_ties)


def test_wrong_fusion_preference(monkeypatch):
    orig = FU.select_fusion_targets

    def bad(imap, v, n, conf, *a):
        return orig(imap, v, n, -np.asarray(conf), *a)   # lowest confidence wins
    monkeypatch.setattr(FU, "select_fusion_targets", bad)
    _fails(T_FU.test_window_search_brute_force_and_update)


def test_flipped_cross_product_in_rigid_jacobian(monkeypatch):
    """y × n_d turned into n_d × y: the finite-difference pin fails."""
    import test_oracle_rigid as T
    from oracle import rigid as R

    def bad_terms(y, n_d, v_d):
        r = np.einsum('ij,ij->i', n_d, y - v_d)
        return r, np.concatenate([np.cross(n_d, y), n_d], axis=1)
    monkeypatch.setattr(R, "rigid_terms", bad_terms)
    with pytest.raises(AssertionError):
        T.test_rigid_jacobian_matches_finite_differences()


def test_eq7_against_live_distances_only(monkeypatch):
    """Eq. 7 with the reference distance replaced by the live one: the hand-worked case fails."""
    import test_oracle_append as T
    from oracle import append as AP

    def bad(knn, p_live32, p_ref32, eps=AP.EPS):
        return AP_consistent(knn, p_live32, p_live32, eps)
    AP_consistent = AP.consistent
    monkeypatch.setattr(AP, "consistent", bad)
    _fails(T.test_eq7_ratio_test_by_hand)


def test_one_sided_strain_difference(monkeypatch):
    """A forward difference divided by 2h halves the strain: the analytic pin fails."""
    import test_oracle_append as T
    from oracle import append as AP

    def bad(x, node_dq, knn, keep, p_live32, sigma, h=AP.FD_STEP):
        x = np.asarray(x, dtype=np.float64)
        out = np.empty(x.shape + (3,))
        zero = np.zeros_like(x)
        r0, _ = AP.inverse_warp_live(x, zero, node_dq, knn, AP.live_weights(x, p_live32, sigma, knn, keep))
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            rp, _ = AP.inverse_warp_live(x + e, zero, node_dq, knn, AP.live_weights(x + e, p_live32, sigma, knn, keep))
            out[:, :, a] = (rp - r0) / (2.0 * h)
        return out
    monkeypatch.setattr(AP, "strain", bad)
    _fails(T.test_strain_matches_analytic_jacobian_and_flags_compression)


def test_forward_instead_of_inverse_warp_on_append(monkeypatch):
    """Appending with the forward warp: the rigid closed form fails."""
    import test_oracle_append as T
    from oracle import append as AP

    def bad(x, n, node_dq, knn, w):
        b = DQ.blend(node_dq, knn, w)
        return DQ.dq_transform_point(b, x), DQ.dq_rotate_vector(b, n)
    monkeypatch.setattr(AP, "inverse_warp_live", bad)
    _fails(T.test_rigid_warp_field_inverts_exactly)


def test_strict_unstable_period(monkeypatch):
    """t_now − t_init > t_low_confid instead of ≥: the boundary table fails."""
    import test_oracle_append as T
    from oracle import append as AP

    def bad(conf, t_init, t_now, stable_conf, t_low=AP.T_LOW_CONFID):
        return (np.asarray(conf) < stable_conf) & (t_now - np.asarray(t_init) > t_low)
    monkeypatch.setattr(AP, "unstable", bad)
    _fails(T.test_unstable_removal_boundaries)


def test_wrong_splat_intersection_depth(monkeypatch):
    """The ray-plane depth taken as (n·v)/(n·q) with q's z dropped: the closed-form disk pin fails."""
    import test_oracle_visibility as T
    from oracle import visibility as V
    orig = V.splat_cover

    def bad(v32, n32, r32, xs, ys, cx, cy, fx, fy):
        qx = (xs.astype(np.float32) - np.float32(cx)) / np.float32(fx)
        qy = (ys.astype(np.float32) - np.float32(cy)) / np.float32(fy)
        nv = ((n32[:, 0] * v32[:, 0]) + (n32[:, 1] * v32[:, 1])) + (n32[:, 2] * v32[:, 2])
        nq = (n32[:, 0] * qx) + (n32[:, 1] * qy) - n32[:, 2]
        with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
            t = nv / nq
            d2 = ((t * qx - v32[:, 0]) ** 2 + (t * qy - v32[:, 1]) ** 2) + (t - v32[:, 2]) ** 2
            return (t > 0) & (d2 <= r32 * r32), t
    monkeypatch.setattr(V, "splat_cover", bad)
    assert orig is not bad
    _fails(T.test_fronto_parallel_disk_closed_form)


def test_splat_ties_to_the_higher_id(monkeypatch):
    import test_oracle_visibility as T
    from oracle import visibility as V
    orig = V.visibility_map

    def bad(v_live, n_live, radius, selected, cam, chunk=4096):
        k = len(v_live)
        rev = orig(np.asarray(v_live)[::-1], np.asarray(n_live)[::-1], np.asarray(radius)[::-1],
                   np.asarray(selected)[::-1], cam, chunk)
        return np.where(rev >= 0, k - 1 - rev, -1)
    monkeypatch.setattr(V, "visibility_map", bad)
    _fails(T.test_equal_depths_go_to_the_lower_id_and_hidden_splats_are_invisible)


def test_subsampling_ignores_accepted_nodes(monkeypatch):
    """Sub-sampling that checks only the old nodes: the hand-worked line gives too many nodes."""
    import test_oracle_append as T
    from oracle import append as AP

    def bad(v_unc, node_p, node_sigma, max_new):
        v32 = np.asarray(v_unc, dtype=np.float32)
        p32 = np.asarray(node_p, dtype=np.float32)
        s32 = np.asarray(node_sigma, dtype=np.float32)
        new_p, new_s = [], []
        for v in v32[:max_new]:
            d_old = AP.d2_fp32(p32, v[None, :])
            j0 = int(np.argmin(d_old))
            if np.any(d_old < s32[j0] * s32[j0]):
                continue
            new_p.append(v)
            new_s.append(s32[j0])
        return np.asarray(new_p, np.float32).reshape(-1, 3), np.asarray(new_s, np.float32)
    monkeypatch.setattr(AP, "subsample_nodes", bad)
    _fails(T.test_coverage_and_greedy_subsampling_by_hand)
