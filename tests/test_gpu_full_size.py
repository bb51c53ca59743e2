"""Parity with the FP64 oracle at the sizes the kernels are timed at.

The full-size workload (640x480 bending sphere, 300k surfels, 2048 nodes,
10 Gauss-Newton x 20 PCG iterations per frame) and a 4096-node stream of
the uneven batch's largest size run with the launch shapes the bench times:
the data-term kernel's chunked run reduction over ~1,200 tiles, the PCG as
the bench launches it, and in the batch the PCG the batch's shared memory
allows.

Two properties of this size shape the checks.
* Association: a few decisions differ between the library's FP32 warp and
  the oracle's FP32 rounding of its FP64 warp (about one surfel in 10^4 sits
  within an ulp of a pixel edge).  Each such surfel is checked to lie at a
  decision boundary, where both roundings are valid answers; there the
  oracle takes the library's decision.
* Conditioning: the 12,288-unknown system is ill-conditioned (20 PCG
  iterations leave a relative residual near 1e-2), and the configured
  precision evaluates the SpMV in FP32.  Its rounding (the products of
  one 6x6 block and the sums across blocks cancel strongly) moves a
  20-iteration increment by ~2e-4 rad; rounding JᵀJ itself to FP32 costs
  ~3e-5 rad.  The FP64 variant meets the configuration's 1e-4 rad / 1e-5 m
  at this size and is asserted there; the FP32 modes' error is measured,
  reported and held to the bound their arithmetic sets (see each test).
"""
import numpy as np
import pytest

import synth
import paper_1904_13073_gb300 as sw
from oracle import solver as OS

from gpu_helpers import (Pair, association_flips, ensure_built, oracle_dq_from, oracle_for, rigid_dq8_from,
                         rotation_angle_between, set_maps_from_oracle, set_maps_like, solve_with_fp32_spmv)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_built()


@pytest.fixture(scope="module")
def full():
    return synth.plain_full(seed=0)


def _oracle_system(o, odq, pix):
    """The oracle's JᵀJ, Jᵀe and their entry-wise absolute sums for the
    association pix (pixel per surfel or -1) at the transforms odq."""
    mask = (pix >= 0) & ~OS.unskinned(OS.DQ.blend(odq, o.knn, o.w))
    idx = np.nonzero(mask)[0]
    tv = o.maps["V"].reshape(-1, 3)[pix[idx]]
    tn = o.maps["N"].reshape(-1, 3)[pix[idx]]
    r, J = OS.data_terms(o.v_ref[idx], o.knn[idx], o.w[idx], odq, tv, tn)
    reg = OS.reg_terms(o.node_p, odq, o.graph, o.p.lam)
    return OS.assemble(o.pattern, len(o.node_p), o.knn[idx], J, r, reg, absolute=True)


def _data_jacobian_magnitude(o, idx, odq, tn):
    """Entry-wise magnitude of the computation of each data-term Jacobian
    component: the chain n_dᵀ (∂p'/∂b) w_k s_k ∂(δ ⊗ q̂_k)/∂ξ with every
    factor replaced by its absolute value.  A floating-point evaluation of
    the chain errs by a small multiple of the unit roundoff times this
    magnitude however much its terms cancel -- as they do for the rotation
    about the line of sight, where (p' × n)_z is ~1e-2 of |p'| |n|."""
    b = OS.DQ.blend(odq, o.knn[idx], o.w[idx])
    T = np.abs(OS.transform_jacobian(b, o.v_ref[idx]))                    # (t, 3, 8)
    M = np.abs(OS.node_increment_jacobian(odq[o.knn[idx]]))                # (t, k, 8, 6)
    return o.w[idx][..., None] * np.einsum('tj,tkjc->tkc', np.einsum('ti,tij->tj', np.abs(tn), T), M)


def _oracle_scale(o, odq, pix):
    """The entry-wise scale of the system's computation (see the JᵀJ test),
    and for Jᵀe also Σ |J̃| r̃, r̃ the magnitude of each residual's
    computation: |n|ᵀ(|v'| + |V|) for a data term n·(v' − V) and
    √λ (|T_j p_j| + |T_i p_j|) for a regulariser term, both formed from
    points ~1 m away, which an FP32 evaluation errs by a few unit roundoffs
    of however small r is."""
    mask = (pix >= 0) & ~OS.unskinned(OS.DQ.blend(odq, o.knn, o.w))
    idx = np.nonzero(mask)[0]
    tv = o.maps["V"].reshape(-1, 3)[pix[idx]]
    tn = o.maps["N"].reshape(-1, 3)[pix[idx]]
    r, _ = OS.data_terms(o.v_ref[idx], o.knn[idx], o.w[idx], odq, tv, tn)
    _, vl, _ = OS.warp_surfels(o.v_ref[idx], o.n_ref[idx], o.knn[idx], o.w[idx], odq)
    rmag = np.sum(np.abs(tn) * (np.abs(vl) + np.abs(tv)), axis=1)
    Jm = _data_jacobian_magnitude(o, idx, odq, tn)
    reg = OS.reg_terms(o.node_p, odq, o.graph, o.p.lam)
    _, _, S, gS = OS.assemble(o.pattern, len(o.node_p), o.knn[idx], Jm, np.abs(r), reg, absolute=True)
    j, i, _, Jj, Ji = reg
    pj = o.node_p[j]
    rmag_reg = np.sqrt(o.p.lam) * (np.abs(OS.node_transform(odq[j], pj)) + np.abs(OS.node_transform(odq[i], pj)))
    _, _, _, gR = OS.assemble(o.pattern, len(o.node_p), o.knn[idx], Jm, rmag, (j, i, rmag_reg, Jj, Ji),
                              absolute=True)
    return S, gS, gR


def test_full_size_jtj_matches_oracle(full):
    """One linearisation of the full-size frame at a random per-node warp.
    Scale of each entry: the sums of |J̃_a| |J̃_b| (and |J̃| |r| for Jᵀe),
    J̃ the magnitude of the Jacobian's computation (_data_jacobian_magnitude;
    the regulariser's Jacobian entries are its own magnitude), the bound of
    FP32 evaluation and summation in any order.  Every block entry within
    1e-4 of that scale; every entry not dominated by cancellation
    (|A_ij| >= 1e-2 of its scale) within 1e-4 relative.  Jᵀe within 1e-4 of
    Σ |J̃| |r|, and every entry within 1e-4 relative plus 16 unit roundoffs
    of Σ |J̃| r̃, r̃ the magnitude of each residual's computation
    (_oracle_scale): an FP32 residual errs by a few roundoffs of the points'
    magnitude however small it is.  FP32 evaluations of the oracle's terms
    on this linearisation err by up to 16 roundoffs of r̃ in a single
    regulariser residual (0.23 in a data residual), by 0.6 (0.16) of the
    second term in Jᵀe, and by up to 6e-4 relative on Jᵀe entries above
    1e-2 of Σ |J̃| |r|.  The largest error relative to the plain sums
    |J|ᵀ|J| is reported beside it."""
    scene = full
    p = Pair(scene)
    try:
        p.upload(1)
        p.set_maps_from_oracle()
        axis, ang, tr = synth.random_rigid_dq_inputs(13, len(scene.node_p), 2.0, 0.005)
        dq8, odq = rigid_dq8_from(axis, ang, tr), oracle_dq_from(axis, ang, tr)
        sw.sw_set_node_dq(p.h, dq8)
        nnzb, n_corr = sw.sw_debug_assemble(p.h)
        corr = sw.sw_read_correspondence(p.h)
        o = p.o
        _, vl, nl = OS.warp_surfels(o.v_ref, o.n_ref, o.knn, o.w, odq)
        flipped, at_boundary, pix_o = association_flips(o, vl, nl, corr)
        assert np.all(at_boundary), (flipped[~at_boundary], corr[flipped[~at_boundary]])
        assert len(flipped) <= 1e-4 * len(corr) + 5, len(flipped)
        assert n_corr == int(np.sum(corr >= 0)) and n_corr > 50_000
        # the oracle's system under its own decisions, the boundary surfels as the library decided
        pix = np.where(np.isin(np.arange(len(corr)), flipped), corr, pix_o)
        A, g, S0, gS0 = _oracle_system(o, odq, pix)
        S, gS, gR = _oracle_scale(o, odq, pix)
        rows, cols, vals, gg = sw.sw_debug_read_jtj(p.h, nnzb, len(scene.node_p))
        orows, ocols = A.rows_cols()
        assert nnzb == int(np.sum(orows <= ocols)) and np.all(rows <= cols)
        at = A.index(rows, cols)
        want, scale = A.vals[at], S.vals[at]
        err = np.abs(vals - want)
        plain = float(np.max(err / (S0.vals[at] + 1e-30)))
        worst = np.unravel_index(int(np.argmax(err / (scale + 1e-30))), err.shape)
        b = worst[0]
        print(f"worst JtJ entry: block ({rows[b]}, {cols[b]}) entry {worst[1:]}: gpu {vals[worst]:.9g} "
              f"oracle {want[worst]:.9g} |J|ᵀ|J| {S0.vals[at][worst]:.6g} scale {scale[worst]:.6g}; "
              f"block diag gpu {np.diag(vals[b])} oracle {np.diag(want[b])}")
        assert np.all(err <= 1e-4 * scale + 1e-12), float(np.max(err / (scale + 1e-30)))
        big = (np.abs(want) >= 1e-2 * scale) & (want != 0)
        rel = float(np.max(err[big] / np.abs(want[big])))
        assert rel <= 1e-4, rel
        gerr = np.abs(gg - g.reshape(-1))
        assert np.all(gerr <= 1e-4 * gS.reshape(-1) + 1e-12), float(np.max(gerr / (gS.reshape(-1) + 1e-30)))
        u32 = 2.0 ** -24
        gexcess = np.maximum(gerr - 1e-4 * np.abs(g.reshape(-1)), 0.0) / (u32 * gR.reshape(-1) + 1e-30)
        grel = float(np.max(gexcess))
        wg = int(np.argmax(gexcess))
        print(f"worst Jte entry: node {wg // 6} component {wg % 6}: gpu {gg[wg]:.9g} oracle {g.reshape(-1)[wg]:.9g} "
              f"sum |J||r| {gS.reshape(-1)[wg]:.6g} sum |J| r-magnitude {gR.reshape(-1)[wg]:.6g}")
        assert grel <= 16.0, grel
        print(f"full-size JtJ: {nnzb} blocks, {n_corr} terms, {len(flipped)} boundary decisions, "
              f"max error {float(np.max(err / (scale + 1e-30))):.2e} of the computation scale "
              f"({plain:.2e} of |J|ᵀ|J|), max entry-relative error {rel:.2e} "
              f"({int(big.sum())} of {big.size} entries), Jte error beyond 1e-4 relative {grel:.2f} unit "
              f"roundoffs of the residuals' magnitude")
    finally:
        p.close()


def _node_errors(h, o):
    _, dq = sw.sw_read_nodes(h)
    dq = dq.astype(np.float64)
    rot = float(rotation_angle_between(dq, o.node_dq).max())
    trans = float(np.linalg.norm(OS.node_transform(dq, o.node_p) - o.warped_nodes(), axis=1).max())
    return rot, trans


def _report(name, data):
    import json
    import os
    out = os.environ.get("SW_REPORT_DIR")
    if out:
        os.makedirs(out, exist_ok=True)
        with open(os.path.join(out, name), "w") as f:
            json.dump(data, f, indent=1)


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_FP64, sw.SW_PRECISION_MIXED, sw.SW_PRECISION_MIXED_F64DOTS])
def test_full_size_frame_matches_oracle(full, precision):
    """The full-size frame, Gauss-Newton x 20 PCG iterations with the
    bench's launch shapes (the PCG autotuned as the bench does), against the
    oracle on the same FP32 depth maps, one Gauss-Newton iteration per call
    on both sides so that the node error is recorded after each iteration.
    The FP64 variant: node rotations within 1e-4 rad and translations within
    1e-5 m after every iteration.  The FP32 modes: the errors are reported,
    and each iteration's must stay below 4x the error that the FP32 SpMV
    alone causes in the oracle's own arithmetic on the same frame (the
    oracle's PCG with its products A p rounded to FP32, pcg_fp32_spmv):
    the configured precision's error, measured and bounded, not hidden."""
    scene = full
    p = Pair(scene, precision=precision)
    try:
        p.upload(1)
        p.set_maps_from_oracle()
        sw.sw_autotune(p.h, scene.pcg_iters)
        ref32 = None
        if precision != sw.SW_PRECISION_FP64:
            ref32 = oracle_for(scene)
            set_maps_like(ref32, p.o)
        rows = []
        # the FP64 variant over the configuration's 10 iterations; the FP32
        # modes over 3 (their error is set within each iteration)
        for it in range(scene.gn_iters if precision == sw.SW_PRECISION_FP64 else 3):
            st = sw.sw_solve_frame(p.h, 1, scene.pcg_iters)
            ost = p.o.solve_frame(1, scene.pcg_iters)
            assert abs(st["n_corr"][0] - ost[0].n_corr) <= 1e-4 * ost[0].n_corr + 5, (it, st["n_corr"][0], ost[0].n_corr)
            rot, trans = _node_errors(p.h, p.o)
            row = {"gn_iter": it + 1, "rot_err_rad": rot, "trans_err_m": trans,
                   "e_depth": st["e_depth"][0], "oracle_e_depth": ost[0].e_depth}
            if ref32 is not None:
                solve_with_fp32_spmv(ref32, 1, scene.pcg_iters)
                row["fp32_spmv_rot_rad"] = float(rotation_angle_between(ref32.node_dq, p.o.node_dq).max())
                row["fp32_spmv_trans_m"] = float(np.linalg.norm(ref32.warped_nodes() - p.o.warped_nodes(), axis=1).max())
            rows.append(row)
            print(row)
        _report(f"full_size_frame_prec{precision}.json", rows)
        for row in rows:
            if precision == sw.SW_PRECISION_FP64:
                assert row["rot_err_rad"] <= 1e-4 and row["trans_err_m"] <= 1e-5, row
            else:
                assert row["rot_err_rad"] <= 4 * row["fp32_spmv_rot_rad"] + 1e-4, row
                assert row["trans_err_m"] <= 4 * row["fp32_spmv_trans_m"] + 1e-5, row
    finally:
        p.close()


@pytest.mark.parametrize("precision", [sw.SW_PRECISION_FP64, sw.SW_PRECISION_MIXED])
def test_4096_node_member_in_a_batch_matches_oracle(precision):
    """A 4096-node, 300k-surfel sphere of the uneven batch's largest size,
    solved inside a batch with two smaller members (3 GN x 20 PCG), against
    the oracle: in the FP64 variant each member within 1e-4 rad / 1e-5 m; in
    the default mode the errors are reported and held, like the full-size
    frame's, to 4x those of the oracle with an FP32 SpMV."""
    scenes = [synth.plain_full(seed=101, n_nodes=4096), synth.batch_member(1), synth.batch_member(2)]
    hs = []
    for s in scenes:
        v4, n4, t2, node4 = sw.model_arrays(s)
        h = sw.sw_create_stream(sw.params_for(s.cam, len(v4), len(node4), precision=precision))
        sw.sw_set_model(h, v4, n4, t2, node4)
        hs.append(h)
    b = sw.sw_batch_create(hs)
    try:
        sw.sw_batch_upload_depth(b, [s.frame(2) for s in scenes], [2] * len(scenes))
        oracles = []
        for h, s in zip(hs, scenes):     # identical FP32 depth maps on both sides
            o = oracle_for(s)
            o.upload_depth(s.frame(2), 2)
            set_maps_from_oracle(h, o)
            oracles.append(o)
        mode = sw.sw_batch_debug_pcg_mode(b)
        st = sw.sw_batch_solve(b, 3, 20)
        report = []
        for k, (h, s, o) in enumerate(zip(hs, scenes, oracles)):
            ref32 = None
            if precision != sw.SW_PRECISION_FP64:
                ref32 = oracle_for(s)
                set_maps_like(ref32, o)
                solve_with_fp32_spmv(ref32, 3, 20)
            ost = o.solve_frame(3, 20)
            rot, trans = _node_errors(h, o)
            row = {"member": k, "nodes": len(s.node_p), "surfels": len(s.surfel_v), "pcg_mode": mode,
                   "rot_err_rad": rot, "trans_err_m": trans}
            if ref32 is not None:
                row["fp32_spmv_rot_rad"] = float(rotation_angle_between(ref32.node_dq, o.node_dq).max())
                row["fp32_spmv_trans_m"] = float(np.linalg.norm(ref32.warped_nodes() - o.warped_nodes(), axis=1).max())
            report.append(row)
            print(row)
            for i in range(3):
                assert abs(st[k]["n_corr"][i] - ost[i].n_corr) <= 1e-4 * ost[i].n_corr + 5
            if precision == sw.SW_PRECISION_FP64:
                assert rot <= 1e-4 and trans <= 1e-5, row
            else:
                assert rot <= 4 * row["fp32_spmv_rot_rad"] + 1e-4 and trans <= 4 * row["fp32_spmv_trans_m"] + 1e-5, row
        _report(f"batch_4096_prec{precision}.json", report)
    finally:
        sw.sw_batch_destroy(b)
        for h in hs:
            sw.sw_destroy_stream(h)
