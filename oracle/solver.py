"""Non-rigid warp-field estimation (Sec. 7, Eq. 9-11; Sec. 8), FP64.

Energy (Eq. 9):  E_total = E_depth + λ E_regulation, λ = 5 (Table 1).

E_depth (Eq. 10) sums (n_depthᵀ (v_model − v_depth))² over the associated
(model surfel, depth pixel) pairs.  E_regulation (Eq. 11) sums
‖T_j p_j − T_i p_j‖² over every node j and every i in its graph
neighbourhood N_j; the directed pairs are taken literally, so a mutual pair
appears twice.  λ is folded into the residual as √λ.

The problem is solved by Gauss-Newton (Sec. 7-8): at each iteration form JᵀJ
and Jᵀe explicitly and solve JᵀJ Δ = −Jᵀe; here the linear solve is block-
Jacobi preconditioned conjugate gradients with a fixed iteration count.

Readings of what the paper leaves open:

* association (the paper defers to another work): each selected surfel is
  warped, projected with the pinhole model to the pixel
  (floor(u + ½), floor(v + ½)), u = fx x / z + cx, and accepted when z > 0,
  the pixel lies in the image and is a usable depth surfel,
  ‖v_live − V(u)‖² < corr_dist² and n_live · N(u) > corr_normal; the
  decision is taken in FP32 with a fixed operation order;
* surfel selection (Sec. 7): confidence c > δ_stable, or recently observed
  (t_now − t_observed ≤ δ_recent);
* parameterisation: each node takes a left increment Δ = (R(ω), τ),
  T ← Δ T, R(ω) by Rodrigues' formula; ξ_j = (ω_j, τ_j) ordered so;
* no robust kernel, no damping; a diagonal block that is not positive
  definite is a solver breakdown;
* PCG: x₀ = 0, exactly ``pcg_iters`` iterations of the standard recurrences,
  stopping early only when rᵀz is exactly zero.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import dq as DQ

_F32 = np.float32


class SolverBreakdown(RuntimeError):
    pass


# ---------------------------------------------------------------------------
# warp (Eq. 1-2)
# ---------------------------------------------------------------------------

def warp_surfels(v_ref, n_ref, knn, w, node_dq):
    """Blend (Eq. 1) and forward warp (Eq. 2) of every surfel.

    Reading: a surfel whose weights are all zero (farther than ~38 σ from
    every node in FP64) has no defined warp and is left in place (identity).
    """
    b = DQ.blend(node_dq, knn, w)
    dead = unskinned(b)
    if np.any(dead):
        b = b.copy()
        b[dead] = DQ.dq_identity(int(dead.sum()))
    return b, DQ.dq_transform_point(b, v_ref), DQ.dq_rotate_vector(b, n_ref)


def unskinned(b):
    """Surfels whose blended real part is exactly zero (no usable weight).

    Reading: such a surfel has no warp to optimise, so it never takes part in
    association; fusion warps it by the identity.
    """
    return np.sum(b[:, :4] * b[:, :4], axis=1) == 0.0


# ---------------------------------------------------------------------------
# projective association (Sec. 7), decisions in FP32
# ---------------------------------------------------------------------------

def project_fp32(v, fx, fy, cx, cy):
    """Pixel of FP32 points: (floor(fx·x/z + cx + ½), floor(fy·y/z + cy + ½)).

    Operation order: ((f * x) / z) + c, then + 0.5, then floor; FP32
    round-to-nearest at every step, IEEE division.  Returns float32 pixel
    coordinates (NaN/inf where z <= 0 must be masked by the caller).
    """
    v = v.astype(_F32)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = ((_F32(fx) * v[:, 0]) / v[:, 2]) + _F32(cx)
        vv = ((_F32(fy) * v[:, 1]) / v[:, 2]) + _F32(cy)
        return np.floor(u + _F32(0.5)), np.floor(vv + _F32(0.5))


def dist2_fp32(a, b):
    a = a.astype(_F32)
    b = b.astype(_F32)
    dx, dy, dz = a[:, 0] - b[:, 0], a[:, 1] - b[:, 1], a[:, 2] - b[:, 2]
    return ((dx * dx) + (dy * dy)) + (dz * dz)


def dot_fp32(a, b):
    a = a.astype(_F32)
    b = b.astype(_F32)
    return ((a[:, 0] * b[:, 0]) + (a[:, 1] * b[:, 1])) + (a[:, 2] * b[:, 2])


def select_surfels(conf, t_obs, t_now, stable_conf, recent_frames):
    """Surfels the solver uses (Sec. 7): stable or recently observed."""
    return (np.asarray(conf, dtype=_F32) > _F32(stable_conf)) | \
        ((t_now - np.asarray(t_obs)) <= recent_frames)


def associate(v_live, n_live, selected, V32, N32, usable, cam, corr_dist, corr_normal):
    """Projective association of warped surfels to depth pixels.

    ``V32``/``N32`` are the FP32 vertex/normal maps (H, W, 3), ``usable`` the
    depth-surfel mask.  Returns (accepted mask, flat pixel index or −1).
    """
    fx, fy, cx, cy, width, height = cam
    v32 = np.asarray(v_live, dtype=_F32)
    n32 = np.asarray(n_live, dtype=_F32)
    ok = np.asarray(selected, dtype=bool) & (v32[:, 2] > 0)
    px, py = project_fp32(v32, fx, fy, cx, cy)
    with np.errstate(invalid="ignore"):
        ok &= (px >= 0) & (px < width) & (py >= 0) & (py < height)
    pix = np.full(len(v32), -1, dtype=np.int64)
    pix[ok] = py[ok].astype(np.int64) * width + px[ok].astype(np.int64)
    flat_ok = usable.reshape(-1)
    ok[ok] &= flat_ok[pix[ok]]
    Vf, Nf = V32.reshape(-1, 3), N32.reshape(-1, 3)
    idx = np.nonzero(ok)[0]
    d2 = dist2_fp32(v32[idx], Vf[pix[idx]])
    dt = dot_fp32(n32[idx], Nf[pix[idx]])
    cd = _F32(corr_dist)
    good = (d2 < cd * cd) & (dt > _F32(corr_normal))
    ok[idx[~good]] = False
    pix[~ok] = -1
    return ok, pix


# ---------------------------------------------------------------------------
# residuals and Jacobians (Eq. 10, Eq. 11)
# ---------------------------------------------------------------------------

def transform_jacobian(b, p):
    """∂p'/∂b (3x8) of p' = W p for the unnormalised blend b (Eq. 1-2).

    With b0 = (W, A), bε = (Wε, Aε), n² = W² + |A|²:
      p' = p + (2/n²) h,  h = A×(A×p) + W A×p + W Aε − Wε A + A×Aε.
    """
    W, A = b[:, 0], b[:, 1:4]
    We, Ae = b[:, 4], b[:, 5:8]
    n2 = W * W + np.sum(A * A, axis=1)
    Axp = np.cross(A, p)
    h = np.cross(A, Axp) + W[:, None] * Axp + W[:, None] * Ae - We[:, None] * A + np.cross(A, Ae)
    eye = np.eye(3)[None]
    dh = np.zeros((len(b), 3, 8))
    dh[:, :, 0] = Axp + Ae
    dh[:, :, 1:4] = (np.sum(A * p, axis=1)[:, None, None] * eye
                     + A[:, :, None] * p[:, None, :]
                     - 2.0 * p[:, :, None] * A[:, None, :]
                     - W[:, None, None] * DQ.skew(p)
                     - We[:, None, None] * eye
                     - DQ.skew(Ae))
    dh[:, :, 4] = -A
    dh[:, :, 5:8] = W[:, None, None] * eye + DQ.skew(A)
    out = (2.0 / n2)[:, None, None] * dh
    out[:, :, 0:4] -= (4.0 / n2 ** 2)[:, None, None] * h[:, :, None] * b[:, None, 0:4]
    return out


def node_increment_jacobian(node_dq_k):
    """∂(δ(ξ) ⊗ q̂)/∂ξ at ξ = 0 (8x6) for node dual quaternions (..., 8).

    δ(ξ) = r(ω) + ε ½ (0, τ) ⊗ r(ω) and r(ω) ≈ (1, ω/2), so
      d real = ½ (0, dω) ⊗ q0,  d dual = ½ (0, dω) ⊗ qe + ½ (0, dτ) ⊗ q0.
    """
    L0 = DQ.left_mult_matrix(node_dq_k[..., :4])
    Le = DQ.left_mult_matrix(node_dq_k[..., 4:])
    out = np.zeros(node_dq_k.shape[:-1] + (8, 6))
    out[..., 0:4, 0:3] = 0.5 * L0
    out[..., 4:8, 0:3] = 0.5 * Le
    out[..., 4:8, 3:6] = 0.5 * L0
    return out


def data_terms(v_ref, knn, w, node_dq, target_v, target_n):
    """Point-to-plane residuals (Eq. 10) and their Jacobians.

    r = n_dᵀ (W(v_ref) v_ref − v_d);
    ∂r/∂ξ_k = n_dᵀ (∂p'/∂b) w_k s_k ∂(δ ⊗ q̂_k)/∂ξ  (1x6 per node slot k).
    Returns (r (T,), J (T, k, 6)).
    """
    b = DQ.blend(node_dq, knn, w)
    p_live = DQ.dq_transform_point(b, v_ref)
    r = np.sum(target_n * (p_live - target_v), axis=1)
    g = np.einsum('ti,tij->tj', target_n, transform_jacobian(b, v_ref))   # (T, 8)
    q = node_dq[knn]                                                         # (T, k, 8)
    s = np.where(np.sum(q[..., :4] * q[:, :1, :4], axis=-1) >= 0.0, 1.0, -1.0)
    M = node_increment_jacobian(q)                                           # (T, k, 8, 6)
    J = (w * s)[..., None] * np.einsum('tj,tkjc->tkc', g, M)
    return r, J


def node_transform(node_dq, p):
    """T_j p for node dual quaternions (rows) and points (rows)."""
    return DQ.dq_transform_point(node_dq, p)


def reg_terms(node_p, node_dq, graph, lam):
    """As-rigid-as-possible residuals (Eq. 11) with √λ folded in.

    For each directed edge (j, i ∈ N_j): r = √λ (T_j p_j − T_i p_j),
    ∂r/∂ξ_j = √λ [−[T_j p_j]× | I],  ∂r/∂ξ_i = −√λ [−[T_i p_j]× | I].
    Returns (j, i, r (E,3), Jj (E,3,6), Ji (E,3,6)).
    """
    nn, k = graph.shape
    j = np.repeat(np.arange(nn), k)
    i = graph.reshape(-1)
    pj = node_p[j]
    xj = node_transform(node_dq[j], pj)
    y = node_transform(node_dq[i], pj)
    sl = np.sqrt(lam)
    r = sl * (xj - y)
    eye = np.broadcast_to(np.eye(3), (len(j), 3, 3))
    Jj = sl * np.concatenate([-DQ.skew(xj), eye], axis=2)
    Ji = -sl * np.concatenate([-DQ.skew(y), eye], axis=2)
    return j, i, r, Jj, Ji


# ---------------------------------------------------------------------------
# block-sparse JᵀJ
# ---------------------------------------------------------------------------

@dataclass
class BlockMatrix:
    """Symmetric block-sparse matrix with 6x6 blocks, both triangles stored."""
    n: int
    keys: np.ndarray                    # sorted row * n + col
    vals: np.ndarray = field(default=None)

    def __post_init__(self):
        if self.vals is None:
            self.vals = np.zeros((len(self.keys), 6, 6))

    @staticmethod
    def pattern(n, knn, graph):
        """Skinning co-occurrence pairs ∪ graph edges ∪ diagonal, both ways."""
        rows, cols = [np.arange(n)], [np.arange(n)]
        for a in range(knn.shape[1]):
            for b in range(knn.shape[1]):
                if a != b:
                    rows.append(knn[:, a])
                    cols.append(knn[:, b])
        j = np.repeat(np.arange(n), graph.shape[1])
        rows += [j, graph.reshape(-1)]
        cols += [graph.reshape(-1), j]
        keys = np.unique(np.concatenate(rows).astype(np.int64) * n
                         + np.concatenate(cols).astype(np.int64))
        return BlockMatrix(n, keys)

    def index(self, rows, cols):
        key = np.asarray(rows, dtype=np.int64) * self.n + np.asarray(cols, dtype=np.int64)
        idx = np.searchsorted(self.keys, key)
        if np.any(idx >= len(self.keys)) or np.any(self.keys[np.minimum(idx, len(self.keys) - 1)] != key):
            raise KeyError("block outside the sparsity pattern")
        return idx

    def add(self, rows, cols, blocks):
        """Accumulate blocks in the given (term) order."""
        np.add.at(self.vals, self.index(rows, cols), blocks)

    def block(self, i, j):
        return self.vals[self.index([i], [j])[0]]

    def rows_cols(self):
        return self.keys // self.n, self.keys % self.n

    def to_scipy(self):
        r, c = self.rows_cols()
        return sp.bsr_matrix((self.vals, c, np.searchsorted(r, np.arange(self.n + 1))),
                             shape=(6 * self.n, 6 * self.n))

    def dense(self):
        out = np.zeros((6 * self.n, 6 * self.n))
        r, c = self.rows_cols()
        for k in range(len(self.keys)):
            out[6 * r[k]:6 * r[k] + 6, 6 * c[k]:6 * c[k] + 6] = self.vals[k]
        return out


def assemble(pattern_keys, n, knn_t, J, r, reg, absolute=False):
    """JᵀJ and Jᵀe of the data terms (rows of ``knn_t``/``J``/``r``) and the
    regulariser terms ``reg`` = (j, i, r, Jj, Ji), accumulated in term order.

    With ``absolute`` the sums of |J_a|ᵀ|J_b| and |J_a| |r| are returned as
    well; they are the natural scale of the rounding error of any summation
    order.
    """
    A = BlockMatrix(n, pattern_keys)
    S = BlockMatrix(n, pattern_keys) if absolute else None
    g = np.zeros((n, 6))
    gS = np.zeros((n, 6))
    k = knn_t.shape[1]
    for a in range(k):
        np.add.at(g, knn_t[:, a], J[:, a] * r[:, None])
        if absolute:
            np.add.at(gS, knn_t[:, a], np.abs(J[:, a] * r[:, None]))
        for b in range(k):
            blk = J[:, a, :, None] * J[:, b, None, :]
            A.add(knn_t[:, a], knn_t[:, b], blk)
            if absolute:
                S.add(knn_t[:, a], knn_t[:, b], np.abs(blk))
    j, i, rr, Jj, Ji = reg
    for (ra, Ja), (rb, Jb) in (((j, Jj), (j, Jj)), ((j, Jj), (i, Ji)),
                               ((i, Ji), (j, Jj)), ((i, Ji), (i, Ji))):
        blk = np.einsum('eri,erj->eij', Ja, Jb)
        A.add(ra, rb, blk)
        if absolute:
            S.add(ra, rb, np.einsum('eri,erj->eij', np.abs(Ja), np.abs(Jb)))
    np.add.at(g, j, np.einsum('eri,er->ei', Jj, rr))
    np.add.at(g, i, np.einsum('eri,er->ei', Ji, rr))
    if absolute:
        np.add.at(gS, j, np.einsum('eri,er->ei', np.abs(Jj), np.abs(rr)))
        np.add.at(gS, i, np.einsum('eri,er->ei', np.abs(Ji), np.abs(rr)))
        return A, g, S, gS
    return A, g


# ---------------------------------------------------------------------------
# block-Jacobi PCG
# ---------------------------------------------------------------------------

def block_jacobi_inverse(A):
    """Inverses of the 6x6 diagonal blocks, by Cholesky factorisation."""
    n = A.n
    diag = A.vals[A.index(np.arange(n), np.arange(n))]
    out = np.empty_like(diag)
    eye = np.eye(6)
    for j in range(n):
        try:
            L = np.linalg.cholesky(diag[j])
        except np.linalg.LinAlgError as exc:
            raise SolverBreakdown(f"diagonal block {j} is not positive definite") from exc
        Li = np.linalg.solve(L, eye)
        out[j] = Li.T @ Li
    return out


def pcg(A, b, Minv, iters):
    """Preconditioned conjugate gradients for A x = b, x₀ = 0.

    Exactly ``iters`` iterations of the standard recurrences; stops early
    only when rᵀz is exactly zero.  Returns (x, final rᵀz, iterations run).
    """
    n = A.n
    As = A.to_scipy()

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
        q = As @ p
        pq = float(p @ q)
        if not pq > 0.0:
            raise SolverBreakdown("pᵀAp <= 0 in PCG")
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        done += 1
    return x, rz, done


def apply_increment(node_dq, x):
    """T_j ← Δ_j T_j for all nodes, then re-normalise each dual quaternion."""
    delta = DQ.increment_dq(x.reshape(-1, 6))
    return DQ.dq_normalize(DQ.dq_mul(delta, node_dq))


# ---------------------------------------------------------------------------
# Gauss-Newton
# ---------------------------------------------------------------------------

@dataclass
class IterStats:
    e_depth: float
    e_reg: float
    n_corr: int
    pcg_rz: float
    corr_mask: np.ndarray = field(repr=False, default=None)


def gauss_newton(v_ref, n_ref, knn, w, node_p, node_dq, graph, pattern_keys,
                 lam, gn_iters, pcg_iters, associate_fn=None, fixed_targets=None,
                 keep_masks=False, linear_solver=None):
    """Gauss-Newton over the node transforms (Sec. 7-8).

    ``associate_fn(v_live, n_live) -> (mask, target_v, target_n)`` finds the
    correspondences at each iteration (the ICP-style re-association of
    Sec. 4); alternatively ``fixed_targets = (mask, target_v, target_n)``
    holds them fixed.  ``linear_solver(A, b, Minv, iters) -> (x, rᵀz, n)``
    replaces ``pcg`` (tests measure how the result depends on the linear
    solve's arithmetic with it).  Returns (node_dq, [IterStats]).
    """
    linear_solver = pcg if linear_solver is None else linear_solver
    n = len(node_p)
    stats = []
    for _ in range(gn_iters):
        b, v_live, n_live = warp_surfels(v_ref, n_ref, knn, w, node_dq)
        if fixed_targets is not None:
            mask, tv, tn = fixed_targets
        else:
            mask, tv, tn = associate_fn(v_live, n_live)
        mask = mask & ~unskinned(DQ.blend(node_dq, knn, w))
        idx = np.nonzero(mask)[0]
        r, J = data_terms(v_ref[idx], knn[idx], w[idx], node_dq, tv[idx], tn[idx])
        reg = reg_terms(node_p, node_dq, graph, lam)
        A, g = assemble(pattern_keys, n, knn[idx], J, r, reg)
        Minv = block_jacobi_inverse(A)
        x, rz, _ = linear_solver(A, -g.reshape(-1), Minv, pcg_iters)
        stats.append(IterStats(float(r @ r), float(np.sum(reg[2] ** 2)), len(idx), rz,
                               mask.copy() if keep_masks else None))
        node_dq = apply_increment(node_dq, x)
    return node_dq, stats
