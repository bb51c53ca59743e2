"""Rigid pre-alignment before the non-rigid solve (Sec. 7: before the
non-rigid estimation the system first aligns rigidly, in the manner of
KinectFusion).

TEST INFRASTRUCTURE ONLY: see the package docstring.

Reading (the paper only names the method): point-to-plane ICP of the warped
model against the live depth.  At each iteration every surfel is warped by
the current warp field (Eq. 1-2) and moved by the current rigid estimate T,
then associated with the depth by the same projective rule as the
non-rigid solve (selection, pixel, distance and normal tests, in FP32).  The
point-to-plane residual r = n_dᵀ(T x − v_d) is linearised in a left
increment ξ = (ω, τ) of T, T ← Δ(ξ) T with Δ = (R(ω) by Rodrigues, τ) as for
the nodes, so that at ξ = 0

    ∂r/∂ω = (T x) × n_d,   ∂r/∂τ = n_d.

The 6x6 normal equations Σ J Jᵀ ξ = −Σ J r are solved by Cholesky in FP64
(a system that is not positive definite ends the iterations with T as it
is), and T is updated.  After `iters` iterations T is composed into every
node transform, T_j ← T T_j, and the non-rigid solve starts from there.
"""
import numpy as np

from . import dq as DQ
from . import solver as S


def rigid_terms(y, n_d, v_d):
    """Residuals r = n_dᵀ(y − v_d) and their 1x6 Jacobians in (ω, τ) at ξ = 0."""
    r = np.einsum('ij,ij->i', n_d, y - v_d)
    J = np.concatenate([np.cross(y, n_d), n_d], axis=1)
    return r, J


def apply_rigid(T, p, n):
    """Points and normals moved by the rigid dual quaternion T."""
    Tb = np.broadcast_to(T, p.shape[:-1] + (8,))
    return DQ.dq_transform_point(Tb, p), DQ.dq_rotate_vector(Tb, n)


def rigid_align(v_ref, n_ref, knn, w, node_dq, associate_fn, iters):
    """Returns (node_dq with T composed in, T, [(correspondences, Σ r²) per iteration])."""
    b, v_live, n_live = S.warp_surfels(v_ref, n_ref, knn, w, node_dq)
    live = ~S.unskinned(b)
    T = DQ.dq_identity(1)[0]
    stats = []
    for _ in range(iters):
        y, ny = apply_rigid(T, v_live, n_live)
        mask, tv, tn = associate_fn(y, ny)
        idx = np.nonzero(mask & live)[0]
        r, J = rigid_terms(y[idx], tn[idx], tv[idx])
        stats.append((len(idx), float(r @ r)))
        A = J.T @ J
        g = J.T @ r
        try:
            L = np.linalg.cholesky(A)
        except np.linalg.LinAlgError:
            break
        xi = -np.linalg.solve(L.T, np.linalg.solve(L, g))
        T = DQ.dq_normalize(DQ.dq_mul(DQ.increment_dq(xi[None])[0], T))
    node_dq = DQ.dq_normalize(DQ.dq_mul(np.broadcast_to(T, node_dq.shape), node_dq))
    return node_dq, T, stats
