"""Quaternion and dual-quaternion algebra in FP64 (Sec. 3, Eq. 1-3).

Conventions
-----------
A quaternion is (w, x, y, z) with the scalar first.  A dual quaternion
q̂ = q0 + ε qe is stored as 8 numbers: the real part q0 then the dual part qe.
A rigid motion x -> R x + t is the dual quaternion (q, ½ (0, t) ⊗ q) with q the
unit rotation quaternion of R (Kavan et al. 2008, cited in Sec. 3).
The product of two dual quaternions composes the motions, the left factor
being applied last.
"""
import numpy as np


def qmul(a, b):
    """Hamilton product a ⊗ b of quaternions (..., 4)."""
    aw, av = a[..., :1], a[..., 1:]
    bw, bv = b[..., :1], b[..., 1:]
    w = aw * bw - np.sum(av * bv, axis=-1, keepdims=True)
    v = aw * bv + bw * av + np.cross(av, bv)
    return np.concatenate([w, v], axis=-1)


def qconj(q):
    return np.concatenate([q[..., :1], -q[..., 1:]], axis=-1)


def qrotate(q, p):
    """R(q) p for a unit quaternion q: p + 2 a × (a × p + w p)."""
    w, a = q[..., :1], q[..., 1:]
    return p + 2.0 * np.cross(a, np.cross(a, p) + w * p)


def qmatrix(q):
    """3x3 rotation matrix of a unit quaternion (columns = rotated axes)."""
    eye = np.broadcast_to(np.eye(3), q.shape[:-1] + (3, 3))
    return np.stack([qrotate(q, eye[..., :, c]) for c in range(3)], axis=-1)


def dq_identity(n):
    out = np.zeros((n, 8))
    out[:, 0] = 1.0
    return out


def dq_from_rt(q, t):
    """Dual quaternion of the motion x -> R(q) x + t."""
    t4 = np.concatenate([np.zeros(t.shape[:-1] + (1,)), t], axis=-1)
    return np.concatenate([q, 0.5 * qmul(t4, q)], axis=-1)


def dq_mul(a, b):
    """(a0 + ε ae)(b0 + ε be) = a0 b0 + ε (a0 be + ae b0)."""
    a0, ae = a[..., :4], a[..., 4:]
    b0, be = b[..., :4], b[..., 4:]
    return np.concatenate([qmul(a0, b0), qmul(a0, be) + qmul(ae, b0)], axis=-1)


def dq_normalize(d):
    """Unit real part and a dual part orthogonal to it (a rigid motion)."""
    q0, qe = d[..., :4], d[..., 4:]
    n = np.linalg.norm(q0, axis=-1, keepdims=True)
    q0 = q0 / n
    qe = qe / n
    qe = qe - np.sum(q0 * qe, axis=-1, keepdims=True) * q0
    return np.concatenate([q0, qe], axis=-1)


def normalized_parts(b):
    """``normalized`` of Eq. 1: both parts divided by the real part's norm."""
    n = np.linalg.norm(b[..., :4], axis=-1, keepdims=True)
    return b[..., :4] / n, b[..., 4:] / n


def dq_translation(c0, ce):
    """t = 2 (w0 aε − wε a0 + a0 × aε) of a dual quaternion with unit real part.

    This is the vector part of 2 cε ⊗ c0*; it is the translation of the
    rigid motion even when cε is not exactly orthogonal to c0 (the blend of
    Eq. 1 is not).
    """
    w0, a0 = c0[..., :1], c0[..., 1:]
    we, ae = ce[..., :1], ce[..., 1:]
    return 2.0 * (w0 * ae - we * a0 + np.cross(a0, ae))


def dq_transform_point(b, p):
    """W(x) x of Eq. 2 for a (possibly unnormalised) blended dual quaternion b."""
    c0, ce = normalized_parts(b)
    return qrotate(c0, p) + dq_translation(c0, ce)


def dq_rotate_vector(b, n):
    """rotation(W(x)) n of Eq. 2."""
    c0, _ = normalized_parts(b)
    return qrotate(c0, n)


def dq_inverse_transform_point(b, p):
    """W(x)^-1 p of Eq. 3: R^T (p − t)."""
    c0, ce = normalized_parts(b)
    return qrotate(qconj(c0), p - dq_translation(c0, ce))


def dq_inverse_rotate_vector(b, n):
    c0, _ = normalized_parts(b)
    return qrotate(qconj(c0), n)


def blend(node_dq, knn, w):
    """Σ_k w_k s_k q̂_k of Eq. 1 over each surfel's k nearest nodes.

    The sign s_k = ±1 puts every real part in the hemisphere of the nearest
    node's real part (slot 0), so that q̂ and −q̂ (the same motion) blend alike
    (antipodality handling of Kavan et al. 2008; sign(0) = +1).
    Returns (n, 8) unnormalised blends.
    """
    q = node_dq[knn]                                   # (n, k, 8)
    ref = q[:, :1, :4]
    s = np.where(np.sum(q[..., :4] * ref, axis=-1) >= 0.0, 1.0, -1.0)
    return np.sum((w * s)[..., None] * q, axis=1)


def rodrigues_quat(omega):
    """Unit quaternion of the rotation vector ω: (cos θ/2, sin θ/2 ω/θ)."""
    theta = np.linalg.norm(omega, axis=-1, keepdims=True)
    safe = np.where(theta > 0.0, theta, 1.0)
    half = 0.5 * theta
    s = np.where(theta > 0.0, np.sin(half) / safe, 0.5)
    return np.concatenate([np.cos(half), s * omega], axis=-1)


def increment_dq(xi):
    """Dual quaternion of the increment ξ = (ω, τ): x -> R(ω) x + τ."""
    return dq_from_rt(rodrigues_quat(xi[..., :3]), xi[..., 3:])


def left_mult_matrix(q):
    """L(q) (4x3) with (0, u) ⊗ q = L(q) u, for q = (w, a): [−aᵀ; w I − [a]×]."""
    w, a = q[..., 0], q[..., 1:]
    out = np.zeros(q.shape[:-1] + (4, 3))
    out[..., 0, :] = -a
    out[..., 1:, :] = w[..., None, None] * np.eye(3) - skew(a)
    return out


def skew(a):
    """[a]× with [a]× b = a × b."""
    out = np.zeros(a.shape[:-1] + (3, 3))
    out[..., 0, 1], out[..., 0, 2] = -a[..., 2], a[..., 1]
    out[..., 1, 0], out[..., 1, 2] = a[..., 2], -a[..., 0]
    out[..., 2, 0], out[..., 2, 1] = -a[..., 1], a[..., 0]
    return out
