// Device math for the SurfelWarp hot path: quaternions, dual-quaternion
// blending (Sec. 3, Eq. 1-2), inverse warp (Sec. 4, Eq. 3), the analytic
// Jacobian of the point-to-plane residual (Sec. 7, Eq. 10) and the
// fixed-order FP32 expressions that decide integers (k-NN selection,
// projection, threshold tests).
//
// Dual quaternion layout: two float4 per node, real part (w, x, y, z) then
// dual part (w, x, y, z).  A rigid motion x -> R x + t is (q, ½ (0, t) ⊗ q).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sw {

// ---------------------------------------------------------------- vectors

__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- exact-order FP32
// These expressions decide integers and are evaluated in FP32
// round-to-nearest with no contraction, in exactly this order, so that any
// implementation doing the same operations on the same inputs gets the same
// bits.

// ((dx*dx) + (dy*dy)) + (dz*dz)
__device__ __forceinline__ float dist2_rn(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by), dz = __fsub_rn(az, bz);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}
// ((ax*bx) + (ay*by)) + (az*bz)
__device__ __forceinline__ float dot_rn(float3 a, float3 b) {
  return __fadd_rn(__fadd_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)), __fmul_rn(a.z, b.z));
}
// ((f * x) / z) + c
__device__ __forceinline__ float project_rn(float f, float x, float z, float c) {
  return __fadd_rn(__fdiv_rn(__fmul_rn(f, x), z), c);
}

// ---------------------------------------------------------------- quaternions

struct DQ {  // an unnormalised dual quaternion b = b0 + ε be
  float W; float3 A;    // real part
  float We; float3 Ae;  // dual part
};

__device__ __forceinline__ float4 qmul(float4 a, float4 b) {
  return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                     a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                     a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                     a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}
// NOTE: float4 quaternions here store (w, x, y, z) in (.x, .y, .z, .w).

__device__ __forceinline__ float qdot(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }

// Σ_k w_k s_k q̂_k over 4 nodes (Eq. 1); s_k = sign(<real_k, real_ref>), sign(0)=+1.
__device__ __forceinline__ DQ blend4(const float4* __restrict__ dq, int4 ids, float4 w, int ref_slot) {
  const int id[4] = {ids.x, ids.y, ids.z, ids.w};
  const float wk[4] = {w.x, w.y, w.z, w.w};
  const float4 qref = __ldg(dq + 2 * id[ref_slot]);
  DQ b;
  b.W = 0.f; b.A = make_float3(0.f, 0.f, 0.f); b.We = 0.f; b.Ae = make_float3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 q0 = __ldg(dq + 2 * id[k]);
    const float4 qe = __ldg(dq + 2 * id[k] + 1);
    const float s = qdot(q0, qref) >= 0.f ? wk[k] : -wk[k];
    b.W += s * q0.x; b.A.x += s * q0.y; b.A.y += s * q0.z; b.A.z += s * q0.w;
    b.We += s * qe.x; b.Ae.x += s * qe.y; b.Ae.y += s * qe.z; b.Ae.z += s * qe.w;
  }
  return b;
}

__device__ __forceinline__ DQ load_dq(const float4* __restrict__ dq, int j) {
  const float4 q0 = dq[2 * j], qe = dq[2 * j + 1];
  DQ b;
  b.W = q0.x; b.A = make_float3(q0.y, q0.z, q0.w);
  b.We = qe.x; b.Ae = make_float3(qe.y, qe.z, qe.w);
  return b;
}

__device__ __forceinline__ float dq_norm2(const DQ& b) { return b.W * b.W + dot3(b.A, b.A); }

// p' = W(x) p with the normalisation of Eq. 1 folded in (n2 = |b0|²):
//   R(c0) p = p + (2/n2) (A × (A × p) + W A × p)
//   t       = (2/n2) (W Aε − Wε A + A × Aε)
__device__ __forceinline__ float3 dq_rotate(const DQ& b, float inv_n2, float3 p) {
  const float3 axp = cross3(b.A, p);
  return p + (2.f * inv_n2) * (cross3(b.A, axp) + b.W * axp);
}
__device__ __forceinline__ float3 dq_translation(const DQ& b, float inv_n2) {
  return (2.f * inv_n2) * (b.W * b.Ae - b.We * b.A + cross3(b.A, b.Ae));
}
__device__ __forceinline__ float3 dq_transform(const DQ& b, float inv_n2, float3 p) {
  return dq_rotate(b, inv_n2, p) + dq_translation(b, inv_n2);
}
// R⁻¹ y: rotation by the conjugate real part (W, −A)
__device__ __forceinline__ float3 dq_inv_rotate(const DQ& b, float inv_n2, float3 y) {
  const float3 axy = cross3(b.A, y);
  return y + (2.f * inv_n2) * (cross3(b.A, axy) - b.W * axy);
}

// g = n_dᵀ ∂p'/∂b (8 values: gW, gA, gWe, gAe) for p' = p + (2/n2) h.
struct DQGrad { float gW; float3 gA; float gWe; float3 gAe; };

__device__ __forceinline__ DQGrad point_plane_grad(const DQ& b, float inv_n2, float3 p, float3 n) {
  const float3 axp = cross3(b.A, p);
  const float3 h = cross3(b.A, axp) + b.W * axp + b.W * b.Ae - b.We * b.A + cross3(b.A, b.Ae);
  const float nh = dot3(n, h);
  const float c2 = 2.f * inv_n2, c4 = 4.f * inv_n2 * inv_n2 * nh;
  const float ap = dot3(b.A, p), na = dot3(n, b.A), np_ = dot3(n, p);
  DQGrad g;
  g.gW = c2 * dot3(n, axp + b.Ae) - c4 * b.W;
  const float3 raw = ap * n + na * p - (2.f * np_) * b.A - b.W * cross3(n, p) - b.We * n - cross3(n, b.Ae);
  g.gA = c2 * raw - c4 * b.A;
  g.gWe = -c2 * na;
  g.gAe = c2 * (b.W * n + cross3(n, b.A));
  return g;
}

// gᵀ L(q) with L(q) = [−aᵀ; w I − [a]×] (4x3): w g_v + a × g_v − g_w a
__device__ __forceinline__ float3 lmul(float gw, float3 gv, float4 q) {
  const float3 a = make_float3(q.y, q.z, q.w);
  return q.x * gv + cross3(a, gv) - gw * a;
}

// ∂r/∂ξ_k (6 values) for the node k with dual quaternion (q0, qe), blend
// coefficient ws = w_k s_k:  ω = ½ (g0ᵀL(q0) + geᵀL(qe)),  τ = ½ geᵀL(q0).
__device__ __forceinline__ void node_jacobian(const DQGrad& g, float4 q0, float4 qe, float ws, float* out6) {
  const float3 om = lmul(g.gW, g.gA, q0) + lmul(g.gWe, g.gAe, qe);
  const float3 ta = lmul(g.gWe, g.gAe, q0);
  const float h = 0.5f * ws;
  out6[0] = h * om.x; out6[1] = h * om.y; out6[2] = h * om.z;
  out6[3] = h * ta.x; out6[4] = h * ta.y; out6[5] = h * ta.z;
}

// The increment Δ = (R(ω), τ) as a dual quaternion, composed on the left and
// re-normalised: unit real part, dual part orthogonal to it.
__device__ __forceinline__ void apply_increment(float4& q0, float4& qe, const float* xi) {
  const float ox = xi[0], oy = xi[1], oz = xi[2];
  const float th2 = ox * ox + oy * oy + oz * oz;
  float4 r;
  if (th2 > 0.f) {
    const float th = sqrtf(th2);
    float s, c;
    sincosf(0.5f * th, &s, &c);
    const float k = s / th;
    r = make_float4(c, k * ox, k * oy, k * oz);
  } else {
    r = make_float4(1.f, 0.f, 0.f, 0.f);
  }
  const float4 t4 = make_float4(0.f, xi[3], xi[4], xi[5]);
  float4 de = qmul(t4, r);
  de.x *= 0.5f; de.y *= 0.5f; de.z *= 0.5f; de.w *= 0.5f;
  float4 n0 = qmul(r, q0);
  const float4 a = qmul(r, qe), b = qmul(de, q0);
  float4 ne = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
  const float inv = 1.f / sqrtf(qdot(n0, n0));   // exact for an exactly unit real part
  n0.x *= inv; n0.y *= inv; n0.z *= inv; n0.w *= inv;
  ne.x *= inv; ne.y *= inv; ne.z *= inv; ne.w *= inv;
  const float d = qdot(n0, ne);
  ne.x -= d * n0.x; ne.y -= d * n0.y; ne.z -= d * n0.z; ne.w -= d * n0.w;
  q0 = n0; qe = ne;
}

}  // namespace sw
