// FP64 device math of the all-FP64 solve variant (SW_PRECISION_FP64): the
// same quantities as sw_math.cuh (dual-quaternion blend and warp, Eq. 1-2;
// the point-to-plane gradient through the normalisation, Eq. 10; the
// increment T ← Δ T) evaluated in double precision from the FP32 inputs.
//
// A dual quaternion is 8 doubles: real part (w, x, y, z), dual part (w, x, y, z).
#pragma once
#include <cuda_runtime.h>

namespace sw {

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 d3(double x, double y, double z) { return D3{x, y, z}; }
__device__ __forceinline__ D3 d3(float4 a) { return D3{(double)a.x, (double)a.y, (double)a.z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return D3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return D3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross3(D3 a, D3 b) {
  return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

struct DQ64 {  // an unnormalised dual quaternion b = b0 + ε be
  double W; D3 A;
  double We; D3 Ae;
};

__device__ __forceinline__ DQ64 load_dq64(const double* dq, int j) {
  const double* q = dq + 8 * (size_t)j;
  return DQ64{q[0], D3{q[1], q[2], q[3]}, q[4], D3{q[5], q[6], q[7]}};
}

// Σ_k w_k s_k q̂_k over 4 nodes (Eq. 1); s_k = sign(<real_k, real_ref>), sign(0) = +1.
__device__ __forceinline__ DQ64 blend4_64(const double* dq, int4 ids, float4 w, int ref_slot) {
  const int id[4] = {ids.x, ids.y, ids.z, ids.w};
  const double wk[4] = {(double)w.x, (double)w.y, (double)w.z, (double)w.w};
  const DQ64 ref = load_dq64(dq, id[ref_slot]);
  DQ64 b{0.0, D3{0.0, 0.0, 0.0}, 0.0, D3{0.0, 0.0, 0.0}};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const DQ64 q = load_dq64(dq, id[k]);
    const double s = (q.W * ref.W + dot3(q.A, ref.A)) >= 0.0 ? wk[k] : -wk[k];
    b.W += s * q.W; b.A = b.A + s * q.A;
    b.We += s * q.We; b.Ae = b.Ae + s * q.Ae;
  }
  return b;
}

__device__ __forceinline__ double dq_norm2(const DQ64& b) { return b.W * b.W + dot3(b.A, b.A); }

// p' = p + (2/n2) (A × (A × p) + W A × p) + (2/n2) (W Aε − Wε A + A × Aε)
__device__ __forceinline__ D3 dq_rotate(const DQ64& b, double inv_n2, D3 p) {
  const D3 axp = cross3(b.A, p);
  return p + (2.0 * inv_n2) * (cross3(b.A, axp) + b.W * axp);
}
__device__ __forceinline__ D3 dq_translation(const DQ64& b, double inv_n2) {
  return (2.0 * inv_n2) * (b.W * b.Ae - b.We * b.A + cross3(b.A, b.Ae));
}
__device__ __forceinline__ D3 dq_transform(const DQ64& b, double inv_n2, D3 p) {
  return dq_rotate(b, inv_n2, p) + dq_translation(b, inv_n2);
}

// g = n_dᵀ ∂p'/∂b for p' = p + (2/n2) h (8 values: gW, gA, gWe, gAe)
struct DQGrad64 { double gW; D3 gA; double gWe; D3 gAe; };

__device__ __forceinline__ DQGrad64 point_plane_grad(const DQ64& b, double inv_n2, D3 p, D3 n) {
  const D3 axp = cross3(b.A, p);
  const D3 h = cross3(b.A, axp) + b.W * axp + b.W * b.Ae - b.We * b.A + cross3(b.A, b.Ae);
  const double nh = dot3(n, h);
  const double c2 = 2.0 * inv_n2, c4 = 4.0 * inv_n2 * inv_n2 * nh;
  const double ap = dot3(b.A, p), na = dot3(n, b.A), np_ = dot3(n, p);
  DQGrad64 g;
  g.gW = c2 * dot3(n, axp + b.Ae) - c4 * b.W;
  const D3 raw = ap * n + na * p - (2.0 * np_) * b.A - b.W * cross3(n, p) - b.We * n - cross3(n, b.Ae);
  g.gA = c2 * raw - c4 * b.A;
  g.gWe = -c2 * na;
  g.gAe = c2 * (b.W * n + cross3(n, b.A));
  return g;
}

// gᵀ L(q) with L(q) = [−aᵀ; w I − [a]×]: w g_v + a × g_v − g_w a
__device__ __forceinline__ D3 lmul(double gw, D3 gv, double qw, D3 qa) {
  return qw * gv + cross3(qa, gv) - gw * qa;
}

// ∂r/∂ξ_k for the node with dual quaternion q (8 doubles) and blend
// coefficient ws = w_k s_k: ω = ½ (g0ᵀL(q0) + geᵀL(qe)), τ = ½ geᵀL(q0).
__device__ __forceinline__ void node_jacobian(const DQGrad64& g, const DQ64& q, double ws, double* out6) {
  const D3 om = lmul(g.gW, g.gA, q.W, q.A) + lmul(g.gWe, g.gAe, q.We, q.Ae);
  const D3 ta = lmul(g.gWe, g.gAe, q.W, q.A);
  const double h = 0.5 * ws;
  out6[0] = h * om.x; out6[1] = h * om.y; out6[2] = h * om.z;
  out6[3] = h * ta.x; out6[4] = h * ta.y; out6[5] = h * ta.z;
}

// Hamilton product of (w, x, y, z) quaternions
__device__ __forceinline__ void qmul64(const double* a, const double* b, double* o) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// T ← Δ T with Δ = (R(ω), τ) by Rodrigues' formula, then re-normalised:
// unit real part, dual part orthogonal to it.
__device__ __forceinline__ void apply_increment64(double* q, const double* xi) {
  const double th2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
  double r[4] = {1.0, 0.0, 0.0, 0.0};
  if (th2 > 0.0) {
    const double th = sqrt(th2);
    double s, c;
    sincos(0.5 * th, &s, &c);
    const double k = s / th;
    r[0] = c; r[1] = k * xi[0]; r[2] = k * xi[1]; r[3] = k * xi[2];
  }
  const double t4[4] = {0.0, xi[3], xi[4], xi[5]};
  double de[4];
  qmul64(t4, r, de);
  for (int c = 0; c < 4; ++c) de[c] *= 0.5;
  double n0[4], a[4], b[4];
  qmul64(r, q, n0);
  qmul64(r, q + 4, a);
  qmul64(de, q, b);
  double ne[4] = {a[0] + b[0], a[1] + b[1], a[2] + b[2], a[3] + b[3]};
  const double inv = 1.0 / sqrt(n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2] + n0[3] * n0[3]);
  for (int c = 0; c < 4; ++c) { n0[c] *= inv; ne[c] *= inv; }
  const double d = n0[0] * ne[0] + n0[1] * ne[1] + n0[2] * ne[2] + n0[3] * ne[3];
  for (int c = 0; c < 4; ++c) { q[c] = n0[c]; q[4 + c] = ne[c] - d * n0[c]; }
}

}  // namespace sw
