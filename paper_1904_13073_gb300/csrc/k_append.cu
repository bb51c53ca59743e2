// Surfel appending after fusion: live skinning with the consistency test of
// Eq. 7 (Sec. 6.2), the compressive-warp bound of Eq. 8 (Sec. 6.3), the
// weight-sum test, appending and the removal of unstable surfels (Sec. 6.4),
// and the GPU selection that compacts the surfel array (Sec. 6.6).
//
//   k_live_nodes    p̂_j = T_j p_j in FP64, rounded to FP32 (the precision the
//                   k-NN and Eq. 7 decide in); w carries σ_j.
//   k_cand_flags    a pixel is a candidate when fusion found it usable with
//                   an empty window (kTargetEmptyWindow).
//   scan + scatter  candidate pixels in row-major order (an exclusive scan of
//                   the flags, then a scatter: order-preserving, deterministic).
//   k_cand_queries  the candidates' depth vertices, for the skinning k-NN
//                   kernel (4 nearest warped nodes, FP32 distances in a fixed
//                   order, ties to the lower id; slot 0 is node_0).
//   k_append_eval   one thread per candidate:
//                     Eq. 7 on squares in exact-order FP32:
//                       (1−ε)² d_ref² < d_live² < (1+ε)² d_ref²;
//                     weights at the live frame, w_i = exp(−‖x − p̂_i‖²/2σ_i²)
//                     for the nodes that stay (FP64); the weight-sum test;
//                     the blend (signs against node_0, Eq. 1) and the inverse
//                     warp (Eq. 3) of the depth vertex and normal (FP64);
//                     the strain ∂x_ref/∂x_live by central differences with
//                     the node set and signs held and the weights
//                     re-evaluated; Eq. 8 as λ_max(JᵀJ) < (1+ε)², i.e.
//                     (1+ε)² I − JᵀJ positive definite, read off the pivots
//                     of its LDLᵀ factorisation.
//   k_stay_flags    an existing surfel stays unless c < δ_stable and
//                   t_now − t_init ≥ t_low_confid (flag at its caller index).
//   k_compose_*     the new model in caller order: the survivors in their
//                   order, then the accepted candidates in pixel order.

#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_math64.cuh"

namespace sw {
namespace {

__device__ __forceinline__ DQ64 node_dq64(const SwDev& d, int j) {
  if (d.dq64) return load_dq64(d.dq64, j);
  const float4 a = d.dq[2 * j], b = d.dq[2 * j + 1];
  return DQ64{a.x, D3{a.y, a.z, a.w}, b.x, D3{b.y, b.z, b.w}};
}

// R⁻¹ y for the rotation of the normalised real part: conjugate (W, −A)
__device__ __forceinline__ D3 inv_rotate64(const DQ64& b, double inv_n2, D3 y) {
  const D3 axy = cross3(b.A, y);
  return y + (2.0 * inv_n2) * (cross3(b.A, axy) - b.W * axy);
}

__device__ __forceinline__ double comp(const D3& v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// The live skinning of one candidate: its 4 nodes' transforms with the signs
// of Eq. 1 folded in, their warped positions, σ and which of them Eq. 7 keeps.
struct LiveSkin {
  DQ64 q[4];
  D3 p[4];
  double s[4];
  bool keep[4];

  __device__ double weights(D3 x, double* w) const {
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const D3 e = x - p[k];
      w[k] = keep[k] ? exp(-dot3(e, e) / (2.0 * s[k] * s[k])) : 0.0;
      sum += w[k];
    }
    return sum;
  }
  // x_ref = b⁻¹ x with b = Σ w_k q_k; an all-zero blend leaves the point in place
  __device__ D3 inverse(D3 x, const double* w, D3* n_in = nullptr, D3* n_out = nullptr) const {
    DQ64 b{0.0, D3{0.0, 0.0, 0.0}, 0.0, D3{0.0, 0.0, 0.0}};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      b.W += w[k] * q[k].W; b.A = b.A + w[k] * q[k].A;
      b.We += w[k] * q[k].We; b.Ae = b.Ae + w[k] * q[k].Ae;
    }
    const double n2 = dq_norm2(b);
    if (!(n2 > 0.0)) {
      if (n_out) *n_out = *n_in;
      return x;
    }
    const double inv = 1.0 / n2;
    if (n_out) *n_out = inv_rotate64(b, inv, *n_in);
    return inv_rotate64(b, inv, x - dq_translation(b, inv));
  }
};

__global__ void k_live_nodes(SwDev d, float4* __restrict__ live) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.n_n) return;
  const DQ64 q = node_dq64(d, j);
  const float4 p = d.node_p[j];
  const double n2 = dq_norm2(q);
  const D3 y = n2 > 0.0 ? dq_transform(q, 1.0 / n2, d3(p)) : d3(p);
  live[j] = make_float4((float)y.x, (float)y.y, (float)y.z, p.w);
}

__global__ void k_cand_flags(SwDev d, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d.W * d.H) flag[i] = d.fuse_target[i] == kTargetEmptyWindow ? 1 : 0;
}

__global__ void k_acc_flags(AppendBufs a, int n_cand, int* __restrict__ flag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cand) flag[c] = (a.flags[c] & kAppAccepted) ? 1 : 0;
}

// out[pos[i]] = i for flagged i; the count goes to *count
__global__ void k_scatter(const int* __restrict__ flag, const int* __restrict__ pos, int n, int* __restrict__ out,
                          int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i] && out) out[pos[i]] = i;
  if (i == n - 1) *count = pos[i] + flag[i];
}

__global__ void k_cand_queries(SwDev d, AppendBufs a, int n_cand) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n_cand) a.query[c] = d.vmap[checked(a.cand[c], (long long)d.W * d.H, d.status)];
}

__global__ void __launch_bounds__(64) k_append_eval(SwDev d, AppendBufs a, AppendParams ap, int n_cand) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cand) return;
  const int pix = checked(a.cand[c], (long long)d.W * d.H, d.status);
  const float4 V = d.vmap[pix], N = d.nmap[pix];
  int id[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) id[k] = checked(a.knn[4 * c + k], d.n_n, d.status);
  LiveSkin sk;
  int flags = 1;
  {   // Eq. 7 on squares, exact-order FP32; node_0 always stays
    const float4 l0 = a.live[id[0]], r0 = d.node_p[id[0]];
    sk.keep[0] = true;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      const float4 l = a.live[id[k]], r = d.node_p[id[k]];
      const float dl = dist2_rn(l.x, l.y, l.z, l0.x, l0.y, l0.z);
      const float dr = dist2_rn(r.x, r.y, r.z, r0.x, r0.y, r0.z);
      sk.keep[k] = dl > __fmul_rn(ap.lo2, dr) && dl < __fmul_rn(ap.hi2, dr);
      if (sk.keep[k]) flags |= 1 << k;
    }
  }
  const DQ64 q0 = node_dq64(d, id[0]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    DQ64 q = node_dq64(d, id[k]);
    if (q.W * q0.W + dot3(q.A, q0.A) < 0.0) {   // sign of Eq. 1 against node_0, sign(0) = +1
      q.W = -q.W; q.A = -1.0 * q.A; q.We = -q.We; q.Ae = -1.0 * q.Ae;
    }
    sk.q[k] = q;
    const float4 l = a.live[id[k]];
    sk.p[k] = d3(l);
    sk.s[k] = (double)l.w;
  }
  const D3 x = d3(V);
  D3 n_in = d3(N), n_ref;
  double w[4];
  const double wsum = sk.weights(x, w);
  const D3 v_ref = sk.inverse(x, w, &n_in, &n_ref);
  // strain: column e is (x_ref(x + h e) − x_ref(x − h e)) / 2h
  double J[9];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const D3 de = D3{e == 0 ? ap.h : 0.0, e == 1 ? ap.h : 0.0, e == 2 ? ap.h : 0.0};
    double wp[4], wm[4];
    const D3 xp = x + de, xm = x - de;
    sk.weights(xp, wp);
    sk.weights(xm, wm);
    const D3 yp = sk.inverse(xp, wp), ym = sk.inverse(xm, wm);
#pragma unroll
    for (int r = 0; r < 3; ++r) J[3 * r + e] = (comp(yp, r) - comp(ym, r)) / (2.0 * ap.h);
  }
  // Eq. 8: M = (1+ε)² I − JᵀJ must be positive definite (LDLᵀ pivots > 0)
  double S[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) S[i][j] = J[i] * J[j] + J[3 + i] * J[3 + j] + J[6 + i] * J[6 + j];
  const double m00 = ap.bound2 - S[0][0], m11 = ap.bound2 - S[1][1], m22 = ap.bound2 - S[2][2];
  const double m10 = -S[1][0], m20 = -S[2][0], m21 = -S[2][1];
  bool pd = m00 > 0.0;
  if (pd) {
    const double d1 = m11 - m10 * m10 / m00;
    pd = d1 > 0.0;
    if (pd) {
      const double l21 = (m21 - m20 * m10 / m00) / d1;
      const double d2 = m22 - m20 * m20 / m00 - l21 * l21 * d1;
      pd = d2 > 0.0;
    }
  }
  const bool low = !(wsum >= ap.delta_nn);
  const bool compressive = !pd;
  if (low) { flags |= kAppLowWeight; atomicAdd(a.counts + kAppNLow, 1); }
  if (compressive) { flags |= kAppCompressive; atomicAdd(a.counts + kAppNComp, 1); }
  if (!low && !compressive) flags |= kAppAccepted;
  a.flags[c] = flags;
  a.wsum[c] = wsum;
#pragma unroll
  for (int k = 0; k < 9; ++k) a.strain[9 * (size_t)c + k] = J[k];
  a.w[c] = make_float4((float)w[0], (float)w[1], (float)w[2], (float)w[3]);
  a.v[c] = make_float4((float)v_ref.x, (float)v_ref.y, (float)v_ref.z, N.w);
  a.n[c] = make_float4((float)n_ref.x, (float)n_ref.y, (float)n_ref.z, V.w);
}

__global__ void k_stay_flags(SwDev d, int t_low, int* __restrict__ stay) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_s) return;
  const float c = d.n_ref[i].w;
  const int age = *d.t_now - d.tt[i].x;
  stay[d.orig_id[i]] = (c < d.stable_conf && age >= t_low) ? 0 : 1;
}

__global__ void k_compose_stay(SwDev d, AppendBufs a, const int4* __restrict__ knn_dist,
                               const float4* __restrict__ w_dist, float4* tv, float4* tn, int2* tt, int4* tknn,
                               float4* tw) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= d.n_s || !a.stay[o]) return;
  const int j = a.pos[o], i = checked(d.inv_perm[o], d.n_s, d.status);
  tv[j] = d.v_ref[i];
  tn[j] = d.n_ref[i];
  tt[j] = d.tt[i];
  tknn[j] = knn_dist[o];
  tw[j] = w_dist[o];
}

__global__ void k_compose_app(SwDev d, AppendBufs a, int n_stay, int n_app, float4* tv, float4* tn, int2* tt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_app) return;
  const int c = a.acc[k], j = n_stay + k;
  tv[j] = a.v[c];
  tn[j] = a.n[c];
  const int t = *d.t_now;
  tt[j] = make_int2(t, t);
}

inline int blocks(int n, int t) { return (n + t - 1) / t; }

// order-preserving compaction of flag[0, n): out[k] = k-th flagged index
cudaError_t compact(const AppendBufs& a, const int* flag, int n, int* out, int* count, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
  if (e != cudaSuccess || n == 0) return e;
  e = scan_sum(flag, a.pos, n, false, a.scan_tmp, a.scan_bytes, st, true);   // cleared at allocation
  if (e != cudaSuccess) return e;
  k_scatter<<<blocks(n, 256), 256, 0, st>>>(flag, a.pos, n, out, count);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ node-graph extension
// (Sec. 6.4, last paragraph): coverage of the appended reference surfels by
// the node radii, greedy sub-sampling of the uncovered ones into new nodes,
// their transforms from the current warp, and each surfel's set compared
// with the new nodes.  Distances that decide are exact-order FP32.

// a warp per appended surfel: 1 when no node j has ‖v − p_j‖² < σ_j²
__global__ void k_node_cover(SwDev d, const float4* __restrict__ tv, int first, int n, int* __restrict__ unc) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= n) return;
  const float4 v = tv[first + k];
  bool cov = false;
  for (int j = lane; j < d.n_n && !cov; j += 32) {
    const float4 p = __ldg(d.node_p + j);
    cov = dist2_rn(v.x, v.y, v.z, p.x, p.y, p.z) < __fmul_rn(p.w, p.w);
  }
  cov = __any_sync(0xffffffffu, cov);
  if (lane == 0) unc[k] = cov ? 0 : 1;
}

// a warp per uncovered surfel: σ of its nearest old node (ties to the lower
// id) and whether some old node lies within that σ
__global__ void k_node_near(SwDev d, const float4* __restrict__ tv, int first, const int* __restrict__ list,
                            const int* __restrict__ n_list, float* __restrict__ sig, int* __restrict__ near) {
  const int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (u >= *n_list) return;
  const float4 v = tv[first + list[u]];
  float bd = __int_as_float(0x7f800000);
  int bi = 0x7fffffff;
  for (int j = lane; j < d.n_n; j += 32) {
    const float4 p = __ldg(d.node_p + j);
    const float d2 = dist2_rn(p.x, p.y, p.z, v.x, v.y, v.z);
    if (d2 < bd || (d2 == bd && j < bi)) { bd = d2; bi = j; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float od = __shfl_xor_sync(0xffffffffu, bd, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (od < bd || (od == bd && oi < bi)) { bd = od; bi = oi; }
  }
  const float s = __ldg(d.node_p + bi).w, s2 = __fmul_rn(s, s);
  bool close = false;
  for (int j = lane; j < d.n_n && !close; j += 32) {
    const float4 p = __ldg(d.node_p + j);
    close = dist2_rn(p.x, p.y, p.z, v.x, v.y, v.z) < s2;
  }
  close = __any_sync(0xffffffffu, close);
  if (lane == 0) { sig[u] = s; near[u] = close ? 1 : 0; }
}

// The greedy pass only needs the uncovered surfels that no old node is near:
// their flag, then (after an order-preserving compaction) their position and
// σ packed as one float4 each.
__global__ void k_node_free_flags(const int* __restrict__ near, const int* __restrict__ n_list, int n,
                                  int* __restrict__ flag) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) flag[u] = (u < *n_list && !near[u]) ? 1 : 0;
}

__global__ void k_node_pack(const float4* __restrict__ tv, int first, const int* __restrict__ list,
                            const float* __restrict__ sig, const int* __restrict__ free_idx,
                            const int* __restrict__ n_free, float4* __restrict__ cand) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= *n_free) return;
  const int u = free_idx[k];
  const float4 v = tv[first + list[u]];
  cand[k] = make_float4(v.x, v.y, v.z, sig[u]);
}

// One warp, in order: candidate k becomes node n_old + count unless a node
// taken before it lies within its σ.  Chunks of 32 candidates (one coalesced
// load, the next chunk's issued before the current one is worked on): each
// lane first tests its candidate against the nodes taken before the chunk
// (kept in shared memory); the survivors are then taken or rejected in lane
// order against the nodes taken inside the chunk.  At most kMaxNewNodes per
// call.
constexpr int kMaxNewNodes = 2048;

__global__ void __launch_bounds__(32) k_node_greedy(SwDev d, const float4* __restrict__ cand,
                                                    const int* __restrict__ n_cand, int n_old, int max_new,
                                                    int* __restrict__ n_new) {
  __shared__ float4 taken[kMaxNewNodes];
  const int lane = threadIdx.x & 31;
  const int n = *n_cand, cap = min(max_new, kMaxNewNodes);
  int count = 0;
  float4 next = lane < n ? cand[lane] : make_float4(0.f, 0.f, 0.f, 0.f);
  for (int base = 0; base < n && count < cap; base += 32) {
    const float4 v = next;
    const bool mine = base + lane < n;
    if (base + 32 + lane < n) next = cand[base + 32 + lane];
    const float s2 = __fmul_rn(v.w, v.w);
    bool close = false;
    for (int k = 0; k < count; ++k) {   // every lane its own candidate against the earlier nodes
      const float4 p = taken[k];
      close = close || dist2_rn(p.x, p.y, p.z, v.x, v.y, v.z) < s2;
    }
    unsigned m = __ballot_sync(0xffffffffu, mine && !close);
    const int count0 = count;
    while (m && count < cap) {
      const int b = __ffs(m) - 1;
      m &= m - 1;
      const float vx = __shfl_sync(0xffffffffu, v.x, b), vy = __shfl_sync(0xffffffffu, v.y, b);
      const float vz = __shfl_sync(0xffffffffu, v.z, b), vs = __shfl_sync(0xffffffffu, v.w, b);
      const float t2 = __fmul_rn(vs, vs);
      bool c2 = false;
      for (int k = count0 + lane; k < count; k += 32) {
        const float4 p = taken[k];
        c2 = c2 || dist2_rn(p.x, p.y, p.z, vx, vy, vz) < t2;
      }
      c2 = __any_sync(0xffffffffu, c2);
      if (!c2) {
        if (lane == 0) {
          taken[count] = make_float4(vx, vy, vz, vs);
          d.node_p[n_old + count] = make_float4(vx, vy, vz, vs);
        }
        ++count;
        __syncwarp();
      }
    }
    __syncwarp();
  }
  if (lane == 0) *n_new = count;
}

// a new node's transform: the normalised blend (Eq. 1, FP64) of its 4 nearest
// old nodes with their weights at its position
__global__ void k_new_node_dq(SwDev d, int n_old, int k_new, const int* __restrict__ ids) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= k_new) return;
  const int j = n_old + k;
  const D3 x = d3(d.node_p[j]);
  DQ64 b{0.0, D3{0.0, 0.0, 0.0}, 0.0, D3{0.0, 0.0, 0.0}};
  const DQ64 q0 = node_dq64(d, checked(ids[4 * k], n_old, d.status));
  for (int a = 0; a < 4; ++a) {
    const int id = checked(ids[4 * k + a], n_old, d.status);
    const float4 p = d.node_p[id];
    const D3 e = x - d3(p);
    const double sg = (double)p.w;
    double w = exp(-dot3(e, e) / (2.0 * sg * sg));
    const DQ64 q = node_dq64(d, id);
    if (q.W * q0.W + dot3(q.A, q0.A) < 0.0) w = -w;
    b.W += w * q.W; b.A = b.A + w * q.A; b.We += w * q.We; b.Ae = b.Ae + w * q.Ae;
  }
  const double inv = 1.0 / sqrt(dq_norm2(b));
  double o[8] = {b.W * inv, b.A.x * inv, b.A.y * inv, b.A.z * inv, b.We * inv, b.Ae.x * inv, b.Ae.y * inv, b.Ae.z * inv};
  const double dd = o[0] * o[4] + o[1] * o[5] + o[2] * o[6] + o[3] * o[7];
  for (int c = 0; c < 4; ++c) o[4 + c] -= dd * o[c];
  if (d.dq64)
    for (int c = 0; c < 8; ++c) d.dq64[8 * (size_t)j + c] = o[c];
  d.dq[2 * j] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)o[3]);
  d.dq[2 * j + 1] = make_float4((float)o[4], (float)o[5], (float)o[6], (float)o[7]);
}

// each surfel's set against the nodes n_old .. n_n − 1: the 4 smallest (d², id)
// of the old set and the new nodes at its position; a changed set is written
// in distance order with its Eq. 1 weights, an unchanged one is left alone
__global__ void k_skin_merge(SwDev d, const float4* __restrict__ tv, int n, int n_old, int4* __restrict__ tknn,
                             float4* __restrict__ tw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 v = tv[i];
  const int4 k0 = tknn[i];
  const int old_ids[4] = {k0.x, k0.y, k0.z, k0.w};
  float bd[4];
  int bi[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) { bd[a] = __int_as_float(0x7f800000); bi[a] = 0x7fffffff; }
  auto offer = [&](int id) {
    const float4 p = __ldg(d.node_p + id);
    float cd = dist2_rn(v.x, v.y, v.z, p.x, p.y, p.z);
    int ci = id;
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (cd < bd[a] || (cd == bd[a] && ci < bi[a])) {
        const float td = bd[a]; const int ti = bi[a];
        bd[a] = cd; bi[a] = ci;
        cd = td; ci = ti;
      }
  };
#pragma unroll
  for (int a = 0; a < 4; ++a) offer(old_ids[a]);
  for (int j = n_old; j < d.n_n; ++j) offer(j);
  bool same = true;
#pragma unroll
  for (int a = 0; a < 4; ++a) same = same && bi[a] < n_old;   // no new node entered: the old set stands
  if (same) return;
  float w[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const float sg = __ldg(&d.node_p[bi[a]].w);
    w[a] = expf(-bd[a] / (2.f * sg * sg));
  }
  tknn[i] = make_int4(bi[0], bi[1], bi[2], bi[3]);
  tw[i] = make_float4(w[0], w[1], w[2], w[3]);
}

// ------------------------------------------------------------------ fast model update
// When no surfel is removed and every appended surfel's 4-node set is already
// in the set table, the pattern of JᵀJ does not change: the appended surfels
// are put after the existing ones in the internal order with their set's id.

__device__ __forceinline__ unsigned long long set_key(const int* a) {
  return ((unsigned long long)a[0] << 48) | ((unsigned long long)a[1] << 32) | ((unsigned long long)a[2] << 16) |
         (unsigned long long)a[3];
}
__device__ __forceinline__ unsigned long long slot_key(const SwDev& d, int set) {
  const int* sl = d.set_slots + (size_t)set * 14 + 10;
  return set_key(sl);
}

// the set of each appended surfel (its 4 ids sorted ascending), searched among
// the sets: the first `sorted_sets` are in increasing key order (binary
// search), the ones added since by fast updates follow (a scan); -1 and the
// key in `keys` (~0 for a found one) when it has none; *missing counts them
__global__ void k_find_sets(SwDev d, int sorted_sets, const int4* __restrict__ tknn, int first, int n_app,
                            int* __restrict__ set_of, unsigned long long* __restrict__ keys, int* __restrict__ missing) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_app) return;
  const int4 q = tknn[first + k];
  int a[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3 - x; ++y)
      if (a[y] > a[y + 1]) { const int t = a[y]; a[y] = a[y + 1]; a[y + 1] = t; }
  const unsigned long long key = set_key(a);
  int lo = 0, hi = sorted_sets - 1, found = -1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const unsigned long long mk = slot_key(d, mid);
    if (mk == key) { found = mid; break; }
    if (mk < key) lo = mid + 1; else hi = mid - 1;
  }
  for (int t = sorted_sets; found < 0 && t < d.n_sets; ++t)
    if (slot_key(d, t) == key) found = t;
  set_of[k] = found;
  keys[k] = found < 0 ? key : ~0ull;
  if (found < 0) atomicAdd(missing, 1);
}

// block (a, b), a <= b, of the pattern, or -1 when it has none
__device__ __forceinline__ int find_block_or_none(const SwDev& d, int a, int b) {
  int lo = d.row_ptr[a], hi = d.row_ptr[a + 1] - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (d.col[mid] < b) lo = mid + 1; else hi = mid;
  }
  return d.col[lo] == b ? lo : -1;
}

// head[k] = 1 where sorted key k starts a run of equal keys
__global__ void k_key_heads(const unsigned long long* __restrict__ sorted, int n, int* __restrict__ head) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) head[k] = (k == 0 || sorted[k] != sorted[k - 1]) ? 1 : 0;
}

// the distinct new sets (rank[k] among the distinct sorted keys), each with
// its 10 blocks found in the pattern and written after the n_sets known ones;
// *no_block is set when a pair of nodes has no block (the pattern would have
// to grow)
__global__ void k_new_sets(SwDev d, const unsigned long long* __restrict__ sorted, const int* __restrict__ head,
                           const int* __restrict__ rank, int n_missing, int* __restrict__ n_new_sets,
                           int* __restrict__ no_block) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_missing) return;
  if (k == n_missing - 1) *n_new_sets = rank[k] + head[k];
  if (!head[k]) return;
  const unsigned long long key = sorted[k];
  const int id[4] = {(int)(key >> 48), (int)((key >> 32) & 0xffff), (int)((key >> 16) & 0xffff), (int)(key & 0xffff)};
  int* out = d.set_slots + (size_t)(d.n_sets + rank[k]) * 14;
  int q = 0;
  for (int x = 0; x < 4; ++x)
    for (int y = x; y < 4; ++y) {
      const int blk = find_block_or_none(d, id[x], id[y]);
      if (blk < 0) atomicOr(no_block, 1);
      out[q++] = blk < 0 ? 0 : blk;
    }
  for (int x = 0; x < 4; ++x) out[10 + x] = id[x];
}

// each surfel without a set takes its new set's id: n_sets + the rank of its key
__global__ void k_assign_new_sets(SwDev d, const unsigned long long* __restrict__ keys,
                                  const unsigned long long* __restrict__ sorted, const int* __restrict__ rank,
                                  int n_missing, int n_app, int* __restrict__ set_of) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_app || set_of[k] >= 0) return;
  const unsigned long long key = keys[k];
  int lo = 0, hi = n_missing - 1;
  while (lo < hi) {   // first position of the key
    const int mid = (lo + hi) >> 1;
    if (sorted[mid] < key) lo = mid + 1; else hi = mid;
  }
  set_of[k] = d.n_sets + rank[lo];
}

// the node ids of sets [0, n) from the set table (entries 10-13 of each row)
__global__ void k_slot_sets(const int* __restrict__ slots, int n, int4* __restrict__ sets) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int* r = slots + (size_t)t * 14 + 10;
  sets[t] = make_int4(r[0], r[1], r[2], r[3]);
}

// appended surfel k becomes internal (and caller) index first + k
__global__ void k_append_internal(SwDev d, const float4* __restrict__ tv, const float4* __restrict__ tn,
                                  const int2* __restrict__ tt, const int4* __restrict__ tknn,
                                  const float4* __restrict__ tw, int first, int n_app, const int* __restrict__ set_of) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_app) return;
  const int o = first + k, i = first + k;
  d.v_ref[i] = tv[o];
  d.n_ref[i] = tn[o];
  d.tt[i] = tt[o];
  d.orig_id[i] = o;
  d.inv_perm[o] = i;
  d.set_id[i] = set_of[k];
  const int4 kk = tknn[o];
  const float4 ww = tw[o];
  int id[4] = {kk.x, kk.y, kk.z, kk.w};
  float w[4] = {ww.x, ww.y, ww.z, ww.w};
  int slot0 = 0;   // where the nearest node (distance slot 0) goes
#pragma unroll
  for (int x = 0; x < 3; ++x)
#pragma unroll
    for (int y = 0; y < 3 - x; ++y)
      if (id[y] > id[y + 1]) {
        const int t = id[y]; id[y] = id[y + 1]; id[y + 1] = t;
        const float u = w[y]; w[y] = w[y + 1]; w[y + 1] = u;
        if (slot0 == y) slot0 = y + 1; else if (slot0 == y + 1) slot0 = y;
      }
  d.knn[i] = make_int4(id[0], id[1], id[2], id[3]);
  d.w[i] = make_float4(w[0], w[1], w[2], w[3]);
  d.ref_slot[i] = slot0;
  d.corr_pix[i] = -1;
}

}  // namespace

void launch_find_sets(const SwDev& d, int sorted_sets, const int4* tknn, int first, int n_app, int* set_of,
                      unsigned long long* keys, int* missing, cudaStream_t st) {
  if (n_app) k_find_sets<<<blocks(n_app, 256), 256, 0, st>>>(d, sorted_sets, tknn, first, n_app, set_of, keys, missing);
}

size_t new_sets_scratch_bytes(int n) { return std::max(sort_scratch_bytes_u64(n, false), scan_scratch_bytes(n)); }

cudaError_t launch_new_sets(const SwDev& d, const unsigned long long* keys, unsigned long long* sorted, int* head,
                            int* rank, int n_app, int n_missing, int* set_of, int* n_new_sets, int* no_block,
                            void* tmp, size_t tmp_bytes, cudaStream_t st) {
  // the found surfels' keys are ~0 and sort last: the first n_missing are the new sets' keys
  cudaError_t e = radix_sort_u64(keys, sorted, nullptr, nullptr, n_app, 0, 64, tmp, tmp_bytes, st);
  if (e != cudaSuccess) return e;
  k_key_heads<<<blocks(n_missing, 256), 256, 0, st>>>(sorted, n_missing, head);
  e = scan_sum(head, rank, n_missing, false, tmp, tmp_bytes, st);
  if (e != cudaSuccess) return e;
  k_new_sets<<<blocks(n_missing, 128), 128, 0, st>>>(d, sorted, head, rank, n_missing, n_new_sets, no_block);
  k_assign_new_sets<<<blocks(n_app, 128), 128, 0, st>>>(d, keys, sorted, rank, n_missing, n_app, set_of);
  return cudaGetLastError();
}

void launch_slot_sets(const int* slots, int n, int4* sets, cudaStream_t st) {
  if (n) k_slot_sets<<<blocks(n, 256), 256, 0, st>>>(slots, n, sets);
}

void launch_append_internal(const SwDev& d, const float4* tv, const float4* tn, const int2* tt, const int4* tknn,
                            const float4* tw, int first, int n_app, const int* set_of, cudaStream_t st) {
  if (n_app) k_append_internal<<<blocks(n_app, 256), 256, 0, st>>>(d, tv, tn, tt, tknn, tw, first, n_app, set_of);
}

void launch_node_cover(const SwDev& d, const float4* tv, int first, int n, int* unc, cudaStream_t st) {
  if (n) k_node_cover<<<(int)(((size_t)n * 32 + 127) / 128), 128, 0, st>>>(d, tv, first, n, unc);
}
cudaError_t launch_node_subsample(const SwDev& d, const AppendBufs& a, const float4* tv, int first, int n_app,
                                  const int* unc_flags, int* unc_list, int* n_unc, float* sig, int* near,
                                  int n_old, int max_new, int* n_new, cudaStream_t st) {
  cudaError_t e = compact(a, unc_flags, n_app, unc_list, n_unc, st);
  if (e != cudaSuccess || n_app == 0) return e;
  k_node_near<<<(int)(((size_t)n_app * 32 + 127) / 128), 128, 0, st>>>(d, tv, first, unc_list, n_unc, sig, near);
  // the free ones (no old node near), packed in order; the scratch after the
  // n_app entries of each buffer holds the packed copies
  int* free_flag = const_cast<int*>(unc_flags);   // the coverage flags are consumed
  int* free_idx = near + n_app;
  int* n_free = n_new + 1;
  float4* cand = reinterpret_cast<float4*>(sig + ((n_app + 3) & ~3));   // 16-byte aligned after the σ
  k_node_free_flags<<<blocks(n_app, 256), 256, 0, st>>>(near, n_unc, n_app, free_flag);
  e = compact(a, free_flag, n_app, free_idx, n_free, st);
  if (e != cudaSuccess) return e;
  k_node_pack<<<blocks(n_app, 256), 256, 0, st>>>(tv, first, unc_list, sig, free_idx, n_free, cand);
  k_node_greedy<<<1, 32, 0, st>>>(d, cand, n_free, n_old, max_new, n_new);
  return cudaGetLastError();
}
void launch_new_node_dq(const SwDev& d, int n_old, int k_new, const int* ids, cudaStream_t st) {
  if (k_new) k_new_node_dq<<<(k_new + 63) / 64, 64, 0, st>>>(d, n_old, k_new, ids);
}
void launch_skin_merge(const SwDev& d, const float4* tv, int n, int n_old, int4* tknn, float4* tw, cudaStream_t st) {
  if (n) k_skin_merge<<<(n + 255) / 256, 256, 0, st>>>(d, tv, n, n_old, tknn, tw);
}

size_t append_scan_bytes(int n_pixels, int n_surfels) { return scan_scratch_bytes(std::max(n_pixels, n_surfels)); }

// Steps up to the candidate list: warped nodes, candidate pixels (count in
// counts[kAppNCand]) and their depth vertices are left in `a`.
cudaError_t launch_append_candidates(const SwDev& d, const AppendBufs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.counts, 0, kAppCounts * sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (d.n_n) k_live_nodes<<<blocks(d.n_n, 128), 128, 0, st>>>(d, a.live);
  const int np = d.W * d.H;
  k_cand_flags<<<blocks(np, 256), 256, 0, st>>>(d, a.stay);
  return compact(a, a.stay, np, a.cand, a.counts + kAppNCand, st);
}

cudaError_t launch_append_eval(const SwDev& d, const AppendBufs& a, const AppendParams& ap, int n_cand,
                               cudaStream_t st) {
  if (n_cand == 0) return cudaMemsetAsync(a.counts + kAppNAcc, 0, sizeof(int), st);
  k_cand_queries<<<blocks(n_cand, 256), 256, 0, st>>>(d, a, n_cand);
  launch_knn4(a.query, n_cand, a.live, d.n_n, a.knn, st);
  k_append_eval<<<blocks(n_cand, 64), 64, 0, st>>>(d, a, ap, n_cand);   // small CTAs: spread over every SM
  k_acc_flags<<<blocks(n_cand, 256), 256, 0, st>>>(a, n_cand, a.stay);
  return compact(a, a.stay, n_cand, a.acc, a.counts + kAppNAcc, st);
}

// stay flags in caller order and the survivors' new indices (count in counts[kAppNStay])
cudaError_t launch_append_removal(const SwDev& d, const AppendBufs& a, int t_low, cudaStream_t st) {
  if (d.n_s) k_stay_flags<<<blocks(d.n_s, 256), 256, 0, st>>>(d, t_low, a.stay);
  return compact(a, a.stay, d.n_s, nullptr, a.counts + kAppNStay, st);
}

void launch_append_compose(const SwDev& d, const AppendBufs& a, const int4* knn_dist, const float4* w_dist,
                           int n_stay, int n_app, float4* tv, float4* tn, int2* tt, int4* tknn, float4* tw,
                           cudaStream_t st) {
  if (d.n_s) k_compose_stay<<<blocks(d.n_s, 256), 256, 0, st>>>(d, a, knn_dist, w_dist, tv, tn, tt, tknn, tw);
  if (n_app) k_compose_app<<<blocks(n_app, 256), 256, 0, st>>>(d, a, n_stay, n_app, tv, tn, tt);
}

}  // namespace sw
