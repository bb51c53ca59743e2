// Rigid pre-alignment before the non-rigid solve (Sec. 7: a rigid alignment
// in the manner of KinectFusion): point-to-plane ICP of the warped model
// against the live depth, one rigid transform T per stream, composed into
// every node transform at the end.
//
//   k_rigid_begin   T = identity.
//   k_rigid_reduce  one thread per surfel: warp (Eq. 1-2), move by T,
//                   associate exactly as the non-rigid solve does, and form
//                   the residual r = n_dᵀ(T x − v_d) and its Jacobian
//                   J = ((T x) × n_d, n_d) in a left increment (ω, τ) of T;
//                   the CTA sums the 21 upper entries of J Jᵀ, the 6 of J r,
//                   the count and r² into one partial row (plain stores, no
//                   atomics).
//   k_rigid_solve   one CTA per stream, a warp per sum: adds its tiles'
//                   partial rows in a fixed order in double-float pairs,
//                   then one thread solves the 6x6 system by Cholesky and
//                   updates T ← Δ(ξ) T (FP64); a system that is not positive
//                   definite stops the iterations with T as it is.
//   k_rigid_fold    T_j ← T T_j for every node.
#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_math64.cuh"
#include "sw_assoc.cuh"
#include "sw_df.cuh"

namespace sw {
namespace {

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ DQ rigid_dq(const double* T) {
  DQ b;
  b.W = (float)T[0]; b.A = make_float3((float)T[1], (float)T[2], (float)T[3]);
  b.We = (float)T[4]; b.Ae = make_float3((float)T[5], (float)T[6], (float)T[7]);
  return b;
}

__global__ void k_rigid_begin(Batch bt) {
  const int s = blockIdx.x;
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  if (threadIdx.x < kRigidSlots) d.rigid[threadIdx.x] = threadIdx.x == 0 ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(kSurfTile) k_rigid_reduce(Batch bt, int it) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int tile = blockIdx.x - __ldg(bt.tile_base + s);
  const int i = tile * kSurfTile + threadIdx.x;
  float v[kRigidSums];
#pragma unroll
  for (int k = 0; k < kRigidSums; ++k) v[k] = 0.f;
  if (d.rigid[8] == 0.0 && i < d.n_s) {   // not stopped
    const DQ b = blend4(d.dq, checked4(d.knn[i], d.n_n, d.status), d.w[i], checked(d.ref_slot[i], 4, d.status));
    const float n2 = dq_norm2(b);
    if (n2 > 0.f) {
      const float inv = 1.f / n2;
      const float4 v4 = d.v_ref[i], n4 = d.n_ref[i];
      const DQ T = rigid_dq(d.rigid);
      const float3 y = dq_transform(T, 1.f, dq_transform(b, inv, f3(v4)));
      const float3 ny = dq_rotate(T, 1.f, dq_rotate(b, inv, f3(n4)));
      int pix = -1;
      if (surfel_selected(d, *d.t_now, n4.w, d.tt[i].y)) pix = associate_one(d, y, ny);
      if (pix >= 0) {
        const float3 V = f3(d.vmap[pix]), N = f3(d.nmap[pix]);
        const float r = dot3(N, y - V);
        const float3 c = cross3(y, N);
        const float J[6] = {c.x, c.y, c.z, N.x, N.y, N.z};
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int bb = a; bb < 6; ++bb) v[k++] = J[a] * J[bb];   // upper triangle, row-major
#pragma unroll
        for (int a = 0; a < 6; ++a) v[21 + a] = J[a] * r;
        v[27] = 1.f;
        v[28] = r * r;
      }
    }
  }
  __shared__ float sw_part[kSurfTile / 32][kRigidSums];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kRigidSums; ++k) {
    const float t = warp_sum_f(v[k]);
    if (lane == 0) sw_part[wid][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < kRigidSums) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kSurfTile / 32; ++w) t += sw_part[w][threadIdx.x];
    d.rigid_part[(size_t)tile * kRigidSums + threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(32 * kRigidSums) k_rigid_solve(Batch bt, int it) {
  const int s = blockIdx.x;
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int tiles = (d.n_s + kSurfTile - 1) / kSurfTile;
  __shared__ double tot[kRigidSums];
  {   // warp w sums value w over the tiles (lanes stride, then a butterfly): a fixed order
    DF acc = df_from(0.f);
    for (int k = lane; k < tiles; k += 32) acc = df_add(acc, df_from(d.rigid_part[(size_t)k * kRigidSums + wid]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = df_add(acc, df_shfl_xor(acc, o));
    if (lane == 0) tot[wid] = df_value(acc);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  d.rigid_stats[2 * it] = tot[27];
  d.rigid_stats[2 * it + 1] = tot[28];
  if (d.rigid[8] != 0.0) return;   // stopped earlier
  double A[6][6], g[6];
  int k = 0;
  for (int a = 0; a < 6; ++a)
    for (int b = a; b < 6; ++b) { A[a][b] = A[b][a] = tot[k++]; }
  for (int a = 0; a < 6; ++a) g[a] = tot[21 + a];
  // Cholesky A = L Lᵀ; a system that is not positive definite stops the iterations
  double L[6][6] = {};
  for (int c = 0; c < 6; ++c) {
    double sum = A[c][c];
    for (int q = 0; q < c; ++q) sum -= L[c][q] * L[c][q];
    if (!(sum > 0.0)) { d.rigid[8] = 1.0; return; }
    L[c][c] = sqrt(sum);
    for (int r = c + 1; r < 6; ++r) {
      double t = A[r][c];
      for (int q = 0; q < c; ++q) t -= L[r][q] * L[c][q];
      L[r][c] = t / L[c][c];
    }
  }
  double y[6], xi[6];
  for (int r = 0; r < 6; ++r) {   // L y = −g
    double t = -g[r];
    for (int q = 0; q < r; ++q) t -= L[r][q] * y[q];
    y[r] = t / L[r][r];
  }
  for (int r = 5; r >= 0; --r) {  // Lᵀ ξ = y
    double t = y[r];
    for (int q = r + 1; q < 6; ++q) t -= L[q][r] * xi[q];
    xi[r] = t / L[r][r];
  }
  double T[8];
  for (int q = 0; q < 8; ++q) T[q] = d.rigid[q];
  apply_increment64(T, xi);
  for (int q = 0; q < 8; ++q) d.rigid[q] = T[q];
}

// T_j ← T T_j (dual quaternion product, T on the left), re-normalised
__global__ void k_rigid_fold(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int j = (blockIdx.x - __ldg(bt.tile_base + s)) * kBlkTile + threadIdx.x;
  if (j >= d.n_n) return;
  const double* T = d.rigid;
  double q[8];
  if (d.dq64) {
    for (int c = 0; c < 8; ++c) q[c] = d.dq64[8 * j + c];
  } else {
    const float4 a = d.dq[2 * j], b = d.dq[2 * j + 1];
    q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w; q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
  }
  double r0[4], ra[4], rb[4], out[8];
  qmul64(T, q, r0);          // real part: T0 q0
  qmul64(T, q + 4, ra);      // dual part: T0 qe + Te q0
  qmul64(T + 4, q, rb);
  for (int c = 0; c < 4; ++c) { out[c] = r0[c]; out[4 + c] = ra[c] + rb[c]; }
  const double inv = 1.0 / sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2] + out[3] * out[3]);
  for (int c = 0; c < 8; ++c) out[c] *= inv;
  const double dd = out[0] * out[4] + out[1] * out[5] + out[2] * out[6] + out[3] * out[7];
  for (int c = 0; c < 4; ++c) out[4 + c] -= dd * out[c];
  if (d.dq64)
    for (int c = 0; c < 8; ++c) d.dq64[8 * j + c] = out[c];
  d.dq[2 * j] = make_float4((float)out[0], (float)out[1], (float)out[2], (float)out[3]);
  d.dq[2 * j + 1] = make_float4((float)out[4], (float)out[5], (float)out[6], (float)out[7]);
}

inline Batch with_kind(const BatchHost& b, int kind) {
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kind];
  return bt;
}

}  // namespace

void launch_rigid_align(const BatchHost& b, int iters, cudaStream_t st) {
  if (!b.bt.n_streams) return;
  k_rigid_begin<<<b.bt.n_streams, 32, 0, st>>>(b.bt);
  for (int it = 0; it < iters; ++it) {
    if (b.total_tiles[kTileSurfels])
      k_rigid_reduce<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels), it);
    k_rigid_solve<<<b.bt.n_streams, 32 * kRigidSums, 0, st>>>(b.bt, it);
  }
  if (b.total_tiles[kTileNodes])
    k_rigid_fold<<<b.total_tiles[kTileNodes], kBlkTile, 0, st>>>(with_kind(b, kTileNodes));
}

}  // namespace sw
