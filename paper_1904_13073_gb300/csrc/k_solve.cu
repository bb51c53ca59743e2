// K4-K8: one Gauss-Newton iteration of the non-rigid solve (Sec. 7-8).
//
//   K6 k_reg_assemble   one thread per upper 6x6 block of JᵀJ: writes the
//                       as-rigid-as-possible part (Eq. 11) of that block, and
//                       of Jᵀe on diagonal blocks, with plain stores.  It runs
//                       first and so also initialises the whole system.
//   K4+K5 k_data_assemble  one thread per surfel: dual-quaternion blend and
//                       forward warp (Eq. 1-2), projective association,
//                       point-to-plane residual (Eq. 10) and its 1x24
//                       Jacobian; the CTA then reduces JᵀJ and Jᵀe over runs
//                       of surfels that share one 4-node set (surfels are
//                       stored sorted by that set) and adds each run's ten
//                       6x6 blocks and four 6-vectors to the system with
//                       atomics.
//   K7 k_pcg_*          block-Jacobi PCG on JᵀJ Δ = −Jᵀe: FP64 Cholesky
//                       inverses of the diagonal blocks, FP32 block SpMV and
//                       vector updates, FP64 dot-product reductions.
//   K8 k_apply_update   T_j ← Δ_j T_j and re-normalisation.
#include "sw_internal.h"
#include "sw_math.cuh"

namespace sw {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ bool surfel_selected(const SwDev& d, float conf, int t_obs) {
  return conf > d.stable_conf || (d.t_now - t_obs) <= d.recent_frames;
}

// Projective association of one warped surfel (Sec. 7); -1 if rejected.
// Every test is an exact-order FP32 expression (see sw_math.cuh).
__device__ __forceinline__ int associate_one(const SwDev& d, float3 vl, float3 nl) {
  if (!(vl.z > 0.f)) return -1;
  const float u = project_rn(d.fx, vl.x, vl.z, d.cx);
  const float v = project_rn(d.fy, vl.y, vl.z, d.cy);
  const float px = floorf(__fadd_rn(u, 0.5f)), py = floorf(__fadd_rn(v, 0.5f));
  if (!(px >= 0.f && px < (float)d.W && py >= 0.f && py < (float)d.H)) return -1;
  const int pix = (int)py * d.W + (int)px;
  const float4 V = d.vmap[pix];
  if (!(V.w > 0.f)) return -1;
  const float4 N = d.nmap[pix];
  const float d2 = dist2_rn(vl.x, vl.y, vl.z, V.x, V.y, V.z);
  if (!(d2 < __fmul_rn(d.corr_dist, d.corr_dist))) return -1;
  if (!(dot_rn(nl, f3(N)) > d.corr_normal)) return -1;
  return pix;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum to one atomicAdd (blockDim multiple of 32, <= 1024)
template <typename T>
__device__ __forceinline__ void block_atomic_sum(T v, T* dst) {
  __shared__ T part[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) part[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    T t = lane < nw ? part[lane] : T(0);
    t = warp_sum(t);
    if (lane == 0 && t != T(0)) atomicAdd(dst, t);
  }
}

// J_aᵀ J_b for J_a = [−[xa]× | I], J_b = [−[xb]× | I] (3x6 each), scaled:
//   [[(xa·xb) I − xb xaᵀ, [xa]×], [−[xb]×, I]]
__device__ __forceinline__ void add_reg_pair(float* acc, float s, float3 xa, float3 xb) {
  const float ab = dot3(xa, xb);
  const float a[3] = {xa.x, xa.y, xa.z}, b[3] = {xb.x, xb.y, xb.z};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) acc[p * 6 + q] += s * ((p == q ? ab : 0.f) - b[p] * a[q]);
  // [a]× = [[0,-a2,a1],[a2,0,-a0],[-a1,a0,0]]
  const float ax[9] = {0.f, -a[2], a[1], a[2], 0.f, -a[0], -a[1], a[0], 0.f};
  const float bx[9] = {0.f, -b[2], b[1], b[2], 0.f, -b[0], -b[1], b[0], 0.f};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      acc[p * 6 + 3 + q] += s * ax[p * 3 + q];
      acc[(3 + p) * 6 + q] -= s * bx[p * 3 + q];
    }
#pragma unroll
  for (int p = 0; p < 3; ++p) acc[(3 + p) * 6 + 3 + p] += s;
}

__device__ __forceinline__ float3 node_apply(const SwDev& d, int j, float3 p) {
  const DQ b = load_dq(d.dq, j);
  return dq_transform(b, 1.f / dq_norm2(b), p);
}

// ------------------------------------------------------------------ K6: regulariser

namespace {

__global__ void __launch_bounds__(kBlkTile) k_reg_assemble(Batch bt, int gn_it) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const int b = (blockIdx.x - __ldg(bt.tile_base + s)) * kBlkTile + threadIdx.x;
  if (b == 0) {
    for (int k = 0; k < kRedSlots; ++k) d.red[k] = 0.0;
  }
  float ereg = 0.f;
  if (b < d.nnzb) {
    const int i = d.blk_row[b], j = d.col[b];
    const float sl = d.sqrt_lambda, l = sl * sl;
    float acc[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) acc[k] = 0.f;
    if (i == j) {
      float gj[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      const float3 pj = f3(d.node_p[j]);
      const float3 x = node_apply(d, j, pj);
      for (int e = 0; e < SW_K_GRAPH; ++e) {      // out-edges j -> m
        const int m = d.graph[j * SW_K_GRAPH + e];
        const float3 y = node_apply(d, m, pj);
        const float3 r = sl * (x - y);
        ereg += dot3(r, r);
        add_reg_pair(acc, l, x, x);
        const float3 xr = cross3(x, r);
        gj[0] += sl * xr.x; gj[1] += sl * xr.y; gj[2] += sl * xr.z;
        gj[3] += sl * r.x; gj[4] += sl * r.y; gj[5] += sl * r.z;
      }
      for (int e = d.in_ptr[j]; e < d.in_ptr[j + 1]; ++e) {   // in-edges m -> j
        const int m = d.in_src[e];
        const float3 pm = f3(d.node_p[m]);
        const float3 y = node_apply(d, j, pm);
        const float3 r = sl * (node_apply(d, m, pm) - y);
        add_reg_pair(acc, l, y, y);
        const float3 yr = cross3(y, r);
        gj[0] -= sl * yr.x; gj[1] -= sl * yr.y; gj[2] -= sl * yr.z;
        gj[3] -= sl * r.x; gj[4] -= sl * r.y; gj[5] -= sl * r.z;
      }
#pragma unroll
      for (int k = 0; k < 6; ++k) d.g[6 * j + k] = gj[k];
    } else {
      const int fl = d.blk_edge[b];
      if (fl & 1) {   // edge i -> j: J_i = sl[−[T_i p_i]×|I], J_j = −sl[−[T_j p_i]×|I]
        const float3 pi = f3(d.node_p[i]);
        add_reg_pair(acc, -l, node_apply(d, i, pi), node_apply(d, j, pi));
      }
      if (fl & 2) {   // edge j -> i: J_j = sl[−[T_j p_j]×|I], J_i = −sl[−[T_i p_j]×|I]
        const float3 pj = f3(d.node_p[j]);
        add_reg_pair(acc, -l, node_apply(d, i, pj), node_apply(d, j, pj));
      }
    }
    float4* dst = reinterpret_cast<float4*>(d.A + (size_t)b * 36);
#pragma unroll
    for (int k = 0; k < 9; ++k) dst[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
  }
  block_atomic_sum<double>((double)ereg, d.e_reg + gn_it);
}

// ------------------------------------------------------------------ K4+K5: data term

constexpr int kJS = 25;   // 24 Jacobian entries + residual per term

__global__ void __launch_bounds__(kAsmTile) k_data_assemble(Batch bt, int gn_it, int write_live) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const int tid = threadIdx.x;
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kAsmTile + tid;

  __shared__ float sJ[kAsmTile * kJS];
  __shared__ int sset[kAsmTile];
  __shared__ int sseg_start[kAsmTile + 1];
  __shared__ int sseg_active[kAsmTile];
  __shared__ int swarp_cnt[kAsmTile / 32];

  float* myJ = sJ + tid * kJS;
  int set = -1;
  bool valid = false;
  float res = 0.f;
  if (i < d.n_s) {
    const float4 v4 = d.v_ref[i], n4 = d.n_ref[i];
    const int4 ids = d.knn[i];
    const float4 w = d.w[i];
    const int rs = d.ref_slot[i];
    set = d.set_id[i];
    const DQ b = blend4(d.dq, ids, w, rs);
    const float n2 = dq_norm2(b);
    int pix = -1;
    float3 vl = f3(v4), nl = f3(n4);
    float inv = 0.f;
    if (n2 > 0.f) {
      inv = 1.f / n2;
      vl = dq_transform(b, inv, f3(v4));
      nl = dq_rotate(b, inv, f3(n4));
      if (surfel_selected(d, n4.w, d.tt[i].y)) pix = associate_one(d, vl, nl);
    }
    d.corr_pix[i] = pix;
    if (write_live) {
      d.v_live[i] = make_float4(vl.x, vl.y, vl.z, v4.w);
      d.n_live[i] = make_float4(nl.x, nl.y, nl.z, n4.w);
    }
    if (pix >= 0) {
      valid = true;
      const float4 V = d.vmap[pix], N = d.nmap[pix];
      const float3 nd = f3(N);
      res = dot3(nd, vl - f3(V));
      const DQGrad gr = point_plane_grad(b, inv, f3(v4), nd);
      const int id[4] = {ids.x, ids.y, ids.z, ids.w};
      const float wk[4] = {w.x, w.y, w.z, w.w};
      const float4 qref = __ldg(d.dq + 2 * id[rs]);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 q0 = __ldg(d.dq + 2 * id[k]), qe = __ldg(d.dq + 2 * id[k] + 1);
        const float ws = qdot(q0, qref) >= 0.f ? wk[k] : -wk[k];
        node_jacobian(gr, q0, qe, ws, myJ + 6 * k);
      }
      myJ[24] = res;
    }
  }
  if (!valid) {
#pragma unroll
    for (int k = 0; k < kJS; ++k) myJ[k] = 0.f;
  }
  sset[tid] = set;

  // statistics
  block_atomic_sum<double>((double)(res * res), d.e_depth + gn_it);
  {
    const int c = __syncthreads_count(valid);
    if (tid == 0 && c) atomicAdd(d.n_corr + gn_it, c);
  }

  // segments: maximal runs of equal set id within the tile
  const bool head = (tid == 0) || (sset[tid] != sset[tid - 1]);
  const unsigned hb = __ballot_sync(0xffffffffu, head);
  const int lane = tid & 31, wid = tid >> 5;
  if (lane == 0) swarp_cnt[wid] = __popc(hb);
  __syncthreads();
  int before = 0, nseg = 0;
#pragma unroll
  for (int k = 0; k < kAsmTile / 32; ++k) {
    const int c = swarp_cnt[k];
    if (k < wid) before += c;
    nseg += c;
  }
  const int seg = before + __popc(hb & ((2u << lane) - 1u)) - 1;
  if (head) { sseg_start[seg] = tid; sseg_active[seg] = 0; }
  if (tid == 0) sseg_start[nseg] = kAsmTile;
  __syncthreads();
  if (valid) sseg_active[seg] = 1;
  __syncthreads();

  // work items: (segment, item) with items 0..9 = upper blocks (a<=b), 10..13 = Jᵀe of node a
  const int nitems = nseg * 14;
  for (int it = tid; it < nitems; it += kAsmTile) {
    const int sg = it / 14, item = it - sg * 14;
    if (!sseg_active[sg]) continue;
    const int t0 = sseg_start[sg], t1 = sseg_start[sg + 1];
    const int st_ = sset[t0];
    if (st_ < 0) continue;
    const int* slots = d.set_slots + (size_t)st_ * 14;
    if (item < 10) {
      // pair index -> (a, b): (0,0)(0,1)(0,2)(0,3)(1,1)(1,2)(1,3)(2,2)(2,3)(3,3)
      const int a = item < 4 ? 0 : item < 7 ? 1 : item < 9 ? 2 : 3;
      const int bb = item < 4 ? item : item < 7 ? item - 3 : item < 9 ? item - 5 : 3;
      float acc[36];
#pragma unroll
      for (int k = 0; k < 36; ++k) acc[k] = 0.f;
      for (int t = t0; t < t1; ++t) {
        const float* Jt = sJ + t * kJS;
        float ja[6], jb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) { ja[k] = Jt[6 * a + k]; jb[k] = Jt[6 * bb + k]; }
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[p * 6 + q] += ja[p] * jb[q];
      }
      float* dst = d.A + (size_t)__ldg(slots + item) * 36;
#pragma unroll
      for (int k = 0; k < 36; ++k) atomicAdd(dst + k, acc[k]);
    } else {
      const int a = item - 10;
      float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      for (int t = t0; t < t1; ++t) {
        const float* Jt = sJ + t * kJS;
        const float rr = Jt[24];
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += Jt[6 * a + k] * rr;
      }
      float* dst = d.g + (size_t)__ldg(slots + 10 + a) * 6;
#pragma unroll
      for (int k = 0; k < 6; ++k) atomicAdd(dst + k, acc[k]);
    }
  }
}

// association alone, on the stored live surfels (stage checks)
__global__ void k_associate_only(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kSurfTile + threadIdx.x;
  if (i >= d.n_s) return;
  const float4 vl = d.v_live[i], nl = d.n_live[i];
  int pix = -1;
  if (surfel_selected(d, d.n_ref[i].w, d.tt[i].y)) pix = associate_one(d, f3(vl), f3(nl));
  d.corr_pix[i] = pix;
}

// ------------------------------------------------------------------ K7: PCG

// 6x6 SPD inverse by Cholesky in FP64; false if not positive definite.
__device__ bool spd_inverse6(const float* a, double* inv) {
  double L[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) L[k] = 0.0;
  for (int c = 0; c < 6; ++c) {
    double s = (double)a[c * 6 + c];
    for (int k = 0; k < c; ++k) s -= L[c * 6 + k] * L[c * 6 + k];
    if (!(s > 0.0)) return false;
    const double lcc = sqrt(s);
    L[c * 6 + c] = lcc;
    for (int r = c + 1; r < 6; ++r) {
      double t = 0.5 * ((double)a[r * 6 + c] + (double)a[c * 6 + r]);
      for (int k = 0; k < c; ++k) t -= L[r * 6 + k] * L[c * 6 + k];
      L[r * 6 + c] = t / lcc;
    }
  }
  // Li = L⁻¹ (lower), inv = Liᵀ Li
  double Li[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) Li[k] = 0.0;
  for (int c = 0; c < 6; ++c) {
    Li[c * 6 + c] = 1.0 / L[c * 6 + c];
    for (int r = c + 1; r < 6; ++r) {
      double t = 0.0;
      for (int k = c; k < r; ++k) t -= L[r * 6 + k] * Li[k * 6 + c];
      Li[r * 6 + c] = t / L[r * 6 + r];
    }
  }
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) {
      double t = 0.0;
      for (int k = (r > c ? r : c); k < 6; ++k) t += Li[k * 6 + r] * Li[k * 6 + c];
      inv[r * 6 + c] = t;
    }
  return true;
}

__global__ void __launch_bounds__(kNodeTile) k_pcg_init(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const int j = (blockIdx.x - __ldg(bt.tile_base + s)) * kNodeTile + threadIdx.x;
  double rz = 0.0;
  if (j < d.n_n) {
    const float* Ajj = d.A + (size_t)d.row_ptr[j] * 36;    // diagonal block leads its row
    double inv[36];
    float* M = d.Minv + (size_t)j * 36;
    if (spd_inverse6(Ajj, inv)) {
#pragma unroll
      for (int k = 0; k < 36; ++k) M[k] = (float)inv[k];
    } else {
      atomicOr(d.status, kStatusBreakdown);
#pragma unroll
      for (int k = 0; k < 36; ++k) { M[k] = 0.f; inv[k] = 0.0; }
    }
    float r[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) { r[k] = -d.g[6 * j + k]; d.r[6 * j + k] = r[k]; d.x[6 * j + k] = 0.f; }
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      float zp = 0.f;
#pragma unroll
      for (int q = 0; q < 6; ++q) zp += M[p * 6 + q] * r[q];
      d.z[6 * j + p] = zp;
      rz += (double)r[p] * (double)zp;
    }
  }
  block_atomic_sum<double>(rz, d.red + 0);
}

// red layout: rz_0 = red[0]; iteration k: pq_k = red[2k+1], rz_{k+1} = red[2k+2]
__global__ void __launch_bounds__(kRowTile) k_pcg_spmv(Batch bt, int k) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const double rzk = *(volatile const double*)(d.red + 2 * k);
  if (rzk == 0.0) return;                      // exact zero residual: the solve is done
  const float beta = k == 0 ? 0.f : (float)(rzk / d.red[2 * k - 2]);
  const float* __restrict__ z = d.z;
  const float* __restrict__ pold = (k & 1) ? d.p0 : d.p1;
  float* __restrict__ pnew = (k & 1) ? d.p1 : d.p0;
  const int t = (blockIdx.x - __ldg(bt.tile_base + s)) * kRowTile + threadIdx.x;
  double pq = 0.0;
  if (t < 6 * d.n_n) {
    const int i = t / 6, c = t - 6 * i;
    float acc = 0.f;
    for (int bk = d.row_ptr[i]; bk < d.row_ptr[i + 1]; ++bk) {
      const int j = d.col[bk];
      const float* B = d.A + (size_t)bk * 36 + c * 6;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float pj = k == 0 ? z[6 * j + q] : z[6 * j + q] + beta * pold[6 * j + q];
        acc += B[q] * pj;
      }
    }
    for (int e = d.low_ptr[i]; e < d.low_ptr[i + 1]; ++e) {
      const int bk = d.low_blk[e];
      const int j = d.blk_row[bk];
      const float* B = d.A + (size_t)bk * 36 + c;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const float pj = k == 0 ? z[6 * j + q] : z[6 * j + q] + beta * pold[6 * j + q];
        acc += B[q * 6] * pj;
      }
    }
    const float pi = k == 0 ? z[t] : z[t] + beta * pold[t];
    pnew[t] = pi;
    d.q[t] = acc;
    pq = (double)pi * (double)acc;
  }
  block_atomic_sum<double>(pq, d.red + 2 * k + 1);
}

__global__ void __launch_bounds__(kNodeTile) k_pcg_update(Batch bt, int k) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const double rzk = d.red[2 * k];
  if (rzk == 0.0) return;
  const double pqk = d.red[2 * k + 1];
  const int j = (blockIdx.x - __ldg(bt.tile_base + s)) * kNodeTile + threadIdx.x;
  if (!(pqk > 0.0)) {
    if (j == 0) atomicOr(d.status, kStatusBreakdown);
    return;
  }
  const float alpha = (float)(rzk / pqk);
  const float* __restrict__ p = (k & 1) ? d.p1 : d.p0;
  double rz = 0.0;
  if (j < d.n_n) {
    float r[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const int t = 6 * j + c;
      d.x[t] += alpha * p[t];
      r[c] = d.r[t] - alpha * d.q[t];
      d.r[t] = r[c];
    }
    const float* M = d.Minv + (size_t)j * 36;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
      float zp = 0.f;
#pragma unroll
      for (int c = 0; c < 6; ++c) zp += M[a * 6 + c] * r[c];
      d.z[6 * j + a] = zp;
      rz += (double)r[a] * (double)zp;
    }
  }
  block_atomic_sum<double>(rz, d.red + 2 * k + 2);
}

// ------------------------------------------------------------------ K8: update

__global__ void __launch_bounds__(kNodeTile) k_apply_update(Batch bt, int gn_it, int pcg_iters) {
  const int s = find_stream(bt, blockIdx.x);
  const SwDev& d = bt.devs[s];
  const int j = (blockIdx.x - __ldg(bt.tile_base + s)) * kNodeTile + threadIdx.x;
  if (j == 0) d.pcg_rz[gn_it] = d.red[2 * pcg_iters];
  if (j >= d.n_n || (*d.status & kStatusBreakdown)) return;
  float xi[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) xi[c] = d.x[6 * j + c];
  float4 q0 = d.dq[2 * j], qe = d.dq[2 * j + 1];
  apply_increment(q0, qe, xi);
  d.dq[2 * j] = q0;
  d.dq[2 * j + 1] = qe;
}

inline Batch with_kind(const BatchHost& b, int kind) {
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kind];
  return bt;
}

}  // namespace

void launch_reg_assemble(const BatchHost& b, int gn_it, cudaStream_t st) {
  if (b.total_tiles[kTileBlocks]) k_reg_assemble<<<b.total_tiles[kTileBlocks], kBlkTile, 0, st>>>(with_kind(b, kTileBlocks), gn_it);
}
void launch_data_assemble(const BatchHost& b, int gn_it, cudaStream_t st) {
  if (b.total_tiles[kTileSurfelsAssembly])
    k_data_assemble<<<b.total_tiles[kTileSurfelsAssembly], kAsmTile, 0, st>>>(with_kind(b, kTileSurfelsAssembly), gn_it, 1);
}
void launch_associate_only(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels]) k_associate_only<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels));
}
void launch_pcg_init(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileNodes]) k_pcg_init<<<b.total_tiles[kTileNodes], kNodeTile, 0, st>>>(with_kind(b, kTileNodes));
}
void launch_pcg_spmv(const BatchHost& b, int k, cudaStream_t st) {
  if (b.total_tiles[kTileRows6]) k_pcg_spmv<<<b.total_tiles[kTileRows6], kRowTile, 0, st>>>(with_kind(b, kTileRows6), k);
}
void launch_pcg_update(const BatchHost& b, int k, cudaStream_t st) {
  if (b.total_tiles[kTileNodes]) k_pcg_update<<<b.total_tiles[kTileNodes], kNodeTile, 0, st>>>(with_kind(b, kTileNodes), k);
}
void launch_apply_update(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st) {
  if (b.total_tiles[kTileNodes])
    k_apply_update<<<b.total_tiles[kTileNodes], kNodeTile, 0, st>>>(with_kind(b, kTileNodes), gn_it, pcg_iters);
}

}  // namespace sw
