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
//   K7+K8 k_pcg         one persistent cooperative launch per Gauss-Newton
//                       iteration runs the whole block-Jacobi PCG on
//                       JᵀJ Δ = −Jᵀe and applies T_j ← Δ_j T_j: FP64 Cholesky
//                       of the diagonal blocks, FP32 block SpMV (a warp per
//                       block row) and vector updates, FP64 dot products
//                       summed from published per-CTA partials in a fixed
//                       order; each reduction is a bounded wait among the
//                       CTAs of one stream.
#include "sw_internal.h"
#include "sw_math.cuh"

namespace sw {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ bool surfel_selected(const SwDev& d, int t_now, float conf, int t_obs) {
  return conf > d.stable_conf || (t_now - t_obs) <= d.recent_frames;
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

__global__ void k_solve_begin(Batch bt) {
  const int s = blockIdx.x;
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  for (int k = threadIdx.x; k < kMaxGn; k += blockDim.x) {
    d.e_depth[k] = 0.0; d.e_reg[k] = 0.0; d.n_corr[k] = 0; d.pcg_rz[k] = 0.0;
  }
  if (threadIdx.x == 0) *d.status = 0;
}

__global__ void __launch_bounds__(kBlkTile) k_reg_assemble(Batch bt, int gn_it) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int b = (blockIdx.x - __ldg(bt.tile_base + s)) * kBlkTile + threadIdx.x;
  // a new epoch for the generation stamps of the PCG launch that follows
  if (b == 0) *d.pcg_epoch += 1;
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
constexpr int kAsmChunks = kAsmTile / 14;                        // 18 chunks x 14 outputs = 252 threads

__global__ void __launch_bounds__(kAsmTile, 4) k_data_assemble(Batch bt, int gn_it, int write_live) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int t_now = *d.t_now;
  const int tid = threadIdx.x;
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kAsmTile + tid;

  __shared__ float sJ[kAsmTile * kJS];
  __shared__ int sset[kAsmTile];
  __shared__ int swarp[kAsmTile / 32];

  float Jr[24];
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
      if (surfel_selected(d, t_now, n4.w, d.tt[i].y)) pix = associate_one(d, vl, nl);
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
        node_jacobian(gr, q0, qe, ws, Jr + 6 * k);
      }
    }
  }

  // statistics: E_depth is a diagnostic (FP32 warp sums, one FP64 atomic per warp)
  const int lane = tid & 31, wid = tid >> 5;
  {
    const float e = warp_sum(res * res);
    if (lane == 0 && e != 0.f) atomicAdd(d.e_depth + gn_it, (double)e);
  }

  // compact the tile's associated terms, in order, into shared memory
  const unsigned vb = __ballot_sync(0xffffffffu, valid);
  if (lane == 0) swarp[wid] = __popc(vb);
  __syncthreads();
  int pos = __popc(vb & ((1u << lane) - 1u)), nvalid = 0;
#pragma unroll
  for (int k = 0; k < kAsmTile / 32; ++k) {
    const int c = swarp[k];
    if (k < wid) pos += c;
    nvalid += c;
  }
  if (valid) {
    float* dst = sJ + pos * kJS;
#pragma unroll
    for (int k = 0; k < 24; ++k) dst[k] = Jr[k];
    dst[24] = res;
    sset[pos] = set;
  }
  if (tid == 0 && nvalid) atomicAdd(d.n_corr + gn_it, nvalid);
  __syncthreads();
  if (nvalid == 0) return;

  // JᵀJ and Jᵀe of the tile's terms, balanced over the threads: thread
  // (item, chunk) owns one of the 14 outputs of a node set -- items 0..9 the
  // upper blocks (a <= b) of its 4 nodes, 10..13 the Jᵀe segments -- over one
  // chunk of consecutive terms.  It accumulates while the set id stays the
  // same and adds the sum to the system (16-byte vector atomics) whenever the
  // set changes or the chunk ends, so node sets of any size cost every thread
  // about the same.
  // item-major: a warp's lanes take the same item on neighbouring chunks (no
  // divergence between block and Jᵀe items); an odd chunk length keeps the
  // lanes' shared-memory rows in different banks
  const int item = tid / kAsmChunks, chunk = tid - item * kAsmChunks;
  const int len = ((nvalid + kAsmChunks - 1) / kAsmChunks) | 1;
  if (item < 14) {
    const int t0 = min(nvalid, chunk * len), t1 = min(nvalid, t0 + len);
    if (t0 >= t1) return;
    if (item < 10) {
      // pair index -> (a, b): (0,0)(0,1)(0,2)(0,3)(1,1)(1,2)(1,3)(2,2)(2,3)(3,3)
      const int a = item < 4 ? 0 : item < 7 ? 1 : item < 9 ? 2 : 3;
      const int bb = item < 4 ? item : item < 7 ? item - 3 : item < 9 ? item - 5 : 3;
      float acc[36];
#pragma unroll
      for (int k = 0; k < 36; ++k) acc[k] = 0.f;
      int cur = sset[t0];
      int slot = __ldg(d.set_slots + (size_t)cur * 14 + item);
      for (int t = t0; t <= t1; ++t) {
        const int st_ = t < t1 ? sset[t] : -1;
        if (st_ != cur) {
          float4* dst = reinterpret_cast<float4*>(d.A + (size_t)slot * 36);
#pragma unroll
          for (int k = 0; k < 9; ++k)
            atomicAdd(dst + k, make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]));
          if (t == t1) break;
#pragma unroll
          for (int k = 0; k < 36; ++k) acc[k] = 0.f;
          cur = st_;
          slot = __ldg(d.set_slots + (size_t)cur * 14 + item);
        }
        const float* Jt = sJ + t * kJS;
        float ja[6], jb[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) { ja[k] = Jt[6 * a + k]; jb[k] = Jt[6 * bb + k]; }
#pragma unroll
        for (int p = 0; p < 6; ++p)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[p * 6 + q] += ja[p] * jb[q];
      }
    } else {
      const int a = item - 10;
      float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      int cur = sset[t0];
      int node = __ldg(d.set_slots + (size_t)cur * 14 + 10 + a);
      for (int t = t0; t <= t1; ++t) {
        const int st_ = t < t1 ? sset[t] : -1;
        if (st_ != cur) {
          float2* dst = reinterpret_cast<float2*>(d.g + (size_t)node * 6);   // 8-byte aligned
#pragma unroll
          for (int k = 0; k < 3; ++k) atomicAdd(dst + k, make_float2(acc[2 * k], acc[2 * k + 1]));
          if (t == t1) break;
#pragma unroll
          for (int k = 0; k < 6; ++k) acc[k] = 0.f;
          cur = st_;
          node = __ldg(d.set_slots + (size_t)cur * 14 + 10 + a);
        }
        const float* Jt = sJ + t * kJS;
        const float rr = Jt[24];
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += Jt[6 * a + k] * rr;
      }
    }
  }
}

// association alone, on the stored live surfels (stage checks)
__global__ void k_associate_only(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kSurfTile + threadIdx.x;
  if (i >= d.n_s) return;
  const float4 vl = d.v_live[i], nl = d.n_live[i];
  int pix = -1;
  if (surfel_selected(d, *d.t_now, d.n_ref[i].w, d.tt[i].y)) pix = associate_one(d, f3(vl), f3(nl));
  d.corr_pix[i] = pix;
}

// ------------------------------------------------------------------ K7+K8: PCG

// Counter barrier over all CTAs of a cooperative launch, with a bounded wait
// (used by the timeout probe).
__device__ __forceinline__ bool grid_sync(GridBarrier* gb, unsigned nblocks, int spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gb->gen;
    const unsigned g = *vgen;
    int ok = 1;
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == nblocks - 1) {
      atomicExch(&gb->count, 0u);
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      int spins = 0;
      while (*vgen == g) {
        if (++spins > spin_limit) { ok = 0; break; }
        if (spins > 64) __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Double-float accumulation of the PCG's dot products: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, which
// carries about 48 significant bits.  Products come from the error-free
// TwoProduct (one FMA recovers the rounding error of a*b, Dekker 1971);
// sums use Knuth's TwoSum on the high and the low parts followed by two
// renormalisations (the "accurate" pair addition analysed by Joldes, Muller
// and Popescu, ACM TOMS 2017: relative error below 3 * 2^-48).  Only FP32
// operations are involved: an FP64 instruction occupies this part's FP64
// pipe for tens of cycles, and the reductions sit on the PCG's critical path.
// The _rn intrinsics are never contracted or reassociated by the compiler.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return DF{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b| or a == 0
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  fast_two_sum(s, e, s, e);
  return DF{s, e};
}

// TwoSum's error term is exact, so df_add(a, b) == df_add(b, a) bit for bit
// and every lane of the butterfly ends with the same pair.
__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = df_add(v, w);
  }
  return v;
}

// a / b of two positive pair totals, rounded to FP32 (the PCG uses its step
// lengths in FP32; dividing the high parts costs at most one more ulp).
__device__ __forceinline__ float df_ratio(DF a, DF b) { return __fdiv_rn(a.hi, b.hi); }

// Packed lower-triangular index (r >= c).
__device__ __forceinline__ int tri(int r, int c) { return r * (r + 1) / 2 + c; }

// Inverse Cholesky factor Li = L⁻¹ of a 6x6 SPD block, in FP64, stored packed
// as FP32; false if the block is not positive definite.
__device__ bool chol_inverse_factor(const float* a, float* li) {
  double L[21], dinv[6];
  for (int c = 0; c < 6; ++c) {
    double s = (double)a[c * 6 + c];
    for (int k = 0; k < c; ++k) s -= L[tri(c, k)] * L[tri(c, k)];
    if (!(s > 0.0)) return false;
    const double lcc = sqrt(s);
    L[tri(c, c)] = lcc;
    dinv[c] = 1.0 / lcc;
    for (int r = c + 1; r < 6; ++r) {
      double t = 0.5 * ((double)a[r * 6 + c] + (double)a[c * 6 + r]);
      for (int k = 0; k < c; ++k) t -= L[tri(r, k)] * L[tri(c, k)];
      L[tri(r, c)] = t * dinv[c];
    }
  }
  for (int c = 0; c < 6; ++c) {
    li[tri(c, c)] = (float)dinv[c];
    double col[6];
    col[c] = dinv[c];
    for (int r = c + 1; r < 6; ++r) {
      double t = 0.0;
      for (int k = c; k < r; ++k) t += L[tri(r, k)] * col[k];
      col[r] = -t * dinv[r];
      li[tri(r, c)] = (float)col[r];
    }
  }
  return true;
}

// z = M⁻¹ r = Liᵀ (Li r)
__device__ __forceinline__ void apply_precond(const float* __restrict__ li, const float* r, float* z) {
  float y[6];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    float t = 0.f;
#pragma unroll
    for (int c = 0; c <= a; ++c) t += li[tri(a, c)] * r[c];
    y[a] = t;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float t = 0.f;
#pragma unroll
    for (int a = c; a < 6; ++a) t += li[tri(a, c)] * y[a];
    z[c] = t;
  }
}

// p_j = z_j (+ β p_old,j) for one neighbour node (6 values, 8-byte aligned)
__device__ __forceinline__ void load_p(const float* __restrict__ z, const float* __restrict__ pold, int j, float beta,
                                       bool first, float* p) {
  const float2* z2 = reinterpret_cast<const float2*>(z + 6 * j);
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const float2 a = __ldcg(z2 + h);
    p[2 * h] = a.x; p[2 * h + 1] = a.y;
  }
  if (!first) {
    const float2* o2 = reinterpret_cast<const float2*>(pold + 6 * j);
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      const float2 b = __ldcg(o2 + h);
      p[2 * h] += beta * b.x; p[2 * h + 1] += beta * b.y;
    }
  }
}

// One reduction among the CTAs of one stream, which is also their only
// synchronisation.  Every CTA publishes its block sum in its slot with
// generation `gen` (value, fence, stamp), then one warp polls the stream's
// slots (plain volatile loads, bounded), fences, and sums the values in a
// fixed order, so the total is deterministic for a given number of CTAs.
// The CTA's global-memory writes before the call are visible to every CTA
// that returns from the same reduction.  Returns false if the wait ran out.
__device__ __forceinline__ bool stream_reduce(DF v, PartSlot* part, int t, int gs, unsigned long long gen,
                                              int spin_limit, DF* total) {
  __shared__ DF s_w[32];
  __shared__ DF s_tot;
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_df(v);
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  PartSlot* buf = part + (gen & 1ull) * kMaxCtaPerStream;
  if (wid == 0) {
    DF b = lane < nw ? s_w[lane] : DF{0.f, 0.f};
    b = warp_sum_df(b);
    if (lane == 0) {
      __threadfence();                       // the CTA's data writes, then the value, then the stamp
      *reinterpret_cast<float2*>(&buf[t].hi) = make_float2(b.hi, b.lo);
      __threadfence();
      *reinterpret_cast<volatile unsigned long long*>(&buf[t].gen) = gen;
    }
    int ok = 1;
    for (int k = lane; k < gs; k += 32) {
      int spins = 0;
      while (*reinterpret_cast<volatile unsigned long long*>(&buf[k].gen) < gen) {
        if (++spins > spin_limit) { ok = 0; break; }
      }
      if (!ok) break;
    }
    ok = __all_sync(0xffffffffu, ok);
    __threadfence();
    DF acc{0.f, 0.f};
    for (int k = lane; k < gs; k += 32) {
      const float2 pv = __ldcg(reinterpret_cast<const float2*>(&buf[k].hi));
      acc = df_add(acc, DF{pv.x, pv.y});
    }
    acc = warp_sum_df(acc);
    if (lane == 0) { s_tot = acc; s_ok = ok; }
  }
  __syncthreads();
  *total = s_tot;
  const bool ok = s_ok != 0;
  __syncthreads();
  return ok;
}

// One persistent launch runs the PCG of every active stream of the batch and
// applies the increments.  Stream s owns the CTAs [tile_base[s],
// tile_base[s+1]) (all co-resident: cooperative launch).  CTA t of a stream
// with G CTAs owns the nodes and block rows i = t + G a (a = 0, 1, ...) and
// keeps everything about them in shared memory for the whole solve: the
// inverse Cholesky factors of their diagonal blocks and their x, r, z, q and
// p.  Global memory carries only what other CTAs read: z and p of every node.
// The two reductions of an iteration (pᵀq, rᵀz) are also its only
// synchronisation, and they are per stream, so streams never wait for one
// another (stream_reduce).  Per iteration:
//   SpMV    a warp per own block row, a lane per 6x6 block of the row: the
//           block times the neighbour's p = z + β p_old (formed on the fly
//           from global memory), a warp sum of the six outputs;
//   update  x += α p, r −= α q, z = M⁻¹ r per own node, in shared memory.
// Dot products are accumulated in double-float pairs (about 48 bits, see DF);
// the 6x6 factorisations are FP64.
constexpr int kPcgThreads = 1024;
constexpr int kPcgWarps = kPcgThreads / 32;
constexpr int kPcgRowFloats = 21 + 5 * 6;   // Li, then x, r, z, q, p

__global__ void __launch_bounds__(kPcgThreads, 1)
k_pcg(Batch bt, int K, int gn_it, int spin_limit, int rows_cap) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int t = blockIdx.x - __ldg(bt.tile_base + s);
  const int Gs = __ldg(bt.tile_base + s + 1) - __ldg(bt.tile_base + s);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = d.n_n;
  const int nr = n > t ? (n - t + Gs - 1) / Gs : 0;   // own rows (<= rows_cap, checked on the host)
  const unsigned long long base = __ldcg(d.pcg_epoch) * 1024ull;
  extern __shared__ float smem_f[];
  float* sli = smem_f;
  float* sx = sli + 21 * rows_cap;
  float* sr = sx + 6 * rows_cap;
  float* sz = sr + 6 * rows_cap;
  float* sq = sz + 6 * rows_cap;
  float* sp = sq + 6 * rows_cap;

  // ---- set-up: preconditioner, r = −g, z = M⁻¹ r, x = 0
  DF acc{0.f, 0.f};
  for (int a = tid; a < nr; a += kPcgThreads) {
    const int j = t + Gs * a;
    float* li = sli + 21 * a;
    if (!chol_inverse_factor(d.A + (size_t)d.row_ptr[j] * 36, li)) {
      atomicOr(d.status, kStatusBreakdown);
#pragma unroll
      for (int k = 0; k < 21; ++k) li[k] = 0.f;
    }
    float r[6], z[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { r[c] = -d.g[6 * j + c]; sr[6 * a + c] = r[c]; sx[6 * a + c] = 0.f; }
    apply_precond(li, r, z);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      sz[6 * a + c] = z[c];
      d.z[6 * j + c] = z[c];
      acc = df_add(acc, df_prod(r[c], z[c]));
    }
  }
  DF rz, rz_prev{1.f, 0.f};
  if (!stream_reduce(acc, d.part, t, Gs, base + 1, spin_limit, &rz)) { atomicOr(d.status, kStatusTimeout); return; }
  bool bad = (__ldcg(d.status) & kStatusBreakdown) != 0;

  for (int k = 0; k < K; ++k) {
    const bool work = !bad && rz.hi != 0.f;
    const float beta = (k == 0 || !work) ? 0.f : df_ratio(rz, rz_prev);
    const float* __restrict__ pold = (k & 1) ? d.p0 : d.p1;
    float* __restrict__ pnew = (k & 1) ? d.p1 : d.p0;
    acc = DF{0.f, 0.f};
    if (work) {
      for (int a = warp; a < nr; a += kPcgWarps) {
        const int i = t + Gs * a;
        float v[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        const int e1 = d.rl_ptr[i + 1];
        for (int e = d.rl_ptr[i] + lane; e < e1; e += 32) {
          const int2 ent = d.rl_ent[e];
          const float2* B2 = reinterpret_cast<const float2*>(d.A + (size_t)(ent.x & 0x7fffffff) * 36);
          float p[6];
          load_p(d.z, pold, ent.y, beta, k == 0, p);
          const bool tr = ent.x < 0;
#pragma unroll
          for (int b = 0; b < 6; ++b) {
            const float2 b0 = __ldg(B2 + 3 * b), b1 = __ldg(B2 + 3 * b + 1), b2 = __ldg(B2 + 3 * b + 2);
            const float row[6] = {b0.x, b0.y, b1.x, b1.y, b2.x, b2.y};
            if (!tr) {
              float u = 0.f;
#pragma unroll
              for (int q = 0; q < 6; ++q) u += row[q] * p[q];
              v[b] += u;
            } else {
#pragma unroll
              for (int q = 0; q < 6; ++q) v[q] += p[b] * row[q];
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] = warp_sum(v[c]);
        if (lane < 6) {
          float vc = v[0];
#pragma unroll
          for (int c = 1; c < 6; ++c) if (lane == c) vc = v[c];
          const float pi = k == 0 ? sz[6 * a + lane] : sz[6 * a + lane] + beta * sp[6 * a + lane];
          sp[6 * a + lane] = pi;
          sq[6 * a + lane] = vc;
          pnew[6 * i + lane] = pi;
          acc = df_add(acc, df_prod(pi, vc));
        }
      }
    }
    DF pq;
    if (!stream_reduce(acc, d.part, t, Gs, base + 2 + 2 * k, spin_limit, &pq)) {
      atomicOr(d.status, kStatusTimeout);
      return;
    }
    acc = DF{0.f, 0.f};
    if (work) {
      if (!(pq.hi > 0.f)) {
        bad = true;
        if (t == 0 && tid == 0) atomicOr(d.status, kStatusBreakdown);
      } else {
        const float alpha = df_ratio(rz, pq);
        for (int a = tid; a < nr; a += kPcgThreads) {
          float r[6], z[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            sx[6 * a + c] += alpha * sp[6 * a + c];
            r[c] = sr[6 * a + c] - alpha * sq[6 * a + c];
            sr[6 * a + c] = r[c];
          }
          apply_precond(sli + 21 * a, r, z);
          const int j = t + Gs * a;
#pragma unroll
          for (int c = 0; c < 6; ++c) {
            sz[6 * a + c] = z[c];
            d.z[6 * j + c] = z[c];
            acc = df_add(acc, df_prod(r[c], z[c]));
          }
        }
      }
    }
    DF rz_new;
    if (!stream_reduce(acc, d.part, t, Gs, base + 3 + 2 * k, spin_limit, &rz_new)) {
      atomicOr(d.status, kStatusTimeout);
      return;
    }
    if (work && !bad) { rz_prev = rz; rz = rz_new; }
  }
  if (t == 0 && tid == 0) d.pcg_rz[gn_it] = (double)rz.hi + (double)rz.lo;
  // ---- T_j ← Δ_j T_j (nothing moves after a breakdown)
  if (bad || (__ldcg(d.status) & kStatusBreakdown)) return;
  for (int a = tid; a < nr; a += kPcgThreads) {
    const int j = t + Gs * a;
    float xi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xi[c] = sx[6 * a + c];
    float4 q0 = d.dq[2 * j], qe = d.dq[2 * j + 1];
    apply_increment(q0, qe, xi);
    d.dq[2 * j] = q0;
    d.dq[2 * j + 1] = qe;
  }
}

// A grid barrier that never completes when fewer CTAs run than it expects:
// used to check that a wait which cannot finish ends by its bound and reports
// a status the host can read.
__global__ void k_barrier_probe(GridBarrier* gb, unsigned expected, int spin_limit, int* status) {
  if (!grid_sync(gb, expected, spin_limit)) {
    if (threadIdx.x == 0) atomicOr(status, kStatusTimeout);
  }
}

inline Batch with_kind(const BatchHost& b, int kind) {
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kind];
  return bt;
}

}  // namespace

void launch_solve_begin(const BatchHost& b, cudaStream_t st) {
  if (b.bt.n_streams) k_solve_begin<<<b.bt.n_streams, 32, 0, st>>>(b.bt);
}
void launch_reg_assemble(const BatchHost& b, int gn_it, cudaStream_t st) {
  if (b.total_tiles[kTileBlocks]) k_reg_assemble<<<b.total_tiles[kTileBlocks], kBlkTile, 0, st>>>(with_kind(b, kTileBlocks), gn_it);
}
void launch_data_assemble(const BatchHost& b, int gn_it, cudaStream_t st) {
  if (b.total_tiles[kTileSurfelsAssembly])
    k_data_assemble<<<b.total_tiles[kTileSurfelsAssembly], kAsmTile, 0, st>>>(with_kind(b, kTileSurfelsAssembly), gn_it, 0);
}
void launch_associate_only(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels]) k_associate_only<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels));
}

int pcg_blocks_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pcg, kPcgThreads, 0) != cudaSuccess) return 0;
  return n;
}

int pcg_threads() { return kPcgThreads; }

size_t pcg_smem_bytes(int rows_cap) { return sizeof(float) * (size_t)kPcgRowFloats * rows_cap; }

// One cooperative launch: every CTA is resident, so the waits of
// stream_reduce always end (and are bounded regardless).
cudaError_t launch_pcg(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st) {
  const int nb = b.total_tiles[kTilePcg];
  if (nb == 0) return cudaSuccess;
  Batch bt = with_kind(b, kTilePcg);
  int spin = b.spin_limit;
  int rows_cap = b.pcg_rows_cap;
  const size_t smem = pcg_smem_bytes(rows_cap);
  static size_t configured = 48 * 1024;
  if (smem > configured) {
    const cudaError_t e = cudaFuncSetAttribute(k_pcg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  void* args[] = {&bt, &pcg_iters, &gn_it, &spin, &rows_cap};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(k_pcg), args);
}

cudaError_t launch_barrier_probe(GridBarrier* gb, int nblocks_launched, int nblocks_expected, int spin_limit,
                                 int* status, cudaStream_t st) {
  unsigned expected = (unsigned)nblocks_expected;
  void* args[] = {&gb, &expected, &spin_limit, &status};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nblocks_launched);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(k_barrier_probe), args);
}
}  // namespace sw
