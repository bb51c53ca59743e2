// K4-K6: the assembly half of one Gauss-Newton iteration of the non-rigid
// solve (Sec. 7-8), one launch (k_assemble) of two kinds of CTA:
//
//   K6 regulariser tiles  the as-rigid-as-possible part (Eq. 11) of every
//                       upper 6x6 block of JᵀJ and of Jᵀe, added by vector
//                       atomics: 8 lanes per node for the diagonal blocks and
//                       Jᵀe, one thread per block for the others.  They also
//                       clear the other of the two system buffers, which the
//                       next iteration assembles into.
//   K4+K5 data tiles    one thread per surfel: dual-quaternion blend and
//                       forward warp (Eq. 1-2), projective association,
//                       point-to-plane residual (Eq. 10) and its 1x24
//                       Jacobian; the CTA then reduces JᵀJ and Jᵀe over runs
//                       of surfels that share one 4-node set (surfels are
//                       stored sorted by that set) and adds each run's ten
//                       6x6 blocks and four 6-vectors to the system with
//                       atomics.
//
// The two kinds run side by side, so the system they add to must be zero
// before the launch: iteration k assembles into buffer k mod 2 (sys_A,
// sys_g), cleared by iteration k - 1's launch or, for the solve's first
// iteration, by k_system_clear.
//   (K7+K8, the PCG and the node update, are in k_pcg.cu.)
#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_assoc.cuh"

namespace sw {

// ------------------------------------------------------------------ helpers

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
// The rotation part's diagonal (xa·xb − xa_p xb_p) is formed as the sum of
// the other two coordinates' products: the difference would cancel when the
// points lie near axis p (near the optical axis for p = z), leaving FP32
// rounding of |xa||xb| in an entry that is far smaller.
__device__ __forceinline__ void add_reg_pair(float* acc, float s, float3 xa, float3 xb) {
  const float a[3] = {xa.x, xa.y, xa.z}, b[3] = {xb.x, xb.y, xb.z};
#pragma unroll
  for (int p = 0; p < 3; ++p)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int p1 = (p + 1) % 3, p2 = (p + 2) % 3;
      acc[p * 6 + q] += s * (p == q ? a[p1] * b[p1] + a[p2] * b[p2] : -b[p] * a[q]);
    }
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
  // the solve's bits; the frame's depth stage keeps its own, and a failed
  // index check (checked build) stays until the model is set again
  if (threadIdx.x == 0) *d.status &= kStatusDepthTimeout | kStatusBounds;
}

// Threads [0, n8), n8 = 8 n_n rounded up to a whole warp: a group of 8
// lanes per node j writes the diagonal block (j, j) and the Jᵀe segment of
// j (the groups past the last node only join the shuffles, which need whole
// warps).  Every edge adds the same form to
// the diagonal block: for the point y = T_j p (p_j on an out-edge, p_m on an
// in-edge) the block of [−[y]×|I]ᵀ[−[y]×|I] is [[|y|²I − y yᵀ, [y]×],
// [−[y]×, I]], so the block needs only the edges' count, Σy and Σ y yᵀ; the
// out-edges all share y = T_j p_j.  Lane q of the group takes out-edge q and
// the in-edges q, q + 8, ...; the group sums its lanes' shares by shuffles.
// Threads [n8, n8 + nnzb): one per block; an off-diagonal one adds its
// block when a graph edge joins its two nodes.  Thread b of the stream's
// n8 + nnzb; returns its share of E_reg.  The system buffer of iteration
// gn_it gets the terms; the other buffer's entries that the thread owns
// (block b - n8, the Jᵀe segment of node j) are cleared for the next.
__device__ __forceinline__ float reg_assemble_thread(const SwDev& d, int b, int gn_it) {
  // a new epoch for the generation stamps of the PCG launch that follows
  if (b == 0) *d.pcg_epoch += 1;
  float* __restrict__ A = sys_A(d, gn_it);
  float* __restrict__ g = sys_g(d, gn_it);
  const float sl = d.sqrt_lambda, l = sl * sl;
  const int n8 = reg_diag_threads(d.n_n);   // a multiple of 32: no warp straddles the two parts
  float ereg = 0.f;
  if (b < n8) {
    const int j = b >> 3, q = b & 7;
    const bool on = j < d.n_n;
    float3 x = make_float3(0.f, 0.f, 0.f);
    // [gj (6), Σy (3), Σyyᵀ (xx xy xz yy yz zz), in-edge count]
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = 0.f;
    static_assert(SW_K_GRAPH == 8, "one out-edge per lane of the group");
    if (on) {   // out-edge j -> m
      const float3 pj = f3(d.node_p[j]);
      x = node_apply(d, j, pj);
      const int m = checked(d.graph[j * SW_K_GRAPH + q], d.n_n, d.status);
      const float3 y = node_apply(d, m, pj);
      const float3 r = sl * (x - y);
      ereg += dot3(r, r);
      const float3 xr = cross3(x, r);
      v[0] += sl * xr.x; v[1] += sl * xr.y; v[2] += sl * xr.z;
      v[3] += sl * r.x; v[4] += sl * r.y; v[5] += sl * r.z;
    }
    const int e1 = on ? d.in_ptr[j + 1] : 0;
    for (int e = (on ? d.in_ptr[j] : 0) + q; e < e1; e += 8) {   // in-edges m -> j
      const int m = checked(d.in_src[e], d.n_n, d.status);
      const float3 pm = f3(d.node_p[m]);
      const float3 y = node_apply(d, j, pm);
      const float3 r = sl * (node_apply(d, m, pm) - y);
      v[6] += y.x; v[7] += y.y; v[8] += y.z;
      v[9] += y.x * y.x; v[10] += y.x * y.y; v[11] += y.x * y.z;
      v[12] += y.y * y.y; v[13] += y.y * y.z; v[14] += y.z * y.z;
      v[15] += 1.f;
      const float3 yr = cross3(y, r);
      v[0] -= sl * yr.x; v[1] -= sl * yr.y; v[2] -= sl * yr.z;
      v[3] -= sl * r.x; v[4] -= sl * r.y; v[5] -= sl * r.z;
    }
    // the group's sums (its 8 lanes are aligned within the warp, and every
    // lane of the warp is here)
#pragma unroll
    for (int o = 4; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (on && q == 0) {
      const float ko = (float)SW_K_GRAPH;
      const float cnt = ko + v[15];
      const float sy[3] = {ko * x.x + v[6], ko * x.y + v[7], ko * x.z + v[8]};
      const float S[9] = {ko * x.x * x.x + v[9],  ko * x.x * x.y + v[10], ko * x.x * x.z + v[11],
                          ko * x.x * x.y + v[10], ko * x.y * x.y + v[12], ko * x.y * x.z + v[13],
                          ko * x.x * x.z + v[11], ko * x.y * x.z + v[13], ko * x.z * x.z + v[14]};
      const float ax[9] = {0.f, -sy[2], sy[1], sy[2], 0.f, -sy[0], -sy[1], sy[0], 0.f};
      float acc[36];
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // Σ(|y|² δ_pc − y_p y_c); on the diagonal the sum of the other two
          // squares, without the cancellation of |y|² − y_p²
          const int p1 = (p + 1) % 3, p2 = (p + 2) % 3;
          acc[p * 6 + c] = l * (p == c ? S[4 * p1] + S[4 * p2] : -S[p * 3 + c]);
          acc[p * 6 + 3 + c] = l * ax[p * 3 + c];
          acc[(3 + p) * 6 + c] = -l * ax[p * 3 + c];
          acc[(3 + p) * 6 + 3 + c] = p == c ? l * cnt : 0.f;
        }
      float4* dst = reinterpret_cast<float4*>(A + (size_t)checked(d.row_ptr[j], d.nnzb, d.status) * 36);
#pragma unroll
      for (int k = 0; k < 9; ++k)
        atomicAdd(dst + k, make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]));
      float2* gj = reinterpret_cast<float2*>(g + 6 * (size_t)j);   // 8-byte aligned
      float2* gn = reinterpret_cast<float2*>(sys_g(d, gn_it + 1) + 6 * (size_t)j);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        atomicAdd(gj + k, make_float2(v[2 * k], v[2 * k + 1]));
        gn[k] = make_float2(0.f, 0.f);
      }
    }
  } else if (b - n8 < d.nnzb) {
    const int bi = b - n8;
    float4* nxt = reinterpret_cast<float4*>(sys_A(d, gn_it + 1) + (size_t)bi * 36);
#pragma unroll
    for (int k = 0; k < 9; ++k) nxt[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int i = checked(d.blk_row[bi], d.n_n, d.status), j = checked(d.col[bi], d.n_n, d.status);
    const int fl = i != j ? d.blk_edge[bi] : 0;
    if (fl) {
      float acc[36];
#pragma unroll
      for (int k = 0; k < 36; ++k) acc[k] = 0.f;
      if (fl & 1) {   // edge i -> j: J_i = sl[−[T_i p_i]×|I], J_j = −sl[−[T_j p_i]×|I]
        const float3 pi = f3(d.node_p[i]);
        add_reg_pair(acc, -l, node_apply(d, i, pi), node_apply(d, j, pi));
      }
      if (fl & 2) {   // edge j -> i: J_j = sl[−[T_j p_j]×|I], J_i = −sl[−[T_i p_j]×|I]
        const float3 pj = f3(d.node_p[j]);
        add_reg_pair(acc, -l, node_apply(d, i, pj), node_apply(d, j, pj));
      }
      float4* dst = reinterpret_cast<float4*>(A + (size_t)bi * 36);
#pragma unroll
      for (int k = 0; k < 9; ++k)
        atomicAdd(dst + k, make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]));
    }
  }
  return ereg;
}

// ------------------------------------------------------------------ K4+K5: data term

constexpr int kJS = 25;   // 24 Jacobian entries + residual per term
// chunks of terms per output third: 6 x 3 x 14 = 252 threads.  Every chunk
// flushes at least once (3 float4 or one float2 vector atomic per third), and
// the atomics cost more than the products (with whole outputs per thread
// over 126 threads, measured on the full-size frame: 18 chunks 39.5 us, 12
// 36.8, 9 35.8, 6 36.2, 5 37.5 per launch)
constexpr int kAsmChunks = 6;
static_assert(3 * kAsmChunks * 14 <= kAsmTile, "one thread per (item, part, chunk)");

// data tile `tile` of the batch (bt.tile_base: the data tiles' table)
__device__ __forceinline__ void data_assemble_tile(const Batch& bt, int tile, int gn_it, int write_live) {
  const int s = find_stream(bt, tile);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  float* __restrict__ A = sys_A(d, gn_it);
  float* __restrict__ g = sys_g(d, gn_it);
  const int t_now = *d.t_now;
  const int tid = threadIdx.x;
  const int i = (tile - __ldg(bt.tile_base + s)) * kAsmTile + tid;

  __shared__ float sJ[kAsmTile * kJS];
  __shared__ int sset[kAsmTile];
  __shared__ int swarp[kAsmTile / 32];

  float Jr[24];
  int set = -1;
  bool valid = false;
  float res = 0.f;
  if (i < d.n_s) {
    const float4 v4 = d.v_ref[i], n4 = d.n_ref[i];
    const int4 ids = checked4(d.knn[i], d.n_n, d.status);
    const float4 w = d.w[i];
    const int rs = checked(d.ref_slot[i], 4, d.status);
    set = checked(d.set_id[i], d.n_sets, d.status);
    const DQ b = blend4(d.dq, ids, w, rs);
    const float n2 = dq_norm2(b);
    int pix = -1;
    float3 vl = f3(v4), nl = f3(n4);
    float inv = 0.f;
    if (n2 > 0.f) {
      inv = 1.f / n2;
      vl = dq_transform(b, inv, f3(v4));
      nl = dq_rotate(b, inv, f3(n4));
      if (surfel_visible(d, i) && surfel_selected(d, t_now, n4.w, d.tt[i].y)) pix = associate_one(d, vl, nl);
    }
    d.corr_pix[i] = pix;
    if (d.corr_rec) d.corr_rec[(size_t)gn_it * d.n_s + i] = pix;
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
  // (item, part, chunk) owns a third of one of the 14 outputs of a node set
  // -- items 0..9 the upper blocks (a <= b) of its 4 nodes, a part two of a
  // block's six rows; items 10..13 the Jᵀe segments, a part two of a
  // segment's six values -- over one chunk of consecutive terms.  It
  // accumulates while the set id stays the same and adds the sum to the
  // system (vector atomics) whenever the set changes or the chunk ends, so
  // node sets of any size cost every thread about the same.  Splitting each
  // output three ways keeps 252 of the 256 threads busy with a third of the
  // products each, over fewer chunks (so fewer flushes).
  // item-major: a warp's lanes take the same item and part on neighbouring
  // chunks (no divergence between block and Jᵀe items); an odd chunk length
  // keeps the lanes' shared-memory rows in different banks
  const int item = tid / (3 * kAsmChunks), rem = tid - item * (3 * kAsmChunks);
  const int part = rem / kAsmChunks, chunk = rem - part * kAsmChunks;
  const int len = ((nvalid + kAsmChunks - 1) / kAsmChunks) | 1;
  if (item < 14) {
    const int t0 = min(nvalid, chunk * len), t1 = min(nvalid, t0 + len);
    if (t0 >= t1) return;
    if (item < 10) {
      // pair index -> (a, b): (0,0)(0,1)(0,2)(0,3)(1,1)(1,2)(1,3)(2,2)(2,3)(3,3)
      const int a = item < 4 ? 0 : item < 7 ? 1 : item < 9 ? 2 : 3;
      const int bb = item < 4 ? item : item < 7 ? item - 3 : item < 9 ? item - 5 : 3;
      const int ra = 6 * a + 2 * part;   // rows 2 part and 2 part + 1 of the block
      // acc[3 r + j]: entries (2 part + r, 2 j) and (2 part + r, 2 j + 1), on packed FP32 pairs
      float2 acc[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) acc[k] = make_float2(0.f, 0.f);
      int cur = sset[t0];
      int slot = checked(__ldg(d.set_slots + (size_t)cur * 14 + item), d.nnzb, d.status);
      for (int t = t0; t <= t1; ++t) {
        const int st_ = t < t1 ? sset[t] : -1;
        if (st_ != cur) {
          float4* dst = reinterpret_cast<float4*>(A + (size_t)slot * 36 + 12 * part);   // 16-byte aligned
#pragma unroll
          for (int k = 0; k < 3; ++k)
            atomicAdd(dst + k, make_float4(acc[2 * k].x, acc[2 * k].y, acc[2 * k + 1].x, acc[2 * k + 1].y));
          if (t == t1) break;
#pragma unroll
          for (int k = 0; k < 6; ++k) acc[k] = make_float2(0.f, 0.f);
          cur = st_;
          slot = checked(__ldg(d.set_slots + (size_t)cur * 14 + item), d.nnzb, d.status);
        }
        const float* Jt = sJ + t * kJS;
        const float2 j0 = make_float2(Jt[ra], Jt[ra]), j1 = make_float2(Jt[ra + 1], Jt[ra + 1]);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const float2 jb = make_float2(Jt[6 * bb + 2 * j], Jt[6 * bb + 2 * j + 1]);
          acc[j] = __ffma2_rn(j0, jb, acc[j]);
          acc[3 + j] = __ffma2_rn(j1, jb, acc[3 + j]);
        }
      }
    } else {
      const int a = item - 10;
      float2 acc = make_float2(0.f, 0.f);   // values 2 part and 2 part + 1 of the segment
      int cur = sset[t0];
      int node = checked(__ldg(d.set_slots + (size_t)cur * 14 + 10 + a), d.n_n, d.status);
      for (int t = t0; t <= t1; ++t) {
        const int st_ = t < t1 ? sset[t] : -1;
        if (st_ != cur) {
          atomicAdd(reinterpret_cast<float2*>(g + (size_t)node * 6 + 2 * part), acc);   // 8-byte aligned
          if (t == t1) break;
          acc = make_float2(0.f, 0.f);
          cur = st_;
          node = checked(__ldg(d.set_slots + (size_t)cur * 14 + 10 + a), d.n_n, d.status);
        }
        const float* Jt = sJ + t * kJS;
        const float rr = Jt[24];
        acc = __ffma2_rn(make_float2(Jt[6 * a + 2 * part], Jt[6 * a + 2 * part + 1]), make_float2(rr, rr), acc);
      }
    }
  }
}

// One Gauss-Newton iteration's assembly: CTAs [0, reg_tiles) are the
// regulariser's tiles (reg_base: their table, kAsmTile threads of a
// stream's n8 + nnzb each), the rest the data tiles (bt.tile_base).  Both
// add to the system buffer of gn_it, cleared before the launch.
__global__ void __launch_bounds__(kAsmTile, 4)
k_assemble(Batch bt, const int* __restrict__ reg_base, int reg_tiles, int gn_it, int write_live) {
  pdl_begin();
  if ((int)blockIdx.x < reg_tiles) {
    Batch rb = bt;
    rb.tile_base = reg_base;
    const int s = find_stream(rb, blockIdx.x);
    if (!stream_active(rb, s)) return;   // CTA-uniform
    const SwDev d = bt.devs[s];
    const int b = (blockIdx.x - __ldg(reg_base + s)) * kAsmTile + threadIdx.x;
    const float ereg = reg_assemble_thread(d, b, gn_it);
    block_atomic_sum<double>((double)ereg, d.e_reg + gn_it);
    return;
  }
  data_assemble_tile(bt, blockIdx.x - reg_tiles, gn_it, write_live);
}

// Zeroes system buffer 0 of every active stream (the solve's first
// iteration assembles into it): one thread per upper block, and the first
// n_n threads the Jᵀe segments.
__global__ void __launch_bounds__(kBlkTile) k_system_clear(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int b = (blockIdx.x - __ldg(bt.tile_base + s)) * kBlkTile + threadIdx.x;
  if (b < d.nnzb) {
    float4* blk = reinterpret_cast<float4*>(d.A + (size_t)b * 36);
#pragma unroll
    for (int k = 0; k < 9; ++k) blk[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (b < d.n_n) {
    float2* gj = reinterpret_cast<float2*>(d.g + 6 * (size_t)b);
#pragma unroll
    for (int k = 0; k < 3; ++k) gj[k] = make_float2(0.f, 0.f);
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
  if (surfel_visible(d, i) && surfel_selected(d, *d.t_now, d.n_ref[i].w, d.tt[i].y)) pix = associate_one(d, f3(vl), f3(nl));
  d.corr_pix[i] = pix;
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
void launch_system_clear(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileBlocks]) k_system_clear<<<b.total_tiles[kTileBlocks], kBlkTile, 0, st>>>(with_kind(b, kTileBlocks));
}
void launch_assemble(const BatchHost& b, int gn_it, cudaStream_t st) {
  const int nr = b.total_tiles[kTileRegAssembly], nd = b.total_tiles[kTileSurfelsAssembly];
  if (nr + nd)
    launch_overlapped(k_assemble, nr + nd, kAsmTile, st, with_kind(b, kTileSurfelsAssembly),
                      (const int*)b.tile_base_dev[kTileRegAssembly], nr, gn_it, 0);
}
void launch_associate_only(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels]) k_associate_only<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels));
}

}  // namespace sw
