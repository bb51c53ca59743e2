// The assembly half of one Gauss-Newton iteration in FP64 (SW_PRECISION_FP64):
// the same regulariser (Eq. 11) and data term (Eq. 10) as k_solve.cu with
// the node transforms, the warp, the residuals, the Jacobians and JᵀJ / Jᵀe
// all in double precision.  The association is decided exactly as in the
// FP32 path, in FP32 from the FP64 warp rounded to FP32.  This variant is a
// precision reference, so it favours plainness over speed: one thread per
// surfel adding its ten 6x6 blocks and four 6-vectors with FP64 atomics.
#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_math64.cuh"
#include "sw_assoc.cuh"

namespace sw {
namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ D3 node_apply64(const SwDev& d, int j, D3 p) {
  const DQ64 b = load_dq64(d.dq64, j);
  return dq_transform(b, 1.0 / dq_norm2(b), p);
}

// s J_aᵀ J_b for J_a = [−[xa]× | I], J_b = [−[xb]× | I] (3x6 each):
//   [[(xa·xb) I − xb xaᵀ, [xa]×], [−[xb]×, I]]
__device__ __forceinline__ void add_reg_pair64(double* acc, double s, D3 xa, D3 xb) {
  const double ab = dot3(xa, xb);
  const double a[3] = {xa.x, xa.y, xa.z}, b[3] = {xb.x, xb.y, xb.z};
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) acc[p * 6 + q] += s * ((p == q ? ab : 0.0) - b[p] * a[q]);
  const double ax[9] = {0.0, -a[2], a[1], a[2], 0.0, -a[0], -a[1], a[0], 0.0};
  const double bx[9] = {0.0, -b[2], b[1], b[2], 0.0, -b[0], -b[1], b[0], 0.0};
  for (int p = 0; p < 3; ++p)
    for (int q = 0; q < 3; ++q) {
      acc[p * 6 + 3 + q] += s * ax[p * 3 + q];
      acc[(3 + p) * 6 + q] -= s * bx[p * 3 + q];
    }
  for (int p = 0; p < 3; ++p) acc[(3 + p) * 6 + 3 + p] += s;
}

// One thread per upper 6x6 block: the regulariser's part of the block (and
// of Jᵀe on diagonal blocks), written with plain stores; it runs first and
// so initialises the whole system.
__global__ void __launch_bounds__(kBlkTile) k_reg_assemble64(Batch bt, int gn_it) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int b = (blockIdx.x - __ldg(bt.tile_base + s)) * kBlkTile + threadIdx.x;
  if (b == 0) *d.pcg_epoch += 1;   // a new epoch for the stamps of the PCG launch that follows
  double ereg = 0.0;
  if (b < d.nnzb) {
    const int i = checked(d.blk_row[b], d.n_n, d.status), j = checked(d.col[b], d.n_n, d.status);
    const double sl = d.sqrt_lambda, l = sl * sl;
    double acc[36];
    for (int k = 0; k < 36; ++k) acc[k] = 0.0;
    if (i == j) {
      double gj[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      const D3 pj = d3(d.node_p[j]);
      const D3 x = node_apply64(d, j, pj);
      for (int e = 0; e < SW_K_GRAPH; ++e) {      // out-edges j -> m
        const int m = checked(d.graph[j * SW_K_GRAPH + e], d.n_n, d.status);
        const D3 r = sl * (x - node_apply64(d, m, pj));
        ereg += dot3(r, r);
        add_reg_pair64(acc, l, x, x);
        const D3 xr = cross3(x, r);
        gj[0] += sl * xr.x; gj[1] += sl * xr.y; gj[2] += sl * xr.z;
        gj[3] += sl * r.x; gj[4] += sl * r.y; gj[5] += sl * r.z;
      }
      for (int e = d.in_ptr[j]; e < d.in_ptr[j + 1]; ++e) {   // in-edges m -> j
        const int m = checked(d.in_src[e], d.n_n, d.status);
        const D3 pm = d3(d.node_p[m]);
        const D3 y = node_apply64(d, j, pm);
        const D3 r = sl * (node_apply64(d, m, pm) - y);
        add_reg_pair64(acc, l, y, y);
        const D3 yr = cross3(y, r);
        gj[0] -= sl * yr.x; gj[1] -= sl * yr.y; gj[2] -= sl * yr.z;
        gj[3] -= sl * r.x; gj[4] -= sl * r.y; gj[5] -= sl * r.z;
      }
      for (int k = 0; k < 6; ++k) d.g64[6 * j + k] = gj[k];
    } else {
      const int fl = d.blk_edge[b];
      if (fl & 1) {   // edge i -> j
        const D3 pi = d3(d.node_p[i]);
        add_reg_pair64(acc, -l, node_apply64(d, i, pi), node_apply64(d, j, pi));
      }
      if (fl & 2) {   // edge j -> i
        const D3 pj = d3(d.node_p[j]);
        add_reg_pair64(acc, -l, node_apply64(d, i, pj), node_apply64(d, j, pj));
      }
    }
    double* dst = d.A64 + (size_t)b * 36;
    for (int k = 0; k < 36; ++k) dst[k] = acc[k];
  }
  ereg = warp_sum_d(ereg);
  if ((threadIdx.x & 31) == 0 && ereg != 0.0) atomicAdd(d.e_reg + gn_it, ereg);
}

// One thread per surfel: FP64 blend and warp (Eq. 1-2), association, the
// point-to-plane residual (Eq. 10) and its 1x24 Jacobian, added to the
// system with FP64 atomics.
__global__ void __launch_bounds__(kSurfTile) k_data_assemble64(Batch bt, int gn_it) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kSurfTile + threadIdx.x;
  double res = 0.0;
  bool valid = false;
  if (i < d.n_s) {
    const float4 v4 = d.v_ref[i], n4 = d.n_ref[i];
    const int4 ids = checked4(d.knn[i], d.n_n, d.status);
    const float4 w = d.w[i];
    const int rs = checked(d.ref_slot[i], 4, d.status);
    const DQ64 b = blend4_64(d.dq64, ids, w, rs);
    const double n2 = dq_norm2(b);
    int pix = -1;
    D3 vl = d3(v4), nl = d3(n4);
    double inv = 0.0;
    if (n2 > 0.0) {
      inv = 1.0 / n2;
      vl = dq_transform(b, inv, d3(v4));
      nl = dq_rotate(b, inv, d3(n4));
      if (surfel_visible(d, i) && surfel_selected(d, *d.t_now, n4.w, d.tt[i].y))
        pix = associate_one(d, make_float3((float)vl.x, (float)vl.y, (float)vl.z),
                            make_float3((float)nl.x, (float)nl.y, (float)nl.z));
    }
    d.corr_pix[i] = pix;
    if (d.corr_rec) d.corr_rec[(size_t)gn_it * d.n_s + i] = pix;
    if (pix >= 0) {
      valid = true;
      const D3 V = d3(d.vmap[pix]), nd = d3(d.nmap[pix]);
      res = dot3(nd, vl - V);
      const DQGrad64 gr = point_plane_grad(b, inv, d3(v4), nd);
      const int id[4] = {ids.x, ids.y, ids.z, ids.w};
      const double wk[4] = {(double)w.x, (double)w.y, (double)w.z, (double)w.w};
      const DQ64 ref = load_dq64(d.dq64, id[rs]);
      double J[24];
      for (int k = 0; k < 4; ++k) {
        const DQ64 q = load_dq64(d.dq64, id[k]);
        const double ws = (q.W * ref.W + dot3(q.A, ref.A)) >= 0.0 ? wk[k] : -wk[k];
        node_jacobian(gr, q, ws, J + 6 * k);
      }
      const int* slots = d.set_slots + (size_t)checked(d.set_id[i], d.n_sets, d.status) * 14;
      int item = 0;
      for (int a = 0; a < 4; ++a)
        for (int c = a; c < 4; ++c, ++item) {
          double* dst = d.A64 + (size_t)checked(__ldg(slots + item), d.nnzb, d.status) * 36;
          for (int p = 0; p < 6; ++p)
            for (int q = 0; q < 6; ++q) atomicAdd(dst + p * 6 + q, J[6 * a + p] * J[6 * c + q]);
        }
      for (int a = 0; a < 4; ++a) {
        double* dst = d.g64 + (size_t)checked(__ldg(slots + 10 + a), d.n_n, d.status) * 6;
        for (int k = 0; k < 6; ++k) atomicAdd(dst + k, J[6 * a + k] * res);
      }
    }
  }
  const double e = warp_sum_d(res * res);
  const int nv = __popc(__ballot_sync(0xffffffffu, valid));
  if ((threadIdx.x & 31) == 0) {
    if (e != 0.0) atomicAdd(d.e_depth + gn_it, e);
    if (nv) atomicAdd(d.n_corr + gn_it, nv);
  }
}

// dq64 = the FP32 node transforms (after the host set them)
__global__ void k_dq_widen(const float4* dq, double* dq64, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const float4 a = dq[2 * j], b = dq[2 * j + 1];
  double* o = dq64 + 8 * (size_t)j;
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}

inline Batch with_kind(const BatchHost& b, int kind) {
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kind];
  return bt;
}

}  // namespace

void launch_reg_assemble64(const BatchHost& b, int gn_it, cudaStream_t st) {
  if (b.total_tiles[kTileBlocks])
    k_reg_assemble64<<<b.total_tiles[kTileBlocks], kBlkTile, 0, st>>>(with_kind(b, kTileBlocks), gn_it);
}
void launch_data_assemble64(const BatchHost& b, int gn_it, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels])
    k_data_assemble64<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels), gn_it);
}
void launch_dq_widen(const SwDev& d, cudaStream_t st) {
  if (d.dq64 && d.n_n > 0) k_dq_widen<<<(d.n_n + 127) / 128, 128, 0, st>>>(d.dq, d.dq64, d.n_n);
}

}  // namespace sw
