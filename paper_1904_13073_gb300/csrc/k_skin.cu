// K2 / K3: brute-force k-nearest-node search (Sec. 6.5 initialisation).
//
// K2 gives every surfel its 4 nearest nodes and the weights of Eq. 1,
// w_k = exp(−‖v − p_k‖² / (2 σ_k²)); K3 gives every node its 8 nearest other
// nodes (the graph of Eq. 11).  The squared distance that decides the
// selection is evaluated in FP32 round-to-nearest in the fixed order
// ((dx·dx) + (dy·dy)) + (dz·dz); candidates are visited in increasing node
// id and only a strictly smaller distance displaces a kept one, so ties go to
// the lower id.  Nodes are staged through shared memory in tiles.
#include "sw_internal.h"
#include "sw_math.cuh"

namespace sw {
namespace {

constexpr int kQThreads = 256;
constexpr int kNodeChunk = 1024;

template <int K>
__global__ void __launch_bounds__(kQThreads)
k_knn(const float4* __restrict__ queries, int n_q, const float4* __restrict__ nodes, int n_n,
      int exclude_self, int* __restrict__ out_ids, float* __restrict__ out_d2) {
  __shared__ float3 sn[kNodeChunk];
  const int qi = blockIdx.x * kQThreads + threadIdx.x;
  float3 q = make_float3(0.f, 0.f, 0.f);
  if (qi < n_q) q = f3(queries[qi]);
  float bd[K];
  int bi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { bd[k] = __int_as_float(0x7f800000); bi[k] = 0x7fffffff; }

  for (int base = 0; base < n_n; base += kNodeChunk) {
    const int cnt = min(kNodeChunk, n_n - base);
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kQThreads) sn[i] = f3(nodes[base + i]);
    __syncthreads();
    if (qi < n_q) {
      for (int i = 0; i < cnt; ++i) {
        const float3 p = sn[i];
        const float d2 = dist2_rn(q.x, q.y, q.z, p.x, p.y, p.z);
        const int id = base + i;
        if (d2 < bd[K - 1] && !(exclude_self && id == qi)) {
          // insert keeping (d2, id) ascending in lexicographic order
          float cd = d2;
          int ci = id;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            if (cd < bd[k] || (cd == bd[k] && ci < bi[k])) {
              const float td = bd[k]; const int ti = bi[k];
              bd[k] = cd; bi[k] = ci;
              cd = td; ci = ti;
            }
          }
        }
      }
    }
  }
  if (qi < n_q) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      out_ids[(size_t)qi * K + k] = bi[k];
      if (out_d2) out_d2[(size_t)qi * K + k] = bd[k];
    }
  }
}

__global__ void k_skin_weights(const float* __restrict__ d2, const int* __restrict__ ids,
                               const float4* __restrict__ nodes, int n_q,
                               int4* __restrict__ knn_out, float4* __restrict__ w_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_q) return;
  float w[4];
  int id[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    id[k] = ids[4 * i + k];
    const float sg = __ldg(&nodes[id[k]].w);
    w[k] = expf(-d2[4 * i + k] / (2.f * sg * sg));
  }
  knn_out[i] = make_int4(id[0], id[1], id[2], id[3]);
  w_out[i] = make_float4(w[0], w[1], w[2], w[3]);
}

}  // namespace

// knn_out / w_out: distance order, caller's surfel order (v_orig).
void launch_knn_skin(const SwDev& d, const float4* v_orig, int n_s, int* ids, float* d2, int4* knn_out,
                     float4* w_out, cudaStream_t st) {
  if (n_s == 0) return;
  k_knn<4><<<(n_s + kQThreads - 1) / kQThreads, kQThreads, 0, st>>>(v_orig, n_s, d.node_p, d.n_n, 0, ids, d2);
  k_skin_weights<<<(n_s + 255) / 256, 256, 0, st>>>(d2, ids, d.node_p, n_s, knn_out, w_out);
}

void launch_knn4(const float4* queries, int n_q, const float4* nodes, int n_n, int* ids, cudaStream_t st) {
  if (n_q == 0) return;
  k_knn<4><<<(n_q + kQThreads - 1) / kQThreads, kQThreads, 0, st>>>(queries, n_q, nodes, n_n, 0, ids, nullptr);
}

void launch_node_graph(const SwDev& d, cudaStream_t st) {
  k_knn<8><<<(d.n_n + kQThreads - 1) / kQThreads, kQThreads, 0, st>>>(d.node_p, d.n_n, d.node_p, d.n_n, 1,
                                                                       d.graph, nullptr);
}

}  // namespace sw
