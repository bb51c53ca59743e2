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
#include "sw_check.cuh"
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

// (d, i) < (e, j) in the order of the selection: distance, then node id
__device__ __forceinline__ bool knn_less(float d, int i, float e, int j) { return d < e || (d == e && i < j); }

__device__ __forceinline__ void knn_cswap(float* d, int* i, int a, int b) {
  if (knn_less(d[b], i[b], d[a], i[a])) {
    const float td = d[a]; d[a] = d[b]; d[b] = td;
    const int ti = i[a]; i[a] = i[b]; i[b] = ti;
  }
}

// The same selection with one warp per query, for few queries: lane l scans
// nodes l, l + 32, ... and keeps its own K best; five butterfly rounds merge
// the lanes' sorted lists (the lower half of a bitonic merge, c_k =
// min(a_k, b_{K-1-k}), then a K-element bitonic sort), so every lane ends
// with the K smallest (d², id) of all nodes: the same unique result as
// k_knn<K>.
template <int K>
__device__ __forceinline__ void knn_bitonic_sort(float* d, int* i) {
  if (K == 8) {
    knn_cswap(d, i, 0, 4); knn_cswap(d, i, 1, 5); knn_cswap(d, i, 2, 6); knn_cswap(d, i, 3, 7);
  }
  knn_cswap(d, i, 0, 2); knn_cswap(d, i, 1, 3);
  if (K == 8) { knn_cswap(d, i, 4, 6); knn_cswap(d, i, 5, 7); }
  knn_cswap(d, i, 0, 1); knn_cswap(d, i, 2, 3);
  if (K == 8) { knn_cswap(d, i, 4, 5); knn_cswap(d, i, 6, 7); }
}

template <int K>
__global__ void __launch_bounds__(kQThreads)
k_knn_warp(const float4* __restrict__ queries, int n_q, const float4* __restrict__ nodes, int n_n, int exclude_self,
           int* __restrict__ out_ids, float* __restrict__ out_d2) {
  static_assert(K == 4 || K == 8, "bitonic network for 4 or 8");
  const int qi = (blockIdx.x * kQThreads + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (qi >= n_q) return;   // uniform across the warp
  const float3 q = f3(queries[qi]);
  float bd[K];
  int bi[K];
#pragma unroll
  for (int k = 0; k < K; ++k) { bd[k] = __int_as_float(0x7f800000); bi[k] = 0x7fffffff; }
  for (int j = lane; j < n_n; j += 32) {
    if (exclude_self && j == qi) continue;
    const float4 p = __ldg(nodes + j);
    float cd = dist2_rn(q.x, q.y, q.z, p.x, p.y, p.z);
    int ci = j;
    if (knn_less(cd, ci, bd[K - 1], bi[K - 1])) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (knn_less(cd, ci, bd[k], bi[k])) {
          const float td = bd[k]; const int ti = bi[k];
          bd[k] = cd; bi[k] = ci;
          cd = td; ci = ti;
        }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float od[K];
    int oi[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      od[k] = __shfl_xor_sync(0xffffffffu, bd[k], o);
      oi[k] = __shfl_xor_sync(0xffffffffu, bi[k], o);
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (knn_less(od[K - 1 - k], oi[K - 1 - k], bd[k], bi[k])) { bd[k] = od[K - 1 - k]; bi[k] = oi[K - 1 - k]; }
    knn_bitonic_sort<K>(bd, bi);
  }
  if (lane < K) {
    int id = bi[0];
    float d = bd[0];
#pragma unroll
    for (int k = 1; k < K; ++k)
      if (lane == k) { id = bi[k]; d = bd[k]; }
    out_ids[(size_t)qi * K + lane] = id;
    if (out_d2) out_d2[(size_t)qi * K + lane] = d;
  }
}

// queries up to which a warp per query beats a thread per query (fills the GPU)
constexpr int kWarpKnnMaxQueries = 40000;

void knn4(const float4* queries, int n_q, const float4* nodes, int n_n, int* ids, float* d2, cudaStream_t st) {
  if (n_q <= kWarpKnnMaxQueries)
    k_knn_warp<4><<<(int)(((size_t)n_q * 32 + kQThreads - 1) / kQThreads), kQThreads, 0, st>>>(queries, n_q, nodes,
                                                                                                n_n, 0, ids, d2);
  else
    k_knn<4><<<(n_q + kQThreads - 1) / kQThreads, kQThreads, 0, st>>>(queries, n_q, nodes, n_n, 0, ids, d2);
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
  knn4(v_orig, n_s, d.node_p, d.n_n, ids, d2, st);
  k_skin_weights<<<(n_s + 255) / 256, 256, 0, st>>>(d2, ids, d.node_p, n_s, knn_out, w_out);
}

void launch_knn4(const float4* queries, int n_q, const float4* nodes, int n_n, int* ids, cudaStream_t st) {
  if (n_q == 0) return;
  knn4(queries, n_q, nodes, n_n, ids, nullptr, st);
}

void launch_node_graph(const SwDev& d, cudaStream_t st) {
  if (d.n_n <= kWarpKnnMaxQueries)
    k_knn_warp<8><<<(int)(((size_t)d.n_n * 32 + kQThreads - 1) / kQThreads), kQThreads, 0, st>>>(
        d.node_p, d.n_n, d.node_p, d.n_n, 1, d.graph, nullptr);
  else
    k_knn<8><<<(d.n_n + kQThreads - 1) / kQThreads, kQThreads, 0, st>>>(d.node_p, d.n_n, d.node_p, d.n_n, 1,
                                                                         d.graph, nullptr);
}

}  // namespace sw
