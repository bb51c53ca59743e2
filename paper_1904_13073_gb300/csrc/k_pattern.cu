// Block-sparse pattern of JᵀJ, built on the device (used by the model set-up
// and by appending): the upper 6x6 blocks (a <= b) of every node pair that
// shares a surfel's 4-node set (the data term, Eq. 10), of every graph edge
// (the regulariser, Eq. 11) and every diagonal block.
//
//   k_pat_keys     a key (a << 16 | b) per upper pair of each set (10), per
//                  node diagonal (1) and per graph edge (8)
//   radix sort, then unique by scan + scatter: the blocks in row-major order
//   k_pat_blocks   row / column of each block and the row pointers (every
//                  row holds its diagonal block, so every row is present)
//   k_pat_edges    graph-edge flags of the off-diagonal blocks (bit 0: the
//                  edge row -> col, bit 1: col -> row), by binary search
//   k_rl_keys      the SpMV lists: block row i multiplies every block (i, j)
//                  and, transposed, every block (j, i) with j < i; one
//                  (row << 32 | block) key per entry, radix-sorted, so each
//                  row lists its blocks in increasing block index
//   k_rl_fill      the entries and the row pointers of those lists
//   k_set_slots    per set, its 10 upper blocks in (0,0)(0,1)(0,2)(0,3)(1,1)
//                  (1,2)(1,3)(2,2)(2,3)(3,3) order, then its 4 node ids

#include "sw_internal.h"
#include "sw_check.cuh"

namespace sw {
namespace {

constexpr int kPatThreads = 256;
inline int pblocks(long long n) { return (int)((n + kPatThreads - 1) / kPatThreads); }

__global__ void k_pat_keys(const int4* __restrict__ sets, int n_sets, const int* __restrict__ graph, int n_n,
                           uint32_t* __restrict__ keys) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n_sets) {
    const int4 s = sets[t];
    const int id[4] = {s.x, s.y, s.z, s.w};
    uint32_t* out = keys + (size_t)t * 10;
    int k = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = a; b < 4; ++b) out[k++] = ((uint32_t)id[a] << 16) | (uint32_t)id[b];
    return;
  }
  const int j = t - n_sets;
  if (j >= n_n) return;
  uint32_t* out = keys + (size_t)n_sets * 10 + (size_t)j * (1 + SW_K_GRAPH);
  out[0] = ((uint32_t)j << 16) | (uint32_t)j;
#pragma unroll
  for (int e = 0; e < SW_K_GRAPH; ++e) {
    const int i = graph[(size_t)j * SW_K_GRAPH + e];
    const int a = min(i, j), b = max(i, j);
    out[1 + e] = ((uint32_t)a << 16) | (uint32_t)b;
  }
}

__global__ void k_pat_head(const uint32_t* __restrict__ k, int n, int* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1 : 0;
}

__global__ void k_pat_unique(const uint32_t* __restrict__ k, const int* __restrict__ flag, const int* __restrict__ pos,
                             int n, uint32_t* __restrict__ out, int* __restrict__ count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) out[pos[i]] = k[i];
  if (i == n - 1) *count = pos[i] + flag[i];
}

__global__ void k_pat_blocks(const uint32_t* __restrict__ ukeys, int nnzb, int n_n, int* __restrict__ row_ptr,
                             int* __restrict__ col, int* __restrict__ blk_row, int* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nnzb) return;
  const int r = checked((int)(ukeys[b] >> 16), n_n, status);
  blk_row[b] = r;
  col[b] = (int)(ukeys[b] & 0xffffu);
  if (b == 0 || (int)(ukeys[b - 1] >> 16) != r) row_ptr[r] = b;
  if (b == nnzb - 1) row_ptr[n_n] = nnzb;
}

// index of block (a, b), a <= b, in row a (it exists by construction)
__device__ __forceinline__ int find_block(const int* __restrict__ row_ptr, const int* __restrict__ col, int a, int b) {
  int lo = row_ptr[a], hi = row_ptr[a + 1] - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (col[mid] < b) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_pat_edges(const int* __restrict__ graph, int n_n, const int* __restrict__ row_ptr,
                            const int* __restrict__ col, int* __restrict__ blk_edge, int* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_n * SW_K_GRAPH) return;
  const int j = t / SW_K_GRAPH, i = checked(graph[t], n_n, status);
  if (i == j) return;
  const int b = find_block(row_ptr, col, min(i, j), max(i, j));
  atomicOr(blk_edge + b, j < i ? 1 : 2);
}

// two keys per block: its own row's entry and, off the diagonal, the
// transposed entry in its column's row; the diagonal's second key sorts last
__global__ void k_rl_keys(const int* __restrict__ blk_row, const int* __restrict__ col, int nnzb,
                          unsigned long long* __restrict__ keys) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nnzb) return;
  const int r = blk_row[b], c = col[b];
  keys[2 * (size_t)b] = ((unsigned long long)r << 32) | (unsigned)b;
  keys[2 * (size_t)b + 1] = r == c ? ~0ull : (((unsigned long long)c << 32) | (unsigned)b);
}

__global__ void k_rl_fill(const unsigned long long* __restrict__ skeys, int n_ent, int n_n,
                          const int* __restrict__ blk_row, const int* __restrict__ col, int* __restrict__ rl_ptr,
                          int2* __restrict__ rl_ent, int nnzb, int* status) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_ent) return;
  const int row = checked((int)(skeys[k] >> 32), n_n, status), b = checked((int)(skeys[k] & 0xffffffffu), nnzb, status);
  rl_ent[k] = blk_row[b] == row ? make_int2(b, col[b]) : make_int2(b | int(0x80000000u), blk_row[b]);
  if (k == 0 || (int)(skeys[k - 1] >> 32) != row) rl_ptr[row] = k;
  if (k == n_ent - 1) rl_ptr[n_n] = n_ent;
}

__global__ void k_set_slots(const int4* __restrict__ sets, int n_sets, const int* __restrict__ row_ptr,
                            const int* __restrict__ col, int* __restrict__ slots) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_sets) return;
  const int4 s = sets[t];
  const int id[4] = {s.x, s.y, s.z, s.w};
  int* out = slots + (size_t)t * 14;
  int k = 0;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) out[k++] = find_block(row_ptr, col, id[a], id[b]);
#pragma unroll
  for (int a = 0; a < 4; ++a) out[10 + a] = id[a];
}

}  // namespace

size_t pattern_scratch_bytes(int n_keys, int n_rl_keys) {
  const size_t a = sort_scratch_bytes_u32(n_keys, false), b = scan_scratch_bytes(n_keys),
               c = sort_scratch_bytes_u64(n_rl_keys, false);
  return std::max(a, std::max(b, c));
}

cudaError_t launch_pattern_blocks(const int4* sets, int n_sets, const int* graph, int n_n, PatternScratch& w,
                                  cudaStream_t st) {
  const int K = 10 * n_sets + (1 + SW_K_GRAPH) * n_n;
  k_pat_keys<<<pblocks(n_sets + n_n), kPatThreads, 0, st>>>(sets, n_sets, graph, n_n, w.keys);
  cudaError_t e = radix_sort_u32(w.keys, w.skeys, nullptr, nullptr, K, 0, 32, w.tmp, w.tmp_bytes, st);
  if (e != cudaSuccess) return e;
  k_pat_head<<<pblocks(K), kPatThreads, 0, st>>>(w.skeys, K, w.flag);
  e = scan_sum(w.flag, w.pos, K, false, w.tmp, w.tmp_bytes, st);
  if (e != cudaSuccess) return e;
  k_pat_unique<<<pblocks(K), kPatThreads, 0, st>>>(w.skeys, w.flag, w.pos, K, w.keys, w.count);
  return cudaGetLastError();
}

cudaError_t launch_pattern_fill(const int4* sets, int n_sets, const int* graph, int n_n, int nnzb,
                                PatternScratch& w, unsigned long long* rl_keys, unsigned long long* rl_skeys,
                                const SwDev& d, cudaStream_t st) {
  k_pat_blocks<<<pblocks(nnzb), kPatThreads, 0, st>>>(w.keys, nnzb, n_n, d.row_ptr, d.col, d.blk_row, d.status);
  cudaError_t e = cudaMemsetAsync(d.blk_edge, 0, (size_t)nnzb * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_pat_edges<<<pblocks((long long)n_n * SW_K_GRAPH), kPatThreads, 0, st>>>(graph, n_n, d.row_ptr, d.col, d.blk_edge, d.status);
  k_rl_keys<<<pblocks(nnzb), kPatThreads, 0, st>>>(d.blk_row, d.col, nnzb, rl_keys);
  e = radix_sort_u64(rl_keys, rl_skeys, nullptr, nullptr, 2 * nnzb, 0, 64, w.tmp, w.tmp_bytes, st);
  if (e != cudaSuccess) return e;
  const int n_ent = 2 * nnzb - n_n;
  k_rl_fill<<<pblocks(n_ent), kPatThreads, 0, st>>>(rl_skeys, n_ent, n_n, d.blk_row, d.col, d.rl_ptr, d.rl_ent, nnzb, d.status);
  if (n_sets) k_set_slots<<<pblocks(n_sets), kPatThreads, 0, st>>>(sets, n_sets, d.row_ptr, d.col, d.set_slots);
  return cudaGetLastError();
}

}  // namespace sw
