// Prefix sums and a stable least-significant-digit radix sort over device
// arrays.  The model set-up sorts the surfels by their 4-node set (Sec. 7's
// JᵀJ is assembled set by set) and numbers the distinct sets with a prefix
// sum; the JᵀJ pattern build sorts and de-duplicates node pairs; appending
// (Sec. 6.2-6.4) compacts flagged pixels, surfels and nodes in order and
// sorts the keys of the new node sets.
//
// Every kernel runs 256 threads on tiles of 4096 items (16 per thread).
//
// Scan (two launches; one when n fits a tile):
//   k_scan_reduce  each CTA sums its tile; the CTA that finishes last (a
//                  ticket counter, no waiting) scans the tile sums in place.
//   k_scan_apply   each CTA scans its tile through shared memory, starting
//                  from its tile's prefix.
//
// Radix sort, 8-bit digits from begin_bit up, per digit (two launches; the
// whole sort in one launch when n fits a tile):
//   k_radix_hist     each CTA counts its tile's digits into a digit-major
//                    table counts[d][tile]; the last CTA turns the table into
//                    exclusive offsets (digit by digit, tiles in order).
//   k_radix_scatter  each warp ranks its 512 keys in order, 32 at a time
//                    (match_any groups the lanes of one digit), the CTA adds
//                    the warps' counts per digit to the tile's offset, and
//                    every key goes to offset + rank.  Equal digits keep
//                    their order, so the sort is stable.
// Keys and values alternate between the output and a scratch copy so that
// the last digit lands in the output; the input is never written.
#include "sw_internal.h"

namespace sw {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // 4096
constexpr int kWarps = kThreads / 32;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kPadded = kTile + kTile / 32;
static_assert(kRadix == kThreads, "one thread per digit in the offset steps");

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
// shared-memory index with one pad word per 32, so that a thread's run of 16
// consecutive items is conflict-free
__device__ __forceinline__ int padi(int i) { return i + (i >> 5); }

// Exclusive scan of one value per thread over the CTA; `total` gets the sum.
__device__ int cta_exclusive_scan(int v, int* s_w, int& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(~0u, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_w[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < kWarps ? s_w[lane] : 0;
#pragma unroll
    for (int o = 1; o < kWarps; o <<= 1) {
      const int y = __shfl_up_sync(~0u, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) s_w[lane] = t;
  }
  __syncthreads();
  total = s_w[kWarps - 1];
  const int before = w ? s_w[w - 1] : 0;
  __syncthreads();   // s_w may be reused
  return before + x - v;
}

// Scans in[0, len) (len <= kTile) into out[0, len), starting from `carry`;
// in and out may be the same array.  Loads bypass L1: the values may have
// been written by other CTAs of the same launch.  Returns the tile's sum.
__device__ int scan_tile(const int* in, int* out, int len, int carry, bool inclusive, int* s, int* s_w) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int i = k * kThreads + tid;
    s[padi(i)] = i < len ? __ldcg(in + i) : 0;
  }
  __syncthreads();
  int v[kItems], sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    v[k] = s[padi(tid * kItems + k)];
    sum += v[k];
  }
  int total;
  int run = cta_exclusive_scan(sum, s_w, total) + carry;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    s[padi(tid * kItems + k)] = inclusive ? run + v[k] : run;
    run += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int i = k * kThreads + tid;
    if (i < len) out[i] = s[padi(i)];
  }
  __syncthreads();
  return total;
}

// Exclusive scan of data[0, n) in place by one CTA, a tile at a time.
__device__ void cta_scan_range(int* data, long long n, int* s, int* s_w) {
  int carry = 0;
  for (long long b = 0; b < n; b += kTile)
    carry += scan_tile(data + b, data + b, (int)(n - b < kTile ? n - b : kTile), carry, false, s, s_w);
}

// True in every thread of the CTA that arrives last at `ticket` (wraps to 0
// after `count` arrivals, so the counter is ready for the next launch).
// Every thread's global writes before the call are visible to that CTA.
__device__ bool last_cta(unsigned* ticket, unsigned count, bool* s_flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_flag = atomicInc(ticket, count - 1) == count - 1;
  __syncthreads();
  const bool last = *s_flag;
  if (last) __threadfence();
  return last;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int* __restrict__ in, int n, int* tile_sum,
                                                          unsigned* ticket, int n_tiles) {
  __shared__ int s[kPadded];
  __shared__ int s_w[kWarps];
  __shared__ bool s_last;
  const long long base = (long long)blockIdx.x * kTile;
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const long long i = base + k * kThreads + threadIdx.x;
    if (i < n) sum += in[i];
  }
  int total;
  cta_exclusive_scan(sum, s_w, total);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
  if (!last_cta(ticket, (unsigned)n_tiles, &s_last)) return;
  cta_scan_range(tile_sum, n_tiles, s, s_w);
}

__global__ void __launch_bounds__(kThreads) k_scan_apply(const int* in, int* out, int n, const int* tile_prefix,
                                                         bool inclusive) {
  __shared__ int s[kPadded];
  __shared__ int s_w[kWarps];
  const long long base = (long long)blockIdx.x * kTile;
  const int carry = tile_prefix ? __ldcg(tile_prefix + blockIdx.x) : 0;
  scan_tile(in + base, out + base, (int)(n - base < kTile ? n - base : kTile), carry, inclusive, s, s_w);
}

template <typename K>
__device__ __forceinline__ int digit_of(K key, int shift, int mask) {
  return (int)((key >> shift) & (K)mask);
}

template <typename K>
__global__ void __launch_bounds__(kThreads) k_radix_hist(const K* __restrict__ keys, int n, int shift, int mask,
                                                         int* counts, unsigned* ticket, int n_tiles) {
  __shared__ int hist[kRadix];
  __shared__ int s[kPadded];
  __shared__ int s_w[kWarps];
  __shared__ bool s_last;
  const int tid = threadIdx.x, lane = tid & 31;
  hist[tid] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
#pragma unroll 4
  for (int k = 0; k < kItems; ++k) {
    const long long i = base + k * kThreads + tid;
    const bool valid = i < n;
    const int d = valid ? digit_of(keys[i], shift, mask) : kRadix;
    const unsigned peers = __match_any_sync(~0u, d);
    if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[d], __popc(peers));
  }
  __syncthreads();
  counts[(long long)tid * n_tiles + blockIdx.x] = hist[tid];
  if (!last_cta(ticket, (unsigned)n_tiles, &s_last)) return;
  cta_scan_range(counts, (long long)kRadix * n_tiles, s, s_w);
}

// Ranks the keys of this CTA's tile: warp w takes the 512 keys from
// base + 512 w, 32 at a time, in order.  On return key/val/rk hold lane's
// keys, values and ranks among the warp's earlier keys of the same digit,
// and wcnt[w][d] the warp's count of digit d.
template <typename K, bool kVals>
__device__ __forceinline__ void rank_tile(const K* kin, const int* vin, long long n, long long base, int shift,
                                          int mask, K (&key)[kItems], int (&val)[kItems], int (&rk)[kItems],
                                          int (*wcnt)[kRadix]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long seg = base + (long long)w * (kItems * 32);
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int c = 0; c < kItems; ++c) {
    const long long i = seg + c * 32 + lane;
    const bool valid = i < n;
    key[c] = valid ? __ldcg(kin + i) : K(0);
    if (kVals) val[c] = valid ? __ldcg(vin + i) : 0;
    const int d = valid ? digit_of(key[c], shift, mask) : kRadix;
    const unsigned peers = __match_any_sync(~0u, d);
    const int before = valid ? wcnt[w][d] : 0;
    rk[c] = before + __popc(peers & lt);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
}

// wcnt[w][d] += the start of digit d's keys of warp w in the output, given
// the start of the tile's digit d (thread d); then every key is written.
template <typename K, bool kVals>
__device__ __forceinline__ void scatter_tile(K* kout, int* vout, long long n, long long base, int shift, int mask,
                                             int tile_start, const K (&key)[kItems], const int (&val)[kItems],
                                             const int (&rk)[kItems], int (*wcnt)[kRadix]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    int run = tile_start;
#pragma unroll
    for (int v = 0; v < kWarps; ++v) {
      const int c = wcnt[v][threadIdx.x];
      wcnt[v][threadIdx.x] = run;
      run += c;
    }
  }
  __syncthreads();
  const long long seg = base + (long long)w * (kItems * 32);
#pragma unroll
  for (int c = 0; c < kItems; ++c) {
    const long long i = seg + c * 32 + lane;
    if (i < n) {
      const int dst = wcnt[w][digit_of(key[c], shift, mask)] + rk[c];
      kout[dst] = key[c];
      if (kVals) vout[dst] = val[c];
    }
  }
}

template <typename K, bool kVals>
__global__ void __launch_bounds__(kThreads) k_radix_scatter(const K* kin, const int* vin, K* kout, int* vout, int n,
                                                            int shift, int mask, const int* offsets, int n_tiles) {
  __shared__ int wcnt[kWarps][kRadix];
  for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kTile;
  K key[kItems];
  int val[kItems], rk[kItems];
  rank_tile<K, kVals>(kin, vin, n, base, shift, mask, key, val, rk, wcnt);
  __syncthreads();
  const int start = __ldcg(offsets + (long long)threadIdx.x * n_tiles + blockIdx.x);
  scatter_tile<K, kVals>(kout, vout, n, base, shift, mask, start, key, val, rk, wcnt);
}

// n <= kTile: every digit in one CTA; keys alternate between the buffers as
// in the multi-tile sort (the CTA's own global writes are visible to it
// after the barrier).
template <typename K, bool kVals>
__global__ void __launch_bounds__(kThreads) k_radix_small(const K* kin, const int* vin, K* kout, int* vout, K* kalt,
                                                          int* valt, int n, int begin_bit, int end_bit) {
  __shared__ int wcnt[kWarps][kRadix];
  __shared__ int s_w[kWarps];
  const int passes = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
  const K* src = kin;
  const int* vsrc = vin;
  for (int p = 0; p < passes; ++p) {
    const int shift = begin_bit + p * kRadixBits;
    const int mask = (1 << min(kRadixBits, end_bit - shift)) - 1;
    const bool to_out = ((passes - 1 - p) & 1) == 0;
    K* dst = to_out ? kout : kalt;
    int* vdst = to_out ? vout : valt;
    for (int i = threadIdx.x; i < kWarps * kRadix; i += kThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    K key[kItems];
    int val[kItems], rk[kItems];
    rank_tile<K, kVals>(src, vsrc, n, 0, shift, mask, key, val, rk, wcnt);
    __syncthreads();
    int count = 0;
#pragma unroll
    for (int v = 0; v < kWarps; ++v) count += wcnt[v][threadIdx.x];
    int total;
    const int start = cta_exclusive_scan(count, s_w, total);
    scatter_tile<K, kVals>(dst, vdst, n, 0, shift, mask, start, key, val, rk, wcnt);
    __threadfence_block();
    __syncthreads();
    src = dst;
    vsrc = vdst;
  }
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
inline int tiles_of(long long n) { return (int)((n + kTile - 1) / kTile); }

template <typename K>
size_t radix_scratch(int n, bool values) {
  if (n <= 0) return 16;
  const size_t t = tiles_of(n);
  return align256((size_t)n * sizeof(K)) + (values ? align256((size_t)n * 4) : 0) + align256(t * kRadix * 4) + 16;
}

template <typename K>
cudaError_t radix_sort(const K* kin, K* kout, const int* vin, int* vout, int n, int begin_bit, int end_bit, void* tmp,
                       size_t tmp_bytes, cudaStream_t st) {
  const bool values = vin != nullptr;
  if (n < 0 || begin_bit < 0 || end_bit > (int)(8 * sizeof(K)) || begin_bit > end_bit || kin == kout ||
      (values && (vout == nullptr || vin == vout)))
    return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  if (begin_bit == end_bit) {
    cudaError_t e = cudaMemcpyAsync(kout, kin, (size_t)n * sizeof(K), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && values) e = cudaMemcpyAsync(vout, vin, (size_t)n * 4, cudaMemcpyDeviceToDevice, st);
    return e;
  }
  if (tmp == nullptr || tmp_bytes < radix_scratch<K>(n, values)) return cudaErrorInvalidValue;
  char* p = static_cast<char*>(tmp);
  K* kalt = reinterpret_cast<K*>(p);
  p += align256((size_t)n * sizeof(K));
  int* valt = nullptr;
  if (values) {
    valt = reinterpret_cast<int*>(p);
    p += align256((size_t)n * 4);
  }
  const int n_tiles = tiles_of(n);
  if (n_tiles == 1) {
    if (values)
      k_radix_small<K, true><<<1, kThreads, 0, st>>>(kin, vin, kout, vout, kalt, valt, n, begin_bit, end_bit);
    else
      k_radix_small<K, false><<<1, kThreads, 0, st>>>(kin, vin, kout, vout, kalt, valt, n, begin_bit, end_bit);
    return cudaGetLastError();
  }
  int* counts = reinterpret_cast<int*>(p);
  p += align256((size_t)n_tiles * kRadix * 4);
  unsigned* ticket = reinterpret_cast<unsigned*>(p);
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int passes = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
  const K* src = kin;
  const int* vsrc = vin;
  for (int pass = 0; pass < passes; ++pass) {
    const int shift = begin_bit + pass * kRadixBits;
    const int mask = (1 << std::min(kRadixBits, end_bit - shift)) - 1;
    const bool to_out = ((passes - 1 - pass) & 1) == 0;
    K* dst = to_out ? kout : kalt;
    int* vdst = to_out ? vout : valt;
    k_radix_hist<K><<<n_tiles, kThreads, 0, st>>>(src, n, shift, mask, counts, ticket, n_tiles);
    if (values)
      k_radix_scatter<K, true><<<n_tiles, kThreads, 0, st>>>(src, vsrc, dst, vdst, n, shift, mask, counts, n_tiles);
    else
      k_radix_scatter<K, false><<<n_tiles, kThreads, 0, st>>>(src, vsrc, dst, vdst, n, shift, mask, counts, n_tiles);
    src = dst;
    vsrc = vdst;
  }
  return cudaGetLastError();
}

}  // namespace

// scratch: the ticket counter in its first 16 bytes, then the tile sums
size_t scan_scratch_bytes(int n) { return n <= kTile ? 16 : 16 + (size_t)tiles_of(n) * 4; }

cudaError_t scan_sum(const int* in, int* out, int n, bool inclusive, void* tmp, size_t tmp_bytes, cudaStream_t st,
                     bool ticket_zero) {
  if (n < 0) return cudaErrorInvalidValue;
  if (n == 0) return cudaSuccess;
  const int n_tiles = tiles_of(n);
  if (n_tiles == 1) {
    k_scan_apply<<<1, kThreads, 0, st>>>(in, out, n, nullptr, inclusive);
    return cudaGetLastError();
  }
  if (tmp == nullptr || tmp_bytes < scan_scratch_bytes(n)) return cudaErrorInvalidValue;
  unsigned* ticket = static_cast<unsigned*>(tmp);
  int* tile_sum = reinterpret_cast<int*>(static_cast<char*>(tmp) + 16);
  if (!ticket_zero) {   // (a completed scan leaves the counter at 0)
    cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  k_scan_reduce<<<n_tiles, kThreads, 0, st>>>(in, n, tile_sum, ticket, n_tiles);
  k_scan_apply<<<n_tiles, kThreads, 0, st>>>(in, out, n, tile_sum, inclusive);
  return cudaGetLastError();
}

size_t sort_scratch_bytes_u32(int n, bool values) { return radix_scratch<uint32_t>(n, values); }
size_t sort_scratch_bytes_u64(int n, bool values) { return radix_scratch<unsigned long long>(n, values); }

cudaError_t radix_sort_u32(const uint32_t* kin, uint32_t* kout, const int* vin, int* vout, int n, int begin_bit,
                           int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t st) {
  return radix_sort<uint32_t>(kin, kout, vin, vout, n, begin_bit, end_bit, tmp, tmp_bytes, st);
}
cudaError_t radix_sort_u64(const unsigned long long* kin, unsigned long long* kout, const int* vin, int* vout, int n,
                           int begin_bit, int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t st) {
  return radix_sort<unsigned long long>(kin, kout, vin, vout, n, begin_bit, end_bit, tmp, tmp_bytes, st);
}

}  // namespace sw
