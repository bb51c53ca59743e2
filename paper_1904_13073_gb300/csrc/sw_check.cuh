// Range checks of gather and scatter indices that kernels read from device
// memory or derive on the device: a pixel from a projection, a node id from
// the skinning, the graph or a set, a surfel id from an index map, a JᵀJ
// block slot from the set table or the pattern, a set id, a PCG table entry.
//
// They are compiled in only with -DSW_BOUNDS_CHECK (the library's checked
// build).  A failed check sets kStatusBounds in the stream's status word and
// yields index 0, so the access stays inside its (non-empty) array; the call
// that reads the status then returns SW_ERR_BOUNDS.  Without the flag every
// check is the identity and costs nothing.
#pragma once
#include "sw_internal.h"

namespace sw {

#ifdef SW_BOUNDS_CHECK
constexpr bool kBoundsChecked = true;
__device__ __forceinline__ bool index_ok(long long i, long long n, int* status) {
  if (i >= 0 && i < n) return true;
  if (status) atomicOr(status, kStatusBounds);
  return false;
}
#else
constexpr bool kBoundsChecked = false;
__device__ __forceinline__ bool index_ok(long long, long long, int*) { return true; }
#endif

__device__ __forceinline__ int checked(int i, long long n, int* status) {
  return index_ok(i, n, status) ? i : 0;
}
__device__ __forceinline__ int4 checked4(int4 v, long long n, int* status) {
  if (kBoundsChecked) {
    v.x = checked(v.x, n, status);
    v.y = checked(v.y, n, status);
    v.z = checked(v.z, n, status);
    v.w = checked(v.w, n, status);
  }
  return v;
}

// a count n that must lie in [0, cap]
__device__ __forceinline__ int checked_count(int n, long long cap, int* status) {
  return index_ok(n, cap + 1, status) ? n : 0;
}
// an SpMV list entry (block | transposed << 31, neighbour node)
__device__ __forceinline__ int2 checked_ent(int2 ent, int nnzb, int n_n, int* status) {
  if (kBoundsChecked) {
    ent.x = (int)((unsigned)ent.x & 0x80000000u) | checked(ent.x & 0x7fffffff, nnzb, status);
    ent.y = checked(ent.y, n_n, status);
  }
  return ent;
}
// a (CTA << 16) | slot pair of the cluster PCG's plan
__device__ __forceinline__ int checked_pair(int v, int n_cta, int n_slot, int* status) {
  if (kBoundsChecked && !(index_ok(v >> 16, n_cta, status) && index_ok(v & 0xffff, n_slot, status))) return 0;
  return v;
}

}  // namespace sw
