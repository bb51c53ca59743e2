// K9-K11: fusion at the live frame (Sec. 6.1, Eq. 5-6) and inverse warp (Eq. 3).
//
//   k_warp_live   S_live = W(S_ref) (Eq. 2) with the solved node transforms.
//   k_index_map   every live surfel is an unsized point in a 4x super-sampled
//                 map; a 64-bit atomicMin on (FP32 depth bits << 32 | caller's
//                 surfel id) keeps the nearest, equal depths going to the
//                 lower id.  Sub-pixel = floor(4 (u + ½)), u = fx x / z + cx,
//                 all in exact-order FP32.
//   k_fuse        one thread per depth pixel scans its own 16 sub-pixels,
//                 keeps candidates within δ_distance and with normal dot
//                 >= δ_normal, takes the highest confidence, then the
//                 smallest distance, then the lowest id; averages it with the
//                 depth surfel (Eq. 5-6), re-normalises the normal, stamps
//                 t_observed and warps it back to the reference frame with
//                 its own skinning (Eq. 3).  Every surfel belongs to exactly
//                 one pixel's window, so no two threads update one surfel.
//                 A usable pixel whose window held no surfel at all is marked
//                 kTargetEmptyWindow: the appending step's candidates.
#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"

namespace sw {
namespace {

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ DQ surfel_blend(const SwDev& d, int i, float& inv_n2) {
  DQ b = blend4(d.dq, checked4(d.knn[i], d.n_n, d.status), d.w[i], checked(d.ref_slot[i], 4, d.status));
  const float n2 = dq_norm2(b);
  if (n2 > 0.f) {
    inv_n2 = 1.f / n2;
  } else {   // no usable weight: identity (see the oracle's reading)
    b.W = 1.f; b.A = make_float3(0.f, 0.f, 0.f); b.We = 0.f; b.Ae = make_float3(0.f, 0.f, 0.f);
    inv_n2 = 1.f;
  }
  return b;
}

__global__ void __launch_bounds__(kSurfTile) k_warp_live(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kSurfTile + threadIdx.x;
  if (i >= d.n_s) return;
  float inv;
  const DQ b = surfel_blend(d, i, inv);
  const float4 v = d.v_ref[i], n = d.n_ref[i];
  const float3 vl = dq_transform(b, inv, f3(v)), nl = dq_rotate(b, inv, f3(n));
  d.v_live[i] = make_float4(vl.x, vl.y, vl.z, v.w);
  d.n_live[i] = make_float4(nl.x, nl.y, nl.z, n.w);
}

__global__ void __launch_bounds__(kSurfTile) k_index_map(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kSurfTile + threadIdx.x;
  if (i >= d.n_s) return;
  const float4 v = d.v_live[i];
  if (!(v.z > 0.f)) return;
  const float u = project_rn(d.fx, v.x, v.z, d.cx);
  const float w = project_rn(d.fy, v.y, v.z, d.cy);
  const float su = floorf(__fmul_rn(4.f, __fadd_rn(u, 0.5f)));
  const float sv = floorf(__fmul_rn(4.f, __fadd_rn(w, 0.5f)));
  if (!(su >= 0.f && su < (float)(4 * d.W) && sv >= 0.f && sv < (float)(4 * d.H))) return;
  const unsigned long long key =
      ((unsigned long long)__float_as_uint(v.z) << 32) | (unsigned long long)(unsigned)d.orig_id[i];
  atomicMin(d.imap + checked((int)sv * (4 * d.W) + (int)su, 16ll * d.W * d.H, d.status), key);
}

__global__ void __launch_bounds__(256) k_fuse(Batch bt, int select_only) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int tile = blockIdx.x - __ldg(bt.tile_base + s);
  const int tiles_x = (d.W + 31) / 32;
  const int x = (tile % tiles_x) * 32 + (threadIdx.x & 31);
  const int y = (tile / tiles_x) * 8 + (threadIdx.x >> 5);
  if (x >= d.W || y >= d.H) return;
  const int pix = y * d.W + x;
  const float4 V = d.vmap[pix];
  int best = -1;
  // This pixel owns its 16 sub-pixels.  In full mode it also leaves them empty
  // for the next frame, so the map is cleared once at creation and never again.
  unsigned long long* row0 = d.imap + (size_t)(4 * y) * (4 * d.W) + 4 * x;
  unsigned long long keys[16];
  bool empty = true;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    keys[k] = row0[(size_t)(k >> 2) * (4 * d.W) + (k & 3)];
    empty = empty && keys[k] == kEmpty;
  }
  if (!select_only) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (keys[k] != kEmpty) row0[(size_t)(k >> 2) * (4 * d.W) + (k & 3)] = kEmpty;
  }
  if (V.w > 0.f) {
    const float4 N = d.nmap[pix];
    const float fd2 = __fmul_rn(d.fuse_dist, d.fuse_dist);
    float bc = -__int_as_float(0x7f800000), bd = __int_as_float(0x7f800000);
    unsigned bo = 0xffffffffu;
#pragma unroll
    for (int sy = 0; sy < 4; ++sy) {
#pragma unroll
      for (int sx = 0; sx < 4; ++sx) {
        const unsigned long long key = keys[sy * 4 + sx];
        if (key == kEmpty) continue;
        const unsigned o = (unsigned)(key & 0xffffffffu);
        const int si = checked(d.inv_perm[checked((int)o, d.n_s, d.status)], d.n_s, d.status);
        const float4 vl = d.v_live[si], nl = d.n_live[si];
        const float d2 = dist2_rn(vl.x, vl.y, vl.z, V.x, V.y, V.z);
        const float dt = dot_rn(f3(nl), f3(N));
        if (!(d2 <= fd2 && dt >= d.fuse_normal)) continue;
        const float c = nl.w;
        if (c > bc || (c == bc && (d2 < bd || (d2 == bd && o < bo)))) {
          bc = c; bd = d2; bo = o; best = si;
        }
      }
    }
    if (best >= 0 && !select_only) {
      const float4 vl = d.v_live[best], nl = d.n_live[best];
      const float c_old = nl.w, cd = V.w, c_new = c_old + cd;
      const float ic = 1.f / c_new;
      const float3 v = ic * (c_old * f3(vl) + cd * f3(V));
      float3 n = ic * (c_old * f3(nl) + cd * f3(N));
      n = rsqrtf(dot3(n, n)) * n;
      const float r = ic * (c_old * vl.w + cd * N.w);
      d.v_live[best] = make_float4(v.x, v.y, v.z, r);
      d.n_live[best] = make_float4(n.x, n.y, n.z, c_new);
      float inv;
      const DQ b = surfel_blend(d, best, inv);
      const float3 vr = dq_inv_rotate(b, inv, v - dq_translation(b, inv));
      const float3 nr = dq_inv_rotate(b, inv, n);
      d.v_ref[best] = make_float4(vr.x, vr.y, vr.z, r);
      d.n_ref[best] = make_float4(nr.x, nr.y, nr.z, c_new);
      d.tt[best].y = *d.t_now;
    }
  }
  d.fuse_target[pix] = best >= 0 ? best : (V.w > 0.f && empty ? kTargetEmptyWindow : kTargetNone);
}

inline Batch with_kind(const BatchHost& b, int kind) {
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kind];
  return bt;
}

}  // namespace

void launch_warp_live(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels]) k_warp_live<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels));
}
void launch_index_map(const BatchHost& b, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels]) k_index_map<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels));
}
void launch_fuse(const BatchHost& b, int select_only, cudaStream_t st) {
  if (b.total_tiles[kTilePixels]) k_fuse<<<b.total_tiles[kTilePixels], 256, 0, st>>>(with_kind(b, kTilePixels), select_only);
}

}  // namespace sw
