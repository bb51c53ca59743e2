// Visibility prediction before the non-rigid solve (Sec. 7): the selected
// live surfels (stable or recently observed) are rendered as opaque disk
// splats spanned by their position, normal and radius into an index map at
// the depth image's resolution; a surfel that keeps at least one pixel is
// visible, and only visible surfels are associated in the frame's
// Gauss-Newton iterations.
//
//   k_vis_splat  one thread per surfel: its live position and normal under
//                the warp the solve starts from (Eq. 1-2; or the stored live
//                surfel), then every pixel within h of the pixel of its
//                centre, h = min(16, ceil(r f / (z − r)) + 1): the pixel ray
//                q = ((x − cx)/fx, (y − cy)/fy, 1) meets the splat's plane at
//                t = (n·v)/(n·q); the pixel is covered when t > 0 and
//                ‖t q − v‖² ≤ r²; a 64-bit atomicMin of (t bits << 32 |
//                caller's id) keeps the nearest splat, equal depths going to
//                the lower id.  All of it in exact-order FP32 (sw_math.cuh).
//   k_vis_mark   one thread per pixel: the winner is visible; the pixel is
//                reset to empty, so the map is cleared once at creation.
#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_assoc.cuh"

namespace sw {
namespace {

constexpr unsigned long long kVisEmpty = ~0ull;
constexpr int kVisMaxHalf = 16;

__global__ void __launch_bounds__(kSurfTile) k_vis_splat(Batch bt, int from_live) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  if (!d.visibility && !from_live) return;
  const int i = (blockIdx.x - __ldg(bt.tile_base + s)) * kSurfTile + threadIdx.x;
  if (i >= d.n_s) return;
  d.visible[i] = 0;
  const float4 nr = d.n_ref[i];
  if (!surfel_selected(d, *d.t_now, nr.w, d.tt[i].y)) return;
  float3 v, n;
  float r;
  if (from_live) {
    const float4 vl = d.v_live[i], nl = d.n_live[i];
    v = f3(vl); n = f3(nl); r = vl.w;
  } else {
    DQ b = blend4(d.dq, checked4(d.knn[i], d.n_n, d.status), d.w[i], checked(d.ref_slot[i], 4, d.status));
    const float n2 = dq_norm2(b);
    const float4 vr = d.v_ref[i];
    r = vr.w;
    if (n2 > 0.f) {
      const float inv = 1.f / n2;
      v = dq_transform(b, inv, f3(vr));
      n = dq_rotate(b, inv, f3(nr));
    } else {   // no usable weight: left in place, as the warp does
      v = f3(vr); n = f3(nr);
    }
  }
  if (!(v.z > 0.f)) return;
  const float den = __fsub_rn(v.z, r);
  if (!(den > 0.f)) return;
  const float hf = fminf(__fadd_rn(ceilf(__fdiv_rn(__fmul_rn(r, fmaxf(d.fx, d.fy)), den)), 1.f), (float)kVisMaxHalf);
  const float pxf = floorf(__fadd_rn(project_rn(d.fx, v.x, v.z, d.cx), 0.5f));
  const float pyf = floorf(__fadd_rn(project_rn(d.fy, v.y, v.z, d.cy), 0.5f));
  if (!(fabsf(pxf) < 1e9f && fabsf(pyf) < 1e9f)) return;
  // the square [p − h, p + h], clipped to the image (in float: p may be far outside)
  const float x0f = fmaxf(pxf - hf, 0.f), x1f = fminf(pxf + hf, (float)(d.W - 1));
  const float y0f = fmaxf(pyf - hf, 0.f), y1f = fminf(pyf + hf, (float)(d.H - 1));
  if (!(x0f <= x1f && y0f <= y1f)) return;
  const int x0 = (int)x0f, x1 = (int)x1f, y0 = (int)y0f, y1 = (int)y1f;
  const float nv = dot_rn(n, v);
  const float r2 = __fmul_rn(r, r);
  const unsigned id = (unsigned)d.orig_id[i];
  for (int y = y0; y <= y1; ++y) {
    const float qy = __fdiv_rn(__fsub_rn((float)y, d.cy), d.fy);
    for (int x = x0; x <= x1; ++x) {
      const float qx = __fdiv_rn(__fsub_rn((float)x, d.cx), d.fx);
      const float nq = __fadd_rn(__fadd_rn(__fmul_rn(n.x, qx), __fmul_rn(n.y, qy)), n.z);
      const float t = __fdiv_rn(nv, nq);
      if (!(t > 0.f)) continue;
      const float d2 = dist2_rn(__fmul_rn(t, qx), __fmul_rn(t, qy), t, v.x, v.y, v.z);
      if (!(d2 <= r2)) continue;
      atomicMin(d.vis_map + checked(y * d.W + x, (long long)d.W * d.H, d.status),
                ((unsigned long long)__float_as_uint(t) << 32) | id);
    }
  }
}

__global__ void __launch_bounds__(256) k_vis_mark(Batch bt, int from_live) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  if (!d.visibility && !from_live) return;
  const int tile = blockIdx.x - __ldg(bt.tile_base + s);
  const int tiles_x = (d.W + 31) / 32;
  const int x = (tile % tiles_x) * 32 + (threadIdx.x & 31);
  const int y = (tile / tiles_x) * 8 + (threadIdx.x >> 5);
  if (x >= d.W || y >= d.H) return;
  unsigned long long* cell = d.vis_map + (size_t)y * d.W + x;
  const unsigned long long key = *cell;
  if (key == kVisEmpty) return;
  *cell = kVisEmpty;
  d.visible[checked(d.inv_perm[checked((int)(key & 0xffffffffu), d.n_s, d.status)], d.n_s, d.status)] = 1;
}

inline Batch with_kind(const BatchHost& b, int kind) {
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kind];
  return bt;
}

}  // namespace

void launch_vis_splat(const BatchHost& b, int from_live, cudaStream_t st) {
  if (b.total_tiles[kTileSurfels])
    k_vis_splat<<<b.total_tiles[kTileSurfels], kSurfTile, 0, st>>>(with_kind(b, kTileSurfels), from_live);
}
void launch_vis_mark(const BatchHost& b, int from_live, cudaStream_t st) {
  if (b.total_tiles[kTilePixels])
    k_vis_mark<<<b.total_tiles[kTilePixels], 256, 0, st>>>(with_kind(b, kTilePixels), from_live);
}

}  // namespace sw
