// K1: depth image processing (Sec. 5, Eq. 4).
//
// One thread per pixel; a CTA covers a 32x8 pixel tile whose depth values
// plus a one-pixel halo are staged in shared memory, so each depth value is
// read from HBM once per tile.  Writes V (x y z, confidence) and N (nx ny nz,
// radius) as float4; confidence 0 marks a pixel that is not a usable depth
// surfel (depth <= 0, image border, a neighbour without depth, or a zero
// cross product).
//
// Traffic per pixel: 4 B depth read (+ halo) and 32 B of maps written.
#include "sw_internal.h"
#include "sw_math.cuh"

namespace sw {
namespace {

constexpr int TX = 32, TY = 8;

__global__ void __launch_bounds__(TX * TY) k_depth_maps(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int tile = blockIdx.x - __ldg(bt.tile_base + s);
  const int tiles_x = (d.W + TX - 1) / TX;
  const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;

  __shared__ float sd[TY + 2][TX + 2];
  const float* __restrict__ D = d.depth;
  for (int i = threadIdx.x; i < (TX + 2) * (TY + 2); i += TX * TY) {
    const int ly = i / (TX + 2), lx = i % (TX + 2);
    const int gx = x0 + lx - 1, gy = y0 + ly - 1;
    sd[ly][lx] = (gx >= 0 && gx < d.W && gy >= 0 && gy < d.H) ? __ldg(D + gy * d.W + gx) : 0.f;
  }
  __syncthreads();

  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int x = x0 + lx, y = y0 + ly;
  if (x >= d.W || y >= d.H) return;

  const float ifx = 1.f / d.fx, ify = 1.f / d.fy;
  auto vert = [&](int dx, int dy) {
    const float z = sd[ly + 1 + dy][lx + 1 + dx];
    return make_float3(z * ((float)(x + dx) - d.cx) * ifx, z * ((float)(y + dy) - d.cy) * ify, z);
  };
  const float z = sd[ly + 1][lx + 1];
  const float3 v = z > 0.f ? vert(0, 0) : make_float3(0.f, 0.f, 0.f);

  float3 n = make_float3(0.f, 0.f, 0.f);
  bool ok = z > 0.f && x > 0 && y > 0 && x < d.W - 1 && y < d.H - 1 &&
            sd[ly + 1][lx] > 0.f && sd[ly + 1][lx + 2] > 0.f && sd[ly][lx + 1] > 0.f && sd[ly + 2][lx + 1] > 0.f;
  if (ok) {
    const float3 dyv = vert(0, 1) - vert(0, -1);
    const float3 dxv = vert(1, 0) - vert(-1, 0);
    const float3 c = cross3(dyv, dxv);
    const float nn = dot3(c, c);
    ok = nn > 0.f;
    if (ok) n = rsqrtf(nn) * c;
  }
  float conf = 0.f, radius = 0.f;
  if (ok) {
    const float ex = (float)x - d.cx, ey = (float)y - d.cy;
    const float g2 = (ex * ex + ey * ey) / (d.cx * d.cx + d.cy * d.cy);
    conf = expf(-g2 / (2.f * 0.36f));                      // φ = 0.6
    const float f = 0.5f * (d.fx + d.fy);
    const float nz = fmaxf(fabsf(n.z), 0.25881904510252074f);   // cos 75°
    radius = 1.41421356237309515f * z / (f * nz);
  }
  const int pix = y * d.W + x;
  d.vmap[pix] = make_float4(v.x, v.y, v.z, conf);
  d.nmap[pix] = make_float4(n.x, n.y, n.z, radius);
}

}  // namespace

void launch_depth_maps(const BatchHost& b, cudaStream_t st) {
  const int n = b.total_tiles[kTilePixels];
  if (n == 0) return;
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kTilePixels];
  k_depth_maps<<<n, TX * TY, 0, st>>>(bt);
}

}  // namespace sw
