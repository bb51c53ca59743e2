// K1: depth image processing (Sec. 5, Eq. 4).
//
// One thread per pixel; a CTA covers a 32x8 pixel tile whose depth values
// plus a one-pixel halo are staged in shared memory, so each depth value is
// read from HBM once per tile.  The staging is one TMA copy when the stream
// has a tensor map of its depth image (width a multiple of 4, so that rows
// are 16-byte aligned): a 40x10 box starting 4 columns and 1 row before the
// tile, so the box's first column stays on a 16-byte boundary, and reading
// zeros (= no depth) outside the image; else plain loads (and plain loads
// too if the copy's bounded wait runs out, which sets kStatusDepthTimeout:
// the maps are still right, the host reports the wait).  Writes V (x y z,
// confidence) and N (nx ny nz, radius) as float4; confidence 0 marks a pixel
// that is not a usable depth surfel (depth <= 0, image border, a neighbour
// without depth, or a zero cross product).
//
// Traffic per pixel: 4 B depth read (+ halo) and 32 B of maps written.
#include "sw_internal.h"
#include "sw_math.cuh"

namespace sw {
namespace {

constexpr int TX = 32, TY = 8;
constexpr int BX = 40, BY = TY + 2, BOX_X0 = 4;   // TMA box and its column offset before the tile
constexpr unsigned kBoxBytes = BX * BY * sizeof(float);

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// failure injection for the test of the bounded wait below: kFaultDepthTma
// withholds the copies (read at every launch)
__device__ int g_depth_fault;

// Bounded wait for phase 0 of the tile's mbarrier; true if it completed.
__device__ __forceinline__ bool wait_box(unsigned b) {
  unsigned done = 0;
  for (int spins = 0; spins < (1 << 16) && !done; ++spins) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(b), "r"(0u)
        : "memory");
  }
  return __syncthreads_and(done != 0) != 0;
}

// One TMA copy of the tile's box into shared memory, completed on an
// mbarrier; false if it did not complete within a bounded wait.
__device__ __forceinline__ bool tma_load_box(float (*box)[BX], unsigned long long* bar, const void* tmap, int x, int y,
                                             bool issue) {
  const unsigned b = smem_u32(bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long state;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;" : "=l"(state) : "r"(b), "r"(kBoxBytes) : "memory");
    (void)state;
    if (issue)
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
              smem_u32(&box[0][0])),
          "l"(tmap), "r"(x), "r"(y), "r"(b)
          : "memory");
  }
  return wait_box(b);
}

__global__ void __launch_bounds__(TX * TY) k_depth_maps(Batch bt) {
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int tile = blockIdx.x - __ldg(bt.tile_base + s);
  const int tiles_x = (d.W + TX - 1) / TX;
  const int x0 = (tile % tiles_x) * TX, y0 = (tile / tiles_x) * TY;

  __shared__ __align__(128) float box[BY][BX];
  __shared__ __align__(8) unsigned long long bar;
  const float* __restrict__ D = d.depth;
  bool staged = false;
  if (d.depth_tmap) {
    // x0 is a multiple of 32, so x0 - BOX_X0 is a multiple of 4 (16 bytes)
    const bool issue = g_depth_fault != kFaultDepthTma;
    staged = tma_load_box(box, &bar, d.depth_tmap, x0 - BOX_X0, y0 - 1, issue);
    if (!staged) {
      if (threadIdx.x == 0) atomicOr(d.status, kStatusDepthTimeout);
      // a copy still in flight writes the same values the plain loads
      // below do; wait for it once more (bounded) so that none is left
      // running when the CTA ends
      if (issue) wait_box(smem_u32(&bar));
    }
  }
  if (!staged) {   // plain loads into the same layout
    for (int i = threadIdx.x; i < BX * BY; i += TX * TY) {
      const int ly = i / BX, lx = i % BX;
      const int gx = x0 - BOX_X0 + lx, gy = y0 - 1 + ly;
      box[ly][lx] = (gx >= 0 && gx < d.W && gy >= 0 && gy < d.H) ? __ldg(D + gy * d.W + gx) : 0.f;
    }
    __syncthreads();
  }

  const int lx = threadIdx.x % TX, ly = threadIdx.x / TX;
  const int x = x0 + lx, y = y0 + ly;
  if (x >= d.W || y >= d.H) return;

  const float ifx = 1.f / d.fx, ify = 1.f / d.fy;
  auto vert = [&](int dx, int dy) {
    const float z = box[ly + 1 + dy][lx + BOX_X0 + dx];
    return make_float3(z * ((float)(x + dx) - d.cx) * ifx, z * ((float)(y + dy) - d.cy) * ify, z);
  };
  const float z = box[ly + 1][lx + BOX_X0];
  const float3 v = z > 0.f ? vert(0, 0) : make_float3(0.f, 0.f, 0.f);

  float3 n = make_float3(0.f, 0.f, 0.f);
  bool ok = z > 0.f && x > 0 && y > 0 && x < d.W - 1 && y < d.H - 1 &&
            box[ly + 1][lx + BOX_X0 - 1] > 0.f && box[ly + 1][lx + BOX_X0 + 1] > 0.f &&
            box[ly][lx + BOX_X0] > 0.f && box[ly + 2][lx + BOX_X0] > 0.f;
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

void set_depth_wait_fault(int kind) { cudaMemcpyToSymbol(g_depth_fault, &kind, sizeof(int)); }

void launch_depth_maps(const BatchHost& b, cudaStream_t st) {
  const int n = b.total_tiles[kTilePixels];
  if (n == 0) return;
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kTilePixels];
  k_depth_maps<<<n, TX * TY, 0, st>>>(bt);
}

}  // namespace sw
