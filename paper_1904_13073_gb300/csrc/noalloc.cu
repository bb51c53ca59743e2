// sw_fusion_targets_static: the index map and fusion-target selection of
// Sec. 6.1 for callers that may not allocate device memory.  Inputs and the
// output are the caller's; the only scratch, the 4x super-sampled index map,
// is a fixed array in this file (see the declaration in surfelwarp.h for the
// limit, the one-time set-up and the rule that overlapping calls race).
#include <mutex>
#include <string>

#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"

namespace sw {
void set_process_error(const std::string& msg);   // capi.cu
}

namespace {

using namespace sw;

constexpr size_t kStaticEntries = size_t(16) * SW_STATIC_MAX_PIXELS;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kMaxDevices = 64;

// Held by every GPU that loads the library, for the life of the process.
static __device__ __align__(256) unsigned long long g_index_map[kStaticEntries];

std::mutex g_mu;
unsigned long long* g_addr[kMaxDevices] = {};

__global__ void k_clear(unsigned long long* imap, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    imap[i] = kEmptyKey;
}

// each surfel with z > 0 lands in at most one sub-pixel; nearest wins, then lower index
__global__ void k_index(const float4* __restrict__ v, int n, unsigned long long* imap, int W, int H, float fx,
                        float fy, float cx, float cy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = v[i];
  if (!(p.z > 0.f)) return;
  const float su = floorf(__fmul_rn(4.f, __fadd_rn(project_rn(fx, p.x, p.z, cx), 0.5f)));
  const float sv = floorf(__fmul_rn(4.f, __fadd_rn(project_rn(fy, p.y, p.z, cy), 0.5f)));
  if (!(su >= 0.f && su < (float)(4 * W) && sv >= 0.f && sv < (float)(4 * H))) return;
  const unsigned long long key = ((unsigned long long)__float_as_uint(p.z) << 32) | (unsigned)i;
  atomicMin(imap + (size_t)(int)sv * (4 * W) + (int)su, key);
}

// per depth pixel: its 16 sub-pixels; distance <= fuse_dist and normal dot >=
// fuse_normal; highest confidence, then nearest, then lowest index
__global__ void k_select(const float4* __restrict__ v, int n, const float4* __restrict__ nl,
                         const float4* __restrict__ vmap, const float4* __restrict__ nmap,
                         const unsigned long long* __restrict__ imap, int W, int H, float fuse_dist,
                         float fuse_normal, int* __restrict__ target) {
  const int pix = blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= W * H) return;
  const int x = pix % W, y = pix / W;
  const float4 V = vmap[pix];
  int best = -1;
  if (V.w > 0.f) {
    const float4 N = nmap[pix];
    const float fd2 = __fmul_rn(fuse_dist, fuse_dist);
    float bc = -__int_as_float(0x7f800000), bd = __int_as_float(0x7f800000);
    unsigned bo = 0xffffffffu;
    for (int sy = 0; sy < 4; ++sy)
      for (int sx = 0; sx < 4; ++sx) {
        const unsigned long long key = imap[(size_t)(4 * y + sy) * (4 * W) + 4 * x + sx];
        if (key == kEmptyKey) continue;
        const unsigned o = (unsigned)(key & 0xffffffffu);
        // checked build: this stream-free call has no status word, so an
        // out-of-range surfel id is skipped without a record
        if (!index_ok((long long)o, n, nullptr)) continue;
        const float4 a = v[o], b = nl[o];
        const float d2 = dist2_rn(a.x, a.y, a.z, V.x, V.y, V.z);
        const float dt = dot_rn(f3(b), f3(N));
        if (!(d2 <= fd2 && dt >= fuse_normal)) continue;
        if (b.w > bc || (b.w == bc && (d2 < bd || (d2 == bd && o < bo)))) {
          bc = b.w; bd = d2; bo = o; best = (int)o;
        }
      }
  }
  target[pix] = best;
}

}  // namespace

sw_status sw_fusion_targets_static(const float* v_live4, const float* n_live4, int n_surfels, const float* vmap4,
                                   const float* nmap4, int width, int height, float fx, float fy, float cx,
                                   float cy, float fuse_dist, float fuse_normal, int* target, void* cuda_stream) {
  if (width <= 0 || height <= 0 || n_surfels < 0) {
    set_process_error("sw_fusion_targets_static: sizes must be positive");
    return SW_ERR_INVALID_ARG;
  }
  if ((long long)width * height > SW_STATIC_MAX_PIXELS) {
    set_process_error("sw_fusion_targets_static: width * height exceeds SW_STATIC_MAX_PIXELS (76800)");
    return SW_ERR_INVALID_ARG;
  }
  if (!vmap4 || !nmap4 || !target || (n_surfels > 0 && (!v_live4 || !n_live4))) {
    set_process_error("sw_fusion_targets_static: null device pointer");
    return SW_ERR_INVALID_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_process_error(std::string("sw_fusion_targets_static: cudaGetDevice: ") + cudaGetErrorString(e));
    return SW_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_process_error("sw_fusion_targets_static: device ordinal " + std::to_string(dev) + " is beyond the " +
                      std::to_string(kMaxDevices) + " this entry point supports");
    return SW_ERR_CUDA;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) {
    set_process_error(std::string("sw_fusion_targets_static: cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    return SW_ERR_CUDA;
  }
  unsigned long long* imap = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
      // outside capture: the address in the current context (it changes
      // after a device reset or in another context), remembered for
      // captured calls
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_index_map);
      if (e != cudaSuccess) {
        set_process_error(std::string("sw_fusion_targets_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return SW_ERR_CUDA;
      }
      g_addr[dev] = static_cast<unsigned long long*>(p);
    } else if (!g_addr[dev]) {
      set_process_error("sw_fusion_targets_static: the first call on a device must not be under stream capture");
      return SW_ERR_CUDA;
    }
    imap = g_addr[dev];
  }
  const size_t entries = size_t(16) * width * height;
  k_clear<<<(unsigned)std::min<size_t>((entries + 255) / 256, 4096), 256, 0, st>>>(imap, entries);
  if (n_surfels > 0)
    k_index<<<(n_surfels + 255) / 256, 256, 0, st>>>(reinterpret_cast<const float4*>(v_live4), n_surfels, imap,
                                                      width, height, fx, fy, cx, cy);
  k_select<<<(width * height + 255) / 256, 256, 0, st>>>(
      reinterpret_cast<const float4*>(v_live4), n_surfels, reinterpret_cast<const float4*>(n_live4),
      reinterpret_cast<const float4*>(vmap4), reinterpret_cast<const float4*>(nmap4), imap, width, height,
      fuse_dist, fuse_normal, target);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_process_error(std::string("sw_fusion_targets_static: launch: ") + cudaGetErrorString(e));
    return SW_ERR_CUDA;
  }
  return SW_OK;
}
