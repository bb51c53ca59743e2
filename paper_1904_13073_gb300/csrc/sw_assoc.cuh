// Surfel selection and projective association (Sec. 7), shared by the FP32
// and the FP64 assembly.  Every test is an exact-order FP32 expression (see
// sw_math.cuh), so the decisions match any implementation that evaluates the
// same operations on the same FP32 inputs.
#pragma once
#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"

namespace sw {

// A surfel takes part in the solve when it is stable (confidence above
// δ_stable) or was observed within the last δ_recent frames.
__device__ __forceinline__ bool surfel_selected(const SwDev& d, int t_now, float conf, int t_obs) {
  return conf > d.stable_conf || (t_now - t_obs) <= d.recent_frames;
}

// With visibility prediction on, only the surfels that kept a pixel of the
// frame's splat index map are associated (k_visibility.cu).
__device__ __forceinline__ bool surfel_visible(const SwDev& d, int i) { return !d.visibility || d.visible[i]; }

// Projective association of one warped surfel; the depth pixel it projects
// to, or -1 if rejected (behind the camera, outside the image, not a usable
// depth surfel, farther than corr_dist, normals within corr_normal).
__device__ __forceinline__ int associate_one(const SwDev& d, float3 vl, float3 nl) {
  if (!(vl.z > 0.f)) return -1;
  const float u = project_rn(d.fx, vl.x, vl.z, d.cx);
  const float v = project_rn(d.fy, vl.y, vl.z, d.cy);
  const float px = floorf(__fadd_rn(u, 0.5f)), py = floorf(__fadd_rn(v, 0.5f));
  if (!(px >= 0.f && px < (float)d.W && py >= 0.f && py < (float)d.H)) return -1;
  const int pix = checked((int)py * d.W + (int)px, (long long)d.W * d.H, d.status);
  const float4 V = d.vmap[pix];
  if (!(V.w > 0.f)) return -1;
  const float4 N = d.nmap[pix];
  const float d2 = dist2_rn(vl.x, vl.y, vl.z, V.x, V.y, V.z);
  if (!(d2 < __fmul_rn(d.corr_dist, d.corr_dist))) return -1;
  if (!(dot_rn(nl, f3(N)) > d.corr_normal)) return -1;
  return pix;
}

}  // namespace sw
