// Internal declarations shared by the kernel translation units and the C-ABI.
//
// Per-stream device state is described by SwDev, a plain struct of device
// pointers and sizes.  Kernels take a pointer to an array of SwDev in device
// memory plus a tile table, so one launch can serve one stream or a batch of
// streams of uneven size (blockIdx.x -> (stream, tile) through a prefix sum
// of tiles per stream).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/surfelwarp.h"

namespace sw {

constexpr int kMaxGn = SW_MAX_GN_ITERS;
constexpr int kMaxPcg = SW_MAX_PCG_ITERS;
constexpr int kRedSlots = 2 * kMaxPcg + 2;   // rz0, then (pq_k, rz_k+1) per PCG iteration

// status bits written by kernels
constexpr int kStatusBreakdown = 1;          // a diagonal block is not positive definite, or pᵀAp <= 0
constexpr int kStatusBadIndex = 2;           // a gather index failed its range check

struct SwDev {
  // camera and parameters
  int W, H;
  float fx, fy, cx, cy;
  float sqrt_lambda, corr_dist, corr_normal, fuse_dist, fuse_normal, stable_conf;
  int recent_frames;
  int t_now;
  // sizes
  int n_s, n_n, n_sets, nnzb;
  // surfels, internal order (sorted by their 4-node set)
  float4* v_ref;      // x y z radius
  float4* n_ref;      // nx ny nz confidence
  int2* tt;           // t_init, t_observed
  int4* knn;          // node ids in ascending order
  float4* w;          // weights in the same order
  int* ref_slot;      // slot of the nearest node (sign reference of Eq. 1)
  int* set_id;        // index of the surfel's 4-node set
  int* orig_id;       // caller's surfel index
  int* inv_perm;      // caller's index -> internal index
  float4* v_live;     // forward-warped position (+ radius)
  float4* n_live;     // forward-warped normal (+ confidence)
  int* corr_pix;      // last association: pixel per surfel or -1
  // nodes
  float4* node_p;     // x y z sigma
  float4* dq;         // 2 per node
  int* graph;         // 8 per node
  int* in_ptr;        // in-edges (m -> j with j in N_m): CSR by j
  int* in_src;
  // depth maps
  float* depth;
  float4* vmap;       // V(u) and the depth-surfel confidence (0 if unusable)
  float4* nmap;       // N(u) and the depth-surfel radius
  unsigned long long* imap;  // 4W x 4H: (z bits << 32) | caller's surfel index
  int* fuse_target;   // per pixel: internal surfel index or -1
  // block-sparse JᵀJ (upper triangle incl. diagonal, 6x6 blocks, row-major)
  int* row_ptr;       // n_n + 1
  int* col;           // nnzb
  int* blk_row;       // nnzb
  int* blk_edge;      // bit0: graph edge row->col, bit1: col->row
  int* low_ptr;       // per row i: blocks (j, i) with j < i
  int* low_blk;
  int* set_slots;     // 14 per set: 10 upper blocks of (a<=b), then 4 node ids
  float* A;           // nnzb * 36
  float* g;           // 6 n_n
  // PCG
  float* Minv;        // n_n * 36
  float* x; float* r; float* z; float* p0; float* p1; float* q;
  double* red;        // kRedSlots
  // per-GN-iteration statistics
  double* e_depth;    // kMaxGn
  double* e_reg;      // kMaxGn
  int* n_corr;        // kMaxGn
  double* pcg_rz;     // kMaxGn
  int* status;
};

// tile table for batched launches: block b serves stream s with
// tile_base[s] <= b < tile_base[s+1]
struct Batch {
  const SwDev* devs;      // device array
  const int* tile_base;   // device array, n_streams + 1
  int n_streams;
};

__device__ __forceinline__ int find_stream(const Batch& bt, int b) {
  int lo = 0, hi = bt.n_streams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(bt.tile_base + mid) <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------ launchers
// Each launcher covers every stream of the batch; `tiles[s]` is the number of
// CTAs stream s needs and is turned into the device tile table by the caller.

enum TileKind { kTilePixels = 0, kTileSurfels, kTileSurfelsAssembly, kTileNodes, kTileBlocks, kTileRows6,
                kTileKinds };

struct BatchHost {
  Batch bt;
  int total_tiles[kTileKinds];
  int* tile_base_dev[kTileKinds];   // device, per kind
};

void launch_depth_maps(const BatchHost& b, cudaStream_t st);
void launch_knn_skin(const SwDev& d, const float4* v_orig, int n_s, int* ids_tmp, float* d2_tmp, int4* knn_out,
                     float4* w_out, cudaStream_t st);
void launch_node_graph(const SwDev& d, cudaStream_t st);
void launch_reg_assemble(const BatchHost& b, int gn_it, cudaStream_t st);
void launch_data_assemble(const BatchHost& b, int gn_it, cudaStream_t st);
void launch_pcg_init(const BatchHost& b, cudaStream_t st);
void launch_pcg_spmv(const BatchHost& b, int k, cudaStream_t st);
void launch_pcg_update(const BatchHost& b, int k, cudaStream_t st);
void launch_apply_update(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st);
void launch_warp_live(const BatchHost& b, cudaStream_t st);
void launch_index_map(const BatchHost& b, cudaStream_t st);
void launch_fuse(const BatchHost& b, int select_only, cudaStream_t st);
void launch_associate_only(const BatchHost& b, cudaStream_t st);

// tile sizes
constexpr int kSurfTile = 256;
constexpr int kAsmTile = 256;
constexpr int kNodeTile = 128;
constexpr int kBlkTile = 128;
constexpr int kRowTile = 192;   // 32 rows x 6 components

inline int tiles_for(int kind, const SwDev& d) {
  switch (kind) {
    case kTilePixels: return ((d.W + 31) / 32) * ((d.H + 7) / 8);   // 32x8 pixel tiles
    case kTileSurfels: return (d.n_s + kSurfTile - 1) / kSurfTile;
    case kTileSurfelsAssembly: return (d.n_s + kAsmTile - 1) / kAsmTile;
    case kTileNodes: return (d.n_n + kNodeTile - 1) / kNodeTile;
    case kTileBlocks: return (d.nnzb + kBlkTile - 1) / kBlkTile;
    case kTileRows6: return (6 * d.n_n + kRowTile - 1) / kRowTile;
  }
  return 0;
}

}  // namespace sw
