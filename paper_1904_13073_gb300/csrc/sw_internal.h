// Internal declarations shared by the kernel translation units and the C-ABI.
//
// Per-stream device state is described by SwDev, a plain struct of device
// pointers and immutable sizes; everything that changes per frame lives behind
// a pointer, so a stream's descriptor can be copied into any number of batch
// tables.  Kernels take a Batch: an array of SwDev in device memory plus a tile
// table, so one launch serves one stream or many streams of uneven size
// (blockIdx.x -> (stream, tile) through a prefix sum of tiles per stream).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/surfelwarp.h"

namespace sw {

constexpr int kMaxGn = SW_MAX_GN_ITERS;
constexpr int kMaxPcg = SW_MAX_PCG_ITERS;
constexpr int kMaxCtaPerStream = 1024;   // CTAs of the persistent PCG that one stream may own
constexpr int kMaxRigid = SW_MAX_RIGID_ITERS;
constexpr int kRigidSlots = 16;          // rigid pre-alignment state: T (8), stopped flag, spare
constexpr int kRigidSums = 29;           // per surfel tile: 21 (J Jᵀ upper) + 6 (J r) + count + Σ r²

// fusion result of a pixel without a target surfel
constexpr int kTargetNone = -1;          // its window held surfels, none passed the tests (or unusable)
constexpr int kTargetEmptyWindow = -2;   // usable, and its window held no surfel: an append candidate

// status bits written by kernels
constexpr int kStatusBreakdown = 1;      // a diagonal block is not positive definite, or pᵀAp <= 0
constexpr int kStatusTimeout = 4;        // a bounded wait of the PCG (a reduction or a neighbour's vector) gave up
constexpr int kStatusDepthTimeout = 8;   // the depth stage's bounded wait for its TMA tile gave up (the tile was
                                         // then loaded with plain loads); cleared by the next depth upload
constexpr int kStatusBounds = 16;       // checked build (-DSW_BOUNDS_CHECK): a device index was out of range

// Failure injection for the tests of the bounded device waits
// (sw_debug_inject_wait_fault): what a kernel withholds so that the waits
// that depend on it must run out.  Each kernel file keeps its own device
// copy of the setting, read at every launch.
enum WaitFault {
  kFaultNone = 0,
  kFaultPcgPartial = 1,   // CTA 1 of the first stream does not publish its share of the PCG's first reduction
  kFaultPcgVector = 2,    // CTA 1 of the first stream does not publish its rows' first PCG vector
  kFaultDepthTma = 3,     // the depth tiles' TMA copies are not issued (their mbarrier waits run out)
};
void set_pcg_wait_fault(int kind, int spin_limit);   // k_pcg.cu
void set_depth_wait_fault(int kind);                 // k_depth.cu

// A CTA's partial of one reduction (the accumulator's bit pattern),
// published with a generation stamp (release pattern: the value, a fence,
// then `gen`); slots are double-buffered by the parity of the reduction's
// index.
struct __align__(16) PartSlot {
  unsigned long long v;
  unsigned long long gen;
};

struct SwDev {
  // camera and parameters
  int W, H;
  float fx, fy, cx, cy;
  float sqrt_lambda, corr_dist, corr_normal, fuse_dist, fuse_normal, stable_conf;
  int recent_frames;
  int precision;      // SW_PRECISION_*
  int visibility;     // 1: splat visibility gates the association
  // sizes
  int n_s, n_n, n_sets, nnzb;
  int* t_now;         // current frame id (device scalar)
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
  int* corr_rec;      // null, or [kMaxGn][n_s]: every Gauss-Newton iteration's association (test hook)
  // nodes
  float4* node_p;     // x y z sigma
  float4* dq;         // 2 per node
  int* graph;         // 8 per node
  int* in_ptr;        // in-edges (m -> j with j in N_m): CSR by j
  int* in_src;
  // depth maps
  float* depth;
  const void* depth_tmap;   // TMA descriptor (CUtensorMap) of `depth`, or null: plain loads
  float4* vmap;       // V(u) and the depth-surfel confidence (0 if unusable)
  float4* nmap;       // N(u) and the depth-surfel radius
  unsigned long long* imap;  // 4W x 4H: (z bits << 32) | caller's surfel index
  int* fuse_target;   // per pixel: internal surfel index, kTargetNone or kTargetEmptyWindow
  unsigned long long* vis_map;   // W x H splat index map: (depth bits << 32) | caller's surfel index
  int* visible;       // per surfel: kept a pixel of the frame's splat index map
  // block-sparse JᵀJ (upper triangle incl. diagonal, 6x6 blocks, row-major)
  int* row_ptr;       // n_n + 1; the diagonal block leads its row
  int* col;           // nnzb
  int* blk_row;       // nnzb
  int* blk_edge;      // bit0: graph edge row->col, bit1: col->row
  int* rl_ptr;        // n_n + 1: per block row, every block that multiplies into it
  int2* rl_ent;       //   (block | transposed << 31, neighbour node)
  int* set_slots;     // 14 per set: 10 upper blocks of (a<=b), then 4 node ids
  // the system JᵀJ (upper blocks) and Jᵀe in two buffers: Gauss-Newton
  // iteration k assembles into buffer k mod 2 (sys_A, sys_g) while
  // clearing the other for iteration k + 1
  float* A;           // nnzb * 36, buffer 0
  float* g;           // 6 n_n, buffer 0
  float* A2;          // buffer 1
  float* g2;
  // PCG
  float* minv;        // n_n * 21: block-Jacobi preconditioner, inverse of each diagonal block, packed lower
  struct PartSlot* part;   // 4 * kMaxCtaPerStream slots for the per-CTA partials of the PCG's reductions
  unsigned long long* xp;  // 12 n_n tagged words: the PCG's u = M⁻¹ r as other CTAs read it, by iteration parity
  unsigned long long* pcg_epoch;   // launches of the persistent PCG so far
  const int* cplan;   // the cluster PCG's plan of this stream (k_pcg_cluster.cu), or null: the cooperative PCG
  // all-FP64 variant only (null otherwise): the system, the PCG's shared
  // vectors (u, m even, m odd) and the authoritative node transforms
  double* A64;        // nnzb * 36
  double* g64;        // 6 n_n
  double* minv64;     // n_n * 21, the preconditioner in the FP64 mode
  double* v64;        // 3 * 6 n_n
  double* dq64;       // 8 per node
  // rigid pre-alignment
  double* rigid;        // kRigidSlots: T as a dual quaternion, then a stopped flag
  float* rigid_part;    // per surfel tile, kRigidSums partial sums
  double* rigid_stats;  // per iteration: correspondences, Σ r²
  // per-GN-iteration statistics
  double* e_depth;    // kMaxGn
  double* e_reg;      // kMaxGn
  int* n_corr;        // kMaxGn
  double* pcg_rz;     // kMaxGn
  int* status;
};

// A launch over several streams: block b serves stream s with
// tile_base[s] <= b < tile_base[s+1]; streams whose active flag is 0 skip
// their tiles (the persistent PCG still takes part in its barriers).
struct Batch {
  const SwDev* devs;      // device array
  const int* tile_base;   // device array, n_streams + 1
  const int* active;      // device array or null (all active)
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

__device__ __forceinline__ bool stream_active(const Batch& bt, int s) { return !bt.active || __ldg(bt.active + s); }

// the system buffers that Gauss-Newton iteration gn_it assembles into and solves
__device__ __forceinline__ float* sys_A(const SwDev& d, int gn_it) { return (gn_it & 1) ? d.A2 : d.A; }
__device__ __forceinline__ float* sys_g(const SwDev& d, int gn_it) { return (gn_it & 1) ? d.g2 : d.g; }

// Programmatic dependent launch along the Gauss-Newton loop: a kernel
// launched by launch_overlapped may begin while the previous launch on the
// stream still runs.  Such a kernel calls pdl_begin first: it waits until
// that launch has completed and its writes are visible (so everything it
// reads is current, and its own completion implies the previous one's),
// then lets the next launch begin.  Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_overlapped(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                                     Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------------ launchers

enum TileKind { kTilePixels = 0, kTileSurfels, kTileSurfelsAssembly, kTileBlocks, kTilePcg, kTileNodes, kTilePrecond,
                kTileRegAssembly, kTileKinds };

struct BatchHost {
  Batch bt;
  int total_tiles[kTileKinds];
  int* tile_base_dev[kTileKinds];   // device, per kind
  int spin_limit;                   // bounded wait of the PCG's reductions (polls)
  int pcg_rows_cap;                 // most rows one PCG CTA owns in the batch
  int precision;                    // SW_PRECISION_* shared by every member
  int pcg_ent_cap;                  // most matrix entries (block-row terms) one PCG CTA owns
  int pcg_mode;                     // how the PCG's SpMV reaches the matrix (k_pcg.cu: SpmvMode)
  int any_visibility;               // some member predicts splat visibility
  // members solved by the cluster PCG (k_pcg_cluster.cu): one cluster of
  // cluster_ctas CTAs each, cluster_smem bytes of shared memory per CTA
  int n_cluster;
  int cluster_ctas;
  size_t cluster_smem;
  const int* cluster_members_dev;   // device, n_cluster stream indices
};

void launch_depth_maps(const BatchHost& b, cudaStream_t st);
void launch_knn_skin(const SwDev& d, const float4* v_orig, int n_s, int* ids_tmp, float* d2_tmp, int4* knn_out,
                     float4* w_out, cudaStream_t st);
void launch_node_graph(const SwDev& d, cudaStream_t st);
void launch_solve_begin(const BatchHost& b, cudaStream_t st);
// zeroes system buffer 0 of every active stream (before a solve's first assembly)
void launch_system_clear(const BatchHost& b, cudaStream_t st);
// Gauss-Newton iteration gn_it's assembly (FP32 modes): regulariser and data
// terms into system buffer gn_it mod 2, which must be zero; clears the other
void launch_assemble(const BatchHost& b, int gn_it, cudaStream_t st);
// the block-Jacobi preconditioner of every active stream (inverse of each
// diagonal block of the system iteration gn_it assembled)
void launch_precond(const BatchHost& b, int gn_it, cudaStream_t st);
cudaError_t launch_pcg(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st);
void launch_reg_assemble64(const BatchHost& b, int gn_it, cudaStream_t st);
void launch_data_assemble64(const BatchHost& b, int gn_it, cudaStream_t st);
void launch_dq_widen(const SwDev& d, cudaStream_t st);
void launch_warp_live(const BatchHost& b, cudaStream_t st);
void launch_rigid_align(const BatchHost& b, int iters, cudaStream_t st);
void launch_index_map(const BatchHost& b, cudaStream_t st);
// splat visibility: from_live = 0 warps each surfel with the current node
// transforms (members without visibility skip), 1 renders the stored live
// surfels of every member
void launch_vis_splat(const BatchHost& b, int from_live, cudaStream_t st);
void launch_vis_mark(const BatchHost& b, int from_live, cudaStream_t st);
void launch_fuse(const BatchHost& b, int select_only, cudaStream_t st);
void launch_associate_only(const BatchHost& b, cudaStream_t st);
// the cluster PCG (k_pcg_cluster.cu): the plan's host
// build (false if the stream does not fit clusters of C CTAs with smem_limit
// bytes each), whether such clusters can run, and the launch over the
// batch's cluster members
bool build_cluster_plan(int C, int n_n, const std::vector<int>& row_ptr, const std::vector<int>& col,
                        const std::vector<float>& node4, size_t smem_limit, std::vector<int>& plan,
                        size_t* smem_out);
bool cluster_pcg_fits(int precision, int C, size_t smem);
int cluster_pcg_active(int precision, int C, size_t smem);   // clusters that can run at once (< 0: CUDA error)
cudaError_t cluster_barrier_cost(int C, double* us_per_barrier);   // one cluster barrier, measured
cudaError_t launch_pcg_cluster(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st);
int pcg_blocks_per_sm(int precision);
int pcg_threads();
size_t pcg_smem_bytes(int rows_cap, int ent_cap, int precision, int mode);
// Wait for a batch's work and turn each member's device status word into
// its sw_status (SW_OK for inactive members); `status` has one entry per member.
sw_status batch_member_status(sw_batch_handle b, int* status);
// the PCG's 6x6 block inverse on n row-major blocks (float, or double with fp64), packed lower out
// mode 0: FP32 blocks, double-float inverse (the default precision's); 1: FP64
// blocks, FP64 inverse; 2: FP32 blocks, FP64 inverse (SW_PRECISION_MIXED_F64DOTS)
cudaError_t launch_debug_block_inverse(const void* blocks, int n, int mode, void* out, int* ok, cudaStream_t st);

// ------------------------------------------------------------------ appending
// Per-candidate records and scratch of the appending step (k_append.cu),
// owned by the stream and sized for W·H candidates.
struct AppendBufs {
  float4* live;       // n_n warped nodes: T_j p_j rounded to FP32, w = σ_j
  int* cand;          // candidate pixels, row-major order
  float4* query;      // the candidates' depth vertices
  int* knn;           // 4 per candidate: nearest warped nodes, distance order
  int* flags;         // per candidate: bits 0-3 the nodes Eq. 7 keeps, then kApp* bits
  double* wsum;       // Σ of the live weights
  double* strain;     // 9 per candidate: ∂x_ref/∂x_live, row-major
  float4* w;          // the live weights (0 for removed nodes)
  float4* v;          // v_ref and the depth surfel's radius
  float4* n;          // n_ref and the depth surfel's confidence
  int* acc;           // accepted candidates, in candidate order
  int* stay;          // per existing surfel, caller order: 1 if it stays
  int* pos;           // its new caller index (exclusive scan of stay)
  int* counts;        // kAppCounts device counters
  void* scan_tmp;     // compaction scan scratch
  size_t scan_bytes;
};
constexpr int kAppAccepted = 16, kAppLowWeight = 32, kAppCompressive = 64;
enum AppCount { kAppNCand = 0, kAppNAcc, kAppNLow, kAppNComp, kAppNStay, kAppCounts = 8 };
struct AppendParams {
  float lo2, hi2;     // (1 − ε)², (1 + ε)² rounded to FP32 (Eq. 7 on squares)
  double bound2;      // (1 + ε)² (Eq. 8 on λ_max(JᵀJ))
  double delta_nn;    // weight-sum threshold
  double h;           // finite-difference step of the strain, metres
  int t_low;          // t_low_confid
};
size_t append_scan_bytes(int n_pixels, int n_surfels);
cudaError_t launch_append_candidates(const SwDev& d, const AppendBufs& a, cudaStream_t st);
cudaError_t launch_append_eval(const SwDev& d, const AppendBufs& a, const AppendParams& ap, int n_cand,
                               cudaStream_t st);
cudaError_t launch_append_removal(const SwDev& d, const AppendBufs& a, int t_low, cudaStream_t st);
// the new model in caller order: survivors, then the first n_app accepted candidates
void launch_append_compose(const SwDev& d, const AppendBufs& a, const int4* knn_dist, const float4* w_dist,
                           int n_stay, int n_app, float4* tv, float4* tn, int2* tt, int4* tknn, float4* tw,
                           cudaStream_t st);
void launch_knn4(const float4* queries, int n_q, const float4* nodes, int n_n, int* ids, cudaStream_t st);
// the fast model update after appending (k_append.cu): each appended surfel's
// existing set (or -1, counted in *missing), then the appended surfels placed
// after the first `first` surfels of the internal order with those sets
void launch_find_sets(const SwDev& d, int sorted_sets, const int4* tknn, int first, int n_app, int* set_of,
                      unsigned long long* keys, int* missing, cudaStream_t st);
// new sets of the appended surfels: the distinct keys among the n_missing
// that `keys` holds (~0 for surfels that have a set) get the ids n_sets,
// n_sets + 1, ... and their 10 blocks of the pattern in set_slots (which must
// have room); *no_block = 1 when a pair of their nodes has no block (scratch:
// sorted n_app keys, head and rank n_app ints each)
size_t new_sets_scratch_bytes(int n);
cudaError_t launch_new_sets(const SwDev& d, const unsigned long long* keys, unsigned long long* sorted, int* head,
                            int* rank, int n_app, int n_missing, int* set_of, int* n_new_sets, int* no_block,
                            void* tmp, size_t tmp_bytes, cudaStream_t st);
// the node ids of the sets [0, n) of a set table (14 ints per set) into sets[n]
void launch_slot_sets(const int* slots, int n, int4* sets, cudaStream_t st);
void launch_append_internal(const SwDev& d, const float4* tv, const float4* tn, const int2* tt, const int4* tknn,
                            const float4* tw, int first, int n_app, const int* set_of, cudaStream_t st);
// node-graph extension after appending (k_append.cu): coverage flags of the
// surfels tv[first, first + n) (1 = uncovered), the greedy sub-sampling that
// writes new nodes to node_p[n_old ..] and their count to *n_new (scratch:
// unc_list n_app ints; near 2 n_app ints; sig 20 n_app + 16 bytes, the σ then
// n_app float4 from a 16-byte boundary; n_new two ints), the new
// transforms from the current warp (ids: their 4 nearest old nodes), and the
// merge of every surfel's set with the new nodes
void launch_node_cover(const SwDev& d, const float4* tv, int first, int n, int* unc, cudaStream_t st);
cudaError_t launch_node_subsample(const SwDev& d, const AppendBufs& a, const float4* tv, int first, int n_app,
                                  const int* unc_flags, int* unc_list, int* n_unc, float* sig, int* near,
                                  int n_old, int max_new, int* n_new, cudaStream_t st);
void launch_new_node_dq(const SwDev& d, int n_old, int k_new, const int* ids, cudaStream_t st);
void launch_skin_merge(const SwDev& d, const float4* tv, int n, int n_old, int4* tknn, float4* tw, cudaStream_t st);

// ------------------------------------------------------------------ JᵀJ pattern
// Device scratch of the pattern build (k_pattern.cu); K = 10 n_sets + 9 n_n keys.
// k_sort.cu: prefix sums and a stable LSD radix sort (8-bit digits) over
// device arrays.  `tmp` is scratch of at least the *_bytes size for n; the
// sort's input is left untouched and must not alias its output.  Errors
// (bad sizes, too little scratch) come back as cudaErrorInvalidValue.
size_t scan_scratch_bytes(int n);
// ticket_zero: the scratch's first word is known to be 0 (a scratch kept
// across calls and cleared once: every completed scan leaves it 0), so no
// clearing is enqueued
cudaError_t scan_sum(const int* in, int* out, int n, bool inclusive, void* tmp, size_t tmp_bytes, cudaStream_t st,
                     bool ticket_zero = false);
size_t sort_scratch_bytes_u32(int n, bool values);
size_t sort_scratch_bytes_u64(int n, bool values);
cudaError_t radix_sort_u32(const uint32_t* kin, uint32_t* kout, const int* vin, int* vout, int n, int begin_bit,
                           int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t st);
cudaError_t radix_sort_u64(const unsigned long long* kin, unsigned long long* kout, const int* vin, int* vout, int n,
                           int begin_bit, int end_bit, void* tmp, size_t tmp_bytes, cudaStream_t st);

struct PatternScratch {
  uint32_t* keys;     // K: the pair keys, then the unique blocks in order
  uint32_t* skeys;    // K: sorted keys
  int* flag;          // K
  int* pos;           // K
  int* count;         // 1: blocks (nnzb)
  void* tmp;          // sort / scan scratch
  size_t tmp_bytes;
};
size_t pattern_scratch_bytes(int n_keys, int n_rl_keys);
// the unique upper blocks of the sets, the diagonal and the graph edges, in
// row-major order, to w.keys[0, *w.count)
cudaError_t launch_pattern_blocks(const int4* sets, int n_sets, const int* graph, int n_n, PatternScratch& w,
                                  cudaStream_t st);
// row_ptr, col, blk_row, blk_edge, rl_ptr, rl_ent and set_slots of `d` from
// the nnzb blocks in w.keys (rl_keys / rl_skeys: 2 nnzb scratch each)
cudaError_t launch_pattern_fill(const int4* sets, int n_sets, const int* graph, int n_n, int nnzb,
                                PatternScratch& w, unsigned long long* rl_keys, unsigned long long* rl_skeys,
                                const SwDev& d, cudaStream_t st);

// tile sizes
constexpr int kSurfTile = 256;
constexpr int kAsmTile = 256;
constexpr int kBlkTile = 128;
// nodes per CTA of the preconditioner launch: few, so that its FP64 work
// spreads over as many SMs as possible
constexpr int kPrecondTile = 16;

// threads of the regulariser assembly's diagonal part: 8 per node, rounded
// up to a whole warp
__host__ __device__ inline int reg_diag_threads(int n_n) { return (8 * n_n + 31) & ~31; }

inline int tiles_for(int kind, const SwDev& d) {
  switch (kind) {
    case kTilePixels: return ((d.W + 31) / 32) * ((d.H + 7) / 8);   // 32x8 pixel tiles
    case kTileSurfels: return (d.n_s + kSurfTile - 1) / kSurfTile;
    case kTileSurfelsAssembly: return (d.n_s + kAsmTile - 1) / kAsmTile;
    case kTileBlocks: return (d.nnzb + kBlkTile - 1) / kBlkTile;
    case kTilePcg: return 0;   // assigned by the runner (share of the persistent grid)
    case kTileNodes: return (d.n_n + kBlkTile - 1) / kBlkTile;
    case kTilePrecond: return (d.n_n + kPrecondTile - 1) / kPrecondTile;
    case kTileRegAssembly: return (reg_diag_threads(d.n_n) + d.nnzb + kAsmTile - 1) / kAsmTile;   // 8 lanes per node, then a thread per block
  }
  return 0;
}

}  // namespace sw
