/*
 * surfelwarp.h -- C ABI of the GB300 (sm_103a) SurfelWarp per-frame hot path.
 *
 * SurfelWarp (Gao & Tedrake 2019) reconstructs a deforming surface from a depth
 * stream.  Per frame it (Sec. 4) re-estimates a node-graph deformation field
 * against the new depth image (Sec. 7-8), fuses the depth surfels into the
 * warped ("live") surfels (Sec. 6.1) and warps the fused surfels back to the
 * reference frame (Sec. 4, Eq. 3).  This library runs that path on one GPU.
 *
 * Conventions (all calls):
 *  - Every call returns an sw_status and never aborts the process.  On an
 *    error the human-readable reason is available from sw_last_error(h).
 *  - The library owns all device state of a stream.  Buffers passed in are
 *    owned by the caller; the library copies what it keeps.
 *  - "host" pointers point to CPU memory; "device" pointers to memory of the
 *    current CUDA device.  Arrays are C-contiguous, row-major, float32 or
 *    int32, indexed by the caller's surfel / node / pixel indices.
 *  - Work is enqueued on the CUDA stream given at creation.  Calls that
 *    return data to the host synchronise that stream; the others return
 *    without waiting for the GPU.
 *  - A stream handle may be used by one host thread at a time.
 *  - Units: metres; pixel (x, y) has its centre at integer coordinates.
 */
#ifndef SURFELWARP_H
#define SURFELWARP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SW_MAX_GN_ITERS 16     /* Sec. 8 caps Gauss-Newton at 10 iterations */
#define SW_MAX_PCG_ITERS 128
#define SW_MAX_RIGID_ITERS 16
#define SW_MAX_NODES 65535     /* node ids are packed in 16 bits */
#define SW_K_SKIN 4            /* nearest nodes per surfel (Eq. 1) */
#define SW_K_GRAPH 8           /* graph neighbours per node (Eq. 11) */

/* Arithmetic of the solve (sw_params.precision).  Depth processing, the
 * association decisions, fusion and the stored surfels are FP32 in every mode.
 *   SW_PRECISION_MIXED         residuals, Jacobians, JᵀJ, SpMV and vectors in
 *                              FP32; PCG inner products accumulated in
 *                              double-float pairs (about 48 significant bits);
 *                              6x6 block inverses (the block-Jacobi
 *                              preconditioner) by Gauss-Jordan sweeps in
 *                              double-float pairs.
 *   SW_PRECISION_FP64          the whole solve in FP64: node transforms, warp,
 *                              residuals, Jacobians, JᵀJ, PCG (the association
 *                              still decided in FP32 from the FP64 warp).
 *   SW_PRECISION_MIXED_F64DOTS as MIXED, with the inner products accumulated
 *                              in FP64 and the block inverses by LDLᵀ in FP64.
 * Every member of one batch must use the same mode. */
#define SW_PRECISION_MIXED 0
#define SW_PRECISION_FP64 1
#define SW_PRECISION_MIXED_F64DOTS 2

typedef struct sw_stream* sw_handle;

typedef enum {
  SW_OK = 0,
  SW_ERR_INVALID_ARG = 1,       /* a null pointer, a size out of range */
  SW_ERR_NO_MEMORY = 2,         /* the device-memory budget refused the stream */
  SW_ERR_NOT_INITIALIZED = 3,   /* no model (sw_set_model) or no depth frame yet */
  SW_ERR_SOLVER_BREAKDOWN = 4,  /* a 6x6 diagonal block is not positive definite, or pᵀAp <= 0 */
  SW_ERR_TIMEOUT = 5,           /* a bounded device-side wait gave up */
  SW_ERR_CUDA = 6,              /* a CUDA runtime error; see sw_last_error */
  SW_ERR_BOUNDS = 7             /* checked build only (-DSW_BOUNDS_CHECK): an index that a kernel read
                                   or derived on the device was out of range; the access was skipped */
} sw_status;

/* Parameters of one stream.  Table 1 fixes lambda, fuse_dist, fuse_normal,
 * stable_conf and recent_frames; corr_dist and corr_normal (the solver's
 * projective-association thresholds) are not given by the paper. */
typedef struct {
  int width, height;            /* depth image size in pixels */
  float fx, fy, cx, cy;         /* pinhole intrinsics K */
  int max_surfels, max_nodes;   /* capacity; device memory is sized from these */
  float lambda;                 /* λ of Eq. 9 (Table 1: 5) */
  float fuse_dist;              /* δ_distance, metres (Table 1: 1 mm) */
  float fuse_normal;            /* δ_normal (Table 1: 0.85) */
  float corr_dist;              /* association distance, metres (0.05) */
  float corr_normal;            /* association normal dot (0.7) */
  float stable_conf;            /* δ_stable (Table 1: 10) */
  int recent_frames;            /* δ_recent (Table 1: 2) */
  int precision;                /* SW_PRECISION_* (default SW_PRECISION_MIXED) */
  int visibility;               /* 1: predict visibility before each solve (Sec. 7): the
                                   selected live surfels are drawn as opaque disk splats
                                   (position, normal, radius) into an index map at the depth
                                   resolution, and only surfels that keep a pixel are
                                   associated; 0 (default): every selected surfel is
                                   associated and occlusion is left to the distance test */
  /* appending (sw_append_frame) */
  float eps;                    /* ε of Eq. 7-8 (Table 1: 0.2) */
  float delta_nn;               /* δ_nn, least sum of a new surfel's live weights (not in Table 1: 0.3) */
  float fd_step;                /* finite-difference step of the Eq. 8 strain, metres (1 mm) */
  int t_low_confid;             /* t_low_confid, frames (Table 1: 30) */
  int extend_nodes;             /* 1 (default): node-graph extension after appending, while the
                                   stream has room below max_nodes (sw_append_frame) */
} sw_params;

/* Per-call statistics of sw_solve_frame; entry i describes Gauss-Newton
 * iteration i at its linearisation point (before its update). */
typedef struct {
  int gn_iters;                         /* iterations run */
  double e_depth[SW_MAX_GN_ITERS];      /* E_depth of Eq. 10 */
  double e_reg[SW_MAX_GN_ITERS];        /* λ E_regulation of Eq. 11 */
  int n_corr[SW_MAX_GN_ITERS];          /* associated (surfel, pixel) pairs */
  double pcg_rz[SW_MAX_GN_ITERS];       /* final rᵀ M⁻¹ r of the linear solve */
} sw_solve_stats;

/* Fill *p with Table 1 values and the association defaults for a camera.
 * Returns SW_ERR_INVALID_ARG for a null p or non-positive sizes. */
sw_status sw_params_default(sw_params* p, int width, int height, float fx, float fy,
                            float cx, float cy, int max_surfels, int max_nodes);

/* Create a stream: validate *p, reserve its device memory under the
 * process-wide budget (SW_ERR_NO_MEMORY if it does not fit) and bind it to
 * cuda_stream (a cudaStream_t; NULL = the legacy default stream).
 * *out receives the handle; it stays valid until sw_destroy_stream. */
sw_status sw_create_stream(const sw_params* p, void* cuda_stream, sw_handle* out);

/* Release every device allocation of the stream (synchronises it). */
sw_status sw_destroy_stream(sw_handle h);

/* Set the process-wide device-memory budget in bytes for sw_create_stream
 * (0 = unlimited) and read the bytes currently held by all streams. */
sw_status sw_set_memory_budget(size_t bytes);
size_t sw_memory_in_use(void);

/* Load the reference surfel model S_ref (= S_live) and the warp-field nodes
 * (Sec. 3), then initialise as Sec. 6.5 does: node transforms to identity,
 * 4-NN skinning of every surfel with weights exp(−‖v − p_k‖² / (2 σ_k²))
 * (Eq. 1), the 8-NN node graph, and the block-sparse pattern of JᵀJ.
 * Host arrays, caller's order:
 *   surfel_v4 [n_surfels][4]: x, y, z, radius
 *   surfel_n4 [n_surfels][4]: nx, ny, nz, confidence
 *   surfel_t2 [n_surfels][2]: t_init, t_observed (int32; NULL = all 0)
 *   node4     [n_nodes][4]  : x, y, z, σ
 * Requires 0 <= n_surfels <= max_surfels and 9 <= n_nodes <= max_nodes.
 * Synchronous. */
sw_status sw_set_model(sw_handle h, const float* surfel_v4, const float* surfel_n4,
                       const int* surfel_t2, int n_surfels, const float* node4, int n_nodes);

/* Upload depth frame `frame_id` (metres, 0 = invalid; [height][width] float32,
 * host or device memory as on_device says) and compute the depth surfels of
 * Sec. 5: vertex map V = D K⁻¹ (u, 1), normal map by central differences,
 * confidence exp(−γ²/(2·0.6²)) and radius √2 d / (f |n_z|) (Eq. 4, |n_z|
 * clamped at cos 75°).  The frame id becomes t_now. */
sw_status sw_upload_depth(sw_handle h, const float* depth, int on_device, int frame_id);

/* Estimate the node transforms for the current frame (Sec. 7-8), starting
 * from the previous frame's: gn_iters Gauss-Newton iterations (1..16), each
 * re-associating the selected surfels (stable c > δ_stable or recent
 * t_now − t_obs <= δ_recent) to the depth map, assembling JᵀJ and Jᵀe of
 * E_depth + λ E_regulation (Eq. 9-11) in a block-sparse 6x6 layout, and
 * solving JᵀJ Δ = −Jᵀe by pcg_iters (1..128) block-Jacobi PCG iterations.
 * stats (host, nullable): when given, the call synchronises and fills it.
 * Returns SW_ERR_SOLVER_BREAKDOWN if a diagonal block was not positive
 * definite (reported when stats is given or at the next synchronising call). */
sw_status sw_solve_frame(sw_handle h, int gn_iters, int pcg_iters, sw_solve_stats* stats);

/* Fuse the current depth frame into the model (Sec. 6.1, Eq. 5-6): forward
 * warp S_ref with the solved field (Eq. 2), render the 4x super-sampled index
 * map of unsized points, pick per depth pixel the corresponding surfel in its
 * 4x4 sub-pixel window (δ_distance, δ_normal; highest confidence, then
 * closest), average it with the depth surfel, and warp the fused surfels back
 * to the reference frame (Eq. 3). */
sw_status sw_fuse_frame(sw_handle h);

/* Copy the node state to the host: pos4 [n][4] = x, y, z, σ and dq8 [n][8] =
 * the dual quaternion (real w x y z, dual w x y z) of each node transform T_j.
 * cap is the capacity of both arrays in nodes; *n_out receives n_nodes.
 * Either array may be NULL.  Synchronous. */
sw_status sw_read_nodes(sw_handle h, float* pos4, float* dq8, int cap, int* n_out);

/* ---------------------------------------------------------------------------
 * Inspection and test hooks (additions to the paper's interface).  All host
 * memory, caller's order, synchronous.
 * ------------------------------------------------------------------------- */

/* Reference surfels: v4 (x y z r), n4 (nx ny nz c), t2 (t_init, t_obs). */
sw_status sw_read_surfels(sw_handle h, float* v4, float* n4, int* t2, int cap, int* n_out);
/* Live surfels of the last forward warp (solve or fuse): v4, n4 as above. */
sw_status sw_read_live_surfels(sw_handle h, float* v4, float* n4, int cap, int* n_out);
/* Skinning: knn4 [n][4] node ids nearest first (ties: lower id), w4 weights. */
sw_status sw_read_skinning(sw_handle h, int* knn4, float* w4, int cap, int* n_out);
/* Node graph: graph8 [n_nodes][8] neighbour ids, nearest first. */
sw_status sw_read_graph(sw_handle h, int* graph8, int cap);
/* Depth surfels of the current frame: V4 [H][W][4] = x y z confidence
 * (confidence 0 = not a usable depth surfel), N4 [H][W][4] = nx ny nz radius. */
sw_status sw_read_maps(sw_handle h, float* V4, float* N4);
/* Replace the current frame's depth surfels by the given maps (same layout as
 * sw_read_maps), so that stages can be checked on fixed FP32 inputs. */
sw_status sw_debug_set_maps(sw_handle h, const float* V4, const float* N4);
/* Set every node's dual quaternion (dq8 [n_nodes][8], not re-normalised). */
sw_status sw_set_node_dq(sw_handle h, const float* dq8, int n_nodes);
/* Association of the last Gauss-Newton iteration: pixel index y*W+x per
 * surfel, or -1. */
sw_status sw_read_correspondence(sw_handle h, int* pix, int cap, int* n_out);
/* Test hook: with enable = 1, every later solve of this stream also keeps
 * each Gauss-Newton iteration's association (device memory for
 * SW_MAX_GN_ITERS x max_surfels ints, from the stream's budget, allocated
 * at the first enable); 0 stops keeping it.  sw_read_correspondence_iter
 * returns iteration gn_iter's (0-based) of the last solve, as
 * sw_read_correspondence does the last one (SW_ERR_NOT_INITIALIZED while
 * recording is off).  A comparison can then give another implementation
 * the library's decisions where the two differ at a rounding boundary. */
sw_status sw_debug_record_correspondence(sw_handle h, int enable);
sw_status sw_read_correspondence_iter(sw_handle h, int gn_iter, int* pix, int cap, int* n_out);
/* Replace the live surfels (v4: x y z r, n4: nx ny nz c; only xyz are used). */
sw_status sw_debug_set_live(sw_handle h, const float* v4, const float* n4, int n);
/* Run projective association on the current live surfels (no warp); the
 * result is read with sw_read_correspondence. */
sw_status sw_debug_associate(sw_handle h);
/* Render the index map of the current live surfels and select each depth
 * pixel's fusion target without updating anything: target [H*W] caller's
 * surfel index or -1; imap [4H][4W] caller's surfel index or -1 (nullable). */
sw_status sw_debug_fusion_targets(sw_handle h, int* target, int* imap);
/* Assemble JᵀJ and Jᵀe at the current node transforms and maps (one
 * Gauss-Newton linearisation, no solve).  Sizes: *nnzb_out upper blocks. */
/* Splat visibility of the live surfels as they are stored (e.g. by
 * sw_debug_set_live; each surfel keeps its own radius): vis_map (W*H, nullable) gets the caller's
 * surfel index drawn at each pixel or -1, visible (n_surfels, caller order,
 * nullable) 1 for the surfels that keep a pixel.  Independent of
 * sw_params.visibility; the call synchronises. */
sw_status sw_debug_visibility(sw_handle h, int* vis_map, int* visible);
sw_status sw_debug_assemble(sw_handle h, int* nnzb_out, int* n_corr_out);
/* Read the last assembled system (sw_debug_assemble's, or the last
 * Gauss-Newton iteration's of the last solve): rows/cols [nnzb] block
 * coordinates (row <= col), vals [nnzb][36] row-major 6x6, g [6 n_nodes]. */
sw_status sw_debug_read_jtj(sw_handle h, int* rows, int* cols, float* vals, float* g, int cap_blocks);

/* ---------------------------------------------------------------------------
 * Batches: several streams of uneven size advanced together, each stage one
 * launch over all of them (additions to the paper's interface, which runs
 * one stream; Sec. 8 names stream-level parallelism as future work).
 *
 * A batch keeps per-stream state where it is (every member stays resident)
 * and runs on its own CUDA stream.  Each Gauss-Newton iteration is a few
 * launches for the whole batch -- the assembly of both terms, the
 * block-Jacobi preconditioner, and the PCG with the update (a thread-block
 * cluster per member whose system fits on chip, one persistent cooperative
 * kernel for the others) -- replayed from a captured CUDA graph.  Members whose active
 * flag is 0 are skipped by every launch (their state is untouched).
 * Results equal those of running each member alone up to floating-point
 * summation order.  Work that a member's own calls enqueued is ordered before
 * the next batch call, and batch work before the member's next own call.
 * When a member's model changes (sw_set_model, sw_import_state,
 * sw_append_frame) the batch rebuilds its tables and solve graphs at its next
 * call, keeping the active flags.  Errors of
 * batch calls are reported by sw_last_error(NULL).
 * ------------------------------------------------------------------------- */
typedef struct sw_batch* sw_batch_handle;

/* streams: n (1..4096) distinct handles with a model; cuda_stream as in
 * sw_create_stream.  All members start active. */
sw_status sw_batch_create(const sw_handle* streams, int n, void* cuda_stream, sw_batch_handle* out);
sw_status sw_batch_destroy(sw_batch_handle b);
/* active: host [n] ints, nonzero = the member takes part in the next calls. */
sw_status sw_batch_set_active(sw_batch_handle b, const int* active);
/* depths: host array of n pointers to [H_i][W_i] float32 depth images (host
 * or device memory as on_device says; NULL entries and inactive members are
 * skipped); frame_ids: host [n].  Computes every active member's depth
 * surfels (Sec. 5) in one launch. */
sw_status sw_batch_upload_depth(sw_batch_handle b, const float* const* depths, int on_device, const int* frame_ids);
/* sw_solve_frame for every active member; stats: host [n] or NULL. */
sw_status sw_batch_solve(sw_batch_handle b, int gn_iters, int pcg_iters, sw_solve_stats* stats);
/* sw_fuse_frame for every active member. */
sw_status sw_batch_fuse(sw_batch_handle b);
/* The PCG's SpMV staging mode of the batch's current launch plan (see
 * sw_debug_set_pcg_mode below); test hook. */
sw_status sw_batch_debug_pcg_mode(sw_batch_handle b, int* mode);

/* ---------------------------------------------------------------------------
 * Stage timing (CUDA events recorded on the launching stream, inside the
 * captured solve graph).  Stages: 0 depth processing, 1 regulariser
 * assembly (SW_PRECISION_FP64 only: the FP32 modes assemble both terms in
 * one launch, timed as stage 2), 2 data-term assembly, 3 PCG + update, 4
 * fusion, 5 visibility prediction (streams with sw_params.visibility).  Enabling or
 * disabling re-captures the solve graph.  sw_read_profile synchronises and
 * returns, per stage, the summed milliseconds and the number of launches of
 * the last upload, solve and fusion.
 * ------------------------------------------------------------------------- */
#define SW_PROFILE_STAGES 6
sw_status sw_set_profiling(sw_handle h, int enable);
sw_status sw_read_profile(sw_handle h, double* ms, int* launches);
sw_status sw_batch_set_profiling(sw_batch_handle b, int enable);
sw_status sw_batch_read_profile(sw_batch_handle b, double* ms, int* launches);

/* Test hook for failure detection (an addition; the paper has no
 * counterpart): make the product's own bounded device waits run out, without
 * any fault on the GPU, by having a kernel withhold what another waits for.
 *   kind 0  off (the default)
 *   kind 1  in the persistent PCG (Sec. 7), CTA 1 of the first stream of a
 *           launch does not publish its share of the first reduction: every
 *           CTA of that stream stops polling after spin_limit polls
 *   kind 2  the same CTA does not publish its rows' first vector u = M⁻¹ r:
 *           the neighbours' waits for those rows run out
 *   kind 3  the depth stage (Sec. 5) does not issue its TMA tile copies: each
 *           CTA's bounded mbarrier wait runs out and it loads the tile with
 *           plain loads instead (the maps stay exact)
 * spin_limit (0..2^22): the poll limit that replaces the PCG's own while the
 * hook is on (0 = keep the PCG's, 2^22 reduction polls); small values keep
 * the test short.  The setting is process-wide on the current device, read
 * by every later launch (captured graphs included), and the call
 * synchronises the device.  A wait that ran out makes the next synchronising
 * call of the stream (sw_solve_frame with stats, sw_batch_solve with stats)
 * return SW_ERR_TIMEOUT; after a PCG wait ran out the node transforms are
 * left as they were.  The CUDA context stays usable. */
sw_status sw_debug_inject_wait_fault(int kind, int spin_limit);

/* Test hooks for the PCG's modes (Sec. 7; additions).  Mode 3: a stream
 * whose JᵀJ fits one thread-block cluster's shared memory (FP32 modes) runs
 * its PCG as one cluster of CTAs that exchange vectors through distributed
 * shared memory.  Otherwise the cooperative PCG keeps what fits of each
 * CTA's share of JᵀJ in shared memory: mode 2 stages the rows' 6x6 blocks
 * and the per-entry products, mode 1 only the products (blocks read from
 * global memory every iteration), mode 0 nothing (a warp per block row).
 * The mode is chosen per stream (per batch for the cooperative kernel) when
 * its launch plan is built, as the highest that fits.  sw_debug_set_pcg_mode
 * caps it (0..3; 3 = no cap) for launch plans built after the call (streams
 * given a model, batches created or rebuilt after it), process-wide.
 * sw_debug_pcg_mode reports the mode a stream's current plan uses;
 * sw_batch_debug_pcg_mode 3 when every member runs on clusters, else the
 * cooperative kernel's mode. */
sw_status sw_debug_set_pcg_mode(int max_mode);
sw_status sw_debug_pcg_mode(sw_handle h, int* mode);

/* The launch plan of the cluster PCG (an addition; host code only, needs no
 * GPU): the PCG of a stream whose JᵀJ fits the shared memory of one
 * thread-block cluster runs as one cluster of `ctas` CTAs, each holding the
 * upper 6x6 blocks of the node rows it owns.  Input (host): the upper block
 * pattern as the library keeps it, row_ptr [n_nodes + 1] and col
 * [row_ptr[n_nodes]] with every row leading with its diagonal block;
 * node4 [n_nodes][4] the node positions (x y z, w unused).  Output: plan
 * (host, cap ints, nullable to ask for the size in *n_out) laid out as
 * header {ctas, most rows, most home blocks, most receive slots of a CTA,
 * n_nodes, most halo rows, most u pushes}; per CTA prefix tables (ctas + 1
 * each) of rows, home blocks, receive slots and u pushes; each CTA's rows
 * (node ids, its local order); per CTA the rows' home-block, receive-slot
 * and u-push offsets (rows + 1 each); per home block its block index, the
 * local u slot of its column (own row, or halo slot after the own rows) and
 * the target of its transposed product ((owner CTA << 16) | receive slot,
 * -1 on the diagonal); per u push (peer CTA << 16) | the peer's u slot.
 * *smem_out: the shared memory a CTA needs.
 * SW_ERR_INVALID_ARG if the system does not fit smem_limit bytes per CTA
 * (or 192 rows per CTA) or the pattern is malformed. */
sw_status sw_debug_cluster_plan(int ctas, int n_nodes, const int* row_ptr, const int* col, const float* node4,
                                size_t smem_limit, int* plan, size_t cap, size_t* n_out, size_t* smem_out);

/* Cluster-PCG inspection (an addition): with h non-null, the cluster size
 * and per-CTA shared memory of the stream's plan (0, 0 if it has none);
 * with active_clusters non-null, how many clusters of `ctas` CTAs with
 * `smem` bytes of shared memory each the device runs at once in the given
 * precision (a negative value is a CUDA error code). */
sw_status sw_debug_pcg_cluster(sw_handle h, int precision, int ctas, size_t smem, int* plan_ctas,
                               size_t* plan_smem, int* active_clusters);

/* The cluster PCG's hop measured alone (an addition): the time of one
 * cluster barrier (barrier.cluster arrive + wait) of `ctas` CTAs of the
 * cluster PCG's size, in microseconds, from two timed launches.  The PCG
 * passes two such barriers per iteration; bench.py states its latency
 * bound in this unit.  Synchronous; needs a GPU. */
sw_status sw_debug_cluster_barrier_us(int ctas, double* us);

/* Splat visibility (Sec. 7) that the last solve of a stream with
 * sw_params.visibility = 1 predicted before its first Gauss-Newton
 * iteration: visible [n_surfels] (host, caller's order) 1 for the surfels
 * that kept a pixel of the splat index map, else 0.  Synchronous. */
sw_status sw_read_visibility(sw_handle h, int* visible, int cap, int* n_out);

/* Test hook for the block-Jacobi preconditioner (Sec. 7): the inverse of
 * each of n symmetric 6x6 blocks (host, row-major, 36 values each) as the
 * PCG forms it -- from its lower triangle -- written to inv21 (host, 21
 * values per block, packed lower triangle row by row: (0,0) (1,0) (1,1)
 * (2,0) ...), same element type as the blocks.  mode 0: float blocks,
 * Gauss-Jordan sweeps in double-float pairs on eight lanes per block (the
 * default precision's); 1: double blocks, LDLᵀ in FP64 (SW_PRECISION_FP64);
 * 2: float blocks, LDLᵀ in FP64 (SW_PRECISION_MIXED_F64DOTS).  ok[i] (host) is 1, or 0 when
 * block i is not positive definite (its inv21 entries are then
 * unspecified).  SW_ERR_INVALID_ARG for another mode.  Needs a GPU;
 * synchronous. */
sw_status sw_debug_block_inverse(const void* blocks36, int n, int mode, void* inv21, int* ok);

/* Test hooks for the library's own prefix sum and radix sort (k_sort.cu;
 * the model set-up sorts surfels by their 4-node set, the JᵀJ pattern
 * build sorts node pairs, appending compacts and sorts new node sets).
 *
 * sw_debug_scan: out[i] (host, n int32) = in[0] + ... + in[i-1], or up to
 * in[i] when inclusive is nonzero (host in, n int32; wraps like int32).
 *
 * sw_debug_radix_sort: a stable sort of n keys (host; key_bytes 4 = uint32
 * or 8 = uint64) by their bits [begin_bit, end_bit), least significant
 * 8-bit digit first.  keys_out (host, n keys) gets the keys in order; when
 * vals (host, n int32) is not NULL, vals_out (host, n int32) gets each key's
 * value, equal keys in input order.  n = 0 is a no-op;
 * SW_ERR_INVALID_ARG for a bad size, key width or bit range.  Both need a
 * GPU and are synchronous. */
/* Test hook for the checked build (-DSW_BOUNDS_CHECK): writes node id
 * `node` as skinning node `slot` (0..3) of surfel `surfel` in the library's
 * internal order, with no other change.  node must lie in [0, max_nodes),
 * inside the node arrays' allocation, but may be >= n_nodes: then the
 * checked build reports the next per-frame call with SW_ERR_BOUNDS, and the
 * normal build reads unused node storage (a wrong warp, no fault).
 * SW_ERR_INVALID_ARG for an argument out of range.  Synchronous. */
sw_status sw_debug_set_skin_node(sw_handle h, int surfel, int slot, int node);

sw_status sw_debug_scan(const int32_t* in, int n, int inclusive, int32_t* out);
sw_status sw_debug_radix_sort(int key_bytes, const void* keys, const int32_t* vals, int n, int begin_bit,
                              int end_bit, void* keys_out, int32_t* vals_out);

/* Whole-stream state to and from host memory (checkpoint / resume):
 * sw_export_state with buf NULL reports the size in *bytes. */
sw_status sw_export_state(sw_handle h, void* buf, size_t* bytes);
sw_status sw_import_state(sw_handle h, const void* buf, size_t bytes);

/* ---------------------------------------------------------------------------
 * Fusion-target selection without any device allocation.
 *
 * The paper has no counterpart to this call; it is an addition for callers
 * that may not call cudaMalloc: code that runs while someone else is
 * capturing its CUDA stream into a graph, real-time loops in which an
 * allocation would stall every stream of the device, and host frameworks
 * that hand out all device memory from their own pool.  It computes what
 * sw_debug_fusion_targets computes (the 4x super-sampled index map of the
 * live surfels, then each depth pixel's fusion target, Sec. 6.1) but takes
 * every input and output as caller-owned device memory and keeps its only
 * scratch buffer, the index map, in a fixed array compiled into the
 * library.
 *
 * Scratch: 16 * SW_STATIC_MAX_PIXELS 64-bit entries (9.8 MB).  Every GPU
 * that loads the library holds this array until the process exits.  A call
 * whose stream is not being captured looks up the array's device address in
 * the current context (cudaGetSymbolAddress) and remembers it per device; a
 * call under stream capture uses the remembered address.  So make one call
 * outside capture before capturing, and again after cudaDeviceReset or
 * after making another context current on the device (SW_ERR_CUDA if a
 * captured call finds no address).  Every call on a device uses the same
 * array and overwrites
 * it (the call clears it first), so calls whose work overlaps on the GPU --
 * on different streams, or from different host threads -- race and give
 * wrong results; serialise them.
 *
 * Arguments (all device pointers, caller's surfel order):
 *   v_live4 [n_surfels][4] x y z (.w unused), n_live4 [n_surfels][4]
 *   nx ny nz confidence; vmap4 / nmap4 [height][width][4] as sw_read_maps
 *   returns them (confidence 0 = not a usable depth surfel); target
 *   [height*width] receives the chosen surfel index or -1.
 * The work is enqueued on cuda_stream (NULL = legacy default stream) and the
 * call returns without waiting.  Returns SW_ERR_INVALID_ARG (with a message
 * in sw_last_error(NULL)) for null pointers, non-positive sizes or
 * width * height > SW_STATIC_MAX_PIXELS, and SW_ERR_CUDA if a launch fails.
 * ------------------------------------------------------------------------- */
#define SW_STATIC_MAX_PIXELS 76800   /* 320 x 240 */
sw_status sw_fusion_targets_static(const float* v_live4, const float* n_live4, int n_surfels,
                                   const float* vmap4, const float* nmap4, int width, int height,
                                   float fx, float fy, float cx, float cy, float fuse_dist,
                                   float fuse_normal, int* target, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Serving: a request loop over many independent streams with continuous
 * batching.  Addition with no counterpart in the paper (one camera there).
 *
 * One worker thread per server owns the GPU.  Streams are opened with their
 * parameters and model and wait for admission until their device state fits
 * the memory budget (sw_server_create sets the process-wide budget of
 * sw_set_memory_budget); admitted streams keep their surfels, node graph and
 * warp field resident on the device.  Each worker step takes the oldest
 * queued frame of every admitted stream that has one and runs depth
 * processing, the Gauss-Newton solve (gn_iters x pcg_iters) and fusion for
 * all of them in one batch; frames submitted while a step runs join the next.
 * Streams leave with sw_server_close once their queued frames are done.
 * The server's streams are used only through these calls.
 * ------------------------------------------------------------------------- */
typedef struct sw_server* sw_server_handle;

/* One completed frame.  Times are milliseconds on the server's host clock
 * (steady, from sw_server_create). */
typedef struct {
  int stream;          /* id from sw_server_open */
  int frame_id;
  int status;          /* sw_status of the frame's work */
  int batch_size;      /* frames processed in the same launches (1: through its stream's own calls) */
  double submit_ms;    /* sw_server_submit took the frame */
  double start_ms;     /* its processing began */
  double done_ms;      /* its fusion (and appending) had finished on the device */
  int appended;        /* surfels the frame appended (sw_server_set_appending) */
  int n_surfels;       /* the stream's surfels after the frame */
} sw_frame_result;

typedef struct {
  int admitted;             /* streams on the device */
  int waiting;              /* opened, waiting for memory */
  long long steps;          /* worker steps with at least one frame */
  long long frames;         /* frames completed */
  double busy_ms;           /* time spent in steps */
  size_t memory_in_use;     /* bytes held by all streams */
  long long steps_alone;    /* steps the adaptive policy ran stream by stream */
} sw_server_stats;

/* Start a server.  memory_budget: bytes for all streams (0 = unlimited);
 * queue_depth: frames a stream may have queued (1..64), each in a pinned
 * host slot.  SW_ERR_INVALID_ARG for out-of-range counts. */
sw_status sw_server_create(size_t memory_budget, int gn_iters, int pcg_iters, int queue_depth,
                           sw_server_handle* out);
/* Stop the worker (after its current step) and release every stream. */
sw_status sw_server_destroy(sw_server_handle s);
/* Open a stream: p and the model as for sw_create_stream / sw_set_model
 * (copied; t2 may be NULL = all zero).  *stream_id is valid at once; frames
 * can be submitted once sw_server_is_admitted reports 1. */
sw_status sw_server_open(sw_server_handle s, const sw_params* p, const float* v4, const float* n4, const int* t2,
                         int n_s, const float* node4, int n_n, int* stream_id);
/* Close a stream: it leaves after its queued frames (or at once if waiting). */
sw_status sw_server_close(sw_server_handle s, int stream_id);
/* 1 in *admitted once the stream's state is on the device. */
sw_status sw_server_is_admitted(sw_server_handle s, int stream_id, int* admitted);
/* Queue one depth frame (host memory, width*height floats, copied before the
 * call returns).  SW_ERR_NOT_INITIALIZED while the stream waits for
 * admission, SW_ERR_NO_MEMORY when its queue is full, SW_ERR_INVALID_ARG for
 * an unknown or closing stream. */
sw_status sw_server_submit(sw_server_handle s, int stream_id, const float* depth, int frame_id);
/* Move up to cap completed frames (oldest first) into out; *n_out = count. */
sw_status sw_server_poll(sw_server_handle s, sw_frame_result* out, int cap, int* n_out);
/* Wait until every submitted frame has completed (SW_ERR_TIMEOUT after timeout_ms). */
sw_status sw_server_wait(sw_server_handle s, int timeout_ms);
/* A stream's node positions and transforms, as sw_read_nodes. */
sw_status sw_server_read_nodes(sw_server_handle s, int stream_id, float* pos4, float* dq8, int cap, int* n_out);
/* Batching window: a step with frames of only some admitted streams waits up
 * to window_ms (0..1000) after its oldest frame arrived for the others'
 * frames (0 = start at once, the default). */
sw_status sw_server_set_batch_window(sw_server_handle s, double window_ms);
/* Appending (sw_append_frame) after every served frame, stream by stream,
 * once the batch's fusion has finished (0 = off, the default).  The model
 * grows within each stream's max_surfels (and max_nodes, with extend_nodes);
 * a frame whose appending fails reports that status. */
sw_status sw_server_set_appending(sw_server_handle s, int enable);
/* Plain serving (1), the reference for continuous batching: each step takes
 * only the oldest queued frame of all admitted streams and runs it through
 * that stream's own calls (sw_upload_depth, sw_solve_frame, sw_fuse_frame),
 * one frame and one stream at a time, with the same admission, queues and
 * time stamps.  0 (the default) batches every admitted stream's oldest
 * frame into one step. */
sw_status sw_server_set_plain(sw_server_handle s, int enable);
/* Adaptive steps (1, the default): every step runs its frames either as one
 * batch or, when the server's measured times say that serving them one by
 * one through their streams' own calls takes less time, only the oldest
 * queued frame alone (as the plain mode does), deciding again at the next
 * step (a batch step is shaped for all admitted streams, so under light load
 * a few frames finish sooner alone).  0 batches every step.  Ignored in the
 * plain mode. */
sw_status sw_server_set_adaptive(sw_server_handle s, int enable);
sw_status sw_server_read_stats(sw_server_handle s, sw_server_stats* out);

/* Rigid pre-alignment of the current frame (Sec. 7: before the non-rigid
 * estimation a rigid alignment in the manner of KinectFusion).  Runs `iters`
 * (0..SW_MAX_RIGID_ITERS) point-to-plane ICP iterations of the warped model
 * against the uploaded depth: association exactly as in sw_solve_frame, the
 * model moved by one rigid transform T solved from 6x6 normal equations
 * (FP64 Cholesky; a system that is not positive definite ends the
 * iterations with T as it is), and finally T composed into every node
 * transform (T_j <- T T_j).  Call between sw_upload_depth and
 * sw_solve_frame.  n_corr / energy (nullable, `iters` entries each) receive
 * each iteration's correspondence count and sum of squared point-to-plane
 * residuals before its update; the call then synchronises. */
sw_status sw_rigid_align(sw_handle h, int iters, int* n_corr, double* energy);
/* The same for every active member of a batch (no statistics). */
sw_status sw_batch_rigid_align(sw_batch_handle b, int iters);

/* ---------------------------------------------------------------------------
 * Appending and removal (Sec. 6.2 live skinning with the consistency test of
 * Eq. 7; Sec. 6.3 the compressive-warp bound of Eq. 8; Sec. 6.4 appending and
 * removal; the GPU selection that compacts the surfel array, Sec. 6.6).
 * Call after sw_fuse_frame (SW_ERR_NOT_INITIALIZED if no fusion ran since
 * the last depth frame).  Candidates are the usable depth pixels whose
 * fusion window (their 16 index-map sub-pixels) held no live surfel.  Each
 * is skinned to its 4 nearest warped nodes T_j p_j; node i != 0 stays when
 * 1-eps < |p^_i - p^_0| / |p_i - p_0| < 1+eps (decided on squares in FP32);
 * the live weights exp(-|x - p^_i|^2 / 2 sigma_i^2) of the nodes that stay
 * must sum to at least delta_nn; the depth vertex and normal are warped back
 * (Eq. 3, FP64) and the strain d x_ref / d x_live, by central differences of
 * step fd_step, must have no singular value above 1+eps.  Accepted
 * candidates become surfels with the depth surfel's radius and confidence,
 * t_init = t_observed = the frame id, and a skinning recomputed at their
 * reference position by the initialisation rule.  Existing surfels with
 * confidence below stable_conf and t_now - t_init >= t_low_confid are
 * removed.  The new caller order is the surviving surfels in their order,
 * then the appended ones in pixel order; appended surfels beyond max_surfels
 * are dropped from the end.  Node positions, the graph and the transforms
 * are unchanged unless the node graph is extended: with extend_nodes and
 * room below max_nodes, appended surfels farther than every node's radius
 * (σ_j, node4.w) from it are sub-sampled in order into new nodes (at least
 * the nearest old node's σ apart from every node; each takes that σ and the
 * current warp at its position as its transform), the 8-NN graph is
 * recomputed and every surfel whose 4 nearest nodes now include a new node
 * is re-skinned.  The model's internal structure is then updated: when
 * nothing was removed, no node was added and few surfels were placed since
 * the last sort, the appended surfels follow the sorted ones and only new
 * node sets are added (the JᵀJ pattern rebuilt only for node pairs it
 * lacked); otherwise the surfels are re-sorted by node set and the pattern
 * rebuilt.  Either way the runner and the solve graphs are re-described
 * (the call synchronises; its scratch and the model's arrays come from a
 * per-stream cache of device blocks that repeated calls reuse).  A
 * batch holding the stream rebuilds its tables at its next call (its active
 * flags are kept).  If the model update fails (SW_ERR_NO_MEMORY under the
 * memory budget, SW_ERR_CUDA), by the fast update or the rebuild, the stream
 * has no model until the next sw_set_model or sw_import_state.  *stats (nullable) receives
 * the counts.
 * ------------------------------------------------------------------------- */
typedef struct {
  int candidates;        /* usable pixels with an empty fusion window */
  int rejected_nn;       /* of those, weight sum below delta_nn */
  int rejected_strain;   /* of those, strain singular value above 1+eps (Eq. 8) */
  int appended;          /* surfels added */
  int removed;           /* unstable surfels removed */
  int n_surfels;         /* surfels after the call */
  double kernel_ms;      /* device time of the appending kernels (CUDA events), model rebuild excluded */
  double rebuild_ms;     /* host time of the model rebuild (set sort, JᵀJ pattern, runner) */
  int new_nodes;         /* nodes added by the node-graph extension */
  int resorted;          /* 1: the surfels were re-sorted by node set and the JᵀJ pattern rebuilt;
                            0: no change, or the appended surfels were placed after the sorted ones
                            (nothing removed, no new node, and the surfels so placed since the last
                            re-sort at most 1/16 of the model), new node sets added to the set table,
                            the JᵀJ pattern kept (every new set's node pairs already blocks of it);
                            2: as 0, with the JᵀJ pattern rebuilt for node pairs it lacked */
} sw_append_stats;
sw_status sw_append_frame(sw_handle h, sw_append_stats* stats);
/* Per-candidate record of the last sw_append_frame, candidate order (row-
 * major pixel order); each pointer nullable; cap entries: pix (1), knn4 (4
 * node ids, live distance order), flags (1: bits 0-3 the nodes Eq. 7 keeps,
 * 16 accepted, 32 weight sum below delta_nn, 64 compressive), wsum (1),
 * strain9 (9, row-major), w4 (4 live weights), v4 (v_ref, radius), n4
 * (n_ref, confidence).  *n_out receives the candidate count; with every
 * array pointer null only the count is returned. */
sw_status sw_debug_read_append(sw_handle h, int* pix, int* knn4, int* flags, double* wsum, double* strain9,
                               float* w4, float* v4, float* n4, int cap, int* n_out);

/* ---------------------------------------------------------------------------
 * Autotuning (addition; no counterpart in the paper).  Chooses the PCG's
 * granularity -- one persistent CTA per rows_per_cta block rows of a stream,
 * from 16, 24, 32, 48, 64, 96; it sets the CTA count, how much of the matrix
 * fits in shared memory and how many CTAs each reduction waits for -- by
 * timing the persistent launch on the stream's (or the batch members')
 * current system.  Needs a model and a depth frame on every stream; the
 * node transforms are restored afterwards and a batch's members are all made
 * active.  Each candidate's launch is timed twelve times (two sweeps of six)
 * and its fastest launch counts.  *rows_per_cta and *pcg_us (nullable)
 * receive the choice and its time per launch in microseconds (that fastest
 * launch).  The choice stays with the stream (or
 * the batch) until the next autotune call.
 * ------------------------------------------------------------------------- */
sw_status sw_autotune(sw_handle h, int pcg_iters, int* rows_per_cta, double* pcg_us);
sw_status sw_batch_autotune(sw_batch_handle b, int pcg_iters, int* rows_per_cta, double* pcg_us);

/* Reason of the last error on this handle ("" if none); NULL handle: the last
 * process-wide error (e.g. of sw_create_stream). */
const char* sw_last_error(sw_handle h);
const char* sw_status_string(sw_status s);

#ifdef __cplusplus
}
#endif
#endif /* SURFELWARP_H */
