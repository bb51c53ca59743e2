// K7+K8 on one thread-block cluster per stream: block-Jacobi preconditioned
// conjugate gradients on JᵀJ Δ = −Jᵀe (Sec. 7's linear solve, x₀ = 0,
// exactly K iterations, stopping early only when rᵀM⁻¹r is exactly zero) and
// the node update T_j ← Δ_j T_j, for streams whose system fits the cluster's
// shared memory (FP32 modes).
//
// Why a cluster.  The solve is small (2048 nodes: 12,288 unknowns, ~17k
// upper 6x6 blocks) and each iteration needs every CTA to agree on two inner
// products, so it is bound by synchronisation, not by HBM.  Here the C CTAs
// of a cluster (C = 16, one per SM, 768 threads each) keep the whole system
// in their shared memory, exchange what they share through distributed
// shared memory, and synchronise with the hardware cluster barrier
// (barrier.cluster arrive.release / wait.acquire): nothing of the iteration
// goes through global memory and nothing polls.
//
// Work split.  The host partitions the nodes into C contiguous ranges of
// their Morton order (a spatially compact share per CTA, balanced by shared
// memory bytes) and gives every upper block (i, j), i <= j, to the CTA that
// owns row i (its "home").  A home block serves both halves of the
// symmetric product: y_i += A_ij u_j and, off the diagonal, y_j += A_ijᵀ u_i.
// Within a CTA, a group of 8 lanes serves up to two rows (the second row of
// group g is row 2 G − 1 − g of the CTA's cost-sorted order, G groups, so
// that the dearest row pairs with the cheapest): in the product phase its
// lanes take the rows' home blocks in turn, in the update phase lane c < 6
// takes component c (r in a register; x, p, s in shared memory).
//
// Exchange, all by the producer into the consumer's shared memory (remote
// stores: st.shared::cluster), so that every read on the critical path is a
// local one:
//   u     each owner writes its rows' new u into the halo slots of the CTAs
//         whose home blocks reference them (a push list per row);
//   A_ijᵀ u_i  each home block writes its transposed product into a receive
//         slot of row j's owner, which sums its slots in a fixed order, so
//         the sums, and the solve, are deterministic;
//   γ, δ  each CTA writes its two partial sums into slot `me` of every CTA.
// One iteration (Chronopoulos-Gear: u = M⁻¹r and w = A u formed, γ = (r, u)
// and δ = (w, u) from one reduction, p and s = A p by recurrence):
//   A  w's home part from the local u and halo, the transposed products out,
//      δ's share blockwise as uᵀA u (each off-diagonal block counts twice),
//      γ's share from the previous step, the partials out;
//                                                   -> cluster barrier
//   B  every CTA sums the C partials in the same order and takes the same
//      step (α, β); own rows add their received products, then p = u + βp,
//      s = w + βs, x += αp, r −= αs, u = M⁻¹r, u out, γ's next share;
//                                                   -> cluster barrier
// Every CTA takes the same decisions from bit-identical totals, so all of
// them pass the same barriers and leave the loop together; after the last
// barrier no CTA touches another's shared memory.  The inner products are
// accumulated in the accumulator type (double-float pairs or FP64) and
// reduced by cascaded summation (sw_pcg.cuh).  The home blocks are staged
// by bulk copies (cp.async.bulk, one per row, on an mbarrier whose wait is
// bounded).
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_pcg.cuh"

namespace sw {

namespace {

constexpr int kCThreads = 768;                 // 24 warps: 80 registers a thread
constexpr int kGroup = 8;                      // lanes per row group
constexpr int kGroups = kCThreads / kGroup;    // 96
constexpr int kMaxRowsPerCta = 2 * kGroups;    // two rows per group at most
constexpr int kMaxCluster = 16;

// ------------------------------------------------------------------ the plan (host-built, device-resident)

// int buffer: header {C, NR, NB, NG, n_n, NH, NP}; per CTA prefix tables
// (C + 1 each) of rows, home blocks, receive slots and u pushes; then
//   rows  [n_n]        the CTAs' rows (global node ids) in local order
//   hb    [n_n + C]    per CTA, its rows' home-block offsets (nr + 1)
//   go    [n_n + C]    per CTA, its rows' receive-slot offsets (nr + 1)
//   po    [n_n + C]    per CTA, its rows' u-push offsets (nr + 1)
//   blk   [nnzb]       per home block (CTA-major, row by row), its index in A
//   col   [nnzb]       per home block, the local u slot of its column (own
//                      row a, or halo slot nr + h)
//   o2t   [nnzb]       per home block off the diagonal, (owner of its column
//                      << 16) | receive slot there; -1 on the diagonal
//   push  [total]      per u push, (peer CTA << 16) | the peer's u slot
// NR, NB, NG, NH and NP are the most rows, home blocks, receive slots, halo
// rows and u pushes of a CTA.
struct PlanOff {
  int rb, bb, gb, pb, rows, hb, go, po, blk, col, o2t, push, total;
};
constexpr int kPlanHeader = 7;
__host__ __device__ inline PlanOff plan_off(int C, int n_n, int nnzb, int n_push) {
  PlanOff o{};
  o.rb = kPlanHeader;
  o.bb = o.rb + C + 1;
  o.gb = o.bb + C + 1;
  o.pb = o.gb + C + 1;
  o.rows = o.pb + C + 1;
  o.hb = o.rows + n_n;
  o.go = o.hb + n_n + C;
  o.po = o.go + n_n + C;
  o.blk = o.po + n_n + C;
  o.col = o.blk + nnzb;
  o.o2t = o.col + nnzb;
  o.push = o.o2t + nnzb;
  o.total = o.push + n_push;
  return o;
}

// shared memory of one CTA, sized by the largest share of any CTA, so that
// the remotely written sections (partials, u, receive slots) sit at the same
// offsets in every CTA
struct SmemPlan {   // byte offsets
  unsigned part, u, recv, a, col, mi, xps, hb, go, po, push, rows, bar, total;
};
__host__ __device__ constexpr unsigned al16(unsigned x) { return (x + 15u) & ~15u; }
__host__ __device__ inline SmemPlan smem_plan(int NR, int NB, int NG, int NH, int NP) {
  SmemPlan L{};
  L.part = 0;                                       // per sender CTA, its two partial sums (16 bytes)
  L.u = 16u * kMaxCluster;                          // u of the own rows, then the halo: 8 floats each
  L.recv = al16(L.u + 32u * (NR + NH));             // received A_ijᵀ u_i: 6 floats per slot
  L.a = al16(L.recv + 24u * NG);                    // home blocks, 36 floats each, row-major
  L.col = al16(L.a + 144u * NB);                    // per home block {column's u slot, transposed target}
  L.mi = al16(L.col + 8u * NB);                     // M⁻¹ of each row, packed lower (21 floats)
  L.xps = al16(L.mi + 84u * NR);                    // x, p, s of each row (3 x 6 floats)
  L.hb = al16(L.xps + 72u * NR);
  L.go = al16(L.hb + 4u * (NR + 1));
  L.po = al16(L.go + 4u * (NR + 1));
  L.push = al16(L.po + 4u * (NR + 1));
  L.rows = al16(L.push + 4u * NP);
  L.bar = al16(L.rows + 4u * NR);                   // the staging copies' mbarrier
  L.total = L.bar + 16u;
  return L;
}

// ------------------------------------------------------------------ distributed shared memory

__device__ __forceinline__ unsigned cta_rank_in_cluster() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// the address of the same shared-memory location in CTA `rank` of the
// cluster (a CTA's own addresses are valid cluster addresses as they are)
__device__ __forceinline__ unsigned at_rank(unsigned a, unsigned rank, unsigned me) {
  if (rank == me) return a;
  unsigned r;
  asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cl_f4(unsigned a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cl_f2(unsigned a, float x, float y) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}
__device__ __forceinline__ void st_cl_u64x2(unsigned a, unsigned long long x, unsigned long long y) {
  asm volatile("st.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(x), "l"(y) : "memory");
}
// one bulk copy global -> this CTA's shared memory, completing on an mbarrier
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// bounded wait for phase 0 of an mbarrier; true if it completed (every thread of the CTA)
__device__ __forceinline__ bool wait_phase0(unsigned bar) {
  unsigned done = 0;
  for (int spins = 0; spins < (1 << 20) && !done; ++spins) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(0u)
        : "memory");
  }
  return __syncthreads_and(done != 0) != 0;
}
// every thread of every CTA of the cluster: the shared-memory writes before
// it, local and remote, are visible to every CTA's reads after it
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The group's sums of six values, reduce-scattered: lane l of the 8-lane
// group (gl = l) returns the sum over the group of value l (l < 6; lanes 6
// and 7 return the sums of two zeros).  Three exchange levels halve the
// values a lane carries (7 shuffles instead of the 18 of six butterflies).
__device__ __forceinline__ float group_reduce_scatter6(const float* v6, int gl) {
  float v[8] = {v6[0], v6[1], v6[2], v6[3], v6[4], v6[5], 0.f, 0.f};
  const bool b4 = gl & 4, b2 = gl & 2, b1 = gl & 1;
  float w[4], x[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {   // keep values 4..7 on lanes with bit 2, 0..3 on the others
    const float keep = b4 ? v[i + 4] : v[i], send = b4 ? v[i] : v[i + 4];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b2 ? w[i + 2] : w[i], send = b2 ? w[i] : w[i + 2];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  const float keep = b1 ? x[1] : x[0], send = b1 ? x[0] : x[1];
  return keep + __shfl_xor_sync(0xffffffffu, send, 1);
}

// The CTA's sums of two accumulators (every thread holds shares), by
// cascaded summation in a fixed order; every lane of warp 0 returns them.
template <typename Acc>
__device__ __forceinline__ void cta_sum2(Acc& a, Acc& b, Acc (*s_w)[32]) {
  using O = AccOps<Acc>;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  a = warp_sum_cascaded(a);
  b = warp_sum_cascaded(b);
  if (lane == 0) { s_w[0][wid] = a; s_w[1][wid] = b; }
  __syncthreads();
  if (wid == 0) {
    constexpr int kWarps = kCThreads / 32;
    a = lane < kWarps ? s_w[0][lane] : O::zero();
    b = lane < kWarps ? s_w[1][lane] : O::zero();
    a = acc_norm(warp_sum_cascaded(a));
    b = acc_norm(warp_sum_cascaded(b));
  }
}

// ------------------------------------------------------------------ the kernel

template <typename Acc>
__global__ void __launch_bounds__(kCThreads, 1)
k_pcg_cluster(Batch bt, const int* __restrict__ members, int C, int K, int gn_it) {
  using O = AccOps<Acc>;
  const unsigned me = cta_rank_in_cluster();
  const int s = __ldg(members + blockIdx.x / C);
  if (!stream_active(bt, s)) {   // the whole cluster leaves together, after the launch it may overlap
    asm volatile("griddepcontrol.wait;" ::: "memory");
    return;
  }
  const SwDev d = bt.devs[s];
  const int* __restrict__ P = d.cplan;
  const int NR = __ldg(P + 1), NB = __ldg(P + 2), NG = __ldg(P + 3), NH = __ldg(P + 5), NP = __ldg(P + 6);
  const int n_push = __ldg(P + kPlanHeader + 4 * (C + 1) - 1);   // the push prefix table's last entry
  const PlanOff off = plan_off(C, d.n_n, d.nnzb, n_push);
  const int row0 = __ldg(P + off.rb + me), nr = checked_count(__ldg(P + off.rb + me + 1) - row0, NR, d.status);
  const int blk0 = __ldg(P + off.bb + me), nb = checked_count(__ldg(P + off.bb + me + 1) - blk0, NB, d.status);
  const int push0 = __ldg(P + off.pb + me), np = checked_count(__ldg(P + off.pb + me + 1) - push0, NP, d.status);
  const SmemPlan L = smem_plan(NR, NB, NG, NH, NP);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Acc* sPart = reinterpret_cast<Acc*>(smem_raw + L.part);   // [sender][2]
  float* sU = reinterpret_cast<float*>(smem_raw + L.u);
  float* sRecv = reinterpret_cast<float*>(smem_raw + L.recv);
  float* sA = reinterpret_cast<float*>(smem_raw + L.a);
  int2* sCol = reinterpret_cast<int2*>(smem_raw + L.col);
  float* sMi = reinterpret_cast<float*>(smem_raw + L.mi);
  float* sXps = reinterpret_cast<float*>(smem_raw + L.xps);   // row a: x at 18a, p at 18a + 6, s at 18a + 12
  int* sHb = reinterpret_cast<int*>(smem_raw + L.hb);
  int* sGo = reinterpret_cast<int*>(smem_raw + L.go);
  int* sPo = reinterpret_cast<int*>(smem_raw + L.po);
  int* sPush = reinterpret_cast<int*>(smem_raw + L.push);
  int* sRows = reinterpret_cast<int*>(smem_raw + L.rows);
  __shared__ Acc s_w[2][32];
  __shared__ float s_alpha, s_beta;
  __shared__ int s_state;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = tid >> 3, gl = tid & 7;           // row group, lane in the group
  const int gbase = lane & ~7;                    // the group's first lane in the warp
  const bool comp = gl < 6;                       // this lane holds component gl of its rows
  const unsigned symoff = sym_offsets(comp ? gl : 0);   // row gl of a packed M⁻¹ block
  const unsigned uBase = smem_u32(sU), recvBase = smem_u32(sRecv), partBase = smem_u32(sPart);
  const unsigned bar = smem_u32(smem_raw + L.bar);

  // ---- set-up: the plan's tables and M⁻¹ by plain loads; the home blocks,
  // contiguous in A row by row, by one bulk copy per row on an mbarrier
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  for (int a = tid; a <= nr; a += kCThreads) {
    if (a < nr) sRows[a] = checked(__ldg(P + off.rows + row0 + a), d.n_n, d.status);
    sHb[a] = checked_count(__ldg(P + off.hb + row0 + me + a), nb, d.status);
    sGo[a] = checked_count(__ldg(P + off.go + row0 + me + a), NG, d.status);
    sPo[a] = checked_count(__ldg(P + off.po + row0 + me + a), np, d.status);
  }
  for (int x = tid; x < np; x += kCThreads) sPush[x] = checked_pair(__ldg(P + off.push + push0 + x), C, NR + NH, d.status);
  for (int e = tid; e < nb; e += kCThreads) {
    const int o2t = __ldg(P + off.o2t + blk0 + e);
    sCol[e] = make_int2(checked(__ldg(P + off.col + blk0 + e), NR + NH, d.status),
                        o2t == -1 ? -1 : checked_pair(o2t, C, NG, d.status));
  }
  for (int t = tid; t < 18 * nr; t += kCThreads) sXps[t] = 0.f;
  __syncthreads();
  if (tid == 0) {
    unsigned long long st;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;" : "=l"(st) : "r"(bar), "r"(144u * nb)
                 : "memory");
    (void)st;
  }
  __syncthreads();
  const float* __restrict__ Ag = sys_A(d, gn_it);
  for (int a = tid; a < nr; a += kCThreads) {
    const int e0 = sHb[a], len = checked_count(sHb[a + 1] - e0, nb - e0, d.status);
    // the row's first block; its others follow it in A
    const int b0 = checked(__ldg(P + off.blk + blk0 + e0), (long long)d.nnzb - len + 1, d.status);
    bulk_g2s(smem_u32(sA + 36 * (size_t)e0), Ag + 36 * (size_t)b0, 144u * (unsigned)len, bar);
  }
  // M⁻¹ comes from the preconditioner launch just before this one, which
  // lets this launch start early (programmatic dependent launch): everything
  // above overlaps it, and this waits until it has completed and its writes
  // are visible (a no-op when launched without the dependency)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int t = tid; t < nr * 21; t += kCThreads) {
    const int a = t / 21, q = t - 21 * a;
    sMi[t] = __ldg(d.minv + 21 * (size_t)sRows[a] + q);
  }
  if (!wait_phase0(bar)) {
    // the copies did not complete within the bound: report it, let them
    // land (bounded), and stage the blocks with plain loads instead
    if (tid == 0) atomicOr(d.status, kStatusTimeout);
    wait_phase0(bar);
    for (int t = tid; t < nb * 36; t += kCThreads) {
      const int e = t / 36;
      sA[t] = __ldg(Ag + 36 * (size_t)checked(__ldg(P + off.blk + blk0 + e), d.nnzb, d.status) + (t - 36 * e));
    }
    __syncthreads();
  }

  // rows of this group: a = g, and a = 2G − 1 − g
  int arow[2];
  arow[0] = g;
  arow[1] = 2 * kGroups - 1 - g;
  float rr[2] = {0.f, 0.f};   // component gl of the rows' r
  float uc[2] = {0.f, 0.f};   // component gl of the rows' u (also in sU for the group's loads)
  Acc gam = O::zero();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int a = arow[h];
    const bool on = a < nr;
    const float* mi = sMi + 21 * (on ? a : 0);
    const float r = (on && comp) ? -__ldg(sys_g(d, gn_it) + 6 * (size_t)sRows[a] + gl) : 0.f;
    float u = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float rk = __shfl_sync(0xffffffffu, r, gbase + k);
      if (comp) u += mi[sym_at(symoff, k)] * rk;
    }
    if (on && comp) {
      rr[h] = r;
      uc[h] = u;
      sU[8 * a + gl] = u;
      // a diagonal block that is not positive definite (its inverse's first
      // entry is a NaN) reaches every CTA through the first reduction
      gam = (mi[0] != mi[0]) ? acc_nan<Acc>() : O::add(gam, O::prod(r, u));
    }
  }
  __syncthreads();
  cluster_barrier();   // every CTA runs: its shared memory may be written now

  // u of the own rows out to the CTAs that hold them as halo (one lane per push)
  auto push_u = [&]() {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int a = arow[h];
      const bool on = a < nr;
      const int x1 = on ? sPo[a + 1] : 0;
      for (int x = (on ? sPo[a] : 0) + gl; x < x1; x += kGroup) {
        const int tg = sPush[x];
        const float4 v = *reinterpret_cast<const float4*>(sU + 8 * a);
        const float2 w2 = *reinterpret_cast<const float2*>(sU + 8 * a + 4);
        const unsigned ta = at_rank(uBase + 32u * (unsigned)(tg & 0xffff), (unsigned)(tg >> 16), me);
        st_cl_f4(ta, v);
        st_cl_f2(ta + 16, w2.x, w2.y);
      }
    }
  };
  push_u();
  float a_prev = 1.f;     // warp 0, lane 0: the previous step's α and γ
  Acc g_prev = O::zero();
  int state = kGearOk;
  cluster_barrier();   // every CTA's halo holds u₀

  // second rows exist only in the upper groups: whole warps without any skip them
  const int hmax = __any_sync(0xffffffffu, arow[1] < nr) ? 2 : 1;
  for (int k = 0; k < K; ++k) {
    // ---- A: w's home part, the transposed products out, δ's share
    Acc del = O::zero();
    float wh[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= hmax) break;   // warp-uniform
      const int a = arow[h];
      const bool on = a < nr;
      const int e0 = on ? sHb[a] : 0, e1 = on ? sHb[a + 1] : 0;
      float ui[6], o1[6];
      {
        const float4 v = *reinterpret_cast<const float4*>(sU + 8 * (on ? a : 0));
        const float2 w2 = *reinterpret_cast<const float2*>(sU + 8 * (on ? a : 0) + 4);
        ui[0] = v.x; ui[1] = v.y; ui[2] = v.z; ui[3] = v.w; ui[4] = w2.x; ui[5] = w2.y;
      }
#pragma unroll
      for (int b = 0; b < 6; ++b) o1[b] = 0.f;
      for (int e = e0 + gl; e < e1; e += kGroup) {
        const int2 co = sCol[e];   // one 8-byte load: the column's u slot and the transposed target
        const int ci = co.x;
        const float4 u4 = *reinterpret_cast<const float4*>(sU + 8 * ci);
        const float2 u2 = *reinterpret_cast<const float2*>(sU + 8 * ci + 4);
        // u_j in component pairs; the products run on packed FP32 pairs
        // (each lane of a pair an ordinary FP32 FMA, rounded alike)
        const float2 uj[3] = {make_float2(u4.x, u4.y), make_float2(u4.z, u4.w), u2};
        const float4* A4 = reinterpret_cast<const float4*>(sA + 36 * (size_t)e);
        float2 o2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        float dt = 0.f;
#pragma unroll
        for (int bp = 0; bp < 3; ++bp) {   // rows 2bp and 2bp + 1 of the block
          const float4 q0 = A4[3 * bp], q1 = A4[3 * bp + 1], q2 = A4[3 * bp + 2];
          const float2 ra[3] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y)};
          const float2 rb[3] = {make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
          // (A u_j) of both rows as pairs of partial sums over even and odd columns
          float2 ta = __fmul2_rn(ra[0], uj[0]), tb = __fmul2_rn(rb[0], uj[0]);
          ta = __ffma2_rn(ra[1], uj[1], ta);
          tb = __ffma2_rn(rb[1], uj[1], tb);
          ta = __ffma2_rn(ra[2], uj[2], ta);
          tb = __ffma2_rn(rb[2], uj[2], tb);
          const float sa = ta.x + ta.y, sb = tb.x + tb.y;
          // (A_ijᵀ u_i): rows 2bp and 2bp + 1 weighted by u_i's components
          const float2 wa = make_float2(ui[2 * bp], ui[2 * bp]), wb = make_float2(ui[2 * bp + 1], ui[2 * bp + 1]);
#pragma unroll
          for (int c = 0; c < 3; ++c) o2[c] = __ffma2_rn(rb[c], wb, __ffma2_rn(ra[c], wa, o2[c]));
          o1[2 * bp] += sa;
          o1[2 * bp + 1] += sb;
          dt += ui[2 * bp] * sa + ui[2 * bp + 1] * sb;
        }
        const int tg = co.y;
        // δ's share: exact times 1 or 2, added by a cascaded (TwoSum) step
        del = acc_add_cascaded(del, acc_from<Acc>(tg < 0 ? dt : 2.f * dt));
        if (tg >= 0) {   // off the diagonal: A_ijᵀ u_i to its receive slot at the column's owner
          const unsigned slot = (unsigned)(tg & 0xffff);
          const unsigned ta = at_rank(recvBase + 24u * slot, (unsigned)(tg >> 16), me);
          // a slot is 24 bytes, 8-byte aligned: three pair stores, the same for every slot
          st_cl_f2(ta, o2[0].x, o2[0].y);
          st_cl_f2(ta + 8, o2[1].x, o2[1].y);
          st_cl_f2(ta + 16, o2[2].x, o2[2].y);
        }
      }
      wh[h] = group_reduce_scatter6(o1, gl);
    }
    Acc ga = gam, da = del;
    cta_sum2(ga, da, s_w);
    if (warp == 0 && lane < C)   // the CTA's partials into slot `me` of every CTA
      st_cl_u64x2(at_rank(partBase + 16u * me, (unsigned)lane, me), O::bits(ga), O::bits(da));
    cluster_barrier();   // 1: partials and transposed products delivered

    // ---- B: the step, the received products, the update, u out
    if (warp == 0) {
      Acc gs = O::zero(), ds = O::zero();
      if (lane < C) {
        gs = sPart[2 * lane];
        ds = sPart[2 * lane + 1];
      }
      // lanes C..31 hold zeros: the butterfly over lanes 0..15 gives the same sums
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        gs = acc_add_cascaded(gs, O::shfl_xor(gs, o));
        ds = acc_add_cascaded(ds, O::shfl_xor(ds, o));
      }
      gs = acc_norm(gs);
      ds = acc_norm(ds);
      if (lane == 0) {
        float al, be;
        const int st = gear_step(k, gs, ds, g_prev, a_prev, &al, &be);
        s_state = st;
        s_alpha = al;
        s_beta = be;
        a_prev = al;
        g_prev = gs;
      }
    }
    // lane c adds component c of the row's received products, in slot order
    float wt[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= hmax) break;   // warp-uniform
      const int a = arow[h];
      const bool on = a < nr && comp;
      float acc = wh[h];
      const int x1 = on ? sGo[a + 1] : 0;
      int x = on ? sGo[a] : 0;
      for (; x + 1 < x1; x += 2) acc = (acc + sRecv[6 * x + gl]) + sRecv[6 * x + 6 + gl];
      if (x < x1) acc += sRecv[6 * x + gl];
      wt[h] = acc;
    }
    __syncthreads();
    state = s_state;
    if (state == kGearOk) {
      const float al = s_alpha, be = s_beta;
      gam = O::zero();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h >= hmax) break;   // warp-uniform
        const int a = arow[h];
        const bool on = a < nr;
        const float* mi = sMi + 21 * (on ? a : 0);
        if (on && comp) {
          float* xps = sXps + 18 * a + gl;
          const float pc = uc[h] + be * xps[6];
          const float sc = wt[h] + be * xps[12];
          xps[6] = pc;
          xps[12] = sc;
          xps[0] += al * pc;
          rr[h] -= al * sc;
        }
        float u = 0.f;
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
          const float rk = __shfl_sync(0xffffffffu, rr[h], gbase + kk);
          if (comp) u += mi[sym_at(symoff, kk)] * rk;
        }
        if (on && comp) {
          uc[h] = u;
          sU[8 * a + gl] = u;
          gam = acc_add_cascaded(gam, O::prod(rr[h], u));
        }
      }
      __syncwarp();   // the group's six components of u written before its lanes push them
      push_u();
    }
    cluster_barrier();   // 2: the new u delivered; partial and receive slots free again
    if (state != kGearOk) break;
  }

  // the next launch (the next iteration's regulariser assembly) may begin;
  // it waits for this launch's completion before reading anything
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  // ---- the final rᵀM⁻¹r (a statistic: one FP64 atomic per CTA, nobody waits)
  if (state == kGearOk || state == kGearConverged) {
    Acc ga = gam, zero = O::zero();
    cta_sum2(ga, zero, s_w);
    if (tid == 0) atomicAdd(d.pcg_rz + gn_it, O::value(ga));
  }
  if (state == kGearBreakdown) {
    if (tid == 0 && me == 0) atomicOr(d.status, kStatusBreakdown);
    return;
  }
  // ---- T_j ← Δ_j T_j for the own rows (nothing moves after a breakdown)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int a = arow[h];
    if (a < nr && gl == 0) {
      float xi[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) xi[c] = sXps[18 * a + c];
      const int j = sRows[a];
      float4 q0 = d.dq[2 * j], qe = d.dq[2 * j + 1];
      apply_increment(q0, qe, xi);
      d.dq[2 * j] = q0;
      d.dq[2 * j + 1] = qe;
    }
  }
}

// The hop the cluster PCG pays twice per iteration, alone: `iters` cluster
// barriers of C CTAs of kCThreads threads (its latency bound's unit).
__global__ void __launch_bounds__(kCThreads, 1) k_cluster_barrier_loop(int iters) {
  for (int k = 0; k < iters; ++k) cluster_barrier();
}

template <typename Acc>
const void* cluster_kernel() {
  return reinterpret_cast<const void*>(k_pcg_cluster<Acc>);
}

const void* cluster_kernel_for(int precision) {
  return precision == SW_PRECISION_MIXED_F64DOTS ? cluster_kernel<double>() : cluster_kernel<DF>();
}

// The function attributes a launch of `smem` bytes in clusters of C needs.
// The shared-memory limit only ever grows (per kernel and device), so a
// query for a small plan never lowers what a large plan's launches rely on.
cudaError_t prepare_cluster_kernel(const void* fn, int C, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set_to;   // (kernel, device) -> bytes
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set_to[{fn, dev}];
  if (smem > cur) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cur = smem;
  }
  if (C > 8) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// Morton code of a point in the unit cube, 10 bits per axis
uint32_t morton3(float x, float y, float z) {
  auto spread = [](uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
  };
  auto q = [](float t) { return (uint32_t)std::min(1023.f, std::max(0.f, t * 1023.f)); };
  return spread(q(x)) | (spread(q(y)) << 1) | (spread(q(z)) << 2);
}

}  // namespace

// The plan of one stream for clusters of C CTAs (see the file comment):
// false if some CTA would need more than kMaxRowsPerCta rows or more than
// smem_limit bytes of shared memory.
bool build_cluster_plan(int C, int n_n, const std::vector<int>& row_ptr, const std::vector<int>& col,
                        const std::vector<float>& node4, size_t smem_limit, std::vector<int>& plan,
                        size_t* smem_out) {
  if (C < 1 || C > kMaxCluster || n_n < 1 || (int)row_ptr.size() != n_n + 1) return false;
  const int nnzb = row_ptr[n_n];
  if ((int)col.size() != nnzb) return false;
  // receive slots: the off-diagonal upper blocks of each column
  std::vector<int> ng_col(n_n, 0);
  for (int i = 0; i < n_n; ++i)
    for (int b = row_ptr[i] + 1; b < row_ptr[i + 1]; ++b) ++ng_col[col[b]];
  // Morton order of the node positions
  float lo[3] = {1e30f, 1e30f, 1e30f}, hi[3] = {-1e30f, -1e30f, -1e30f};
  for (int j = 0; j < n_n; ++j)
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(lo[a], node4[4 * j + a]);
      hi[a] = std::max(hi[a], node4[4 * j + a]);
    }
  const float ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-12f});
  std::vector<uint32_t> code(n_n);
  for (int j = 0; j < n_n; ++j)
    code[j] = morton3((node4[4 * j] - lo[0]) / ext, (node4[4 * j + 1] - lo[1]) / ext,
                      (node4[4 * j + 2] - lo[2]) / ext);
  std::vector<int> order(n_n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return code[a] < code[b]; });
  // contiguous ranges of that order, balanced by shared-memory bytes (a
  // row's u, x, p, s, M⁻¹ and tables; each home block's 36 values and
  // tables; each receive slot)
  auto bytes = [&](int j) { return 230.0 + 152.0 * (row_ptr[j + 1] - row_ptr[j]) + 24.0 * ng_col[j]; };
  double total = 0;
  for (int j = 0; j < n_n; ++j) total += bytes(j);
  std::vector<int> cut(C + 1, n_n);
  cut[0] = 0;
  {
    double acc = 0;
    int c = 1;
    for (int t = 0; t < n_n && c < C; ++t) {
      acc += bytes(order[t]);
      if (acc >= total * c / C) cut[c++] = t + 1;
    }
  }
  // per CTA: rows sorted by cost, placed so that group g serves positions g and 2G − 1 − g
  std::vector<int> owner(n_n), local(n_n);
  std::vector<std::vector<int>> rows(C);
  int NR = 0;
  for (int c = 0; c < C; ++c) {
    std::vector<int> r(order.begin() + cut[c], order.begin() + cut[c + 1]);
    if ((int)r.size() > kMaxRowsPerCta) return false;
    auto cost = [&](int j) { return (row_ptr[j + 1] - row_ptr[j] + kGroup - 1) / kGroup; };
    std::stable_sort(r.begin(), r.end(), [&](int a, int b) { return cost(a) > cost(b); });
    for (size_t a = 0; a < r.size(); ++a) {
      owner[r[a]] = c;
      local[r[a]] = (int)a;
    }
    NR = std::max(NR, (int)r.size());
    rows[c] = std::move(r);
  }
  // halos: per CTA, the other CTAs' rows its home blocks reference, in
  // (owner, local row) order; each gets a u slot after the CTA's own rows
  // (halo_slot[c n_n + j], -1 where row j is not in CTA c's halo)
  std::vector<int> halo_slot((size_t)C * n_n, -1);
  std::vector<std::vector<int>> halo_rows(C);   // per CTA, its halo rows in slot order
  int NH = 0, NB = 0, NG = 0;
  for (int c = 0; c < C; ++c) {
    std::vector<long long> ext;
    int nb = 0, ng = 0;
    int* hs = halo_slot.data() + (size_t)c * n_n;
    for (int i : rows[c]) {
      nb += row_ptr[i + 1] - row_ptr[i];
      ng += ng_col[i];
      for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        const int j = col[b];
        if (owner[j] != c && hs[j] == -1) {
          hs[j] = -2;
          ext.push_back(((long long)owner[j] << 32) | local[j]);
        }
      }
    }
    std::sort(ext.begin(), ext.end());
    const int nr = (int)rows[c].size();
    halo_rows[c].resize(ext.size());
    for (size_t h = 0; h < ext.size(); ++h) {
      const int j = rows[ext[h] >> 32][ext[h] & 0xffffffff];
      hs[j] = nr + (int)h;
      halo_rows[c][h] = j;
    }
    NH = std::max(NH, (int)ext.size());
    NB = std::max(NB, nb);
    NG = std::max(NG, ng);
  }
  // u pushes: per own row, the CTAs holding it as halo (in CTA order), with their slot
  std::vector<int> push_ptr(n_n + 1, 0), push_tg;
  for (int c = 0; c < C; ++c)
    for (int j : halo_rows[c]) ++push_ptr[j + 1];
  for (int j = 0; j < n_n; ++j) push_ptr[j + 1] += push_ptr[j];
  push_tg.resize(push_ptr[n_n]);
  {
    std::vector<int> fill(push_ptr.begin(), push_ptr.end() - 1);
    for (int c = 0; c < C; ++c)
      for (int j : halo_rows[c]) push_tg[fill[j]++] = (c << 16) | halo_slot[(size_t)c * n_n + j];
  }
  int NP = 0, n_push = 0;
  for (int c = 0; c < C; ++c) {
    int np = 0;
    for (int i : rows[c]) np += push_ptr[i + 1] - push_ptr[i];
    NP = std::max(NP, np);
    n_push += np;
  }
  if (NG >= (1 << 16) || NR + NH >= (1 << 16)) return false;
  const SmemPlan L = smem_plan(NR, NB, NG, NH, NP);
  if (L.total > smem_limit) return false;
  const PlanOff o = plan_off(C, n_n, nnzb, n_push);
  plan.assign(o.total, 0);
  plan[0] = C; plan[1] = NR; plan[2] = NB; plan[3] = NG; plan[4] = n_n; plan[5] = NH; plan[6] = NP;
  // home block index of each block within its CTA
  std::vector<int> home(nnzb, 0);
  for (int c = 0; c < C; ++c) {
    int e = 0;
    for (int i : rows[c])
      for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) home[b] = e++;
  }
  // receive slots of each row j at its owner: its column's off-diagonal
  // blocks (i, j) in (home CTA, home block index) order, which is the order
  // of the CTAs, their rows and the rows' blocks
  std::vector<int> inc_ptr(n_n + 1, 0), inc_blk;
  for (int j = 0; j < n_n; ++j) inc_ptr[j + 1] = inc_ptr[j] + ng_col[j];
  inc_blk.resize(inc_ptr[n_n]);
  {
    std::vector<int> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int c = 0; c < C; ++c)
      for (int i : rows[c])
        for (int b = row_ptr[i] + 1; b < row_ptr[i + 1]; ++b) inc_blk[fill[col[b]]++] = b;
  }
  std::vector<int> slot_of(nnzb, -1);
  int rb = 0, bb = 0, gb = 0, pb = 0;
  for (int c = 0; c < C; ++c) {
    plan[o.rb + c] = rb;
    plan[o.bb + c] = bb;
    plan[o.gb + c] = gb;
    plan[o.pb + c] = pb;
    int e = 0, x = 0, y = 0;
    const int nr = (int)rows[c].size();
    for (int a = 0; a < nr; ++a) {
      const int i = rows[c][a];
      plan[o.rows + rb + a] = i;
      plan[o.hb + rb + c + a] = e;
      plan[o.go + rb + c + a] = x;
      plan[o.po + rb + c + a] = y;
      e += row_ptr[i + 1] - row_ptr[i];
      for (int q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) slot_of[inc_blk[q]] = x++;
      for (int q = push_ptr[i]; q < push_ptr[i + 1]; ++q) plan[o.push + pb + y++] = push_tg[q];
    }
    plan[o.hb + rb + c + nr] = e;
    plan[o.go + rb + c + nr] = x;
    plan[o.po + rb + c + nr] = y;
    rb += nr;
    bb += e;
    gb += x;
    pb += y;
  }
  plan[o.rb + C] = rb;
  plan[o.bb + C] = bb;
  plan[o.gb + C] = gb;
  plan[o.pb + C] = pb;
  // per home block: A's index, its column's u slot, its transposed product's target
  for (int c = 0; c < C; ++c) {
    const int base = plan[o.bb + c];
    for (int i : rows[c])
      for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        const int e = home[b], j = col[b];
        plan[o.blk + base + e] = b;
        plan[o.col + base + e] = owner[j] == c ? local[j] : halo_slot[(size_t)c * n_n + j];
        plan[o.o2t + base + e] = b == row_ptr[i] ? -1 : ((owner[j] << 16) | slot_of[b]);
      }
  }
  *smem_out = L.total;
  return true;
}

// How many clusters of C CTAs with `smem` bytes each can run at once (0 if
// none, or a negative CUDA error code).
int cluster_pcg_active(int precision, int C, size_t smem) {
  const void* fn = cluster_kernel_for(precision);
  cudaError_t pe = prepare_cluster_kernel(fn, C, smem);
  if (pe != cudaSuccess) {
    cudaGetLastError();
    return -(int)pe;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, fn, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -(int)e;
  }
  return n;
}

bool cluster_pcg_fits(int precision, int C, size_t smem) { return cluster_pcg_active(precision, C, smem) >= 1; }

cudaError_t launch_pcg_cluster(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st) {
  if (b.n_cluster == 0) return cudaSuccess;
  const int C = b.cluster_ctas;
  const void* fn = cluster_kernel_for(b.precision);
  const cudaError_t pe = prepare_cluster_kernel(fn, C, b.cluster_smem);
  if (pe != cudaSuccess) return pe;
  Batch bt = b.bt;
  const int* members = b.cluster_members_dev;
  int c = C, kk = pcg_iters, it = gn_it;
  void* args[] = {&bt, &members, &c, &kk, &it};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C * b.n_cluster);
  cfg.blockDim = dim3(kCThreads);
  cfg.dynamicSmemBytes = b.cluster_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  // may start while the preconditioner launch before it runs (the kernel
  // waits for it before reading M⁻¹)
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Seconds of one cluster barrier of C CTAs (kCThreads threads each), from
// two timed launches of n1 and n2 barriers (the difference removes the
// launch): the unit of the cluster PCG's latency bound.
cudaError_t cluster_barrier_cost(int C, double* us_per_barrier) {
  const void* fn = reinterpret_cast<const void*>(k_cluster_barrier_loop);
  cudaError_t e = C > 8 ? cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) : cudaSuccess;
  if (e != cudaSuccess) return e;
  cudaEvent_t ev[4];
  for (auto& x : ev) cudaEventCreate(&x);
  float ms[2] = {0.f, 0.f};
  const int n[2] = {64, 1064};
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      int it = n[k];
      void* args[] = {&it};
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(kCThreads);
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaEventRecord(ev[2 * k], 0);
      e = cudaLaunchKernelExC(&cfg, fn, args);
      cudaEventRecord(ev[2 * k + 1], 0);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev[2 * k + 1]);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[2 * k], ev[2 * k + 1]);
      if (rep > 0) ms[k] += t;   // the first round warms up
    }
  for (auto& x : ev) cudaEventDestroy(x);
  if (e == cudaSuccess && us_per_barrier) *us_per_barrier = 1000.0 * (ms[1] - ms[0]) / 2.0 / (n[1] - n[0]);
  return e;
}

}  // namespace sw
