// K7+K8: block-Jacobi preconditioned conjugate gradients on JᵀJ Δ = −Jᵀe
// and the node update T_j ← Δ_j T_j (Sec. 7), one persistent cooperative
// launch per Gauss-Newton iteration for every stream of a batch, after the
// preconditioner's own launch (k_precond: the FP64 inverse of every
// diagonal block).
//
// Both kernels run x₀ = 0 and exactly K iterations, stopping early only when
// rᵀM⁻¹r is exactly zero; pᵀAp <= 0 (or a diagonal block that is not
// positive definite) is a breakdown and leaves the node transforms as they
// were.
//
// Work split.  Stream s owns the CTAs [tile_base[s], tile_base[s+1]), all
// co-resident.  CTA t of a stream with G CTAs owns the block rows and nodes
// i = t + G a (a = 0, 1, ...) and keeps everything about them in shared
// memory for the whole solve: the 6x6 block of M⁻¹ (from k_precond) and the
// rows' vectors.  Global memory carries only the vector other CTAs read for
// the SpMV.  The reductions are per stream, so streams never wait for one
// another.
//
//   k_pcg_gear (FP32 modes)  Chronopoulos-Gear arrangement: one reduction
//       per iteration; the SpMV's input is exchanged as tagged words that
//       the readers wait for, with no fences and no barrier.
//   k_pcg_f64 (SW_PRECISION_FP64)  the standard recurrences, two reductions
//       per iteration with a release / acquire protocol; readers form the
//       neighbour's p = z + β p_old from published z and p_old.
//
// Inner products accumulate in the Acc type: DF (double-float pairs, the
// default) or FP64.
#include <type_traits>

#include "sw_internal.h"
#include "sw_check.cuh"
#include "sw_math.cuh"
#include "sw_math64.cuh"
#include "sw_df.cuh"
#include "sw_pcg.cuh"

namespace sw {
namespace {

// failure injection for the tests of the bounded waits: {WaitFault kind,
// poll limit that replaces the launch's (0: the launch's)}; read at every
// launch, so captured graphs follow the current setting
__device__ int g_wait_fault[2];

// ------------------------------------------------------------------ 6x6 blocks


// 1/x for a positive FP64 x: the FP32 reciprocal as the seed, refined by
// kSteps Newton-Raphson steps r <- r + r (1 - x r), each of which about
// doubles the number of correct bits (24 -> 46 -> the FP64 rounding limit).
// A division in FP64 is a chain of several hundred cycles on this part; this
// is 2 + 2 kSteps dependent FP64 operations.  Outside the range where the
// FP32 seed is accurate, the plain division.
template <int kSteps>
__device__ __forceinline__ double recip64(double x) {
  const float xf = (float)x;
  if (!(xf >= 1e-30f && xf <= 1e30f)) return 1.0 / x;
  double r = (double)__frcp_rn(xf);
#pragma unroll
  for (int k = 0; k < kSteps; ++k) {
    const double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
  }
  return r;
}

__device__ __forceinline__ int sl(int r, int c) { return r * (r - 1) / 2 + c; }   // strict lower, r > c

// M⁻¹ of one diagonal block (symmetric, packed lower) in FP64 by the
// factorisation A = L D Lᵀ (L unit lower triangular): M⁻¹ = L⁻ᵀ D⁻¹ L⁻¹,
// from the block's lower triangle (the assembly writes the upper one equal
// up to the rounding order of its atomics).  No square roots, and the six
// pivots' reciprocals by recip64 -- one Newton step for an FP32 result (about
// 46 correct bits), two for an FP64 one -- so the dependent chain, and the
// FP64 instruction stream that bounds a warp here, stay short.  False if the
// block is not positive definite (a pivot <= 0).
template <typename Real>
__device__ bool block_inverse(const Real* a, Real* out) {
  // every loop has a constant trip count (bounds as predicates), so that all
  // of them unroll and the arrays live in registers.
  // S: the lower triangle (packed); its strict lower part is then
  // overwritten by E = L D (E_rc = L_rc d_c) and finally by Y = D⁻¹ L⁻¹
  constexpr int kSteps = std::is_same<Real, float>::value ? 1 : 2;
  double S[21], L[15], Di[6];
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c)
      if (c <= r) S[tri(r, c)] = (double)a[r * 6 + c];
  // column by column: d_c = a_cc − Σ_{k<c} L_ck E_ck, E_rc = a_rc − Σ_{k<c} L_rk E_ck, L_rc = E_rc / d_c
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double dc = S[tri(c, c)];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      if (k < c) dc = fma(-L[sl(c, k)], S[tri(c, k)], dc);
    if (!(dc > 0.0)) return false;
    Di[c] = recip64<kSteps>(dc);
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      if (r <= c) continue;
      double e = S[tri(r, c)];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k < c) e = fma(-L[sl(r, k)], S[tri(c, k)], e);
      S[tri(r, c)] = e;
      L[sl(r, c)] = e * Di[c];
    }
  }
  // X = L⁻¹ (unit lower), over L column by column (column c reads only
  // columns > c of L): X_rc = −L_rc − Σ_{c<k<r} L_rk X_kc
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      if (r <= c) continue;
      double x = -L[sl(r, c)];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k > c && k < r) x = fma(-L[sl(r, k)], L[sl(k, c)], x);
      L[sl(r, c)] = x;
    }
  // M⁻¹_rc = Σ_{k>=r} X_kr D⁻¹_k X_kc (r >= c, X_kk = 1) = Y_rc + Σ_{k>r} X_kr Y_kc, Y = D⁻¹ X
#pragma unroll
  for (int c = 0; c < 6; ++c)
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (k == c) S[tri(c, c)] = Di[c];
      if (k > c) S[tri(k, c)] = Di[k] * L[sl(k, c)];
    }
#pragma unroll
  for (int r = 0; r < 6; ++r)
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      if (c > r) continue;
      double m = S[tri(r, c)];
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k > r) m = fma(L[sl(k, r)], S[tri(k, c)], m);
      out[tri(r, c)] = (Real)m;
    }
  return true;
}

// ------------------------------------------------------------------ exchange

// FP32 kernel: every shared value travels as one 8-byte word {FP32 bits,
// 32-bit generation tag}, written and read with single 8-byte accesses, so a
// reader that sees the expected tag also sees the value written with it and
// no fence is needed (the writer never waits for its stores to reach L2).  A
// reader that finds an older tag reads again, a bounded number of times.
// FP64 kernel: plain values, published with a release pattern (values, one
// acq_rel fence, a relaxed store of a stamp) and read after acquire loads of
// the stamps.

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_v2(unsigned long long* p, unsigned long long a, unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ ulonglong2 ld_relaxed_v2(const unsigned long long* p) {
  ulonglong2 v;
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long tagged(unsigned bits, unsigned tag) {
  return (unsigned long long)bits | ((unsigned long long)tag << 32);
}
__device__ __forceinline__ unsigned tag_of(unsigned long long w) { return (unsigned)(w >> 32); }

__device__ __forceinline__ void put_tagged(unsigned long long* buf, size_t i, float v, unsigned tag) {
  st_relaxed_u64(buf + i, tagged(__float_as_uint(v), tag));
}

// the 6 values of node j carrying the given tag; false if they did not
// arrive within `spins` further reads
__device__ __forceinline__ bool get6_tagged(const unsigned long long* buf, int j, unsigned tag, float* v, int spins) {
  const unsigned long long* src = buf + 6 * (size_t)j;
  for (int n = 0;; ++n) {
    ulonglong2 a[3];
#pragma unroll
    for (int h = 0; h < 3; ++h) a[h] = ld_relaxed_v2(src + 2 * h);
    unsigned bad = 0;
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      bad |= (tag_of(a[h].x) ^ tag) | (tag_of(a[h].y) ^ tag);
      v[2 * h] = __uint_as_float((unsigned)a[h].x);
      v[2 * h + 1] = __uint_as_float((unsigned)a[h].y);
    }
    if (bad == 0) return true;
    if (n >= spins) return false;
  }
}

// p_j = z_j (+ β p_old,j) from two FP64 vectors published before the last reduction
__device__ __forceinline__ void get_p64(const double* z, const double* po, bool with_old, double beta, int j,
                                        double* p) {
  const double2* z2 = reinterpret_cast<const double2*>(z + 6 * (size_t)j);
  const double2* o2 = reinterpret_cast<const double2*>(po + 6 * (size_t)j);
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const double2 a = __ldcg(z2 + h);
    p[2 * h] = a.x; p[2 * h + 1] = a.y;
  }
  if (with_old) {
#pragma unroll
    for (int h = 0; h < 3; ++h) {
      const double2 o = __ldcg(o2 + h);
      p[2 * h] += beta * o.x; p[2 * h + 1] += beta * o.y;
    }
  }
}

// one row of a 6x6 block of the matrix (read-only for the whole launch)
__device__ __forceinline__ void load6_ro(const float* p, float* v) {
  const float2* p2 = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const float2 a = __ldg(p2 + h);
    v[2 * h] = a.x; v[2 * h + 1] = a.y;
  }
}
__device__ __forceinline__ void load6_ro(const double* p, double* v) {
  const double2* p2 = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int h = 0; h < 3; ++h) {
    const double2 a = __ldg(p2 + h);
    v[2 * h] = a.x; v[2 * h + 1] = a.y;
  }
}

template <typename Real>
__device__ __forceinline__ Real warp_sum_r(Real v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ reductions

// A reduction among the CTAs of one stream is also their synchronisation.
// Precondition: within each warp only lanes below `lanes` (a power of two)
// hold nonzero values.  Every CTA publishes its block sums for generation
// `gen` (slots double-buffered by its parity); one warp polls the stream's
// slots (bounded) and sums them in a fixed order, so the totals are
// deterministic for a given number of CTAs.  `on_total` runs on one thread
// before the CTA continues (the step-length arithmetic, done once).  Both
// return false if the wait ran out.

// Two values, tagged: CTA t writes each value's two 32-bit halves as tagged
// words into slots 2t and 2t+1 of the generation's half of `part`
// (2 kMaxCtaPerStream slots per parity); pollers check all four tags at once.
// A tag is the generation's low 31 bits; its top bit says that the
// publishing CTA's wait for a neighbour's vector ran out (*late nonzero),
// and on_total(a, b, any_late) learns whether any CTA of the stream was late.
template <typename Acc, typename F>
__device__ __forceinline__ bool stream_reduce_pair(Acc va, Acc vb, int lanes, PartSlot* part, int t, int gs,
                                                   unsigned long long gen, int spin_limit, bool publish,
                                                   const int* late, F&& on_total) {
  using O = AccOps<Acc>;
  __shared__ Acc s_w[2][32];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = lanes >> 1; o > 0; o >>= 1) {
    va = O::add(va, O::shfl_xor(va, o));
    vb = O::add(vb, O::shfl_xor(vb, o));
  }
  if (lane == 0) { s_w[0][wid] = va; s_w[1][wid] = vb; }
  __syncthreads();
  PartSlot* buf = part + (gen & 1ull) * 2 * kMaxCtaPerStream;
  constexpr unsigned kLateBit = 0x80000000u;
  const unsigned tag = (unsigned)gen & ~kLateBit;
  if (wid == 0) {
    Acc a = lane < nw ? s_w[0][lane] : O::zero();
    Acc b = lane < nw ? s_w[1][lane] : O::zero();
    a = warp_sum_acc(a);
    b = warp_sum_acc(b);
    if (lane == 0 && publish) {   // (publish is false only under failure injection)
      const unsigned long long ba = O::bits(a), bb = O::bits(b);
      const unsigned tg = tag | (*late ? kLateBit : 0u);
      st_relaxed_v2(&buf[2 * t].v, tagged((unsigned)ba, tg), tagged((unsigned)(ba >> 32), tg));
      st_relaxed_v2(&buf[2 * t + 1].v, tagged((unsigned)bb, tg), tagged((unsigned)(bb >> 32), tg));
    }
    int ok = 1;
    unsigned any_late = 0;
    Acc ca = O::zero(), cb = O::zero();
    for (int k = lane; k < gs; k += 32) {
      ulonglong2 wa, wb;
      int spins = 0;
      for (;;) {
        wa = ld_relaxed_v2(&buf[2 * k].v);
        wb = ld_relaxed_v2(&buf[2 * k + 1].v);
        const unsigned m = ~kLateBit;
        if ((((tag_of(wa.x) & m) ^ tag) | ((tag_of(wa.y) & m) ^ tag) | ((tag_of(wb.x) & m) ^ tag) |
             ((tag_of(wb.y) & m) ^ tag)) == 0)
          break;
        if (++spins > spin_limit) { ok = 0; break; }
      }
      if (!ok) break;
      any_late |= tag_of(wa.x) & kLateBit;
      ca = O::add(ca, O::from_bits((wa.x & 0xffffffffull) | (wa.y << 32)));
      cb = O::add(cb, O::from_bits((wb.x & 0xffffffffull) | (wb.y << 32)));
    }
    ok = __all_sync(0xffffffffu, ok);
    any_late = __any_sync(0xffffffffu, any_late != 0);
    ca = warp_sum_acc(ca);
    cb = warp_sum_acc(cb);
    if (lane == 0) {
      s_ok = ok;
      on_total(ca, cb, any_late != 0);
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// The CTA's sum of v (nonzero only in lanes below `lanes` of each warp, a
// power of two) added to *dst with one FP64 atomic.
template <typename Acc>
__device__ __forceinline__ void block_add_value(Acc v, int lanes, double* dst) {
  using O = AccOps<Acc>;
  __shared__ Acc s_w[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = lanes >> 1; o > 0; o >>= 1) v = O::add(v, O::shfl_xor(v, o));
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  if (wid == 0) {
    Acc b = lane < nw ? s_w[lane] : O::zero();
    b = warp_sum_acc(b);
    if (lane == 0) atomicAdd(dst, O::value(b));
  }
}

// One value, release / acquire: the value, one acq_rel fence and a relaxed
// store of the stamp, so the CTA's global writes before the call go with it;
// pollers take acquire loads of the stamps.
template <typename Acc, typename F>
__device__ __forceinline__ bool stream_reduce_fenced(Acc v, int lanes, PartSlot* part, int t, int gs,
                                                     unsigned long long gen, int spin_limit, bool publish,
                                                     F&& on_total) {
  using O = AccOps<Acc>;
  __shared__ Acc s_w[32];
  __shared__ int s_ok;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = lanes >> 1; o > 0; o >>= 1) v = O::add(v, O::shfl_xor(v, o));
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  PartSlot* buf = part + (gen & 1ull) * kMaxCtaPerStream;
  if (wid == 0) {
    Acc b = lane < nw ? s_w[lane] : O::zero();
    b = warp_sum_acc(b);
    if (lane == 0 && publish) {   // (publish is false only under failure injection)
      buf[t].v = O::bits(b);
      fence_acq_rel_gpu();
      st_relaxed_u64(&buf[t].gen, gen);
    }
    int ok = 1;
    for (int k = lane; k < gs; k += 32) {
      int spins = 0;
      while (ld_acquire_u64(&buf[k].gen) < gen) {
        if (++spins > spin_limit) { ok = 0; break; }
      }
      if (!ok) break;
    }
    ok = __all_sync(0xffffffffu, ok);
    Acc c = O::zero();
    for (int k = lane; k < gs; k += 32) c = O::add(c, O::from_bits(__ldcg(&buf[k].v)));
    c = warp_sum_acc(c);
    if (lane == 0) {
      s_ok = ok;
      on_total(c);
    }
  }
  __syncthreads();
  return s_ok != 0;
}

// ------------------------------------------------------------------ shared pieces of the two kernels

constexpr int kPcgThreads = 1024;
constexpr int kPcgWarps = kPcgThreads / 32;

template <typename Real, typename Acc>
struct Scalars {
  Real alpha, beta;
  Acc rz;      // current rᵀM⁻¹r
  int work;    // rᵀM⁻¹r != 0 and no breakdown
  int bad;     // breakdown seen
};

// How the SpMV reaches the matrix (chosen per batch by what fits in shared
// memory):
//   kSpmvSmemA   the CTA copies its rows' blocks into shared memory at set-up;
//   kSpmvSmemOut the blocks are read from global memory each iteration;
// both take one thread per matrix entry of the CTA's rows (all of them in
// flight at once) with six outputs per entry in shared memory, then a warp
// per row sums its entries;
//   kSpmvRows    a warp per row, a lane per entry, nothing staged.
enum SpmvMode { kSpmvRows = 0, kSpmvSmemOut = 1, kSpmvSmemA = 2 };

// Shared memory of one CTA: per own row M⁻¹ (21) and `row_vecs` 6-vectors;
// in the staged modes the six outputs of every entry and, with kSpmvSmemA,
// the entries' blocks (36 values each), both stored entry-minor (value q of
// entry e at q * ent_cap + e, so threads on consecutive entries hit
// consecutive banks) with every block already turned to multiply the
// neighbour's vector directly; then per entry its neighbour (kSpmvSmemA) or
// its block and neighbour (kSpmvSmemOut); then the rows' entry offsets.
// Byte offsets of the sections, each rounded up to 16 bytes.
struct SmemLayout {
  size_t mi, vec, a, out, ent, off, total;
};
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <typename Real>
__host__ __device__ constexpr SmemLayout pcg_layout(int rows_cap, int ent_cap, int mode, int row_vecs) {
  SmemLayout L{};
  const size_t R = sizeof(Real), rc = (size_t)rows_cap, ec = (size_t)ent_cap;
  L.mi = 0;
  L.vec = align16(L.mi + R * 21 * rc);
  L.a = align16(L.vec + R * 6 * (size_t)row_vecs * rc);
  L.out = align16(L.a + (mode == kSpmvSmemA ? R * 36 * ec : 0));
  L.ent = align16(L.out + (mode != kSpmvRows ? R * 6 * ec : 0));
  L.off = align16(L.ent + (mode == kSpmvSmemA ? sizeof(int) * ec : mode == kSpmvSmemOut ? sizeof(int2) * ec : 0));
  L.total = align16(L.off + sizeof(int) * (rc + 1));
  return L;
}

// Staged modes, at set-up, by the warps [w0, kPcgWarps) of the CTA (the
// others may be busy with other set-up work): the rows' entry offsets (warp
// w0, an exclusive scan of the row lengths), then per entry its block turned
// to multiply the neighbour's vector (kSpmvSmemA) or where to find it
// (kSpmvSmemOut).  The participating warps meet at named barrier 1.
template <int kMode, typename Real>
__device__ __forceinline__ void stage_entries(const SwDev& d, const Real* A, int t, int Gs, int nr, int ent_cap,
                                              Real* sA, int* sj, int2* sent, int* soff, int w0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = kPcgWarps - w0;
  if (warp == w0) {
    int run = 0;
    for (int a0 = 0; a0 < nr; a0 += 32) {
      const int a = a0 + lane;
      const int i = t + Gs * a;
      const int len = a < nr ? __ldg(d.rl_ptr + i + 1) - __ldg(d.rl_ptr + i) : 0;
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      if (a < nr) soff[a + 1] = run + incl;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) soff[0] = 0;
  }
  asm volatile("bar.sync 1, %0;" ::"r"(nw * 32) : "memory");
  for (int a = warp - w0; a < nr; a += nw) {
    const int i = t + Gs * a;
    const int r0 = __ldg(d.rl_ptr + i), len = __ldg(d.rl_ptr + i + 1) - r0, e0 = soff[a];
    for (int k = lane; k < len; k += 32) {
      const int2 ent = checked_ent(__ldg(d.rl_ent + r0 + k), d.nnzb, d.n_n, d.status);
      const int e = e0 + k;
      if constexpr (kMode == kSpmvSmemA) {
        const Real* B = A + (size_t)(ent.x & 0x7fffffff) * 36;
        const bool tr = ent.x < 0;
        sj[e] = ent.y;
#pragma unroll
        for (int q = 0; q < 36; ++q) {
          const int dst = tr ? (q % 6) * 6 + q / 6 : q;
          sA[(size_t)dst * ent_cap + e] = __ldg(B + q);
        }
      } else {
        sent[e] = ent;
      }
    }
  }
}

// One entry's product: the block of entry `ent` (or entry e of sA) times p, six outputs.
template <int kMode, typename Real>
__device__ __forceinline__ void entry_product(const Real* A, const Real* sA, int ent_cap, int e, int2 ent,
                                              const Real* p, Real* out) {
  if constexpr (kMode == kSpmvSmemA) {
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      Real v = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q) v += sA[(size_t)(6 * b + q) * ent_cap + e] * p[q];
      out[b] = v;
    }
  } else {
    const Real* B = A + (size_t)(ent.x & 0x7fffffff) * 36;
    const bool tr = ent.x < 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) out[b] = 0;
#pragma unroll
    for (int b = 0; b < 6; ++b) {
      Real row[6];
      load6_ro(B + 6 * b, row);
      if (!tr) {
        Real v = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v += row[q] * p[q];
        out[b] += v;
      } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) out[q] += p[b] * row[q];
      }
    }
  }
}

// ------------------------------------------------------------------ FP64 solver, standard recurrences

enum { kX = 0, kR, kZ, kP, kQ, kRowVecs };

template <int kMode>
__global__ void __launch_bounds__(kPcgThreads, 1)
k_pcg_f64(Batch bt, int K, int gn_it, int spin_arg, int rows_cap, int ent_cap) {
  using Acc = double;
  using O = AccOps<Acc>;
  constexpr bool kStaged = kMode != kSpmvRows;
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int t = blockIdx.x - __ldg(bt.tile_base + s);
  const int Gs = __ldg(bt.tile_base + s + 1) - __ldg(bt.tile_base + s);
  const int spin_limit = g_wait_fault[1] > 0 ? g_wait_fault[1] : spin_arg;
  const bool withhold_first = g_wait_fault[0] == kFaultPcgPartial && s == 0 && t == 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = d.n_n;
  const int nr = n > t ? (n - t + Gs - 1) / Gs : 0;   // own rows (<= rows_cap, checked on the host)
  const unsigned long long base = __ldcg(d.pcg_epoch) * 1024ull;
  const double* __restrict__ A = d.A64;
  const size_t n6 = 6 * (size_t)n;
  double* const gz = d.v64;                                   // z of every node
  double* const pbuf[2] = {d.v64 + n6, d.v64 + 2 * n6};       // p by iteration parity
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SmemLayout L = pcg_layout<double>(rows_cap, ent_cap, kMode, kRowVecs);
  double* sMi = reinterpret_cast<double*>(smem_raw + L.mi);
  double* svec = reinterpret_cast<double*>(smem_raw + L.vec);
  double* sA = reinterpret_cast<double*>(smem_raw + L.a);
  double* sOut = reinterpret_cast<double*>(smem_raw + L.out);
  int* sj = reinterpret_cast<int*>(smem_raw + L.ent);
  int2* sent = reinterpret_cast<int2*>(smem_raw + L.ent);
  int* soff = reinterpret_cast<int*>(smem_raw + L.off);
  auto V = [&](int v, int a) { return svec + ((size_t)v * rows_cap + a) * 6; };
  __shared__ Scalars<double, Acc> sc;

  // ---- set-up, a thread per own row: M⁻¹, r = −g, z = M⁻¹ r (published), x = p = 0
  Acc pa = O::zero();
  bool broken = false;
  for (int a = tid; a < nr; a += kPcgThreads) {
    const int j = t + Gs * a;
    double* mi = sMi + 21 * a;
    const double* src = d.minv64 + 21 * (size_t)j;
#pragma unroll
    for (int k = 0; k < 21; ++k) mi[k] = __ldg(src + k);
    if (mi[0] != mi[0]) {   // not positive definite (flagged by the preconditioner launch)
      broken = true;
#pragma unroll
      for (int k = 0; k < 21; ++k) mi[k] = 0;
    }
    double r[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) r[c] = -d.g64[6 * j + c];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      double z = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) z += mi[sym(c, k)] * r[k];
      V(kR, a)[c] = r[c];
      V(kZ, a)[c] = z;
      V(kX, a)[c] = 0;
      V(kP, a)[c] = 0;
      gz[6 * (size_t)j + c] = z;
      pa = O::add(pa, O::prod(r[c], z));
    }
  }
  if (broken) pa = acc_nan<Acc>();   // reaches every CTA through the first reduction
  if constexpr (kStaged) stage_entries<kMode>(d, A, t, Gs, nr, ent_cap, sA, sj, sent, soff, 0);
  if (!stream_reduce_fenced(pa, 32, d.part, t, Gs, base + 1, spin_limit, !withhold_first, [&](Acc rz) {
        sc.rz = rz;
        sc.bad = acc_is_nan(rz);
        sc.work = !sc.bad && O::nonzero(rz);
        sc.alpha = 0;
        sc.beta = 0;
      })) {
    atomicOr(d.status, kStatusTimeout);
    return;
  }

  for (int k = 0; k < K; ++k) {
    const bool work = sc.work;
    const double beta = sc.beta;
    const double* __restrict__ pold = pbuf[(k + 1) & 1];
    double* __restrict__ pnew = pbuf[k & 1];
    // ---- q = A p with the neighbour's p = z + β p_old, and the shares of pᵀq (lanes 0-5)
    pa = O::zero();
    if (work) {
      if constexpr (kStaged) {
        const int ne = soff[nr];
        for (int e = tid; e < ne; e += kPcgThreads) {
          const int2 ent = kMode == kSpmvSmemA ? make_int2(0, sj[e]) : sent[e];
          double p[6], out[6];
          get_p64(gz, pold, k > 0, beta, ent.y, p);
          entry_product<kMode>(A, sA, ent_cap, e, ent, p, out);
#pragma unroll
          for (int b = 0; b < 6; ++b) sOut[(size_t)b * ent_cap + e] = out[b];
        }
        __syncthreads();
      }
      for (int a = warp; a < nr; a += kPcgWarps) {
        const int i = t + Gs * a;
        double acc[6] = {0, 0, 0, 0, 0, 0};
        if constexpr (kStaged) {
          const int e1 = soff[a + 1];
          for (int e = soff[a] + lane; e < e1; e += 32) {
#pragma unroll
            for (int b = 0; b < 6; ++b) acc[b] += sOut[(size_t)b * ent_cap + e];
          }
        } else {
          const int e1 = __ldg(d.rl_ptr + i + 1);
          for (int e = __ldg(d.rl_ptr + i) + lane; e < e1; e += 32) {
            const int2 ent = checked_ent(__ldg(d.rl_ent + e), d.nnzb, d.n_n, d.status);
            double p[6], out[6];
            get_p64(gz, pold, k > 0, beta, ent.y, p);
            entry_product<kSpmvRows>(A, sA, ent_cap, e, ent, p, out);
#pragma unroll
            for (int b = 0; b < 6; ++b) acc[b] += out[b];
          }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] = warp_sum_r(acc[c]);
        if (lane < 6) {
          double qc = acc[0];
#pragma unroll
          for (int c = 1; c < 6; ++c)
            if (lane == c) qc = acc[c];
          const double pc = k == 0 ? V(kZ, a)[lane] : V(kZ, a)[lane] + beta * V(kP, a)[lane];
          V(kP, a)[lane] = pc;
          V(kQ, a)[lane] = qc;
          pnew[6 * (size_t)i + lane] = pc;
          pa = O::add(pa, O::prod(pc, qc));
        }
      }
    }
    if (!stream_reduce_fenced(pa, 8, d.part, t, Gs, base + 2 + 2 * k, spin_limit, true, [&](Acc pq) {
          if (!sc.work) return;
          if (!(pq > 0.0)) {   // pᵀAp <= 0: nothing moves from here on
            sc.bad = 1;
            sc.work = 0;
            atomicOr(d.status, kStatusBreakdown);
            return;
          }
          sc.alpha = sc.rz / pq;
        })) {
      atomicOr(d.status, kStatusTimeout);
      return;
    }
    // ---- x += α p, r −= α q, z = M⁻¹ r (published), and the shares of rᵀz (lanes 0-5)
    pa = O::zero();
    if (sc.work) {
      const double alpha = sc.alpha;
      for (int a = warp; a < nr; a += kPcgWarps) {
        if (lane < 6) {
          V(kX, a)[lane] += alpha * V(kP, a)[lane];
          V(kR, a)[lane] -= alpha * V(kQ, a)[lane];
        }
        __syncwarp();
        if (lane < 6) {
          const double* mi = sMi + 21 * a;
          const double* r = V(kR, a);
          double z = 0;
#pragma unroll
          for (int c = 0; c < 6; ++c) z += mi[sym(lane, c)] * r[c];
          V(kZ, a)[lane] = z;
          gz[6 * (size_t)(t + Gs * a) + lane] = z;
          pa = O::add(pa, O::prod(r[lane], z));
        }
        __syncwarp();
      }
    }
    if (!stream_reduce_fenced(pa, 8, d.part, t, Gs, base + 3 + 2 * k, spin_limit, true, [&](Acc rz) {
          if (!sc.work) return;
          sc.beta = rz / sc.rz;
          sc.rz = rz;
          sc.work = O::nonzero(rz);
        })) {
      atomicOr(d.status, kStatusTimeout);
      return;
    }
  }
  if (t == 0 && tid == 0) d.pcg_rz[gn_it] = sc.rz;

  // ---- T_j ← Δ_j T_j in FP64 (nothing moves after a breakdown); the FP32 copy follows
  if (sc.bad) return;
  for (int a = tid; a < nr; a += kPcgThreads) {
    const int j = t + Gs * a;
    double xi[6], q[8];
#pragma unroll
    for (int c = 0; c < 6; ++c) xi[c] = V(kX, a)[c];
#pragma unroll
    for (int c = 0; c < 8; ++c) q[c] = d.dq64[8 * j + c];
    apply_increment64(q, xi);
#pragma unroll
    for (int c = 0; c < 8; ++c) d.dq64[8 * j + c] = q[c];
    d.dq[2 * j] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
    d.dq[2 * j + 1] = make_float4((float)q[4], (float)q[5], (float)q[6], (float)q[7]);
  }
}

// ------------------------------------------------------------------ FP32 solver, one reduction per iteration

// The FP32 modes run PCG in the Chronopoulos-Gear arrangement (Chronopoulos
// & Gear, J. Comput. Appl. Math. 27, 1989): u = M⁻¹ r and w = A u are formed
// explicitly every iteration, both inner products γ = (r, u) and δ = (w, u)
// come from ONE reduction, and p, s = A p follow by recurrence:
//   β = γ / γ_prev,  α = γ / (δ − β γ / α_prev)   (first: β = 0, α = γ / δ)
//   p = u + β p,  s = w + β s,  x += α p,  r −= α s.
// The iterates are those of standard PCG in exact arithmetic; with w
// computed, not recurred, FP32 accuracy stays close to the standard
// recurrences (unlike the pipelined variants).  The denominator is pᵀAp; a
// value <= 0 is a breakdown.  A row's owner publishes its u (tagged words)
// as soon as it is formed; the SpMV waits for its neighbours' tags, so the
// exchange of u needs no barrier and an iteration has one synchronisation.
enum { kGx = 0, kGr, kGu, kGw, kGp, kGs, kGearVecs };

template <typename Acc, int kMode>
__global__ void __launch_bounds__(kPcgThreads, 1)
k_pcg_gear(Batch bt, int K, int gn_it, int spin_arg, int rows_cap, int ent_cap) {
  using O = AccOps<Acc>;
  using Real = float;
  constexpr bool kStaged = kMode != kSpmvRows;
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  const int t = blockIdx.x - __ldg(bt.tile_base + s);
  const int Gs = __ldg(bt.tile_base + s + 1) - __ldg(bt.tile_base + s);
  // failure injection (tests only): CTA 1 of the first stream withholds its
  // first partial or its rows' first u, and the waits get a small poll limit
  const int fault = (s == 0 && t == 1) ? g_wait_fault[0] : kFaultNone;
  const int spin_limit = g_wait_fault[1] > 0 ? g_wait_fault[1] : spin_arg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = d.n_n;
  const int nr = n > t ? (n - t + Gs - 1) / Gs : 0;   // own rows (<= rows_cap, checked on the host)
  const unsigned long long base = __ldcg(d.pcg_epoch) * 1024ull;
  const float* __restrict__ A = sys_A(d, gn_it);
  const float* __restrict__ gsys = sys_g(d, gn_it);
  unsigned long long* const ub[2] = {d.xp, d.xp + 6 * (size_t)n};   // u by iteration parity
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SmemLayout L = pcg_layout<Real>(rows_cap, ent_cap, kMode, kGearVecs);
  Real* sMi = reinterpret_cast<Real*>(smem_raw + L.mi);
  Real* svec = reinterpret_cast<Real*>(smem_raw + L.vec);
  Real* sA = reinterpret_cast<Real*>(smem_raw + L.a);
  Real* sOut = reinterpret_cast<Real*>(smem_raw + L.out);
  int* sj = reinterpret_cast<int*>(smem_raw + L.ent);
  int2* sent = reinterpret_cast<int2*>(smem_raw + L.ent);
  int* soff = reinterpret_cast<int*>(smem_raw + L.off);
  auto V = [&](int v, int a) { return svec + ((size_t)v * rows_cap + a) * 6; };
  __shared__ Scalars<Real, Acc> sc;
  __shared__ Acc s_gprev;
  __shared__ Real s_aprev;
  __shared__ int s_late;
  const int data_spins = spin_limit >> 6;

  // ---- set-up, a thread per own row: M⁻¹, r = −g, u = M⁻¹ r (published), x = p = s = 0
  if (tid == 0) s_late = 0;
  bool broken = false;
  // a thread per row (M⁻¹ from the preconditioner launch); the other warps
  // stage the matrix entries meanwhile
  const int inv_warps = min(kPcgWarps - 1, (rows_cap + 31) >> 5);
  if (warp < inv_warps) {
    for (int a = tid; a < nr; a += inv_warps * 32) {
      const int j = t + Gs * a;
      Real* mi = sMi + 21 * a;
      const Real* src = d.minv + 21 * (size_t)j;
#pragma unroll
      for (int k = 0; k < 21; ++k) mi[k] = __ldg(src + k);
      if (mi[0] != mi[0]) {   // not positive definite (flagged by the preconditioner launch)
        broken = true;
#pragma unroll
        for (int k = 0; k < 21; ++k) mi[k] = 0;
      }
      Real r[6];
#pragma unroll
      for (int c = 0; c < 6; ++c) r[c] = -gsys[6 * j + c];
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        Real u = 0;
#pragma unroll
        for (int k = 0; k < 6; ++k) u += mi[sym(c, k)] * r[k];
        V(kGr, a)[c] = r[c];
        V(kGu, a)[c] = u;
        V(kGx, a)[c] = 0;
        V(kGp, a)[c] = 0;
        V(kGs, a)[c] = 0;
        if (fault != kFaultPcgVector) put_tagged(ub[0], 6 * (size_t)j + c, u, (unsigned)(base + 1));
      }
    }
  } else if constexpr (kStaged) {
    stage_entries<kMode>(d, A, t, Gs, nr, ent_cap, sA, sj, sent, soff, inv_warps);
  }
  if (tid == 0) {
    sc.alpha = 0; sc.beta = 0; sc.rz = O::zero(); sc.bad = 0; sc.work = 1;
    s_gprev = O::zero(); s_aprev = 1.f;
  }
  __syncthreads();
  // a broken diagonal block reaches every CTA through the first reduction
  Acc carry = broken ? acc_nan<Acc>() : O::zero();
  __syncthreads();

  for (int k = 0; k <= K; ++k) {
    // ---- w = A u (u of iteration k, from the rows' owners) and the shares of γ = (r, u), δ = (w, u)
    const bool last = k == K;   // the final pass only measures γ for the statistics
    const unsigned tu = (unsigned)(base + 1 + k);
    const unsigned long long* ucur = ub[k & 1];
    Acc pg = carry, pd = O::zero();
    carry = O::zero();
    bool late = false;
    const bool spmv = sc.work && !last;
    if (spmv && kStaged) {
      const int ne = soff[nr];
      for (int e = tid; e < ne; e += kPcgThreads) {
        Real p[6], out[6];
        if constexpr (kMode == kSpmvSmemA) {
          late |= !get6_tagged(ucur, sj[e], tu, p, data_spins);
          entry_product<kMode>(A, sA, ent_cap, e, make_int2(0, 0), p, out);
        } else {
          // the block's loads go out before the wait for u: one L2 round trip per entry
          const int2 ent = sent[e];
          const float4* B4 = reinterpret_cast<const float4*>(A + (size_t)(ent.x & 0x7fffffff) * 36);
          float B[36];
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            const float4 v = __ldg(B4 + q);
            B[4 * q] = v.x; B[4 * q + 1] = v.y; B[4 * q + 2] = v.z; B[4 * q + 3] = v.w;
          }
          late |= !get6_tagged(ucur, ent.y, tu, p, data_spins);
          if (ent.x >= 0) {
#pragma unroll
            for (int b = 0; b < 6; ++b) {
              Real v = 0;
#pragma unroll
              for (int q = 0; q < 6; ++q) v += B[6 * b + q] * p[q];
              out[b] = v;
            }
          } else {
#pragma unroll
            for (int q = 0; q < 6; ++q) {
              Real v = 0;
#pragma unroll
              for (int b = 0; b < 6; ++b) v += B[6 * b + q] * p[b];
              out[q] = v;
            }
          }
        }
#pragma unroll
        for (int b = 0; b < 6; ++b) sOut[(size_t)b * ent_cap + e] = out[b];
      }
      __syncthreads();
    }
    for (int a = warp; a < nr; a += kPcgWarps) {
      const int i = t + Gs * a;
      Real acc[6] = {0, 0, 0, 0, 0, 0};
      if (spmv) {
        if constexpr (kStaged) {
          const int e1 = soff[a + 1];
          for (int e = soff[a] + lane; e < e1; e += 32) {
#pragma unroll
            for (int b = 0; b < 6; ++b) acc[b] += sOut[(size_t)b * ent_cap + e];
          }
        } else {
          const int e1 = __ldg(d.rl_ptr + i + 1);
          for (int e = __ldg(d.rl_ptr + i) + lane; e < e1; e += 32) {
            const int2 ent = checked_ent(__ldg(d.rl_ent + e), d.nnzb, d.n_n, d.status);
            Real p[6], out[6];
            late |= !get6_tagged(ucur, ent.y, tu, p, data_spins);
            entry_product<kSpmvRows>(A, sA, ent_cap, e, ent, p, out);
#pragma unroll
            for (int b = 0; b < 6; ++b) acc[b] += out[b];
          }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] = warp_sum_r(acc[c]);
      }
      if (lane < 6) {
        Real wc = acc[0];
#pragma unroll
        for (int c = 1; c < 6; ++c)
          if (lane == c) wc = acc[c];
        const Real uc = V(kGu, a)[lane];
        pg = O::add(pg, O::prod(V(kGr, a)[lane], uc));
        if (spmv) {
          V(kGw, a)[lane] = wc;
          pd = O::add(pd, O::prod(wc, uc));
        }
      }
    }
    if (late) s_late = 1;   // every CTA stops iterating; the host gets a timeout
    if (last) {
      // the final γ is only a statistic: each CTA adds its share with one
      // FP64 atomic and nobody waits (the order of the additions varies)
      block_add_value(pg, 8, d.pcg_rz + gn_it);
      break;
    }
    // ---- one reduction: γ and δ together
    if (!stream_reduce_pair(pg, pd, k == 0 ? 32 : 8, d.part, t, Gs, base + 1 + k, spin_limit,
                            !(k == 0 && fault == kFaultPcgPartial), &s_late, [&](Acc g, Acc dl, bool any_late) {
          if (!sc.work) return;
          Real alpha, beta;
          const int step = any_late ? kGearLate : gear_step(k, g, dl, s_gprev, s_aprev, &alpha, &beta);
          if (step == kGearBreakdown || step == kGearLate) {   // nothing moves from here on
            sc.bad = 1; sc.work = 0;
            atomicOr(d.status, step == kGearLate ? kStatusTimeout : kStatusBreakdown);
            return;
          }
          sc.rz = g;
          if (step == kGearConverged) { sc.work = 0; return; }
          sc.alpha = alpha;
          sc.beta = beta;
          s_aprev = alpha;
          s_gprev = g;
        })) {
      atomicOr(d.status, kStatusTimeout);
      return;
    }
    // ---- p = u + β p, s = w + β s, x += α p, r −= α s, then u = M⁻¹ r (published)
    if (sc.work) {
      const Real alpha = sc.alpha, beta = sc.beta;
      const unsigned tn = (unsigned)(base + 2 + k);
      unsigned long long* unext = ub[(k + 1) & 1];
      // five rows per warp at a time, six lanes each (lanes 30 and 31 idle)
      const int grp = lane / 6, c = lane - 6 * grp;
      for (int a0 = warp; a0 < nr; a0 += 5 * kPcgWarps) {
        const int a = a0 + grp * kPcgWarps;
        const bool on = grp < 5 && a < nr;
        if (on) {
          const Real pc = V(kGu, a)[c] + beta * V(kGp, a)[c];
          const Real sc_ = V(kGw, a)[c] + beta * V(kGs, a)[c];
          V(kGp, a)[c] = pc;
          V(kGs, a)[c] = sc_;
          V(kGx, a)[c] += alpha * pc;
          V(kGr, a)[c] -= alpha * sc_;
        }
        __syncwarp();
        if (on) {
          const Real* mi = sMi + 21 * a;
          const Real* r = V(kGr, a);
          Real u = 0;
#pragma unroll
          for (int k2 = 0; k2 < 6; ++k2) u += mi[sym(c, k2)] * r[k2];
          V(kGu, a)[c] = u;
          put_tagged(unext, 6 * (size_t)(t + Gs * a) + c, u, tn);
        }
        __syncwarp();
      }
    }
  }
  if (tid == 0 && s_late) atomicOr(d.status, kStatusTimeout);

  // ---- T_j ← Δ_j T_j (nothing moves after a breakdown)
  if (sc.bad) return;
  for (int a = tid; a < nr; a += kPcgThreads) {
    const int j = t + Gs * a;
    float xi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) xi[c] = V(kGx, a)[c];
    float4 q0 = d.dq[2 * j], qe = d.dq[2 * j + 1];
    apply_increment(q0, qe, xi);
    d.dq[2 * j] = q0;
    d.dq[2 * j + 1] = qe;
  }
}

// The inverse of an FP32 block in double-float pairs (sw_df.cuh, about 48
// bits), all in the FP32 pipe: the default precision's preconditioner (an
// FP64 instruction issues once per 64 cycles per warp on this part).  It
// runs the sweep operator -- Gauss-Jordan elimination in place on the
// symmetric block, pivots in order without exchanges -- on eight lanes per
// block: lane c < 6 holds column c, every step sends the pivot column to the
// segment by shuffles, and each lane updates its own column (the pivot lane:
// −v/d off the pivot, 1/d on it; another lane j: t = a_kj/d, then
// a_ij −= a_ik t off the pivot row, a_kj = t).  After the six steps the block
// holds its inverse.  The pivots are the LDLᵀ pivots (Schur complements), so
// the block is positive definite exactly when every one is positive.  One
// thread per block ran this as a serial LDLᵀ chain of ~3,800 instructions;
// here a lane's chain is six steps of five independent updates.  The block
// (its lower triangle: element (r, c) is read at (max, min)) is first scaled
// by the power of two that brings its largest diagonal entry to [0.5, 1) --
// exact -- so that no pair's low part falls below FP32's normal range; M⁻¹
// is scaled back the same way.  Every lane of the 8-lane segment calls it
// (`on` false where the segment has no block); every lane gets whether the
// block is positive definite.
__device__ bool block_inverse_df8(const float* a, float* out, int c, bool on) {
  constexpr unsigned kAll = 0xffffffffu;
  const int cc = c < 6 ? c : 0;
  float col0[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) col0[r] = on ? a[(r > cc ? r : cc) * 6 + (r > cc ? cc : r)] : 0.f;
  float amax = (on && c < 6) ? fabsf(a[7 * cc]) : 0.f;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(kAll, amax, o, 8));
  bool good = on && amax > 0.f && amax < 3.0e38f;
  int ex = 0;
  if (good) frexpf(amax, &ex);
  DF col[6];
#pragma unroll
  for (int r = 0; r < 6; ++r) col[r] = DF{good ? ldexpf(col0[r], -ex) : 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    DF v[6];   // the pivot column, from lane k
#pragma unroll
    for (int i = 0; i < 6; ++i)
      v[i] = DF{__shfl_sync(kAll, col[i].hi, k, 8), __shfl_sync(kAll, col[i].lo, k, 8)};
    good = good && v[k].hi > 0.f;
    const DF inv = df_recip(good ? v[k] : DF{1.f, 0.f});
    const bool piv = c == k;
    const DF t = piv ? inv : df_mul(col[k], inv);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i != k) col[i] = df_fnma(v[i], t, piv ? DF{0.f, 0.f} : col[i]);
    col[k] = t;
  }
  if (on && good && c < 6) {
#pragma unroll
    for (int r = 0; r < 6; ++r)
      if (r >= c) out[tri(r, c)] = ldexpf(__fadd_rn(col[r].hi, col[r].lo), -ex);
  }
  return good;
}

// The block-Jacobi preconditioner for every active stream, launched between
// the assembly and the PCG: its own launch spreads the inversions over many
// SMs, kPrecondTile nodes per CTA.  M⁻¹_j, packed lower, to minv (FP32
// modes) or minv64 (FP64 mode); with kPairs the double-float sweep on eight
// lanes per node (the default precision), else the FP64 LDLᵀ, one thread
// per node (its own launch gives it the registers that the 1024-thread PCG
// cannot).  A
// diagonal block that is not positive definite sets kStatusBreakdown and
// leaves a NaN in its first entry, which the PCG turns into a breakdown of
// the whole solve.
template <typename Real, bool kPairs>
__global__ void __launch_bounds__(8 * kPrecondTile) k_precond(Batch bt, int gn_it) {
  // after the assembly's completion, the cluster PCG launched next may
  // start: it stages its tables and matrix meanwhile and waits for this
  // launch before reading M⁻¹
  pdl_begin();
  const int s = find_stream(bt, blockIdx.x);
  if (!stream_active(bt, s)) return;
  const SwDev d = bt.devs[s];
  if constexpr (kPairs) {   // eight lanes per node
    const int j = (blockIdx.x - __ldg(bt.tile_base + s)) * kPrecondTile + (threadIdx.x >> 3);
    const bool on = j < d.n_n;
    const float* blk = sys_A(d, gn_it) + (on ? (size_t)checked(__ldg(d.row_ptr + j), d.nnzb, d.status) * 36 : 0);
    float* out = d.minv + 21 * (size_t)(on ? j : 0);
    const bool ok = block_inverse_df8(blk, out, threadIdx.x & 7, on);
    if (on && !ok && (threadIdx.x & 7) == 0) {
      atomicOr(d.status, kStatusBreakdown);
      out[0] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const int j = (blockIdx.x - __ldg(bt.tile_base + s)) * kPrecondTile + threadIdx.x;
  if (j >= d.n_n) return;
  const Real* A;
  Real* out;
  if constexpr (std::is_same<Real, double>::value) {
    A = d.A64; out = d.minv64 + 21 * (size_t)j;
  } else {
    A = sys_A(d, gn_it); out = d.minv + 21 * (size_t)j;
  }
  const bool ok = block_inverse(A + (size_t)__ldg(d.row_ptr + j) * 36, out);
  if (!ok) {
    atomicOr(d.status, kStatusBreakdown);
    out[0] = (Real)__longlong_as_double(0x7ff8000000000000ll);
  }
}

// the preconditioner's block inverse alone (stage checks)
template <typename Real, bool kPairs>
__global__ void k_debug_block_inverse(const Real* blocks, int n, Real* out, int* ok) {
  if constexpr (kPairs) {   // eight lanes per block, as in k_precond
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    const bool on = i < n;
    const bool good = block_inverse_df8(blocks + 36 * (size_t)(on ? i : 0), out + 21 * (size_t)(on ? i : 0),
                                        threadIdx.x & 7, on);
    if (on && (threadIdx.x & 7) == 0) ok[i] = good ? 1 : 0;
    return;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  ok[i] = block_inverse(blocks + (size_t)i * 36, out + (size_t)i * 21) ? 1 : 0;
}

template <typename Acc>
const void* pcg_gear_fn(int mode) {
  switch (mode) {
    case kSpmvSmemA: return reinterpret_cast<const void*>(k_pcg_gear<Acc, kSpmvSmemA>);
    case kSpmvSmemOut: return reinterpret_cast<const void*>(k_pcg_gear<Acc, kSpmvSmemOut>);
    default: return reinterpret_cast<const void*>(k_pcg_gear<Acc, kSpmvRows>);
  }
}

const void* pcg_kernel(int precision, int mode) {
  switch (precision) {
    case SW_PRECISION_FP64:
      switch (mode) {
        case kSpmvSmemA: return reinterpret_cast<const void*>(k_pcg_f64<kSpmvSmemA>);
        case kSpmvSmemOut: return reinterpret_cast<const void*>(k_pcg_f64<kSpmvSmemOut>);
        default: return reinterpret_cast<const void*>(k_pcg_f64<kSpmvRows>);
      }
    case SW_PRECISION_MIXED_F64DOTS: return pcg_gear_fn<double>(mode);
    default: return pcg_gear_fn<DF>(mode);
  }
}

}  // namespace

void set_pcg_wait_fault(int kind, int spin_limit) {
  const int v[2] = {kind, spin_limit};
  cudaMemcpyToSymbol(g_wait_fault, v, sizeof(v));
}

int pcg_blocks_per_sm(int precision) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pcg_kernel(precision, kSpmvRows), kPcgThreads, 0) !=
      cudaSuccess)
    return 0;
  return n;
}

int pcg_threads() { return kPcgThreads; }

size_t pcg_smem_bytes(int rows_cap, int ent_cap, int precision, int mode) {
  return precision == SW_PRECISION_FP64 ? pcg_layout<double>(rows_cap, ent_cap, mode, kRowVecs).total
                                        : pcg_layout<float>(rows_cap, ent_cap, mode, kGearVecs).total;
}

// One cooperative launch: every CTA is resident, so the waits of
// stream_reduce always end (and are bounded regardless).
cudaError_t launch_pcg(const BatchHost& b, int gn_it, int pcg_iters, cudaStream_t st) {
  const int nb = b.total_tiles[kTilePcg];
  if (nb == 0) return cudaSuccess;
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kTilePcg];
  int spin = b.spin_limit;
  int rows_cap = b.pcg_rows_cap;
  int ent_cap = b.pcg_ent_cap;
  const int prec = b.precision;
  const int mode = b.pcg_mode;
  const void* fn = pcg_kernel(prec, mode);
  const size_t smem = pcg_smem_bytes(rows_cap, ent_cap, prec, mode);
  static size_t configured[3][3] = {};
  const int slot = prec < 0 || prec > 2 ? 0 : prec;
  if (smem > 48 * 1024 && smem > configured[slot][mode]) {
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[slot][mode] = smem;
  }
  void* args[] = {&bt, &pcg_iters, &gn_it, &spin, &rows_cap, &ent_cap};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(kPcgThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

void launch_precond(const BatchHost& b, int gn_it, cudaStream_t st) {
  const int nb = b.total_tiles[kTilePrecond];
  if (nb == 0) return;
  Batch bt = b.bt;
  bt.tile_base = b.tile_base_dev[kTilePrecond];
  // the default precision's double-float inverse may begin during the data
  // assembly's tail (programmatic dependent launch); the FP64 one does not:
  // overlapped with the assembly it cost the full-size frame 0.1 ms more
  if (b.precision == SW_PRECISION_FP64) k_precond<double, false><<<nb, kPrecondTile, 0, st>>>(bt, gn_it);
  else if (b.precision == SW_PRECISION_MIXED_F64DOTS) k_precond<float, false><<<nb, kPrecondTile, 0, st>>>(bt, gn_it);
  else launch_overlapped(k_precond<float, true>, nb, 8 * kPrecondTile, st, bt, gn_it);
}

cudaError_t launch_debug_block_inverse(const void* blocks, int n, int mode, void* out, int* ok, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + 127) / 128;
  if (mode == 1)
    k_debug_block_inverse<double, false>
        <<<nb, 128, 0, st>>>(static_cast<const double*>(blocks), n, static_cast<double*>(out), ok);
  else if (mode == 2)
    k_debug_block_inverse<float, false>
        <<<nb, 128, 0, st>>>(static_cast<const float*>(blocks), n, static_cast<float*>(out), ok);
  else
    k_debug_block_inverse<float, true><<<(n + 15) / 16, 128, 0, st>>>(static_cast<const float*>(blocks), n,
                                                                       static_cast<float*>(out), ok);
  return cudaGetLastError();
}

}  // namespace sw
