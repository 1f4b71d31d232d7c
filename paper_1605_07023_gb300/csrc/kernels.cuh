// Device kernels of the GB300 convolutional gridder.
//
// Gridding (Merry 2016, Sec. 2.2): each visibility is a delta, convolved with
// an oversampled separable GCF and accumulated on the grid.
//
// Work distribution (Sec. 2.2, Fig. 1; Sec. 3, Fig. 2):
//  - The grid is covered by bins of N_bu x N_bv cells. The bin is at least
//    S + B - 1 wide per axis and a multiple of the block size B (Sec. 3).
//  - A "team" of nu*nv threads covers one bin. Thread (au, av) owns every
//    block of Bu x Bv cells whose block coordinates are congruent to
//    (au, av) modulo (nu, nv).
//  - For each visibility the bin-sized bounding box is aligned to blocks and
//    contains the footprint. Each thread owns exactly one block inside it.
//  - A thread keeps register accumulators for its current block and flushes
//    them with atomic adds when the box moves so that it owns a different
//    block.
//  - A team processes one chunk of consecutive visibilities (ordered by
//    baseline, Sec. 4). Records are staged through shared memory in batches,
//    each thread loading one record (Sec. 4).
//  - The separable GCF (Sec. 4) is held in shared memory as zero-padded 1-D
//    tables, one per (table row, block phase), so that a thread reads its Bu
//    taps as one aligned vector and forms the Bu*Bv products in registers
//    (Sec. 4, last paragraph).
//
// The complex FMAs use the packed FP32x2 FMA of sm_100+ (__ffma2_rn): one
// instruction updates the real and imaginary parts of one accumulator, which
// leaves issue slots for the address arithmetic.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gbg {

constexpr unsigned kInvalid = 0xFFFFFFFFu;
constexpr int kRB = 32;   // records per team per staged batch (gridding)
constexpr int kRBB = 16;  // records per team per staged batch (batched gridding: smaller buffers, more CTAs)
constexpr int kRBD = 8;   // records per team per batch (degridding; bounded by the reduction buffer)
constexpr int kSlots = 8; // flush slots per warp (lanes parked per cooperative-flush round)

enum { FMT_F32 = 0, FMT_BF16 = 1, FMT_F16 = 2 };

struct Geometry {
  int G, S, O, log2O, h, P;
  int nbu, nbv;   // bin width in cells per axis
  int nu, nv;     // blocks per bin per axis
  int ts;         // team size nu*nv
  int tpc;        // teams per CTA
  int nuB, nvB;   // nu*Bu, nv*Bv: a bin's width in table entries
  unsigned mu, mv;  // floor(2^31/nu) + 1, floor(2^31/nv) + 1: exact division of block indices < 2^15
  unsigned mbu, mbv;  // floor(2^31/nbu) + 1, floor(2^31/nbv) + 1: exact cell index mod bin width
};

// Bin and team shape for blocks of Bu x Bv cells (Sec. 3): the bin is the
// smallest multiple of the block that holds S + B - 1 cells per axis.
__host__ __device__ inline void finish_geometry(Geometry& g, int BU, int BV) {
  g.nbu = ((g.S + BU - 1 + BU - 1) / BU) * BU;
  g.nbv = ((g.S + BV - 1 + BV - 1) / BV) * BV;
  g.nu = g.nbu / BU;
  g.nv = g.nbv / BV;
  g.ts = g.nu * g.nv;
  g.nuB = g.nu * BU;
  g.nvB = g.nv * BV;
  g.mu = (unsigned)((1ull << 31) / (unsigned)g.nu + 1);
  g.mv = (unsigned)((1ull << 31) / (unsigned)g.nv + 1);
  g.mbu = (unsigned)((1ull << 31) / (unsigned)g.nbu + 1);
  g.mbv = (unsigned)((1ull << 31) / (unsigned)g.nbv + 1);
}

// q mod n for 0 <= q < 2^31/n (so for q < 2^15 with any n <= 2^16), with
// m = floor(2^31/n) + 1: floor(q*m / 2^31) = floor(q/n + q*e/2^31) with
// 0 < e <= 1, and q*e/2^31 < 1/n, so the quotient is exact.
__device__ __forceinline__ int mod_small(int q, int n, unsigned m) {
  return q - n * (int)__umulhi((unsigned)q << 1, m);
}

struct Args {
  Geometry g;
  long long n_vis;
  const double2* uv;
  const void* vis;        // gridding input, [n][P] complex in vis_fmt
  int vis_fmt;
  const float* weights;   // may be null
  const void* table;      // [O][S] in tab_fmt
  int tab_fmt;
  float2* grid;           // [P][G][G]
  float2* vis_out;        // degridding output, [n][P] complex64
  int chunk_len;          // visibilities per chunk
  long long n_chunks;
  const int* chunk_order; // patch schedule: chunk ids ordered by patch; null = identity
  const int4* work;       // patch schedule: {patch_u0, patch_v0, first, last} into chunk_order
  const int* n_work;      // device count of work items
  int* work_next;         // device work counter (persistent CTAs)
  int win;                // patch window side in cells (patch + halo); 0 = chunked schedule
  int warp_sync;          // 1: every team lies inside one warp (team size divides 32), teams sync per warp
  int seg;                // lazy-box gridder: lanes per team slot (a power of two >= team size, <= 32)
  unsigned* status;       // lazy-box gridder: bit 0 set when a bulk copy did not complete in time
  unsigned long long* skipped;
};

// ---------------------------------------------------------------------------
// Index rule, exact and FP64-free: f = floor(x*O + 1/2) on the exact value of
// the double x (O = 2^log2O). x*O = +-m * 2^-sh with an integer mantissa m, so
// f = (+-m + 2^(sh-1)) >> sh with an arithmetic (flooring) shift. Valid
// positions have |x*O| < 2^26; anything larger, or inf/nan, is invalid.
// Returns false for an invalid coordinate. On success, C is the absolute
// centre cell and row the table row.
__device__ __forceinline__ bool fine_cell(double x, int log2O, int halfG, int& C, int& row) {
  const long long bits = __double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  long long f = 0;
  if (e == 0x7FF) return false;
  if (e != 0) {
    const int sh = 1075 - log2O - e;
    if (sh < 27) return false;
    if (sh <= 54) {
      const long long m = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
      const long long v = bits < 0 ? -m : m;
      f = (v + (1LL << (sh - 1))) >> sh;
    }
  }
  const int fi = (int)f;
  const int half = (1 << log2O) >> 1;
  const int c = (fi + half) >> log2O;
  row = fi - (c << log2O) + half;
  C = c + halfG;
  return true;
}

// L2 cache policies. The degridder's inputs (uv) and outputs stream through
// L2 (evict first, no L1 allocation). Grid reads use plain non-coherent
// loads: an evict-last hint on them was measured 8-11% slower.
__device__ __forceinline__ unsigned long long policy_stream() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(policy_stream()));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(policy_stream()));
  return v;
}
// A hint that brings bytes [p, p + n) into L2 ahead of their first use: bulk
// prefetches (8 KB at most each) of the whole 16-byte units inside the range.
// No registers are held and nothing waits for them.
__device__ __forceinline__ void prefetch_l2(const void* p, size_t n) {
  const uintptr_t s = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + n) & ~(uintptr_t)15;
  for (uintptr_t q = s; q < e; q += 8192) {
    const unsigned len = (unsigned)(e - q < 8192 ? e - q : 8192);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(len) : "memory");
  }
}

// Bulk asynchronous copies (cp.async.bulk, the TMA unit's untiled form) and
// mbarriers. Shared-memory addresses are 32-bit. Every wait is bounded.
constexpr int kWaitLimit = 1 << 20;  // mbarrier polls before a copy is given up

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
// Polls the mbarrier's phase `parity` at most kWaitLimit times (each poll may
// suspend the thread for a while); false if it did not complete.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// output visibilities (degridding): written once
__device__ __forceinline__ void st_stream(float* p, float v) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(policy_stream()) : "memory");
}

__device__ __forceinline__ float load_tap(const void* table, int fmt, int idx) {
  if (fmt == FMT_BF16) return __bfloat162float(((const __nv_bfloat16*)table)[idx]);
  if (fmt == FMT_F16) return __half2float(((const __half*)table)[idx]);
  return ((const float*)table)[idx];
}

__device__ __forceinline__ float2 splat(float x) { return make_float2(x, x); }

// Zero-padded, phase-expanded 1-D tables: tab[(r*B + rem)*nb + k] = T[r][k - rem]
// for 0 <= k - rem < S, else 0. A thread at block position t reads taps
// tab[(r*B + rem)*nb + t*B + i], i < B, as one aligned vector. (Storing each
// tap twice, as a ready (T, T) operand pair for the packed FMA, was measured
// 3-12% slower: the doubled shared-memory loads cost more than the pairing.)
template <int B>
__device__ __forceinline__ void build_table(float* tab, const Args& a, int nb) {
  const Geometry& g = a.g;
  const int n = g.O * B * nb;
  for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
    const int k = idx % nb;
    const int rr = idx / nb;
    const int rem = rr % B;
    const int r = rr / B;
    const int i = k - rem;
    tab[idx] = (i >= 0 && i < g.S) ? load_tap(a.table, a.tab_fmt, r * g.S + i) : 0.f;
  }
}

// Per-visibility record, built once per visibility while staging, so that
// each team thread needs only a few instructions per visibility:
//  x = M = (qu - rqu) | (qv - rqv) << 16: the block index of the bin-aligned
//      origin below the box (q = footprint start / B, rq = q mod n);
//  y = rqu | rqv << 16: the thread position that holds the box's first block;
//  z, w = table offset of (row, phase) minus rq*B, per axis.
// Thread (au, av) owns block (b_u, b_v) = (M_u + au + [au < rqu]*nu, ...),
// the one block of its residue class inside the box (Fig. 2), and reads its
// taps at z + (au + [au < rqu]*nu)*Bu.
template <int BU, int BV>
__device__ __forceinline__ bool make_meta(const Args& a, double2 x, int4& meta) {
  const Geometry& g = a.g;
  int Cu, ru, Cv, rv;
  bool ok = fine_cell(x.x, g.log2O, g.G >> 1, Cu, ru);
  ok = fine_cell(x.y, g.log2O, g.G >> 1, Cv, rv) && ok;
  const int cu0 = Cu - g.h, cv0 = Cv - g.h;
  ok = ok && cu0 >= 0 && cu0 + g.S <= g.G && cv0 >= 0 && cv0 + g.S <= g.G;
  if (!ok) {
    meta.x = (int)kInvalid;
    return false;
  }
  const int qu = cu0 / BU, remu = cu0 - qu * BU;
  const int qv = cv0 / BV, remv = cv0 - qv * BV;
  const int rqu = mod_small(qu, g.nu, g.mu), rqv = mod_small(qv, g.nv, g.mv);
  meta = make_int4((qu - rqu) | ((qv - rqv) << 16), rqu | (rqv << 16), (ru * BU + remu) * g.nbu - rqu * BU,
                   (rv * BV + remv) * g.nbv - rqv * BV);
  return true;
}

// A thread's fixed place in its team.
struct TeamPos {
  int au, av;    // block position in the bin
  unsigned A;    // au | av << 16
  int ou, ov;    // au*Bu, av*Bv
};

template <int BU, int BV>
__device__ __forceinline__ TeamPos team_pos(int l, const Geometry& g) {
  TeamPos t;
  t.au = l % g.nu;
  t.av = l / g.nu;
  t.A = (unsigned)t.au | ((unsigned)t.av << 16);
  t.ou = t.au * BU;
  t.ov = t.av * BV;
  return t;
}

// The thread's block for record m (its key, u | v << 16) and its tap offsets.
__device__ __forceinline__ unsigned box_key(const int4 m, const TeamPos& t, const Geometry& g, int& offu, int& offv) {
  const bool wu = t.au < (m.y & 0xFFFF);
  const bool wv = t.av < (int)((unsigned)m.y >> 16);
  offu = m.z + t.ou + (wu ? g.nuB : 0);
  offv = m.w + t.ov + (wv ? g.nvB : 0);
  return (unsigned)m.x + t.A + (wu ? (unsigned)g.nu : 0u) + (wv ? ((unsigned)g.nv << 16) : 0u);
}

// The raw words of one record's P values (2P words for FP32 pairs, P words
// for 16-bit pairs), loaded apart from their conversion so that staging can
// issue every load of a pass before it waits on any of them.
template <int P>
struct VisWords {
  uint32_t w[2 * P];
};

template <int P>
__device__ __forceinline__ void load_vis_words(const Args& a, long long k, VisWords<P>& q) {
  if (a.vis_fmt == FMT_F32) {
    const float2* src = (const float2*)a.vis + k * P;
    if constexpr (P % 2 == 0) {
#pragma unroll
      for (int p = 0; p < P; p += 2) {
        const uint4 t = *(const uint4*)(src + p);
        q.w[2 * p] = t.x; q.w[2 * p + 1] = t.y; q.w[2 * p + 2] = t.z; q.w[2 * p + 3] = t.w;
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const uint2 t = *(const uint2*)(src + p);
        q.w[2 * p] = t.x; q.w[2 * p + 1] = t.y;
      }
    }
  } else {
    const uint32_t* src = (const uint32_t*)a.vis + k * P;
    if constexpr (P == 4) {
      const uint4 t = *(const uint4*)src;
      q.w[0] = t.x; q.w[1] = t.y; q.w[2] = t.z; q.w[3] = t.w;
    } else if constexpr (P == 2) {
      const uint2 t = *(const uint2*)src;
      q.w[0] = t.x; q.w[1] = t.y;
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) q.w[p] = src[p];
    }
  }
}

// w * V_p for the loaded words (16-bit pairs widened to FP32 first).
template <int P>
__device__ __forceinline__ void vis_values(const Args& a, const VisWords<P>& q, float w, float2 (&val)[P]) {
  if (a.vis_fmt == FMT_F32) {
#pragma unroll
    for (int p = 0; p < P; ++p) val[p] = make_float2(__uint_as_float(q.w[2 * p]) * w, __uint_as_float(q.w[2 * p + 1]) * w);
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      float2 f;
      if (a.vis_fmt == FMT_BF16) {
        __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.w[p]);
        f = __bfloat1622float2(b);
      } else {
        __half2 hh = *reinterpret_cast<const __half2*>(&q.w[p]);
        f = __half22float2(hh);
      }
      val[p] = make_float2(f.x * w, f.y * w);
    }
  }
}

template <int P>
__device__ __forceinline__ void load_vis(const Args& a, long long k, float w, float2 (&val)[P]) {
  VisWords<P> q;
  load_vis_words<P>(a, k, q);
  vis_values<P>(a, q, w, val);
}

template <int B>
__device__ __forceinline__ void load_taps(const float* p, float (&t)[B]) {
  if constexpr (B % 4 == 0) {
#pragma unroll
    for (int i = 0; i < B; i += 4) {
      const float4 q = *(const float4*)(p + i);
      t[i] = q.x; t[i + 1] = q.y; t[i + 2] = q.z; t[i + 3] = q.w;
    }
  } else if constexpr (B % 2 == 0) {
#pragma unroll
    for (int i = 0; i < B; i += 2) {
      const float2 q = *(const float2*)(p + i);
      t[i] = q.x; t[i + 1] = q.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < B; ++i) t[i] = p[i];
  }
}

// ---------------------------------------------------------------------------
// Shared-memory layouts (computed identically on host and device).

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Patch window: P planes of `win` rows; a row holds `win` complex cells as
// interleaved (re, im) floats. win is a multiple of 16, so the row stride
// 2*win + 4 is 4 (mod 32) floats and the plane stride is 8 (mod 32) floats:
// the 2 x 2 cells x 4 polarizations of one block, flushed by one warp
// instruction, fall in 32 different banks. Rows start on 16-byte boundaries.
__host__ __device__ inline int win_row_stride(int win) { return 2 * win + 4; }
__host__ __device__ inline int win_plane_stride(int win) {
  const int x = win * win_row_stride(win);
  return x + ((8 - x % 32) + 32) % 32;
}

// Degridding team reduction buffer. The 2P partial sums of one record are
// split into groups of QW floats (QW = 4 when P is even, else 2). Thread t of a
// team stores group q of record r at r*R + q*Q + t*QW: the group stride Q is
// ts*QW padded to QW (mod 32) floats and the record stride is R = (2P/QW)*Q.
// A quarter-warp of float4 stores (or a half-warp of float2 stores) then
// writes consecutive words, and the reducing threads, which read group
// (r, q) at r*R + q*Q, start in distinct banks. The team stride adds 16 so
// that two teams in one store phase use opposite halves of the banks.
__host__ __device__ constexpr int degrid_qw(int P) { return (P % 2 == 0) ? 4 : 2; }
__host__ __device__ inline int degrid_group_stride(int ts, int P) {
  const int qw = degrid_qw(P);
  const int x = ts * qw;
  return x + ((qw - x % 32) + 32) % 32;
}
__host__ __device__ inline int degrid_rec_stride(int ts, int P) { return (2 * P / degrid_qw(P)) * degrid_group_stride(ts, P); }
__host__ __device__ inline int degrid_team_stride(int ts, int P) { return kRBD * degrid_rec_stride(ts, P) + 16; }

struct SmemLayout {
  size_t tabU, tabV, meta, vals, win, slots, keys, red, total;
};

template <int BU, int BV, int P>
__host__ __device__ inline SmemLayout grid_layout(const Geometry& g, int nthreads, int win) {
  SmemLayout L{};
  size_t off = 0;
  L.tabU = off; off += align16((size_t)g.O * BU * g.nbu * 4);
  L.tabV = off; off += align16((size_t)g.O * BV * g.nbv * 4);
  L.meta = off; off += align16((size_t)2 * g.tpc * kRB * 16);
  L.vals = off; off += align16((size_t)2 * g.tpc * kRB * P * 8);
  if (win > 0) {
    const int nw = (nthreads + 31) / 32;
    L.win = off; off += align16((size_t)P * win_plane_stride(win) * 4);
    L.slots = off; off += align16((size_t)nw * kSlots * 2 * P * BU * BV * 4);
    L.keys = off; off += align16((size_t)nw * kSlots * 4);
  }
  L.total = off;
  return L;
}

template <int BU, int BV, int P>
__host__ __device__ inline SmemLayout degrid_layout(const Geometry& g, int nthreads, int win) {
  SmemLayout L{};
  size_t off = 0;
  L.tabU = off; off += align16((size_t)g.O * BU * g.nbu * 4);
  L.tabV = off; off += align16((size_t)g.O * BV * g.nbv * 4);
  L.meta = off; off += align16((size_t)2 * g.tpc * kRBD * 16);
  L.red = off; off += align16((size_t)g.tpc * degrid_team_stride(g.ts, P) * 4);
  (void)nthreads;
  (void)win;
  L.total = off;
  return L;
}

// ---------------------------------------------------------------------------
// Flushes.

// Adds a thread's block to the grid with vector atomics (no per-vector zero
// test: with B <= 3 no block lies wholly in the padding, and with larger B such
// a block only adds zeros, which costs less than testing every vector). A
// block wholly inside the grid takes the unguarded path: one 64-bit pointer to
// its first cell, and every cell at that pointer plus kernel-uniform row and
// plane strides (a 32-bit cell index per access measured 3% more warp
// instructions in the gridder, 6% more in the degridder's reload, which
// addresses its block the same way). Blocks at the far edge
// address cells by a 32-bit index from the grid base (P*G*G <= 2^32 for
// G <= 32768) and skip their cells outside the grid, which hold exact zeros
// (the footprint of a gridded visibility is inside the grid). With ZERO the
// accumulators are cleared afterwards; the chunked loops instead assign the
// next block.
template <int BU, int BV, int P, bool ZERO = true>
__device__ __forceinline__ void flush_global(float2 (&acc)[P][BV][BU], unsigned key, float2* __restrict__ grid, int G) {
  const unsigned u0 = (key & 0xFFFFu) * BU;
  const unsigned v0 = (key >> 16) * BV;
  const unsigned GG = (unsigned)G * (unsigned)G;
  const unsigned base = v0 * (unsigned)G + u0;
  if (u0 + BU <= (unsigned)G && v0 + BV <= (unsigned)G) {
    char* const bp = (char*)(grid + base);
    const size_t rowB = (size_t)G * 8, planeB = (size_t)GG * 8;
#pragma unroll
    for (int j = 0; j < BV; ++j)
#pragma unroll
      for (int p = 0; p < P; ++p) {
        char* const rp = bp + (size_t)p * planeB + (size_t)j * rowB;
        if constexpr (BU % 2 == 0) {
#pragma unroll
          for (int i = 0; i < BU; i += 2)
            atomicAdd((float4*)(rp + i * 8),
                      make_float4(acc[p][j][i].x, acc[p][j][i].y, acc[p][j][i + 1].x, acc[p][j][i + 1].y));
        } else {
#pragma unroll
          for (int i = 0; i < BU; ++i) atomicAdd((float2*)(rp + i * 8), acc[p][j][i]);
        }
      }
  } else {
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      if (v0 + j >= (unsigned)G) continue;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const unsigned row = base + (unsigned)p * GG + (unsigned)j * (unsigned)G;
        if constexpr (BU % 2 == 0) {
#pragma unroll
          for (int i = 0; i < BU; i += 2)
            if (u0 + i + 1 < (unsigned)G)
              atomicAdd((float4*)(grid + (row + i)),
                        make_float4(acc[p][j][i].x, acc[p][j][i].y, acc[p][j][i + 1].x, acc[p][j][i + 1].y));
        } else {
#pragma unroll
          for (int i = 0; i < BU; ++i)
            if (u0 + i < (unsigned)G) atomicAdd(grid + (row + i), acc[p][j][i]);
        }
      }
    }
  }
  if constexpr (ZERO) {
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int j = 0; j < BV; ++j)
#pragma unroll
        for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);
  }
}

struct WindowCtx {
  float* buf;        // shared window
  int win, ws, ps;   // side, row stride, plane stride (floats)
  int wu0, wv0;      // grid cell of window (0, 0)
  float* slots;      // this warp's flush slots
  unsigned* keys;    // this warp's slot keys
  unsigned wmask;    // lanes of this warp that exist
};

// Cooperative flush into the shared window. Each lane with need=true owns a
// block (key) whose accumulators must be added. Blocks outside the window go
// straight to global memory from their owner. The others are parked in the
// warp's slots, kSlots at a time. Then all 32 lanes add them element by
// element, so every shared atomic instruction runs with all lanes active
// (the cost of a shared atomic is per instruction, not per active lane).
// Must be called by every lane of the warp (warp-uniform).
template <int BU, int BV, int P>
__device__ __forceinline__ void window_flush(bool need, unsigned key, float2 (&acc)[P][BV][BU], float2* grid, int G,
                                             const WindowCtx& w, int4& dirty) {
  constexpr int F = 2 * P * BU * BV;
  if (need) {
    const int lu = (int)(key & 0xFFFFu) * BU - w.wu0;
    const int lv = (int)(key >> 16) * BV - w.wv0;
    if (lu < 0 || lv < 0 || lu + BU > w.win || lv + BV > w.win) {
      flush_global<BU, BV, P>(acc, key, grid, G);
      need = false;
    } else {
      dirty.x = min(dirty.x, lu);
      dirty.y = min(dirty.y, lv);
      dirty.z = max(dirty.z, lu + BU);
      dirty.w = max(dirty.w, lv + BV);
    }
  }
  unsigned m = __ballot_sync(w.wmask, need);
  const int lane = threadIdx.x & 31;
  while (m) {
    unsigned take = 0, mm = m;
#pragma unroll
    for (int k = 0; k < kSlots; ++k) {
      const unsigned b = mm & (0u - mm);
      take |= b;
      mm &= ~b;
    }
    const int cnt = __popc(take);
    if ((take >> lane) & 1u) {
      const int rank = __popc(take & ((1u << lane) - 1u));
      float* dst = w.slots + rank * F;
      if constexpr (BU % 2 == 0) {
        // slot base is 16-byte aligned (kSlots * F floats per warp, F even) and
        // e is a multiple of 4 here, so the float4 stores are aligned
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int j = 0; j < BV; ++j)
#pragma unroll
            for (int i = 0; i < BU; i += 2) {
              const int e = ((p * BV + j) * BU + i) * 2;
              *(float4*)(dst + e) = make_float4(acc[p][j][i].x, acc[p][j][i].y, acc[p][j][i + 1].x, acc[p][j][i + 1].y);
            }
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p)
#pragma unroll
          for (int j = 0; j < BV; ++j)
#pragma unroll
            for (int i = 0; i < BU; ++i) *(float2*)(dst + ((p * BV + j) * BU + i) * 2) = acc[p][j][i];
      }
      w.keys[rank] = key;
#pragma unroll
      for (int p = 0; p < P; ++p)
#pragma unroll
        for (int j = 0; j < BV; ++j)
#pragma unroll
          for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);
    }
    __syncwarp(w.wmask);
    // the last warp of a CTA whose size is not a multiple of 32 has fewer
    // lanes (wmask holds the low ones), so the stride is the lane count
    const int nl = __popc(w.wmask);
    constexpr bool kSmallF = F <= 32 && 32 % F == 0;
    constexpr bool kBigF = F % 32 == 0 && F > 32;
    if ((kSmallF || kBigF) && nl == 32) {
      // Fast path: element e of every slot always lands at the same offset
      // from the slot's block origin, so each lane's offsets are fixed.
      if constexpr (kSmallF) {
        const int e = lane % F;
        const int c = e & 1, q = e >> 1;
        const int eoff = (q / (BU * BV)) * w.ps + ((q / BU) % BV) * w.ws + 2 * (q % BU) + c;
        for (int sl = lane / F; sl < cnt; sl += 32 / F) {
          const float v = w.slots[sl * F + e];
          if (v != 0.f) {
            const unsigned k2 = w.keys[sl];
            const int base = ((int)(k2 >> 16) * BV - w.wv0) * w.ws + 2 * ((int)(k2 & 0xFFFFu) * BU - w.wu0);
            atomicAdd(w.buf + base + eoff, v);
          }
        }
      } else if constexpr (kBigF) {
        int eoff[F / 32 > 0 ? F / 32 : 1];
#pragma unroll
        for (int t = 0; t < F / 32; ++t) {
          const int e = lane + 32 * t;
          const int c = e & 1, q = e >> 1;
          eoff[t] = (q / (BU * BV)) * w.ps + ((q / BU) % BV) * w.ws + 2 * (q % BU) + c;
        }
        for (int sl = 0; sl < cnt; ++sl) {
          const unsigned k2 = w.keys[sl];
          const int base = ((int)(k2 >> 16) * BV - w.wv0) * w.ws + 2 * ((int)(k2 & 0xFFFFu) * BU - w.wu0);
#pragma unroll
          for (int t = 0; t < F / 32; ++t) {
            const float v = w.slots[sl * F + lane + 32 * t];
            if (v != 0.f) atomicAdd(w.buf + base + eoff[t], v);
          }
        }
      }
    } else
    for (int idx = lane; idx < cnt * F; idx += nl) {
      const int s = idx / F;
      const int e = idx - s * F;
      const float v = w.slots[idx];
      if (v != 0.f) {
        const unsigned k2 = w.keys[s];
        const int c = e & 1, q = e >> 1;
        const int i = q % BU, j = (q / BU) % BV, p = q / (BU * BV);
        const int lu = (int)(k2 & 0xFFFFu) * BU - w.wu0 + i;
        const int lv = (int)(k2 >> 16) * BV - w.wv0 + j;
        atomicAdd(w.buf + p * w.ps + lv * w.ws + 2 * lu + c, v);
      }
    }
    __syncwarp(w.wmask);
    m &= ~take;
  }
}

// ---------------------------------------------------------------------------
// Staging: batch b of a team's chunk goes into shared memory. Each team
// thread stages records l, l+ts, ... of the batch (Sec. 4: "each work-item
// loads one visibility"). A thread issues a record's three loads (position,
// weight, values) together, before the index conversion, so it waits for one
// memory latency per record rather than two dependent ones. Values are thus
// loaded for every record in range, valid or not. (Two records per pass, all
// six loads first, needs 112 registers instead of 80.)
template <int BU, int BV, int P>
__device__ __forceinline__ void stage_record(const Args& a, bool have, double2 x, float w, const VisWords<P>& q,
                                             int4* meta, float2* vals) {
  int4 m;
  m.x = (int)kInvalid;
  if (have && !make_meta<BU, BV>(a, x, m)) atomicAdd(a.skipped, 1ULL);
  *meta = m;
  if (m.x != (int)kInvalid) {
    float2 val[P];
    vis_values<P>(a, q, w, val);
#pragma unroll
    for (int p = 0; p < P; ++p) vals[p] = val[p];
  }
}

template <int BU, int BV, int P, int RB = kRB>
__device__ __forceinline__ void stage_batch(const Args& a, long long vbeg, long long vend, int b, int l, int4* meta,
                                            float2* vals) {
  const Geometry& g = a.g;
  const long long kb = vbeg + (long long)b * RB;
  for (int r = l; r < RB; r += g.ts) {
    const bool h = kb + r < vend;
    double2 x = make_double2(0.0, 0.0);
    float w = 1.f;
    VisWords<P> q;
    if (h) {
      x = a.uv[kb + r];
      if (a.weights) w = a.weights[kb + r];
      load_vis_words<P>(a, kb + r, q);
    }
    if (kb + RB + r < vend) {
      // the record this thread stages next batch goes to L1 meanwhile
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a.uv + kb + RB + r));
      asm volatile("prefetch.global.L1 [%0];" ::"l"((const char*)a.vis + (kb + RB + r) * (long long)P * (a.vis_fmt == FMT_F32 ? 8 : 4)));
    }
    stage_record<BU, BV, P>(a, h, x, w, q, meta + r, vals + r * P);
  }
}

// How a thread forms its Bu x Bv x P products t_u[i] t_v[j] V_p (Sec. 6
// remark on the separable product). Each product is one packed FMA either way;
// the forms differ in the multiplies spent beforehand:
//  - TAP_PRODUCT: Bu*Bv scalar products w_ij = t_u[i] t_v[j];
//  - TAP_FACTOR_V: Bv*P packed products Y_jp = t_v[j] V_p, then t_u[i] Y_jp;
//  - TAP_FACTOR_U: Bu*P packed products X_ip = t_u[i] V_p, then t_v[j] X_ip.
// The cheapest is chosen per instantiation (factoring wins when P < max(Bu, Bv),
// e.g. for single polarization with Bu or Bv >= 2).
enum { TAP_PRODUCT = 0, TAP_FACTOR_V = 1, TAP_FACTOR_U = 2 };
template <int BU, int BV, int P>
struct TapForm {
  static constexpr int kProduct = BU * BV, kFactorV = BV * P, kFactorU = BU * P;
  static constexpr int value = (kProduct <= kFactorV && kProduct <= kFactorU) ? TAP_PRODUCT
                               : (kFactorV <= kFactorU ? TAP_FACTOR_V : TAP_FACTOR_U);
};

// The convolution of one visibility into the thread's block (Sec. 3), in two
// steps so that the part common to every lane is done before the branch on
// whether the block changed:
//  - Contribution::prepare: Bu + Bv taps from the padded tables, the values,
//    and the products the chosen form needs;
//  - Contribution::apply: Bu*Bv*P packed FMAs into the accumulators, or (ADD =
//    false) packed multiplies that assign a fresh block after a flush.
template <int BU, int BV, int P>
struct Contribution {
  static constexpr int form = TapForm<BU, BV, P>::value;
  static constexpr int NA = form == TAP_PRODUCT ? BV * BU : (form == TAP_FACTOR_V ? BV * P : BU * P);
  static constexpr int NB = form == TAP_PRODUCT ? 1 : (form == TAP_FACTOR_V ? BU : BV);
  // PRODUCT: A = tap products t_u t_v (scalars), V = values.
  // FACTOR_V: A = t_v V (pairs), t = t_u.  FACTOR_U: A = t_u V (pairs), t = t_v.
  float a[form == TAP_PRODUCT ? NA : 1];
  float2 A[form == TAP_PRODUCT ? 1 : NA];
  float2 V[form == TAP_PRODUCT ? P : 1];
  float t[NB];

  __device__ __forceinline__ void prepare(int offu, int offv, const float2* __restrict__ vals,
                                          const float* __restrict__ tabU, const float* __restrict__ tabV) {
    float wu[BU], wv[BV];
    load_taps<BU>(tabU + offu, wu);
    load_taps<BV>(tabV + offv, wv);
    from_taps(wu, wv, vals);
  }

  // The products of the chosen form from taps and values already loaded.
  __device__ __forceinline__ void from_taps(const float (&wu)[BU], const float (&wv)[BV], const float2* vals) {
    if constexpr (form == TAP_PRODUCT) {
#pragma unroll
      for (int j = 0; j < BV; ++j)
#pragma unroll
        for (int i = 0; i < BU; ++i) a[j * BU + i] = wu[i] * wv[j];
#pragma unroll
      for (int p = 0; p < P; ++p) V[p] = vals[p];
    } else if constexpr (form == TAP_FACTOR_V) {
#pragma unroll
      for (int j = 0; j < BV; ++j)
#pragma unroll
        for (int p = 0; p < P; ++p) A[j * P + p] = __fmul2_rn(splat(wv[j]), vals[p]);
#pragma unroll
      for (int i = 0; i < BU; ++i) t[i] = wu[i];
    } else {
#pragma unroll
      for (int i = 0; i < BU; ++i)
#pragma unroll
        for (int p = 0; p < P; ++p) A[i * P + p] = __fmul2_rn(splat(wu[i]), vals[p]);
#pragma unroll
      for (int j = 0; j < BV; ++j) t[j] = wv[j];
    }
  }

  template <bool ADD>
  __device__ __forceinline__ void apply(float2 (&acc)[P][BV][BU]) const {
    auto term = [](float2 x, float2 y, float2 c) { return ADD ? __ffma2_rn(x, y, c) : __fmul2_rn(x, y); };
#pragma unroll
    for (int p = 0; p < P; ++p)
#pragma unroll
      for (int j = 0; j < BV; ++j)
#pragma unroll
        for (int i = 0; i < BU; ++i) {
          if constexpr (form == TAP_PRODUCT) acc[p][j][i] = term(splat(a[j * BU + i]), V[p], acc[p][j][i]);
          else if constexpr (form == TAP_FACTOR_V) acc[p][j][i] = term(splat(t[i]), A[j * P + p], acc[p][j][i]);
          else acc[p][j][i] = term(splat(t[j]), A[i * P + p], acc[p][j][i]);
        }
  }
};

template <int BU, int BV, int P, bool ADD = true>
__device__ __forceinline__ void accumulate(int offu, int offv, const float2* __restrict__ vals,
                                           const float* __restrict__ tabU, const float* __restrict__ tabV,
                                           float2 (&acc)[P][BV][BU]) {
  Contribution<BU, BV, P> c;
  c.prepare(offu, offv, vals, tabU, tabV);
  c.template apply<ADD>(acc);
}

// The adjoint product for degridding: s_p = sum_ij t_u[i] t_v[j] g[p][j][i],
// in the same three forms (the factored ones sum along one axis first). s is
// assigned, not accumulated: the first term is a multiply, so the caller
// needs no zeroing.
template <int BU, int BV, int P>
__device__ __forceinline__ void block_dot(const float (&wu)[BU], const float (&wv)[BV], const float2 (&gb)[P][BV][BU],
                                          float2 (&s)[P]) {
  constexpr int form = TapForm<BU, BV, P>::value;
  if constexpr (form == TAP_PRODUCT) {
#pragma unroll
    for (int j = 0; j < BV; ++j) {
#pragma unroll
      for (int i = 0; i < BU; ++i) {
        const float2 w2 = splat(wu[i] * wv[j]);
#pragma unroll
        for (int p = 0; p < P; ++p)
          s[p] = (i == 0 && j == 0) ? __fmul2_rn(w2, gb[p][j][i]) : __ffma2_rn(w2, gb[p][j][i], s[p]);
      }
    }
  } else if constexpr (form == TAP_FACTOR_V) {
    // rows first: r_jp = sum_i t_u[i] g[p][j][i], then s_p += t_v[j] r_jp
#pragma unroll
    for (int j = 0; j < BV; ++j) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        float2 r = __fmul2_rn(splat(wu[0]), gb[p][j][0]);
#pragma unroll
        for (int i = 1; i < BU; ++i) r = __ffma2_rn(splat(wu[i]), gb[p][j][i], r);
        s[p] = j == 0 ? __fmul2_rn(splat(wv[j]), r) : __ffma2_rn(splat(wv[j]), r, s[p]);
      }
    }
  } else {
    // columns first: c_ip = sum_j t_v[j] g[p][j][i], then s_p += t_u[i] c_ip
#pragma unroll
    for (int i = 0; i < BU; ++i) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        float2 c = __fmul2_rn(splat(wv[0]), gb[p][0][i]);
#pragma unroll
        for (int j = 1; j < BV; ++j) c = __ffma2_rn(splat(wv[j]), gb[p][j][i], c);
        s[p] = i == 0 ? __fmul2_rn(splat(wu[i]), c) : __ffma2_rn(splat(wu[i]), c, s[p]);
      }
    }
  }
}

__device__ __forceinline__ void group_sync(const Args& a, unsigned wmask) {
  if (a.warp_sync) __syncwarp(wmask);
  else __syncthreads();
}

__device__ __forceinline__ unsigned warp_lane_mask() {
  const int base = threadIdx.x & ~31;
  const int n = (int)blockDim.x - base;
  return n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u);
}

// ---------------------------------------------------------------------------
// Gridding kernel.
//  - Chunked schedule (win == 0): one chunk per team, flushes to global
//    memory with vector atomics (Sec. 4).
//  - Patch schedule (win > 0): persistent CTAs take work items (a patch plus
//    a range of its chunks). A CTA accumulates the patch window in shared
//    memory through cooperative warp flushes, then adds the touched part of
//    the window to the grid and leaves it zeroed for the next item.
// Teams whose size divides 32 sit inside one warp and synchronise per warp
// (warp_sync). Otherwise all teams of the CTA step through batches together.
template <int BU, int BV, int P, bool PATCH>
__global__ void grid_kernel(Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const SmemLayout L = grid_layout<BU, BV, P>(g, blockDim.x, a.win);
  float* tabU = (float*)(smem + L.tabU);
  float* tabV = (float*)(smem + L.tabV);
  int4* meta = (int4*)(smem + L.meta);
  float2* vals = (float2*)(smem + L.vals);

  build_table<BU>(tabU, a, g.nbu);
  build_table<BV>(tabV, a, g.nbv);

  const int team = threadIdx.x / g.ts;
  const int l = threadIdx.x - team * g.ts;
  const TeamPos tp = team_pos<BU, BV>(l, g);
  const int nb = (a.chunk_len + kRB - 1) / kRB;
  const unsigned wmask = warp_lane_mask();
  int4* const mt0 = meta + team * kRB;
  int4* const mt1 = meta + (g.tpc + team) * kRB;
  float2* const vl0 = vals + (size_t)team * kRB * P;
  float2* const vl1 = vals + (size_t)(g.tpc + team) * kRB * P;

  float2 acc[P][BV][BU];
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < BV; ++j)
#pragma unroll
      for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);

  if constexpr (!PATCH) {
    // ---- chunked schedule: one chunk per team
    const long long chunk = (long long)blockIdx.x * g.tpc + team;
    const long long vbeg = chunk * a.chunk_len;
    const long long vend = chunk < a.n_chunks ? min(vbeg + a.chunk_len, a.n_vis) : vbeg;
    __syncthreads();  // tables ready
    unsigned cur = kInvalid;
    for (int b = 0; b < nb; ++b) {
      int4* const mtb = (b & 1) ? mt1 : mt0;
      float2* const vlb = (b & 1) ? vl1 : vl0;
      stage_batch<BU, BV, P>(a, vbeg, vend, b, l, mtb, vlb);
      group_sync(a, wmask);
      // single polarization: few packed FMAs per record, so the loop is unrolled to
      // overlap records (measured 3-4% faster on the S=15 workload); otherwise not
#pragma unroll (P == 1 ? 4 : 1)
      for (int r = 0; r < kRB; ++r) {
        const int4 m = mtb[r];
        if (m.x == (int)kInvalid) continue;
        int offu, offv;
        const unsigned key = box_key(m, tp, g, offu, offv);
        // the box moved: flush the old block, then start the new one with this
        // visibility (the contribution is prepared by all lanes between the two)
        const bool moved = key != cur;
        if (moved && cur != kInvalid) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
        Contribution<BU, BV, P> c;
        c.prepare(offu, offv, vlb + r * P, tabU, tabV);
        if (moved) {
          cur = key;
          c.template apply<false>(acc);
        } else {
          c.template apply<true>(acc);
        }
      }
    }
    if (cur != kInvalid) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
  } else {
  // ---- patch schedule
  __shared__ int s_item;
  __shared__ int s_next;  // next unclaimed chunk of the current item (warp_sync mode)
  __shared__ int s_dirty[4];
  WindowCtx w;
  w.buf = (float*)(smem + L.win);
  w.win = a.win;
  w.ws = win_row_stride(a.win);
  w.ps = win_plane_stride(a.win);
  w.slots = (float*)(smem + L.slots) + (threadIdx.x >> 5) * kSlots * (2 * P * BU * BV);
  w.keys = (unsigned*)(smem + L.keys) + (threadIdx.x >> 5) * kSlots;
  w.wmask = wmask;
  const int plane_floats = P * w.ps;
  for (int i = threadIdx.x; i < plane_floats; i += blockDim.x) w.buf[i] = 0.f;
  const int n_work = *a.n_work;
  int batch = 0;  // running batch counter: selects the staging buffer
  for (;;) {
    __syncthreads();  // previous item flushed, window zero, tables ready
    if (threadIdx.x == 0) {
      s_item = atomicAdd(a.work_next, 1);
      s_next = 0;
      s_dirty[0] = a.win; s_dirty[1] = a.win; s_dirty[2] = 0; s_dirty[3] = 0;
    }
    __syncthreads();
    const int item = s_item;
    if (item >= n_work) break;
    const int4 wk = a.work[item];
    w.wu0 = wk.x;
    w.wv0 = wk.y;
    int4 dirty = make_int4(a.win, a.win, 0, 0);
    const int n_item_chunks = wk.w - wk.z;
    // Warp-synchronous teams claim chunks a warp at a time from a shared
    // counter, so a warp with nothing left to do leaves at once. Otherwise all
    // teams of the CTA step through rounds together.
    const int lane_id = threadIdx.x & 31;
    const int tpw = __popc(wmask) / g.ts;           // teams in this warp (warp_sync mode)
    const int team_in_warp = lane_id / g.ts;
    const int rounds = a.warp_sync ? 0x7FFFFFFF : (n_item_chunks + g.tpc - 1) / g.tpc;
    for (int rd = 0; rd < rounds; ++rd) {
      int ci;
      if (a.warp_sync) {
        int base = 0;
        if (lane_id == 0) base = atomicAdd(&s_next, tpw);
        base = __shfl_sync(wmask, base, 0);
        if (base >= n_item_chunks) break;
        ci = base + team_in_warp;
      } else {
        ci = rd * g.tpc + team;
      }
      long long vbeg = 0, vend = 0;
      if (ci < n_item_chunks) {
        const long long chunk = a.chunk_order[wk.z + ci];
        vbeg = chunk * a.chunk_len;
        vend = min(vbeg + a.chunk_len, a.n_vis);
      }
      unsigned cur = kInvalid;
      for (int b = 0; b < nb; ++b, ++batch) {
        int4* const mtb = (batch & 1) ? mt1 : mt0;
        float2* const vlb = (batch & 1) ? vl1 : vl0;
        stage_batch<BU, BV, P>(a, vbeg, vend, b, l, mtb, vlb);
        group_sync(a, wmask);
#pragma unroll 1
        for (int r = 0; r < kRB; ++r) {
          const int4 m = mtb[r];
          const bool valid = m.x != (int)kInvalid;
          int offu = 0, offv = 0;
          unsigned key = cur;
          if (valid) key = box_key(m, tp, g, offu, offv);
          window_flush<BU, BV, P>(valid && key != cur && cur != kInvalid, cur, acc, a.grid, g.G, w, dirty);
          if (valid) {
            cur = key;
            accumulate<BU, BV, P>(offu, offv, vlb + r * P, tabU, tabV, acc);
          }
        }
      }
      window_flush<BU, BV, P>(cur != kInvalid, cur, acc, a.grid, g.G, w, dirty);
    }
    if (dirty.z > dirty.x) {
      atomicMin(&s_dirty[0], dirty.x);
      atomicMin(&s_dirty[1], dirty.y);
      atomicMax(&s_dirty[2], dirty.z);
      atomicMax(&s_dirty[3], dirty.w);
    }
    __syncthreads();
    // add the touched rectangle of the window to the grid (float4 = two cells,
    // coalesced vector atomics, all-zero vectors skipped) and zero it again
    const int u_lo = s_dirty[0] & ~1, u_hi = (s_dirty[2] + 1) & ~1;
    const int v_lo = s_dirty[1], v_hi = s_dirty[3];
    if (u_hi > u_lo && v_hi > v_lo) {
      const int cols = (u_hi - u_lo) >> 1, rows = v_hi - v_lo;
      const int total = P * rows * cols;
      for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int c = i % cols;
        const int rr = i / cols;
        const int vv = v_lo + rr % rows;
        const int p = rr / rows;
        const int lu = u_lo + 2 * c;
        float4* src = (float4*)(w.buf + p * w.ps + vv * w.ws + 2 * lu);
        const float4 q = *src;
        const bool nz = (q.x != 0.f) | (q.y != 0.f) | (q.z != 0.f) | (q.w != 0.f);
        if (nz) {
          const int gu = w.wu0 + lu, gv = w.wv0 + vv;
          if (gu >= 0 && gv >= 0 && gu + 1 < g.G && gv < g.G)
            atomicAdd((float4*)(a.grid + ((size_t)p * g.G + gv) * g.G + gu), q);
          *src = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    }
  }
  }  // PATCH
}

// ---------------------------------------------------------------------------
// Degridding: the adjoint. Each thread keeps the grid values of its current
// block in registers and reloads them only when the box moves (the read-side
// analogue of a flush). Per visibility it forms P complex partial sums over
// its block. The team reduces them through shared memory: each thread stores
// its partials, then each thread sums whole columns of (record, component)
// outputs.
template <int BU, int BV, int P>
__device__ __forceinline__ void load_block(float2 (&gb)[P][BV][BU], unsigned key, const float2* __restrict__ grid, int G) {
  const unsigned u0 = (key & 0xFFFFu) * BU;
  const unsigned v0 = (key >> 16) * BV;
  const unsigned GG = (unsigned)G * (unsigned)G;
  const unsigned base = v0 * (unsigned)G + u0;
  const bool inside = u0 + BU <= (unsigned)G && v0 + BV <= (unsigned)G;
  const char* const bp = (const char*)(grid + base);
  const size_t rowB = (size_t)G * 8, planeB = (size_t)GG * 8;
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const char* const rp = bp + (size_t)p * planeB + (size_t)j * rowB;
      const bool vin = inside || v0 + j < (unsigned)G;
      if constexpr (BU % 2 == 0) {
#pragma unroll
        for (int i = 0; i < BU; i += 2) {
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (inside || (vin && u0 + i + 1 < (unsigned)G)) q = __ldg((const float4*)(rp + i * 8));
          gb[p][j][i] = make_float2(q.x, q.y);
          gb[p][j][i + 1] = make_float2(q.z, q.w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < BU; ++i) {
          float2 q = make_float2(0.f, 0.f);
          if (inside || (vin && u0 + i < (unsigned)G)) q = __ldg((const float2*)(rp + i * 8));
          gb[p][j][i] = q;
        }
      }
    }
  }
}

template <int BU, int BV, int P>
__global__ void degrid_kernel(Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const SmemLayout L = degrid_layout<BU, BV, P>(g, blockDim.x, 0);
  float* tabU = (float*)(smem + L.tabU);
  float* tabV = (float*)(smem + L.tabV);
  int4* meta = (int4*)(smem + L.meta);

  build_table<BU>(tabU, a, g.nbu);
  build_table<BV>(tabV, a, g.nbv);

  const int team = threadIdx.x / g.ts;
  const int l = threadIdx.x - team * g.ts;
  const TeamPos tp = team_pos<BU, BV>(l, g);
  const unsigned wmask = warp_lane_mask();
  const long long chunk = (long long)blockIdx.x * g.tpc + team;
  const long long vbeg = chunk * a.chunk_len;
  const long long vend = chunk < a.n_chunks ? min(vbeg + a.chunk_len, a.n_vis) : vbeg;
  if (l == 0 && vend > vbeg) {
    // the chunk's positions and weights go to L2 now, so that the staging of
    // every batch after the first waits for L2 rather than HBM
    prefetch_l2(a.uv + vbeg, (size_t)(vend - vbeg) * sizeof(double2));
    if (a.weights) prefetch_l2(a.weights + vbeg, (size_t)(vend - vbeg) * sizeof(float));
  }
  int4* const mt0 = meta + team * kRBD;
  int4* const mt1 = meta + (g.tpc + team) * kRBD;
  constexpr int QW = degrid_qw(P);
  const int Q = degrid_group_stride(g.ts, P);
  const int R = degrid_rec_stride(g.ts, P);
  float* red = (float*)(smem + L.red) + (size_t)team * degrid_team_stride(g.ts, P);
  const int nb = (a.chunk_len + kRBD - 1) / kRBD;

  float2 gb[P][BV][BU];
  unsigned cur = kInvalid;
  __syncthreads();
  for (int b = 0; b < nb; ++b) {
    int4* const mtb = (b & 1) ? mt1 : mt0;
    for (int r = l; r < kRBD; r += g.ts) {
      const long long k = vbeg + (long long)b * kRBD + r;
      int4 m;
      m.x = (int)kInvalid;
      if (k < vend && !make_meta<BU, BV>(a, ld_stream(a.uv + k), m)) atomicAdd(a.skipped, 1ULL);
      mtb[r] = m;
    }
    group_sync(a, wmask);
#pragma unroll 1
    for (int r = 0; r < kRBD; ++r) {
      const int4 m = mtb[r];
      float2 s[P];
      if (m.x == (int)kInvalid) {
#pragma unroll
        for (int p = 0; p < P; ++p) s[p] = make_float2(0.f, 0.f);
      } else {
        int offu, offv;
        const unsigned key = box_key(m, tp, g, offu, offv);
        if (key != cur) {
          load_block<BU, BV, P>(gb, key, a.grid, g.G);
          cur = key;
        }
        float wu[BU], wv[BV];
        load_taps<BU>(tabU + offu, wu);
        load_taps<BV>(tabV + offv, wv);
        block_dot<BU, BV, P>(wu, wv, gb, s);
      }
      float* dst = red + r * R + l * QW;
      if constexpr (QW == 4) {
#pragma unroll
        for (int p = 0; p < P; p += 2) *(float4*)(dst + (p / 2) * Q) = make_float4(s[p].x, s[p].y, s[p + 1].x, s[p + 1].y);
      } else {
#pragma unroll
        for (int p = 0; p < P; ++p) *(float2*)(dst + p * Q) = s[p];
      }
    }
    group_sync(a, wmask);
    // Each team thread reduces whole groups of QW components over the team.
    {
      constexpr int GPR = 2 * P / QW;
      for (int gi = l; gi < kRBD * GPR; gi += g.ts) {
        const int r = gi / GPR;
        const int q = gi - r * GPR;
        const long long k = vbeg + (long long)b * kRBD + r;
        if (k >= vend) continue;
        const float* col = red + r * R + q * Q;
        float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll 4  // measured 1% faster than the compiler's default here
        for (int t = 0; t < g.ts; ++t) {
          if constexpr (QW == 4) {
            const float4 v4 = *(const float4*)(col + t * QW);
            s0 = __fadd2_rn(s0, make_float2(v4.x, v4.y));
            s1 = __fadd2_rn(s1, make_float2(v4.z, v4.w));
          } else {
            s0 = __fadd2_rn(s0, *(const float2*)(col + t * QW));
          }
        }
        if (a.weights) {
          const float wk = ld_stream(a.weights + k);
          s0 = make_float2(s0.x * wk, s0.y * wk);
          s1 = make_float2(s1.x * wk, s1.y * wk);
        }
        float* out = (float*)a.vis_out + k * 2 * P + q * QW;
        st_stream(out, s0.x);
        st_stream(out + 1, s0.y);
        if constexpr (QW == 4) {
          st_stream(out + 2, s1.x);
          st_stream(out + 3, s1.y);
        }
      }
    }
    // the next batch stages into the other meta buffer; its group_sync
    // separates these reads of `red` from the next writes
  }
}

// Function table entry for one (Bu, Bv, P) instantiation, with its
// shared-memory layout functions.
struct KernelEntry {
  int bu, bv, p;
  int form;                   // TapForm<bu, bv, p>::value: how the kernels form the tap products
  const void* grid_fn;        // chunked schedule
  const void* grid_patch_fn;  // patch schedule
  const void* degrid_fn;
  size_t (*grid_smem)(const Geometry&, int nthreads, int win);
  size_t (*degrid_smem)(const Geometry&, int nthreads, int win);
};

template <int BU, int BV, int P>
size_t grid_smem_bytes(const Geometry& g, int nthreads, int win) {
  return grid_layout<BU, BV, P>(g, nthreads, win).total;
}

template <int BU, int BV, int P>
size_t degrid_smem_bytes(const Geometry& g, int nthreads, int win) {
  return degrid_layout<BU, BV, P>(g, nthreads, win).total;
}

}  // namespace gbg

namespace gbg {

// ---------------------------------------------------------------------------
// Batched gridding: many independent grids (channels x w-planes, Sec. 5 grids
// each w-slice with its own kernel instance) in ONE persistent launch. Every
// item has its own visibilities, GCF support S, kernel table and grid; G, O,
// P, the block shape and the storage format are common. Work units are runs of
// chunks of one item, sorted by cost on the host; persistent CTAs take them
// from an atomic counter, rebuild their padded tables when the item changes,
// and grid with the chunked schedule (flushes to global memory).
struct BatchItem {
  const double2* uv;
  const void* vis;
  const float* weights;
  const void* table;
  float2* grid;
  long long n_vis;
  int S;
  int shape;  // block shape: 0 = (BU1, BV1), 1 = (BU2, BV2) of a two-shape kernel
};

struct BatchArgs {
  int G, O, log2O, P;
  int fmt;
  int chunk_len;
  int nb_max;           // table capacity: largest bin width over the items
  int tpc_max;          // record-buffer capacity in teams
  const BatchItem* items;
  const int4* units;    // {item, first chunk, chunks, 0}
  int n_units;
  int* unit_next;
  unsigned long long* skipped;
};

template <int BU, int BV, int P>
__host__ __device__ inline SmemLayout batch_layout(int O, int nb_max, int tpc_max) {
  SmemLayout L{};
  size_t off = 0;
  L.tabU = off; off += align16((size_t)O * BU * nb_max * 4);
  L.tabV = off; off += align16((size_t)O * BV * nb_max * 4);
  L.meta = off; off += align16((size_t)2 * tpc_max * kRBB * 16);
  L.vals = off; off += align16((size_t)2 * tpc_max * kRBB * P * 8);
  L.total = off;
  return L;
}

// One work unit of the batched kernel (up to tpc chunks of one item) with
// blocks of BU x BV cells. `loaded` caches which item's tables are in shared
// memory (uniform across the CTA).
template <int BU, int BV, int P>
__device__ __forceinline__ void batch_unit(const BatchArgs& b, const int4 u, const BatchItem& it, unsigned char* smem,
                                           int& loaded) {
  const SmemLayout L = batch_layout<BU, BV, P>(b.O, b.nb_max, b.tpc_max);
  float* tabU = (float*)(smem + L.tabU);
  float* tabV = (float*)(smem + L.tabV);
  int4* meta = (int4*)(smem + L.meta);
  float2* vals = (float2*)(smem + L.vals);
  const int nbat = (b.chunk_len + kRBB - 1) / kRBB;
  Args a;
  a.g.G = b.G; a.g.S = it.S; a.g.O = b.O; a.g.log2O = b.log2O; a.g.h = (it.S - 1) / 2; a.g.P = P;
  finish_geometry(a.g, BU, BV);
  a.g.tpc = min(b.tpc_max, (int)blockDim.x / a.g.ts);
  a.n_vis = it.n_vis;
  a.uv = it.uv;
  a.vis = it.vis;
  a.vis_fmt = b.fmt;
  a.weights = it.weights;
  a.table = it.table;
  a.tab_fmt = b.fmt;
  a.grid = it.grid;
  a.chunk_len = b.chunk_len;
  a.n_chunks = (it.n_vis + b.chunk_len - 1) / b.chunk_len;
  a.warp_sync = 0;
  a.skipped = b.skipped;
  const Geometry& g = a.g;
  if (u.x != loaded) {
    build_table<BU>(tabU, a, g.nbu);
    build_table<BV>(tabV, a, g.nbv);
    loaded = u.x;
    __syncthreads();
  }
  const int team = threadIdx.x / g.ts;
  const int l = threadIdx.x - team * g.ts;
  const bool active = team < u.z;  // u.z <= tpc chunks in this unit
  const TeamPos tp = team_pos<BU, BV>(l, g);
  const long long chunk = (long long)u.y + team;
  const long long vbeg = chunk * b.chunk_len;
  const long long vend = active ? min(vbeg + b.chunk_len, it.n_vis) : vbeg;
  int4* const mt0 = meta + team * kRBB;
  int4* const mt1 = meta + (b.tpc_max + team) * kRBB;
  float2* const vl0 = vals + (size_t)team * kRBB * P;
  float2* const vl1 = vals + (size_t)(b.tpc_max + team) * kRBB * P;
  float2 acc[P][BV][BU];
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < BV; ++j)
#pragma unroll
      for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);
  unsigned cur = kInvalid;
  for (int bt = 0; bt < nbat; ++bt) {
    int4* const mtb = (bt & 1) ? mt1 : mt0;
    float2* const vlb = (bt & 1) ? vl1 : vl0;
    if (team < g.tpc) stage_batch<BU, BV, P, kRBB>(a, vbeg, vend, bt, l, mtb, vlb);
    __syncthreads();
    if (active) {
#pragma unroll (P == 1 ? 4 : 1)
      for (int r = 0; r < kRBB; ++r) {
        const int4 m = mtb[r];
        if (m.x == (int)kInvalid) continue;
        int offu, offv;
        const unsigned key = box_key(m, tp, g, offu, offv);
        // the box moved: flush the old block, then start the new one with this
        // visibility (the contribution is prepared by all lanes between the two)
        const bool moved = key != cur;
        if (moved && cur != kInvalid) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
        Contribution<BU, BV, P> c;
        c.prepare(offu, offv, vlb + r * P, tabU, tabV);
        if (moved) {
          cur = key;
          c.template apply<false>(acc);
        } else {
          c.template apply<true>(acc);
        }
      }
    }
  }
  if (active && cur != kInvalid) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
}

// Batched gridding (many grids in one persistent launch): CTAs take work
// units from an atomic counter. Each item is gridded with block shape
// (BU1, BV1) or, when its shape flag is set, (BU2, BV2): larger supports
// favour larger blocks. A one-shape kernel has BU2 = BU1, BV2 = BV1.
template <int BU1, int BV1, int BU2, int BV2, int P>
__global__ void grid_batch_kernel(BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_unit;
  int loaded = -1;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_unit = atomicAdd(b.unit_next, 1);
    __syncthreads();
    const int unit = s_unit;
    if (unit >= b.n_units) break;
    const int4 u = b.units[unit];
    const BatchItem it = b.items[u.x];
    if constexpr (BU1 == BU2 && BV1 == BV2) {
      batch_unit<BU1, BV1, P>(b, u, it, smem, loaded);
    } else {
      if (it.shape == 0) batch_unit<BU1, BV1, P>(b, u, it, smem, loaded);
      else batch_unit<BU2, BV2, P>(b, u, it, smem, loaded);
    }
  }
}

template <int BU1, int BV1, int BU2, int BV2, int P>
size_t batch_smem_bytes(int O, int nb_max, int tpc_max) {
  const size_t a = batch_layout<BU1, BV1, P>(O, nb_max, tpc_max).total;
  const size_t b = batch_layout<BU2, BV2, P>(O, nb_max, tpc_max).total;
  return a > b ? a : b;
}

struct BatchKernelEntry {
  int bu, bv, bu2, bv2, p;
  const void* fn;
  size_t (*smem)(int O, int nb_max, int tpc_max);
};

}  // namespace gbg
