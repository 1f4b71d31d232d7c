// Gridding with a widened bin and a lazily placed box.
//
// Romein's work distribution with thread coarsening (Sec. 2.2, Fig. 1;
// Sec. 3, Fig. 2) gives thread (au, av) of a team every block of Bu x Bv cells
// whose block coordinates are congruent to (au, av) modulo the bin of nu x nv
// blocks. For each visibility the team uses one bin-sized box of blocks that
// contains the footprint, and each thread owns exactly one block of that box.
//
// With the paper's bin (nu*Bu = roundup(S + Bu - 1, Bu), Sec. 3 and Sec. 5)
// the box is forced: it starts at the block holding the footprint's first
// cell. With a wider bin the box may start at any block b with
//   hi - nu + 1 <= b <= lo
// (lo, hi: the first and last block the footprint touches). Here the box stays
// where it is while the footprint fits, and otherwise moves by the fewest
// blocks:  b <- min(max(b, hi - nu + 1), lo).  For the paper's bin this is the
// paper's rule. A move by k blocks changes the block of k thread columns (or
// rows), which flush; a track that turns back within the slack flushes
// nothing. The price is padding: more cells per visibility whose taps are 0.
//
// Data flow per team (a team sits in one aligned lane segment of a warp; a
// segment's lanes beyond the team only stage records):
//  - loading: one lane copies the raw records (uv, weights, values) of the
//    team's next batch of 32 consecutive visibilities into shared memory with
//    bulk asynchronous copies (cp.async.bulk, completion on an mbarrier),
//    while the team works on the current batch. A batch that is not whole or
//    not 16-byte aligned is loaded by the lanes instead;
//  - staging: each segment lane converts records l, l + seg, ... of the batch
//    in place (exact index rule, clamp bounds, table offsets) and writes the
//    weighted values;
//  - per record: the box update is two packed 16-bit clamps and one compare.
//    Only when the box moves does a thread recompute its block, and only if
//    its block changed does it flush and restart;
//  - contribution: both tables hold every tap twice, (t, t), so one packed
//    multiply gives a cell's tap product as a ready (w, w) operand and each
//    packed FMA updates the (re, im) accumulator of one cell:
//      acc(i, j, p) += (w_ij, w_ij) * (Re V_p, Im V_p).
//    The accumulators then sit in the grid's (re, im) order, so a flush adds
//    two cells per vector atomic straight from them.
#pragma once

#include "kernels.cuh"

namespace gbg {

constexpr int kRBL = 32;                     // records per team per batch
constexpr unsigned kBoxNone = 0x7FFF7FFFu;   // no box yet
constexpr unsigned kClampLoNone = 0x80008000u;  // clamp bounds of an invalid record: the box stays
constexpr unsigned kClampHiNone = 0x7FFF7FFFu;
constexpr int kOffNone = 0x3FFFFFFF;         // table offset of an invalid record (clamped to the table)

template <int B>
struct Log2B {
  static_assert(B == 1 || B == 2 || B == 4 || B == 8, "block sides are powers of two");
  static constexpr int value = B == 1 ? 0 : B == 2 ? 1 : B == 4 ? 2 : 3;
};

// Per-team shared memory of the lazy gridder: two raw batch buffers, the
// weighted values of the current batch, and one mbarrier per raw buffer.
// A raw buffer holds uv [32] (16 B each; overwritten in place by the record
// metadata), weights [32] and values [32][P] in the input format.
__host__ __device__ constexpr int lazy_raw_bytes(int P) { return kRBL * 16 + kRBL * 4 + kRBL * 8 * P; }
__host__ __device__ constexpr int lazy_team_bytes(int P) { return 2 * lazy_raw_bytes(P) + kRBL * 8 * P + 16; }

struct LazyLayout {
  size_t tabU, tabV, teams, total;
};

// Shared memory: tables (u: [O][Bu][2nu-1][Bu] and v: [O][Bv][2nv-1][Bv], each
// tap as a duplicated pair), then the teams' buffers.
template <int BU, int BV, int P>
__host__ __device__ inline LazyLayout lazy_layout(const Geometry& g, int teams) {
  LazyLayout L{};
  size_t off = 0;
  L.tabU = off; off += align16((size_t)g.O * BU * (2 * g.nu - 1) * BU * 8);
  L.tabV = off; off += align16((size_t)g.O * BV * (2 * g.nv - 1) * BV * 8);
  L.teams = off; off += (size_t)teams * lazy_team_bytes(P);
  L.total = off;
  return L;
}

// Tap tables indexed by (table row r, footprint phase ph = first cell mod B,
// block distance m = thread block - footprint's first block in [-(n-1), n-1]):
//   tabU[((r*BU + ph)*(2nu-1) + m + nu-1)*BU + i]     = (t, t), t = T[r][m*BU + i - ph]
//   tabV[((r*BV + ph)*(2nv-1) + m + nv-1)*BV + j]     = (t, t), t = T[r][m*BV + j - ph]
// and (0, 0) where the tap index falls outside [0, S).
template <int BU, int BV>
__device__ __forceinline__ void lazy_tables(float2* tabU, float2* tabV, const Args& a) {
  const Geometry& g = a.g;
  const int wu = 2 * g.nu - 1, wv = 2 * g.nv - 1;
  const int nU = g.O * BU * wu * BU;
  for (int idx = threadIdx.x; idx < nU; idx += blockDim.x) {
    const int i = idx % BU;
    int q = idx / BU;
    const int mm = q % wu;
    q /= wu;
    const int ph = q % BU, r = q / BU;
    const int k = (mm - g.nu + 1) * BU + i - ph;
    tabU[idx] = splat((k >= 0 && k < g.S) ? load_tap(a.table, a.tab_fmt, r * g.S + k) : 0.f);
  }
  const int nV = g.O * BV * wv * BV;
  for (int idx = threadIdx.x; idx < nV; idx += blockDim.x) {
    const int j = idx % BV;
    int q = idx / BV;
    const int mm = q % wv;
    q /= wv;
    const int ph = q % BV, r = q / BV;
    const int k = (mm - g.nv + 1) * BV + j - ph;
    tabV[idx] = splat((k >= 0 && k < g.S) ? load_tap(a.table, a.tab_fmt, r * g.S + k) : 0.f);
  }
}

// Bytes of one record's values in the input format.
__device__ __forceinline__ int vis_record_bytes(const Args& a, int P) { return (a.vis_fmt == FMT_F32 ? 8 : 4) * P; }

// Whether batch [kb, kb + 32) can be bulk-copied: wholly inside the team's
// range, and every source 16-byte aligned (uv always is).
__device__ __forceinline__ bool lazy_bulk_ok(const Args& a, long long kb, long long vend, int vb) {
  if (kb + kRBL > vend) return false;
  const uintptr_t v = (uintptr_t)a.vis + (uintptr_t)(kb * vb);
  const uintptr_t w = a.weights ? (uintptr_t)(a.weights + kb) : 0;
  return ((v | w) & 15) == 0;
}

// One lane: the bulk copies of batch kb into raw buffer rb, completing on mbar.
__device__ __forceinline__ void lazy_issue(const Args& a, long long kb, unsigned char* rb, uint32_t mbar, int vb) {
  const uint32_t vbytes = (uint32_t)(kRBL * vb);
  mbar_expect(mbar, kRBL * 16 + vbytes + (a.weights ? kRBL * 4 : 0));
  bulk_load(smem_addr(rb), a.uv + kb, kRBL * 16, mbar);
  bulk_load(smem_addr(rb + kRBL * 20), (const char*)a.vis + kb * vb, vbytes, mbar);
  if (a.weights) bulk_load(smem_addr(rb + kRBL * 16), a.weights + kb, kRBL * 4, mbar);
}

// The lanes' copy of a batch that is not bulk-copied: records in range only.
template <int P>
__device__ __forceinline__ void lazy_load_lanes(const Args& a, long long kb, long long vend, unsigned char* rb, int l,
                                                int seg, int vb) {
  for (int r = l; r < kRBL; r += seg) {
    const long long k = kb + r;
    if (k >= vend) continue;
    ((double2*)rb)[r] = a.uv[k];
    if (a.weights) ((float*)(rb + kRBL * 16))[r] = a.weights[k];
    const uint32_t* src = (const uint32_t*)((const char*)a.vis + k * vb);
    uint32_t* dst = (uint32_t*)(rb + kRBL * 20 + r * vb);
    for (int i = 0; i < vb / 4; ++i) dst[i] = src[i];
  }
}

// Record r of a raw buffer, converted in place: the 16 bytes of its uv become
//   x = clamp lower bounds (hi - n + 1) as int16 pairs (u low, v high),
//   y = clamp upper bounds (lo),
//   z / w = table offsets with the footprint's first block removed (a thread
//           adds own_u*Bu / own_v*Bv),
// and its weighted values go to vals. A record outside the team's range or
// with an invalid footprint gets bounds that keep any box where it is, table
// offsets that clamp into the table, and zero values: it adds nothing.
template <int BU, int BV, int P>
__device__ __forceinline__ void lazy_convert(const Args& a, unsigned char* rb, int r, bool have, float2* vals) {
  const Geometry& g = a.g;
  int4 m = make_int4((int)kClampLoNone, (int)kClampHiNone, kOffNone, kOffNone);
  float2 val[P];
#pragma unroll
  for (int p = 0; p < P; ++p) val[p] = make_float2(0.f, 0.f);
  if (have) {
    const double2 x = ((const double2*)rb)[r];
    int Cu, ru, Cv, rv;
    bool ok = fine_cell(x.x, g.log2O, g.G >> 1, Cu, ru);
    ok = fine_cell(x.y, g.log2O, g.G >> 1, Cv, rv) && ok;
    const int cu0 = Cu - g.h, cv0 = Cv - g.h;
    ok = ok && cu0 >= 0 && cu0 + g.S <= g.G && cv0 >= 0 && cv0 + g.S <= g.G;
    if (ok) {
      const int lu = cu0 >> Log2B<BU>::value, pu = cu0 & (BU - 1), hu = (cu0 + g.S - 1) >> Log2B<BU>::value;
      const int lv = cv0 >> Log2B<BV>::value, pv = cv0 & (BV - 1), hv = (cv0 + g.S - 1) >> Log2B<BV>::value;
      const int Au = hu - g.nu + 1, Av = hv - g.nv + 1;
      m.x = (int)(((unsigned)Au & 0xFFFFu) | ((unsigned)Av << 16));
      m.y = (int)((unsigned)lu | ((unsigned)lv << 16));
      m.z = ((ru * BU + pu) * (2 * g.nu - 1) + g.nu - 1 - lu) * BU;
      m.w = ((rv * BV + pv) * (2 * g.nv - 1) + g.nv - 1 - lv) * BV;
      const float w = a.weights ? ((const float*)(rb + kRBL * 16))[r] : 1.f;
      VisWords<P> q;
      const uint32_t* src = (const uint32_t*)(rb + kRBL * 20 + r * vis_record_bytes(a, P));
      if (a.vis_fmt == FMT_F32) {
#pragma unroll
        for (int i = 0; i < 2 * P; ++i) q.w[i] = src[i];
      } else {
#pragma unroll
        for (int i = 0; i < P; ++i) q.w[i] = src[i];
      }
      vis_values<P>(a, q, w, val);
    } else {
      atomicAdd(a.skipped, 1ULL);
    }
  }
  ((int4*)rb)[r] = m;
#pragma unroll
  for (int p = 0; p < P; ++p) vals[p] = val[p];
}

// n consecutive pairs from 16-byte aligned shared memory (8-byte aligned if n is odd).
template <int N>
__device__ __forceinline__ void load_pairs(const float2* p, float2 (&v)[N]) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 2) {
      const float4 q = *(const float4*)(p + i);
      v[i] = make_float2(q.x, q.y);
      v[i + 1] = make_float2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = p[i];
  }
}

// The lazy-box gridder, chunked schedule: team t of CTA c grids visibilities
// [L*(c*teams + t), +L) in order (Sec. 4). a.g holds the widened bin (nu, nv,
// ts = nu*nv <= seg), a.seg the lanes per team slot (a power of two <= 32).
template <int BU, int BV, int P>
__global__ void grid_lazy_kernel(Args a) {
  static_assert(BU % 2 == 0, "a flush adds two cells per vector atomic");
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const int seg = a.seg;
  const int tpw = 32 / seg;
  const int teams = (int)(blockDim.x >> 5) * tpw;
  const LazyLayout L = lazy_layout<BU, BV, P>(g, teams);
  float2* const tabU = (float2*)(smem + L.tabU);
  float2* const tabV = (float2*)(smem + L.tabV);
  const int maxU = g.O * BU * (2 * g.nu - 1) * BU - BU;  // last table offset a thread may read from
  const int maxV = g.O * BV * (2 * g.nv - 1) * BV - BV;

  const int lane = threadIdx.x & 31;
  const int team = (int)(threadIdx.x >> 5) * tpw + lane / seg;
  const int l = lane & (seg - 1);
  const bool worker = l < g.ts;  // lanes past the team stage records but never flush
  const int au = worker ? l % g.nu : 0, av = worker ? l / g.nu : 0;
  unsigned char* const tb = smem + L.teams + (size_t)team * lazy_team_bytes(P);
  unsigned char* const raw0 = tb;
  unsigned char* const raw1 = tb + lazy_raw_bytes(P);
  float2* const vl = (float2*)(tb + 2 * lazy_raw_bytes(P));
  const uint32_t mbar0 = smem_addr(tb + 2 * lazy_raw_bytes(P) + kRBL * 8 * P);
  const uint32_t mbar1 = mbar0 + 8;
  const long long chunk = (long long)blockIdx.x * teams + team;
  const long long vbeg = chunk * a.chunk_len;
  const long long vend = chunk < a.n_chunks ? min(vbeg + a.chunk_len, a.n_vis) : vbeg;
  const int vb = vis_record_bytes(a, P);
  const int nb = (a.chunk_len + kRBL - 1) / kRBL;

  if (l == 0) {
    mbar_init(mbar0);
    mbar_init(mbar1);
    fence_mbar_init();
  }
  lazy_tables<BU, BV>(tabU, tabV, a);
  __syncthreads();  // tables and mbarriers ready
  uint32_t phase = 0;    // bit b: parity of raw buffer b's next completion
  uint32_t pending = 0;  // bit b: a bulk copy into raw buffer b is in flight
  bool failed = false;
  if (l == 0 && nb > 0 && lazy_bulk_ok(a, vbeg, vend, vb)) lazy_issue(a, vbeg, raw0, mbar0, vb);
  if (nb > 0 && lazy_bulk_ok(a, vbeg, vend, vb)) pending = 1;

  float2 acc[P][BV][BU];
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < BV; ++j)
#pragma unroll
      for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);
  unsigned box = kBoxNone;  // box origin in blocks, int16 pair (u low, v high)
  unsigned cur = kInvalid;  // the thread's block, u | v << 16
  int ownU = 0, ownV = 0;   // its first tap offsets in pairs: own_u*Bu, own_v*Bv

  // every team of the grid steps through the same number of batches (a short or empty chunk
  // stages invalid records), so the whole warp stays converged and syncs as one
  for (int bt = 0; bt < nb; ++bt) {
    const int b = bt & 1;
    unsigned char* const rb = b ? raw1 : raw0;
    const long long kb = vbeg + (long long)bt * kRBL;
    if ((pending >> b) & 1u) {
      if (!mbar_wait(b ? mbar1 : mbar0, (phase >> b) & 1u) && !failed) {
        failed = true;
        if (l == 0) atomicOr(a.status, 1u);
      }
      if (!failed) {
        phase ^= 1u << b;
        pending &= ~(1u << b);
      }
    } else if (!failed) {
      lazy_load_lanes<P>(a, kb, vend, rb, l, seg, vb);  // each lane converts what it loaded
    }
    // the next batch goes into the other raw buffer, free since its conversion ended last batch
    const long long kn = kb + kRBL;
    if (!failed && bt + 1 < nb && lazy_bulk_ok(a, kn, vend, vb)) {
      if (l == 0) {
        fence_proxy_async();
        lazy_issue(a, kn, b ? raw0 : raw1, b ? mbar0 : mbar1, vb);
      }
      pending |= 1u << (b ^ 1);
    }
    for (int r = l; r < kRBL; r += seg) lazy_convert<BU, BV, P>(a, rb, r, !failed && kb + r < vend, vl + r * P);
    __syncwarp();
    const int4* const mt = (const int4*)rb;
#pragma unroll 2
    for (int r = 0; r < kRBL; ++r) {
      const int4 m = mt[r];
      const unsigned nbox = __vmins2(__vmaxs2(box, (unsigned)m.x), (unsigned)m.y);
      if (nbox != box) {
        // the box moved: this thread's block changes only if the block it owned left the box
        box = nbox;
        const int bu = (int)(short)(box & 0xFFFFu), bv = (int)(short)(box >> 16);
        // (a - b) mod n with a < n <= 32 and 0 <= b < 2^15: shifted to a non-negative value below
        // 2^21, where the multiply-high division is exact
        const int pu = mod_small(au - bu + (g.nu << 15), g.nu, g.mu);
        const int pv = mod_small(av - bv + (g.nv << 15), g.nv, g.mv);
        const unsigned key = (unsigned)(bu + pu) | ((unsigned)(bv + pv) << 16);
        if (key != cur) {
          if (cur != kInvalid && worker) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
#pragma unroll
          for (int p = 0; p < P; ++p)
#pragma unroll
            for (int j = 0; j < BV; ++j)
#pragma unroll
              for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);
          cur = key;
          ownU = (bu + pu) * BU;
          ownV = (bv + pv) * BV;
        }
      }
      // taps as (t, t) pairs: Bu from the u table, Bv from the v table; each cell's tap
      // product is formed just before its P packed FMAs. An invalid record reads the
      // table's last entries and adds zero values.
      float2 tu[BU], tv[BV], V[P];
      load_pairs<BU>(tabU + min(m.z + ownU, maxU), tu);
      load_pairs<BV>(tabV + min(m.w + ownV, maxV), tv);
      load_pairs<P>(vl + r * P, V);
#pragma unroll
      for (int j = 0; j < BV; ++j)
#pragma unroll
        for (int i = 0; i < BU; ++i) {
          const float2 w2 = __fmul2_rn(tu[i], tv[j]);
#pragma unroll
          for (int p = 0; p < P; ++p) acc[p][j][i] = __ffma2_rn(w2, V[p], acc[p][j][i]);
        }
    }
    __syncwarp();
  }
  if (cur != kInvalid && worker && !failed) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
  // a batch given up on may still have a copy in flight into this CTA's shared memory
  if (failed) {
    if (pending & 1u) mbar_wait(mbar0, phase & 1u);
    if (pending & 2u) mbar_wait(mbar1, (phase >> 1) & 1u);
  }
}

struct LazyEntry {
  int bu, bv, p;
  const void* fn;
  size_t (*smem)(const Geometry&, int teams);
};

template <int BU, int BV, int P>
size_t lazy_smem_bytes(const Geometry& g, int teams) {
  return lazy_layout<BU, BV, P>(g, teams).total;
}

}  // namespace gbg
