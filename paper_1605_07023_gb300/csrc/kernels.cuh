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
constexpr int kRB = 16;   // records per team per staged batch (gridding)
constexpr int kRBD = 8;   // records per team per batch (degridding; bounded by the reduction buffer)

enum { FMT_F32 = 0, FMT_BF16 = 1, FMT_F16 = 2 };

struct Geometry {
  int G, S, O, log2O, h, P;
  int nbu, nbv;   // bin width in cells per axis
  int nu, nv;     // blocks per bin per axis
  int ts;         // team size nu*nv
  int tpc;        // teams per CTA
};

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

__device__ __forceinline__ float load_tap(const void* table, int fmt, int idx) {
  if (fmt == FMT_BF16) return __bfloat162float(((const __nv_bfloat16*)table)[idx]);
  if (fmt == FMT_F16) return __half2float(((const __half*)table)[idx]);
  return ((const float*)table)[idx];
}

// Zero-padded, phase-expanded 1-D tables: tab[(r*B + rem)*nb + k] = T[r][k - rem]
// for 0 <= k - rem < S, else 0. A thread at block position t reads taps
// tab[(r*B + rem)*nb + t*B + i], i < B.
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

// Per-visibility record: meta = {qu | qv<<16, rqu | rqv<<16, table offset u, table offset v}.
//  - q: block index of the box origin (footprint start / B).
//  - rq: q mod n, the thread position that holds the box's first block.
//  - table offsets select (row, phase) in the padded tables.
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
  const int rqu = qu % g.nu, rqv = qv % g.nv;
  meta = make_int4(qu | (qv << 16), rqu | (rqv << 16), (ru * BU + remu) * g.nbu, (rv * BV + remv) * g.nbv);
  return true;
}

template <int P>
__device__ __forceinline__ void load_vis(const Args& a, long long k, float w, float2 (&val)[P]) {
  if (a.vis_fmt == FMT_F32) {
    const float2* src = (const float2*)a.vis + k * P;
    if constexpr (P % 2 == 0) {
#pragma unroll
      for (int p = 0; p < P; p += 2) {
        const float4 q = *(const float4*)(src + p);
        val[p] = make_float2(q.x * w, q.y * w);
        val[p + 1] = make_float2(q.z * w, q.w * w);
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float2 q = src[p];
        val[p] = make_float2(q.x * w, q.y * w);
      }
    }
  } else {
    // 16-bit pairs: P complex values = P 32-bit words
    const uint32_t* src = (const uint32_t*)a.vis + k * P;
    uint32_t wds[P];
    if constexpr (P == 4) {
      const uint4 q = *(const uint4*)src;
      wds[0] = q.x; wds[1] = q.y; wds[2] = q.z; wds[3] = q.w;
    } else if constexpr (P == 2) {
      const uint2 q = *(const uint2*)src;
      wds[0] = q.x; wds[1] = q.y;
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) wds[p] = src[p];
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
      float2 f;
      if (a.vis_fmt == FMT_BF16) {
        __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&wds[p]);
        f = __bfloat1622float2(b);
      } else {
        __half2 hh = *reinterpret_cast<const __half2*>(&wds[p]);
        f = __half22float2(hh);
      }
      val[p] = make_float2(f.x * w, f.y * w);
    }
  }
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

// Flush one block of register accumulators to the grid in global memory with
// vector atomic adds, then zero them. Cells past the grid's high edge (the
// box can overhang it) hold exact zeros and are not written. All-zero
// vectors are skipped.
template <int BU, int BV, int P>
__device__ __forceinline__ void flush_global(float2 (&acc)[P][BV][BU], unsigned key, float2* __restrict__ grid, int G) {
  const int u0 = (int)(key & 0xFFFFu) * BU;
  const int v0 = (int)(key >> 16) * BV;
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int v = v0 + j;
      float2* row = grid + ((size_t)p * G + v) * G + u0;
      if constexpr (BU % 2 == 0) {
#pragma unroll
        for (int i = 0; i < BU; i += 2) {
          const float4 q = make_float4(acc[p][j][i].x, acc[p][j][i].y, acc[p][j][i + 1].x, acc[p][j][i + 1].y);
          const bool nz = (q.x != 0.f) | (q.y != 0.f) | (q.z != 0.f) | (q.w != 0.f);
          if (nz && v < G && u0 + i + 1 < G) atomicAdd((float4*)(row + i), q);
        }
      } else {
#pragma unroll
        for (int i = 0; i < BU; ++i) {
          const float2 q = acc[p][j][i];
          const bool nz = (q.x != 0.f) | (q.y != 0.f);
          if (nz && v < G && u0 + i < G) atomicAdd(row + i, q);
        }
      }
#pragma unroll
      for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);
    }
  }
}

// Shared-memory patch flush: the block lies inside the CTA's window
// [wu0, wu0+win) x [wv0, wv0+win). Window layout: [P][win] rows of
// win_stride(win) = 2*win + 1 floats (interleaved re, im). The odd stride
// puts the rows that different threads flush at once in different banks.
__host__ __device__ inline int win_stride(int win) { return 2 * win + 1; }

template <int BU, int BV, int P>
__device__ __forceinline__ void flush_window(float2 (&acc)[P][BV][BU], int lu, int lv, float* __restrict__ win_buf, int win) {
  const int ws = win_stride(win);
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      float* row = win_buf + ((size_t)p * win + lv + j) * ws + 2 * lu;
#pragma unroll
      for (int i = 0; i < BU; ++i) {
        const float2 q = acc[p][j][i];
        if (q.x != 0.f) atomicAdd(row + 2 * i, q.x);
        if (q.y != 0.f) atomicAdd(row + 2 * i + 1, q.y);
        acc[p][j][i] = make_float2(0.f, 0.f);
      }
    }
  }
}

template <int BU, int BV, int P>
__device__ __forceinline__ void flush_any(float2 (&acc)[P][BV][BU], unsigned key, float2* grid, int G, float* win_buf, int win,
                                          int wu0, int wv0) {
  if (key == kInvalid) return;
  if (win > 0) {
    const int lu = (int)(key & 0xFFFFu) * BU - wu0;
    const int lv = (int)(key >> 16) * BV - wv0;
    if (lu >= 0 && lv >= 0 && lu + BU <= win && lv + BV <= win) {
      flush_window<BU, BV, P>(acc, lu, lv, win_buf, win);
      return;
    }
  }
  flush_global<BU, BV, P>(acc, key, grid, G);
}

template <int BU, int BV>
__host__ __device__ constexpr int tab_floats_align() { return 4; }

// Shared-memory layout helpers (bytes, 16-aligned).
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <int BU, int BV, int P>
__host__ __device__ inline size_t grid_smem_tables(const Geometry& g) {
  return align16((size_t)g.O * BU * g.nbu * 4) + align16((size_t)g.O * BV * g.nbv * 4);
}

template <int BU, int BV, int P>
__host__ __device__ inline size_t grid_smem_records(const Geometry& g) {
  // two buffers x teams x kRB x (meta + P values)
  return 2 * (size_t)g.tpc * kRB * (16 + 8 * P);
}

// ---------------------------------------------------------------------------
// The team's per-visibility step (shared by both schedules).
template <int BU, int BV, int P>
__device__ __forceinline__ void grid_step(const int4 m, const float2* __restrict__ vals, int au, int av, const Geometry& g,
                                          const float* __restrict__ tabU, const float* __restrict__ tabV,
                                          float2 (&acc)[P][BV][BU], unsigned& cur, float2* grid, float* win_buf, int win,
                                          int wu0, int wv0) {
  if (m.x == (int)kInvalid) return;
  const int qu = m.x & 0xFFFF, qv = (int)((unsigned)m.x >> 16);
  const int rqu = m.y & 0xFFFF, rqv = (int)((unsigned)m.y >> 16);
  int tu = au - rqu;
  tu += (tu < 0) ? g.nu : 0;
  int tv = av - rqv;
  tv += (tv < 0) ? g.nv : 0;
  const unsigned key = (unsigned)(qu + tu) | ((unsigned)(qv + tv) << 16);
  if (key != cur) {
    flush_any<BU, BV, P>(acc, cur, grid, g.G, win_buf, win, wu0, wv0);
    cur = key;
  }
  float wu[BU], wv[BV];
  load_taps<BU>(tabU + m.z + tu * BU, wu);
  load_taps<BV>(tabV + m.w + tv * BV, wv);
  float2 V[P];
#pragma unroll
  for (int p = 0; p < P; ++p) V[p] = vals[p];
#pragma unroll
  for (int j = 0; j < BV; ++j) {
#pragma unroll
    for (int i = 0; i < BU; ++i) {
      const float w = wu[i] * wv[j];
      const float2 w2 = make_float2(w, w);
#pragma unroll
      for (int p = 0; p < P; ++p) acc[p][j][i] = __ffma2_rn(w2, V[p], acc[p][j][i]);
    }
  }
}

// Stage batch b of a team's chunk into shared memory: each team thread loads
// records l, l+ts, ... of the batch (Sec. 4: "each work-item loads one
// visibility").
template <int BU, int BV, int P>
__device__ __forceinline__ void stage_batch(const Args& a, long long vbeg, long long vend, int b, int l, int4* meta,
                                            float2* vals) {
  const Geometry& g = a.g;
  for (int r = l; r < kRB; r += g.ts) {
    const long long k = vbeg + (long long)b * kRB + r;
    int4 m;
    m.x = (int)kInvalid;
    float2 val[P];
    if (k < vend) {
      if (make_meta<BU, BV>(a, a.uv[k], m)) {
        const float w = a.weights ? a.weights[k] : 1.f;
        load_vis<P>(a, k, w, val);
      } else {
        atomicAdd(a.skipped, 1ULL);
      }
    }
    meta[r] = m;
    if (m.x != (int)kInvalid) {
#pragma unroll
      for (int p = 0; p < P; ++p) vals[r * P + p] = val[p];
    }
  }
}

// ---------------------------------------------------------------------------
// Gridding kernel. The chunked schedule (win == 0) gives one chunk per team
// with flushes to global memory (Sec. 4). The patch schedule (win > 0) uses
// persistent CTAs that take work items (one patch plus a range of its
// chunks), accumulate the patch window in shared memory and add it to the
// grid at the end of each item.
template <int BU, int BV, int P>
__global__ void grid_kernel(Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  float* tabU = (float*)smem;
  float* tabV = (float*)(smem + align16((size_t)g.O * BU * g.nbu * 4));
  unsigned char* rec = smem + grid_smem_tables<BU, BV, P>(g);
  int4* meta0 = (int4*)rec;
  int4* meta1 = meta0 + g.tpc * kRB;
  float2* vals0 = (float2*)(meta1 + g.tpc * kRB);
  float2* vals1 = vals0 + (size_t)g.tpc * kRB * P;
  float* win_buf = (float*)(vals1 + (size_t)g.tpc * kRB * P);

  build_table<BU>(tabU, a, g.nbu);
  build_table<BV>(tabV, a, g.nbv);

  const int team = threadIdx.x / g.ts;
  const int l = threadIdx.x - team * g.ts;
  const bool active = team < g.tpc;
  const int au = l % g.nu, av = l / g.nu;
  const int nb = (a.chunk_len + kRB - 1) / kRB;

  float2 acc[P][BV][BU];
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < BV; ++j)
#pragma unroll
      for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);

  if (a.win == 0) {
    // ---- chunked schedule: one chunk per team
    const long long chunk = (long long)blockIdx.x * g.tpc + team;
    const long long vbeg = chunk * a.chunk_len;
    const long long vend = (active && chunk < a.n_chunks) ? min(vbeg + a.chunk_len, a.n_vis) : vbeg;
    int4* mt = meta0 + team * kRB;
    float2* vl = vals0 + (size_t)team * kRB * P;
    __syncthreads();  // tables ready
    unsigned cur = kInvalid;
    for (int b = 0; b < nb; ++b) {
      int4* mtb = (b & 1) ? mt + g.tpc * kRB : mt;
      float2* vlb = (b & 1) ? vl + (size_t)g.tpc * kRB * P : vl;
      if (active) stage_batch<BU, BV, P>(a, vbeg, vend, b, l, mtb, vlb);
      __syncthreads();
      if (active) {
#pragma unroll 1
        for (int r = 0; r < kRB; ++r) {
          const int4 m = mtb[r];
          grid_step<BU, BV, P>(m, vlb + r * P, au, av, g, tabU, tabV, acc, cur, a.grid, nullptr, 0, 0, 0);
        }
      }
    }
    if (active) flush_global<BU, BV, P>(acc, cur, a.grid, g.G);
    return;
  }

  // ---- patch schedule
  __shared__ int s_item;
  const int win = a.win;
  const int ws = win_stride(win);
  const int win_floats = P * win * ws;
  const int n_work = *a.n_work;
  for (;;) {
    __syncthreads();  // previous item fully flushed; tables ready on the first pass
    if (threadIdx.x == 0) s_item = atomicAdd(a.work_next, 1);
    for (int i = threadIdx.x; i < win_floats; i += blockDim.x) win_buf[i] = 0.f;
    __syncthreads();
    const int item = s_item;
    if (item >= n_work) break;
    const int4 wk = a.work[item];
    const int wu0 = wk.x, wv0 = wk.y;
    // teams take the item's chunks round-robin, all in lockstep batches
    const int n_item_chunks = wk.w - wk.z;
    const int rounds = (n_item_chunks + g.tpc - 1) / g.tpc;
    int4* mt = meta0 + team * kRB;
    float2* vl = vals0 + (size_t)team * kRB * P;
    for (int rd = 0; rd < rounds; ++rd) {
      const int ci = rd * g.tpc + team;
      long long vbeg = 0, vend = 0;
      if (active && ci < n_item_chunks) {
        const long long chunk = a.chunk_order[wk.z + ci];
        vbeg = chunk * a.chunk_len;
        vend = min(vbeg + a.chunk_len, a.n_vis);
      }
      unsigned cur = kInvalid;
      for (int b = 0; b < nb; ++b) {
        int4* mtb = (b & 1) ? mt + g.tpc * kRB : mt;
        float2* vlb = (b & 1) ? vl + (size_t)g.tpc * kRB * P : vl;
        if (active) stage_batch<BU, BV, P>(a, vbeg, vend, b, l, mtb, vlb);
        __syncthreads();
        if (active) {
#pragma unroll 1
          for (int r = 0; r < kRB; ++r) {
            const int4 m = mtb[r];
            grid_step<BU, BV, P>(m, vlb + r * P, au, av, g, tabU, tabV, acc, cur, a.grid, win_buf, win, wu0, wv0);
          }
        }
      }
      if (active) flush_any<BU, BV, P>(acc, cur, a.grid, g.G, win_buf, win, wu0, wv0);
    }
    __syncthreads();
    // add the window to the grid: coalesced float4 atomics, all-zero vectors skipped
    const int rowf4 = win / 2;  // float4 (two cells) per window row (win even)
    const int total = P * win * rowf4;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      const int c4 = i % rowf4;
      const int rowi = i / rowf4;
      const int vv = rowi % win;
      const int p = rowi / win;
      const int gu = wu0 + 2 * c4, gv = wv0 + vv;
      const float* src = win_buf + (size_t)rowi * ws + 4 * c4;
      const float4 q = make_float4(src[0], src[1], src[2], src[3]);
      const bool nz = (q.x != 0.f) | (q.y != 0.f) | (q.z != 0.f) | (q.w != 0.f);
      if (nz && gu >= 0 && gv >= 0 && gu + 1 < g.G && gv < g.G)
        atomicAdd((float4*)(a.grid + ((size_t)p * g.G + gv) * g.G + gu), q);
    }
  }
}

// ---------------------------------------------------------------------------
// Degridding: the adjoint. Each thread keeps the grid values of its current
// block in registers and reloads them only when the box moves (the read-side
// analogue of a flush). Per visibility it forms P complex partial sums over
// its block. The team reduces them through shared memory: each thread stores
// its partials, then each thread sums one column of (record, component)
// outputs.
template <int BU, int BV, int P>
__device__ __forceinline__ void load_block(float2 (&gb)[P][BV][BU], unsigned key, const float2* __restrict__ grid, int G) {
  const int u0 = (int)(key & 0xFFFFu) * BU;
  const int v0 = (int)(key >> 16) * BV;
#pragma unroll
  for (int p = 0; p < P; ++p) {
#pragma unroll
    for (int j = 0; j < BV; ++j) {
      const int v = v0 + j;
      const float2* row = grid + ((size_t)p * G + v) * G + u0;
      if constexpr (BU % 2 == 0) {
#pragma unroll
        for (int i = 0; i < BU; i += 2) {
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          if (v < G && u0 + i + 1 < G) q = __ldg((const float4*)(row + i));
          gb[p][j][i] = make_float2(q.x, q.y);
          gb[p][j][i + 1] = make_float2(q.z, q.w);
        }
      } else {
#pragma unroll
        for (int i = 0; i < BU; ++i) {
          float2 q = make_float2(0.f, 0.f);
          if (v < G && u0 + i < G) q = __ldg(row + i);
          gb[p][j][i] = q;
        }
      }
    }
  }
}

template <int BU, int BV, int P>
__host__ __device__ inline size_t degrid_smem_bytes(const Geometry& g) {
  const int tsp = g.ts | 1;
  return grid_smem_tables<BU, BV, P>(g) + (size_t)g.tpc * kRBD * 16 + align16((size_t)g.tpc * kRBD * 2 * P * tsp * 4);
}

template <int BU, int BV, int P>
__global__ void degrid_kernel(Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  float* tabU = (float*)smem;
  float* tabV = (float*)(smem + align16((size_t)g.O * BU * g.nbu * 4));
  int4* meta_all = (int4*)(smem + grid_smem_tables<BU, BV, P>(g));
  float* red_all = (float*)(meta_all + g.tpc * kRBD);
  const int tsp = g.ts | 1;

  build_table<BU>(tabU, a, g.nbu);
  build_table<BV>(tabV, a, g.nbv);

  const int team = threadIdx.x / g.ts;
  const int l = threadIdx.x - team * g.ts;
  const bool active = team < g.tpc;
  const int au = l % g.nu, av = l / g.nu;
  const long long chunk = (long long)blockIdx.x * g.tpc + team;
  const long long vbeg = chunk * a.chunk_len;
  const long long vend = (active && chunk < a.n_chunks) ? min(vbeg + a.chunk_len, a.n_vis) : vbeg;
  int4* mt = meta_all + team * kRBD;
  float* red = red_all + (size_t)team * kRBD * 2 * P * tsp;
  const int nb = (a.chunk_len + kRBD - 1) / kRBD;

  float2 gb[P][BV][BU];
  unsigned cur = kInvalid;
  __syncthreads();
  for (int b = 0; b < nb; ++b) {
    if (active) {
      for (int r = l; r < kRBD; r += g.ts) {
        const long long k = vbeg + (long long)b * kRBD + r;
        int4 m;
        m.x = (int)kInvalid;
        if (k < vend && !make_meta<BU, BV>(a, a.uv[k], m)) atomicAdd(a.skipped, 1ULL);
        mt[r] = m;
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll 1
      for (int r = 0; r < kRBD; ++r) {
        const int4 m = mt[r];
        float2 s[P];
#pragma unroll
        for (int p = 0; p < P; ++p) s[p] = make_float2(0.f, 0.f);
        if (m.x != (int)kInvalid) {
          const int qu = m.x & 0xFFFF, qv = (int)((unsigned)m.x >> 16);
          const int rqu = m.y & 0xFFFF, rqv = (int)((unsigned)m.y >> 16);
          int tu = au - rqu;
          tu += (tu < 0) ? g.nu : 0;
          int tv = av - rqv;
          tv += (tv < 0) ? g.nv : 0;
          const unsigned key = (unsigned)(qu + tu) | ((unsigned)(qv + tv) << 16);
          if (key != cur) {
            load_block<BU, BV, P>(gb, key, a.grid, g.G);
            cur = key;
          }
          float wu[BU], wv[BV];
          load_taps<BU>(tabU + m.z + tu * BU, wu);
          load_taps<BV>(tabV + m.w + tv * BV, wv);
#pragma unroll
          for (int j = 0; j < BV; ++j) {
#pragma unroll
            for (int i = 0; i < BU; ++i) {
              const float w = wu[i] * wv[j];
              const float2 w2 = make_float2(w, w);
#pragma unroll
              for (int p = 0; p < P; ++p) s[p] = __ffma2_rn(w2, gb[p][j][i], s[p]);
            }
          }
        }
#pragma unroll
        for (int p = 0; p < P; ++p) {
          red[(r * 2 * P + 2 * p) * tsp + l] = s[p].x;
          red[(r * 2 * P + 2 * p + 1) * tsp + l] = s[p].y;
        }
      }
    }
    __syncthreads();
    if (active) {
      // each team thread sums whole columns: output o = (record, component)
      for (int o = l; o < kRBD * 2 * P; o += g.ts) {
        const int r = o / (2 * P);
        const long long k = vbeg + (long long)b * kRBD + r;
        if (k < vend) {
          const float* col = red + (size_t)o * tsp;
          float sum = 0.f;
          for (int t = 0; t < g.ts; ++t) sum += col[t];
          if (a.weights) sum *= a.weights[k];
          ((float*)a.vis_out)[k * 2 * P + (o - r * 2 * P)] = sum;
        }
      }
    }
    __syncthreads();
  }
}

// Function table entry for one (Bu, Bv, P) instantiation.
struct KernelEntry {
  int bu, bv, p;
  const void* grid_fn;
  const void* degrid_fn;
};

}  // namespace gbg
