// Device code of the tile-gather degridder (see degrid_tile.cu for the
// schedule). Included by the translation units that instantiate its kernels:
// degrid_tile.cu (one lane per visibility, groups of 32) and degrid_tile_q.cu
// (four lanes per visibility, groups of 8).
#pragma once

#include <cuda.h>

#include "kernels.cuh"
#include "internal.h"

namespace gbg {
namespace {

// The smallest even row stride >= w cells that is 6 or 10 mod 16.
__host__ __device__ constexpr int spread_stride(int w) {
  while (w % 16 != 6 && w % 16 != 10) ++w;
  return w;
}

// Tile side in cells. With one lane per visibility, the box of 32 consecutive
// visibilities on a baseline track fits unless the track is fast (a larger
// tile measured faster than S + 9, whose misses cost more than the lost
// occupancy). Groups of 8 are for fast tracks: S + 21 holds 93% of them on
// the S=15 precision workload, against 68% for S + 13.
__host__ __device__ constexpr int tile_side(int S, int lpv) { return S + (lpv == 1 ? 13 : 21); }

// Plane stride in cells for row stride rs: a multiple of 16 (128 bytes), the
// alignment of a tensor copy's destination.
__host__ __device__ constexpr int tile_plane(int S, int lpv, int rs) { return (tile_side(S, lpv) * rs + 15) / 16 * 16; }

template <int S, int P, int LPV>
struct TileShape {
  static constexpr int TW = tile_side(S, LPV);
  // Row stride in cells. It is even, so that rows start on 16-byte boundaries
  // (the box is copied in 16-byte pieces). A cell is two 4-byte banks, so cell
  // (row, col) starts at bank pair (RS*row + col) mod 16; with RS = 6 or 10
  // mod 16, lanes whose footprints are a cell or two apart in any direction
  // read different banks (a stride of TW + 1 = 1 mod 16 made every pair one
  // cell apart along a diagonal collide).
  static constexpr int RS = spread_stride(TW);
  static constexpr int PS = tile_plane(S, LPV, RS);
  static constexpr int CELLS = P * PS;  // complex cells per warp
};

// Box heights of the three tensor maps: the smallest that holds a group's rows
// is used (a group of 32 baseline-ordered visibilities usually spans a few
// rows more than S).
__host__ __device__ constexpr int tile_height(int S, int lpv, int i) {
  return i == 2 ? tile_side(S, lpv) : lpv == 1 ? (i == 0 ? S + 3 : S + 7) : (i == 0 ? S + 5 : S + 11);
}

__device__ __forceinline__ void tensor_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(z), "r"(mbar) : "memory");
}

// s_p for one visibility whose footprint starts at base (cell (x0, y0) of
// plane 0), with rows RSTRIDE and planes PSTRIDE cells apart.
template <int S, int P, typename Ptr, typename Stride>
__device__ __forceinline__ void footprint_dot(Ptr base, Stride rstride, Stride pstride, const float (&tu)[S],
                                              const float (&tv)[S], float2 (&s)[P]) {
#pragma unroll
  for (int j = 0; j < S; ++j) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const Ptr row = base + (Stride)p * pstride + (Stride)j * rstride;
      float2 r = __fmul2_rn(splat(tu[0]), row[0]);
#pragma unroll
      for (int i = 1; i < S; ++i) r = __ffma2_rn(splat(tu[i]), row[i], r);
      s[p] = j == 0 ? __fmul2_rn(splat(tv[0]), r) : __ffma2_rn(splat(tv[j]), r, s[p]);
    }
  }
}

// The part of those sums over the footprint rows q, q + LPV, ... (nrows of
// them): base points at row q, rstride is LPV rows, tv holds the rows' v taps.
// s must be zero on entry.
template <int S, int P, int ROWS, typename Ptr, typename Stride>
__device__ __forceinline__ void footprint_rows(Ptr base, Stride rstride, Stride pstride, const float (&tu)[S],
                                               const float (&tv)[ROWS], int nrows, float2 (&s)[P]) {
#pragma unroll
  for (int jj = 0; jj < ROWS; ++jj) {
    if (jj < nrows) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const Ptr row = base + (Stride)p * pstride + (Stride)jj * rstride;
        float2 r = __fmul2_rn(splat(tu[0]), row[0]);
#pragma unroll
        for (int i = 1; i < S; ++i) r = __ffma2_rn(splat(tu[i]), row[i], r);
        s[p] = __ffma2_rn(splat(tv[jj]), r, s[p]);
      }
    }
  }
}

// The same sums for a support known only at run time, with the taps read
// from the shared-memory table (tu: the visibility's u row; tv: its v taps
// for the rows summed here, tvs apart), each u tap once per row for all P
// planes. Rows: nrows of them from base, rstride apart. s must be zero on
// entry.
template <int P, typename Ptr, typename Stride>
__device__ __forceinline__ void footprint_dot_any(Ptr base, Stride rstride, Stride pstride, const float* tu,
                                                  const float* tv, int tvs, int nrows, int S, float2 (&s)[P]) {
#pragma unroll 1
  for (int j = 0; j < nrows; ++j) {
    const Ptr row = base + (Stride)j * rstride;
    float2 r[P];
#pragma unroll
    for (int p = 0; p < P; ++p) r[p] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int i = 0; i < S; ++i) {
      const float2 t = splat(tu[i]);
#pragma unroll
      for (int p = 0; p < P; ++p) r[p] = __ffma2_rn(t, row[(Stride)p * pstride + i], r[p]);
    }
    const float2 t = splat(tv[j * tvs]);
#pragma unroll
    for (int p = 0; p < P; ++p) s[p] = __ffma2_rn(t, r[p], s[p]);
  }
}

// The direct paths for a group whose box does not fit the tile: kept out
// of line so that they add no registers to the tile path.
template <int S, int P>
__device__ __noinline__ void footprint_dot_global(const float2* base, int G, const float (&tu)[S],
                                                  const float (&tv)[S], float2 (&s)[P]) {
  footprint_dot<S, P>(base, (size_t)G, (size_t)G * G, tu, tv, s);
}

template <int S, int P, int ROWS>
__device__ __noinline__ void footprint_rows_global(const float2* base, size_t rstride, size_t pstride,
                                                   const float (&tu)[S], const float (&tv)[ROWS], int nrows,
                                                   float2 (&s)[P]) {
  footprint_rows<S, P, ROWS>(base, rstride, pstride, tu, tv, nrows, s);
}

template <int P>
__device__ __noinline__ void footprint_dot_global_any(const float2* base, size_t rstride, size_t pstride,
                                                      const float* tu, const float* tv, int tvs, int nrows, int S,
                                                      float2 (&s)[P]) {
  footprint_dot_any<P>(base, rstride, pstride, tu, tv, tvs, nrows, S, s);
}

// SC > 0: support SC, fully unrolled, taps in registers. SC = 0: the plan's
// support (any S), taps read from the shared-memory table.
// LPV lanes per visibility: 1 (a warp group of 32 visibilities) or 4 (a group
// of 8; lane q of a visibility's four sums its footprint rows q, q + 4, ...
// and the four partial sums are added by shuffles).
template <int SC, int P, int LPV>
__global__ void degrid_tile_kernel(Args a, const __grid_constant__ TileMaps maps) {
  static_assert(LPV == 1 || LPV == 4, "one or four lanes per visibility");
  constexpr int GS = 32 / LPV;                             // visibilities per group
  constexpr int ROWS = SC > 0 ? (SC + LPV - 1) / LPV : 1;  // footprint rows per lane (unrolled kernels)
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const int S = SC > 0 ? SC : g.S;
  const int TW = SC > 0 ? TileShape<SC, P, LPV>::TW : tile_side(S, LPV);
  const int RS = SC > 0 ? TileShape<SC, P, LPV>::RS : spread_stride(TW);
  const int PS = SC > 0 ? TileShape<SC, P, LPV>::PS : tile_plane(S, LPV, RS);
  const int CELLS = P * PS;
  float* tab = (float*)smem;
  const int ntab = g.O * S;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) tab[i] = load_tap(a.table, a.tab_fmt, i);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int vi = lane / LPV, q = lane % LPV;  // the lane's visibility in its group, and its row phase
  const int nrows = (S - q + LPV - 1) / LPV;  // footprint rows this lane sums
  // the tiles start on a 128-byte boundary (the host adds 128 bytes of slack)
  const uint32_t tiles0 = (smem_addr(smem) + (uint32_t)align16((size_t)ntab * 4) + 127u) & ~127u;
  unsigned char* const tiles = smem + (tiles0 - smem_addr(smem));
  float2* tile = (float2*)tiles + (size_t)warp * CELLS;
  // one mbarrier per warp, after all the tiles
  const uint32_t mbar = tiles0 + (uint32_t)((blockDim.x >> 5) * CELLS * sizeof(float2)) + 8u * warp;
  if (lane == 0) {
    mbar_init(mbar);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t phase = 0;   // parity of the mbarrier's next completion
  bool failed = false;  // a copy did not complete in time: later groups read the grid directly

  const int G = g.G;
  const long long n_groups = (a.n_vis + GS - 1) / GS;
  const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
  // Persistent warps: the position of the next group's visibility is loaded
  // one group ahead, so its memory latency overlaps the current group.
  long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  double2 xn = make_double2(0.0, 0.0);
  if (c < n_groups && c * GS + vi < a.n_vis) xn = ld_stream(a.uv + c * GS + vi);
  for (; c < n_groups; c += stride) {
    const long long k = c * GS + vi;
    const double2 x = xn;
    if (c + stride < n_groups && (c + stride) * GS + vi < a.n_vis) xn = ld_stream(a.uv + (c + stride) * GS + vi);
    int x0 = 0, y0 = 0, ru = 0, rv = 0;
    bool ok = false;
    if (k < a.n_vis) {
      int Cu, Cv;
      ok = fine_cell(x.x, g.log2O, G >> 1, Cu, ru);
      ok = fine_cell(x.y, g.log2O, G >> 1, Cv, rv) && ok;
      x0 = Cu - g.h;
      y0 = Cv - g.h;
      ok = ok && x0 >= 0 && x0 + S <= G && y0 >= 0 && y0 + S <= G;
      if (!ok && q == 0) atomicAdd(a.skipped, 1ULL);
    }
    float2 s[P];
#pragma unroll
    for (int p = 0; p < P; ++p) s[p] = make_float2(0.f, 0.f);
    // u taps: the whole row; v taps: this lane's rows
    float tu[SC > 0 ? SC : 1], tv[SC > 0 ? ROWS : 1];
    if constexpr (SC > 0) {
#pragma unroll
      for (int i = 0; i < SC; ++i) tu[i] = tab[ru * SC + i];
#pragma unroll
      for (int jj = 0; jj < ROWS; ++jj) tv[jj] = (LPV == 1 || jj < nrows) ? tab[rv * SC + q + jj * LPV] : 0.f;
    }
    const int xmin = __reduce_min_sync(0xFFFFFFFFu, ok ? x0 : 0x7FFFFFFF);
    const int ymin = __reduce_min_sync(0xFFFFFFFFu, ok ? y0 : 0x7FFFFFFF);
    const int xmax = __reduce_max_sync(0xFFFFFFFFu, ok ? x0 : -1);
    const int ymax = __reduce_max_sync(0xFFFFFFFFu, ok ? y0 : -1);
    if (xmax >= 0) {
      // The box starts at an even column, so that each row is whole 16-byte
      // cell pairs (G is even and the grid 16-byte aligned); it lies inside
      // the grid (a union of valid footprints, widened by at most one cell at
      // each end of a row; the right end is checked).
      const int xe = xmin & ~1;                    // first column of the copy
      const int npair = (xmax + S - xe + 1) >> 1;  // cell pairs per row
      const int sy = ymax - ymin + S;
      if (!failed && maps.ok && 2 * npair <= TW && sy <= TW) {
        // One tensor copy per plane of an RS x H box from (xe, ymin); the last group's reads of
        // the tile are ordered before these writes (syncwarp, then a proxy fence in every
        // issuing lane), and lane 0 announces the byte count first.
        const int mi = sy <= maps.h[0] ? 0 : (sy <= maps.h[1] ? 1 : 2);
        if (lane == 0) mbar_expect(mbar, (uint32_t)(P * maps.h[mi] * RS) * 8u);
        __syncwarp();
        if (lane < P) {
          fence_proxy_async();
          tensor_load_3d(smem_addr(tile + lane * PS), &maps.m[mi], 2 * xe, ymin, lane, mbar);
        }
        if (!mbar_wait(mbar, phase)) {
          failed = true;
          if (lane == 0 && a.status) atomicOr(a.status, 1u);
        }
        phase ^= 1u;
        __syncwarp();
        if (ok && !failed) {
          const float2* base = (const float2*)tile + (y0 - ymin + q) * RS + (x0 - xe);
          if constexpr (SC > 0 && LPV == 1) footprint_dot<SC, P>(base, RS, PS, tu, tv, s);
          else if constexpr (SC > 0) footprint_rows<SC, P, ROWS>(base, RS * LPV, PS, tu, tv, nrows, s);
          else footprint_dot_any<P>(base, RS * LPV, PS, tab + ru * S, tab + rv * S + q, LPV, nrows, S, s);
        }
        __syncwarp();  // the tile is refilled for the next group
      } else if (ok) {
        const float2* base = (const float2*)a.grid + (size_t)(y0 + q) * G + x0;
        if constexpr (SC > 0 && LPV == 1) footprint_dot_global<SC, P>(base, G, tu, tv, s);
        else if constexpr (SC > 0) footprint_rows_global<SC, P, ROWS>(base, (size_t)G * LPV, (size_t)G * G, tu, tv, nrows, s);
        else footprint_dot_global_any<P>(base, (size_t)G * LPV, (size_t)G * G, tab + ru * S, tab + rv * S + q, LPV, nrows, S, s);
      }
    }
    if constexpr (LPV > 1) {
      // every lane is here (xmax is the warp's): add the partial sums of a visibility's lanes
#pragma unroll
      for (int o = 1; o < LPV; o <<= 1)
#pragma unroll
        for (int p = 0; p < P; ++p) {
          s[p].x += __shfl_xor_sync(0xFFFFFFFFu, s[p].x, o);
          s[p].y += __shfl_xor_sync(0xFFFFFFFFu, s[p].y, o);
        }
    }
    if (k < a.n_vis && q == 0) {
      const float w = (a.weights && ok) ? a.weights[k] : 1.f;
      float2* out = a.vis_out + k * P;
#pragma unroll
      for (int p = 0; p < P; ++p) __stcs(out + p, make_float2(s[p].x * w, s[p].y * w));
    }
  }
  // a copy given up on may still be landing in this CTA's shared memory
  if (failed) mbar_wait(mbar, phase ^ 1u);
}

template <int S, int P, int LPV>
TileKernel tile_entry() {
  return TileKernel{S, P, LPV, (const void*)&degrid_tile_kernel<S, P, LPV>, TileShape<S, P, LPV>::CELLS,
                    TileShape<S, P, LPV>::RS,
                    {tile_height(S, LPV, 0), tile_height(S, LPV, 1), tile_height(S, LPV, 2)}};
}

#define GB_TILE_ROW(P, LPV)                                                                                  \
  tile_entry<1, P, LPV>(), tile_entry<3, P, LPV>(), tile_entry<5, P, LPV>(), tile_entry<7, P, LPV>(),     \
      tile_entry<9, P, LPV>(), tile_entry<11, P, LPV>(), tile_entry<13, P, LPV>(), tile_entry<15, P, LPV>()

}  // namespace
}  // namespace gbg
