// Degridding by tile gather: a second schedule for the adjoint of gridding.
//
// The sliding-window degridder mirrors the gridder: each thread keeps one
// block of grid values in registers and a team reduces its partial sums
// through shared memory for every visibility. Here each warp instead takes
// 32 consecutive visibilities (one per lane). Consecutive visibilities of a
// baseline lie close together on the grid (Sec. 2.2: the footprints of a
// track almost entirely overlap), so the warp copies the bounding box of their
// 32 footprints into a shared-memory tile once. Then every lane forms its own
// visibility's P sums over the S x S footprint from the tile, with no
// reduction between threads:
//   s_p = sum_j t_v[j] * sum_i t_u[i] * g[p][y0 + j][x0 + i]
// (the separable form of the Sec. 6 remark, rows first). A group whose box is
// larger than the tile (fast tracks, unordered input) reads its footprints
// from global memory instead, with the same arithmetic. (Splitting such a
// group into two halves with a smaller tile measured slower.) Warps are
// persistent and load the next group's positions one group ahead.
//
// The box reaches shared memory by tiled bulk tensor copies (the TMA unit,
// cp.async.bulk.tensor) through 3-D tensor maps over this GPU's own [P][G][G]
// grid: one copy per polarization plane of a box RS cells wide and H rows high
// (the smallest of three heights that holds the group's rows), completing on
// the warp's mbarrier. Cells of the box outside the grid are filled with zeros
// and never read.
//
// Supports S = 1, 3, ..., 15 have fully unrolled kernels (taps in registers);
// every other support up to 64 runs one kernel per P that reads S from the
// plan and its taps from the shared-memory table.
//
// The index rule, validity, skipped count and output layout are those of the
// sliding-window degridder.
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.cuh"
#include "internal.h"

namespace gbg {
namespace {

// The smallest even row stride >= w cells that is 6 or 10 mod 16.
__host__ __device__ constexpr int spread_stride(int w) {
  while (w % 16 != 6 && w % 16 != 10) ++w;
  return w;
}

// Tile side in cells: the box of 32 consecutive visibilities on a baseline
// track fits unless the track is fast (a larger tile measured faster than
// S + 9, whose misses cost more than the lost occupancy).
__host__ __device__ constexpr int tile_side(int S) { return S + 13; }

// Plane stride in cells for row stride rs: a multiple of 16 (128 bytes), the
// alignment of a tensor copy's destination.
__host__ __device__ constexpr int tile_plane(int S, int rs) { return (tile_side(S) * rs + 15) / 16 * 16; }

template <int S, int P>
struct TileShape {
  static constexpr int TW = tile_side(S);
  // Row stride in cells. It is even, so that rows start on 16-byte boundaries
  // (the box is copied in 16-byte pieces). A cell is two 4-byte banks, so cell
  // (row, col) starts at bank pair (RS*row + col) mod 16; with RS = 6 or 10
  // mod 16, lanes whose footprints are a cell or two apart in any direction
  // read different banks (a stride of TW + 1 = 1 mod 16 made every pair one
  // cell apart along a diagonal collide).
  static constexpr int RS = spread_stride(TW);
  static constexpr int PS = tile_plane(S, RS);
  static constexpr int CELLS = P * PS;  // complex cells per warp
};

// Box heights of the three tensor maps: the smallest that holds a group's rows
// is used (a group of 32 baseline-ordered visibilities usually spans a few
// rows more than S).
__host__ __device__ constexpr int tile_height(int S, int i) {
  return i == 0 ? S + 3 : i == 1 ? S + 7 : tile_side(S);
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

// The same sums for a support known only at run time, with the taps read
// from the shared-memory table (tu, tv: the visibility's two table rows),
// each u tap once per row for all P planes. s must be zero on entry.
template <int P, typename Ptr, typename Stride>
__device__ __forceinline__ void footprint_dot_any(Ptr base, Stride rstride, Stride pstride, const float* tu,
                                                  const float* tv, int S, float2 (&s)[P]) {
#pragma unroll 1
  for (int j = 0; j < S; ++j) {
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
    const float2 t = splat(tv[j]);
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

template <int P>
__device__ __noinline__ void footprint_dot_global_any(const float2* base, int G, const float* tu, const float* tv,
                                                      int S, float2 (&s)[P]) {
  footprint_dot_any<P>(base, (size_t)G, (size_t)G * G, tu, tv, S, s);
}

// SC > 0: support SC, fully unrolled, taps in registers. SC = 0: the plan's
// support (any S), taps read from the shared-memory table.
template <int SC, int P>
__global__ void degrid_tile_kernel(Args a, const __grid_constant__ TileMaps maps) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const int S = SC > 0 ? SC : g.S;
  const int TW = SC > 0 ? TileShape<SC, P>::TW : tile_side(S);
  const int RS = SC > 0 ? TileShape<SC, P>::RS : spread_stride(TW);
  const int PS = SC > 0 ? TileShape<SC, P>::PS : tile_plane(S, RS);
  const int CELLS = P * PS;
  float* tab = (float*)smem;
  const int ntab = g.O * S;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) tab[i] = load_tap(a.table, a.tab_fmt, i);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
  const long long n_groups = (a.n_vis + 31) >> 5;
  const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
  // Persistent warps: the position of the next group's visibility is loaded
  // one group ahead, so its memory latency overlaps the current group.
  long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
  double2 xn = make_double2(0.0, 0.0);
  if (c < n_groups && c * 32 + lane < a.n_vis) xn = ld_stream(a.uv + c * 32 + lane);
  for (; c < n_groups; c += stride) {
    const long long k = c * 32 + lane;
    const double2 x = xn;
    if (c + stride < n_groups && (c + stride) * 32 + lane < a.n_vis) xn = ld_stream(a.uv + (c + stride) * 32 + lane);
    int x0 = 0, y0 = 0, ru = 0, rv = 0;
    bool ok = false;
    if (k < a.n_vis) {
      int Cu, Cv;
      ok = fine_cell(x.x, g.log2O, G >> 1, Cu, ru);
      ok = fine_cell(x.y, g.log2O, G >> 1, Cv, rv) && ok;
      x0 = Cu - g.h;
      y0 = Cv - g.h;
      ok = ok && x0 >= 0 && x0 + S <= G && y0 >= 0 && y0 + S <= G;
      if (!ok) atomicAdd(a.skipped, 1ULL);
    }
    float2 s[P];
#pragma unroll
    for (int p = 0; p < P; ++p) s[p] = make_float2(0.f, 0.f);
    float tu[SC > 0 ? SC : 1], tv[SC > 0 ? SC : 1];
    if constexpr (SC > 0) {
#pragma unroll
      for (int i = 0; i < SC; ++i) {
        tu[i] = tab[ru * SC + i];
        tv[i] = tab[rv * SC + i];
      }
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
          const float2* base = (const float2*)tile + (y0 - ymin) * RS + (x0 - xe);
          if constexpr (SC > 0) footprint_dot<SC, P>(base, RS, PS, tu, tv, s);
          else footprint_dot_any<P>(base, RS, PS, tab + ru * S, tab + rv * S, S, s);
        }
        __syncwarp();  // the tile is refilled for the next group
      } else if (ok) {
        const float2* base = (const float2*)a.grid + (size_t)y0 * G + x0;
        if constexpr (SC > 0) footprint_dot_global<SC, P>(base, G, tu, tv, s);
        else footprint_dot_global_any<P>(base, G, tab + ru * S, tab + rv * S, S, s);
      }
    }
    if (k < a.n_vis) {
      const float w = (a.weights && ok) ? a.weights[k] : 1.f;
      float2* out = a.vis_out + k * P;
#pragma unroll
      for (int p = 0; p < P; ++p) __stcs(out + p, make_float2(s[p].x * w, s[p].y * w));
    }
  }
  // a copy given up on may still be landing in this CTA's shared memory
  if (failed) mbar_wait(mbar, phase ^ 1u);
}

template <int S, int P>
TileKernel tile_entry() {
  return TileKernel{S, P, (const void*)&degrid_tile_kernel<S, P>, TileShape<S, P>::CELLS, TileShape<S, P>::RS,
                    {tile_height(S, 0), tile_height(S, 1), tile_height(S, 2)}};
}

#define GB_TILE_ROW(P) \
  tile_entry<1, P>(), tile_entry<3, P>(), tile_entry<5, P>(), tile_entry<7, P>(), tile_entry<9, P>(), \
      tile_entry<11, P>(), tile_entry<13, P>(), tile_entry<15, P>()

const TileKernel kTileKernels[] = {GB_TILE_ROW(1), GB_TILE_ROW(2), GB_TILE_ROW(4)};

}  // namespace

const TileKernel* find_tile_kernel(int S, int P) {
  for (const TileKernel& t : kTileKernels)
    if (t.S == S && t.P == P) return &t;
  return nullptr;
}

int tile_kernel_any(int S, int P, TileKernel* out) {
  const void* fn = P == 1 ? (const void*)&degrid_tile_kernel<0, 1>
                 : P == 2 ? (const void*)&degrid_tile_kernel<0, 2>
                 : P == 4 ? (const void*)&degrid_tile_kernel<0, 4> : nullptr;
  if (!fn || S < 1 || S > 64) return -1;
  const int rs = spread_stride(tile_side(S));
  *out = TileKernel{S, P, fn, P * tile_plane(S, rs), rs, {tile_height(S, 0), tile_height(S, 1), tile_height(S, 2)}};
  return 0;
}

size_t tile_smem_bytes(const TileKernel& t, int O, int warps) {
  return align16((size_t)O * t.S * 4) + 128 + (size_t)warps * t.cells * sizeof(float2) + (size_t)warps * 8;
}

int tile_maps(const TileKernel& t, const void* grid, int G, int P, TileMaps* out) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  memset(out, 0, sizeof *out);
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return -1;
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  // [P][G][G] complex64 as FP32 elements: x = 2G floats, y = G rows, z = P planes
  const cuuint64_t dims[3] = {(cuuint64_t)2 * G, (cuuint64_t)G, (cuuint64_t)P};
  const cuuint64_t strides[2] = {(cuuint64_t)G * 8, (cuuint64_t)G * G * 8};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int i = 0; i < 3; ++i) {
    const cuuint32_t box[3] = {(cuuint32_t)(2 * t.rs), (cuuint32_t)t.h[i], 1};
    out->h[i] = t.h[i];
    if (encode(&out->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(grid), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return -2;
  }
  out->ok = 1;
  return 0;
}

}  // namespace gbg
