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
// Groups of 32 visibilities (one lane each) suit baseline tracks that move
// a fraction of a cell per visibility. For tracks that move several cells
// per visibility a plan can take groups of 8 with four lanes per visibility
// (each lane sums every fourth footprint row) and a tile 8 cells wider; their
// kernels are built in degrid_tile_q.cu.
//
// The index rule, validity, skipped count and output layout are those of the
// sliding-window degridder.
#include <cstring>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "degrid_tile.cuh"

namespace gbg {
namespace {

const TileKernel kTileKernels[] = {GB_TILE_ROW(1, 1), GB_TILE_ROW(2, 1), GB_TILE_ROW(4, 1)};

}  // namespace

const TileKernel* find_tile_kernel(int S, int P, int lpv) {
  int n = 0;
  const TileKernel* tab = kTileKernels;
  if (lpv == 1) n = (int)(sizeof(kTileKernels) / sizeof(kTileKernels[0]));
  else if (lpv == 4) tab = tile_kernels_q(&n);
  for (int i = 0; i < n; ++i)
    if (tab[i].S == S && tab[i].P == P) return &tab[i];
  return nullptr;
}

int tile_kernel_any(int S, int P, int lpv, TileKernel* out) {
  const void* fn = nullptr;
  if (lpv == 1)
    fn = P == 1 ? (const void*)&degrid_tile_kernel<0, 1, 1>
       : P == 2 ? (const void*)&degrid_tile_kernel<0, 2, 1>
       : P == 4 ? (const void*)&degrid_tile_kernel<0, 4, 1> : nullptr;
  else if (lpv == 4)
    fn = tile_kernel_any_q(P);
  if (!fn || S < 1 || S > 64) return -1;
  const int rs = spread_stride(tile_side(S, lpv));
  *out = TileKernel{S, P, lpv, fn, P * tile_plane(S, lpv, rs), rs,
                    {tile_height(S, lpv, 0), tile_height(S, lpv, 1), tile_height(S, lpv, 2)}};
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
