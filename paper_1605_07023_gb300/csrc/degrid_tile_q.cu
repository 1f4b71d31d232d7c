// Tile-gather degridding kernels with four lanes per visibility (warp groups
// of 8 visibilities, for tracks that move several cells per visibility),
// built apart from the one-lane kernels so that the two compile in parallel.
#include "degrid_tile.cuh"

namespace gbg {
namespace {

const TileKernel kTileKernelsQ[] = {GB_TILE_ROW(1, 4), GB_TILE_ROW(2, 4), GB_TILE_ROW(4, 4)};

}  // namespace

const TileKernel* tile_kernels_q(int* n) {
  *n = (int)(sizeof(kTileKernelsQ) / sizeof(kTileKernelsQ[0]));
  return kTileKernelsQ;
}

const void* tile_kernel_any_q(int P) {
  return P == 1 ? (const void*)&degrid_tile_kernel<0, 1, 4>
       : P == 2 ? (const void*)&degrid_tile_kernel<0, 2, 4>
       : P == 4 ? (const void*)&degrid_tile_kernel<0, 4, 4> : nullptr;
}

}  // namespace gbg
