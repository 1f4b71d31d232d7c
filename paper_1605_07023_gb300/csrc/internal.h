// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "lazy.cuh"
#include "rotated.cuh"

namespace gbg {

struct PatchScratch {
  int patch;        // patch side in cells
  int n_pu;         // patches per grid axis
  int n_patches;
  int halo_lo;      // window origin = patch origin - halo_lo
  int win;          // window side in cells
  int max_chunks;   // chunks per work item
  int max_work;
  int* patch_count;
  int* patch_off;
  int* chunk_patch;
  int* chunk_slot;
  int* chunk_order;
  int4* work;
  int* n_work;
  int* work_next;
};

// Kernel tables, one per polarization count (defined in inst_p*.cu).
const KernelEntry* kernels_p1(int* n);
const KernelEntry* kernels_p2(int* n);
const KernelEntry* kernels_p4(int* n);

// Rotated-table chunked gridders (inst_rot_p*.cu), one entry per (Bu, Bv).
const RotEntry* rot_kernels_p1(int* n);
const RotEntry* rot_kernels_p2(int* n);
const RotEntry* rot_kernels_p4(int* n);

// Lazy-box gridders (inst_lazy_p*.cu), one per (Bu, Bv, P) that is built.
const LazyEntry* lazy_kernels_p1(int* n);
const LazyEntry* lazy_kernels_p2(int* n);
const LazyEntry* lazy_kernels_p4(int* n);

// Tile-gather degridding (degrid_tile.cu), one kernel per (S, P).
struct TileKernel {
  int S, P;
  int lpv;          // lanes per visibility: 1 (groups of 32 visibilities per warp) or 4 (groups of 8)
  const void* fn;   // degrid_tile_kernel(Args, TileMaps)
  int cells;        // complex cells of one warp's tile
  int rs;           // tile row stride in cells: the width of a tensor copy's box
  int h[3];         // box heights of the three tensor maps
};
// Tensor maps over one [P][G][G] grid, one per box height (kernel parameter).
struct TileMaps {
  CUtensorMap m[3];
  int h[3];
  int ok;  // 0: no maps (encoding refused, e.g. a grid smaller than a box): every group reads the grid directly
};
const TileKernel* find_tile_kernel(int S, int P, int lpv);
// The run-time-support tile kernel for (S, P, lpv), 1 <= S <= 64: 0, or -1 when P is not 1, 2 or 4
// or lpv not 1 or 4.
int tile_kernel_any(int S, int P, int lpv, TileKernel* out);
// The unrolled tile kernels with four lanes per visibility (groups of 8), from their own translation unit.
const TileKernel* tile_kernels_q(int* n);
const void* tile_kernel_any_q(int P);
size_t tile_smem_bytes(const TileKernel& t, int O, int warps);
// Encodes the tensor maps of a tile kernel for this grid (host call); 0 on success. On failure
// out->ok is 0 and the kernel reads every group's footprints from the grid directly.
int tile_maps(const TileKernel& t, const void* grid, int G, int P, TileMaps* out);

cudaError_t launch_fma_peak(int blocks, int threads, int iters, cudaStream_t st);
double fma_peak_flops_per_launch(int blocks, int threads, int iters);
cudaError_t launch_kb_table(int S, int O, double beta, int fmt, void* out, cudaStream_t st);
cudaError_t launch_indices(const Args& a, int32_t* cell, int32_t* sub, cudaStream_t st);
cudaError_t launch_patch_binning(const Args& a, const PatchScratch& ps, cudaStream_t st);

// Compression (compress.cu).
size_t compress_scratch_bytes(long long n, int P);
cudaError_t launch_compress(const Args& a, void* scratch, double2* uv_out, float2* vis_out, long long* run_of,
                            long long* n_out, int sm_count, cudaStream_t st);
cudaError_t launch_expand(int P, long long n, const long long* run_of, long long n_c, const float2* vis_c,
                          const float* weights, float2* vis_out, int sm_count, cudaStream_t st);

}  // namespace gbg
