// Auxiliary kernels: the Kaiser-Bessel table, the index hook, and patch
// binning for the patch schedule.
#include "kernels.cuh"
#include "internal.h"

namespace gbg {

// Oversampled Kaiser-Bessel table (Sec. 2.2: a precomputed, oversampled GCF
// table). Entry (r, i) is the GCF at distance d = i - h - (r - O/2)/O from
// the visibility. It is evaluated in FP64 with CUDA's cyl_bessel_i0 and
// rounded once to the storage format.
__global__ void kb_table_kernel(int S, int O, double beta, int fmt, void* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= O * S) return;
  const int r = idx / S, i = idx - r * S;
  const int h = (S - 1) / 2;
  const double d = (double)(i - h) - (double)(r - O / 2) / (double)O;
  const double x = 2.0 * d / (double)S;
  double val = 0.0;
  if (fabs(x) <= 1.0) val = cyl_bessel_i0(beta * sqrt(1.0 - x * x)) / cyl_bessel_i0(beta);
  if (fmt == FMT_BF16) ((__nv_bfloat16*)out)[idx] = __double2bfloat16(val);
  else if (fmt == FMT_F16) ((__half*)out)[idx] = __double2half(val);
  else ((float*)out)[idx] = (float)val;
}

// FP32 FMA throughput probe for the roofline denominator: every thread runs
// kPeakChains independent chains of packed FFMA2 (two FMAs per instruction).
// The result is stored only when out is not null, so the loop cannot be
// removed; callers pass null.
constexpr int kPeakChains = 8;
__global__ void fma_peak_kernel(int iters, float2 m, float2 c, float2* out) {
  float2 acc[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) acc[k] = make_float2((float)threadIdx.x * 1e-7f + (float)k, (float)k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) acc[k] = __ffma2_rn(acc[k], m, c);
  }
  if (out) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kPeakChains; ++k) s = __fadd2_rn(s, acc[k]);
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
  }
}

cudaError_t launch_fma_peak(int blocks, int threads, int iters, cudaStream_t st) {
  fma_peak_kernel<<<blocks, threads, 0, st>>>(iters, make_float2(0.9999f, 0.9999f), make_float2(1e-4f, 1e-4f), nullptr);
  return cudaGetLastError();
}

double fma_peak_flops_per_launch(int blocks, int threads, int iters) {
  return (double)blocks * threads * iters * kPeakChains * 2 /* FMAs per FFMA2 */ * 2 /* flop per FMA */;
}

// Per-visibility indices exactly as the gridding kernels stage them.
__global__ void indices_kernel(Args a, int32_t* cell, int32_t* sub) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n_vis) return;
  const Geometry& g = a.g;
  const double2 x = a.uv[k];
  int Cu, ru, Cv, rv;
  bool ok = fine_cell(x.x, g.log2O, g.G >> 1, Cu, ru);
  ok = fine_cell(x.y, g.log2O, g.G >> 1, Cv, rv) && ok;
  ok = ok && Cu - g.h >= 0 && Cu - g.h + g.S <= g.G && Cv - g.h >= 0 && Cv - g.h + g.S <= g.G;
  if (ok) {
    ((int2*)cell)[k] = make_int2(Cu, Cv);
    ((int2*)sub)[k] = make_int2(ru, rv);
  } else {
    ((int2*)cell)[k] = make_int2(-1, -1);
    ((int2*)sub)[k] = make_int2(-1, -1);
  }
}

// Patch binning, step 1: every chunk is assigned to the patch that holds the
// footprint start of its middle visibility (or of its first one, if the
// middle one is invalid). The chunk also takes a slot in that patch's list.
__global__ void chunk_patch_kernel(Args a, int patch, int n_pu, int* chunk_patch, int* chunk_slot, int* patch_count) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.n_chunks) return;
  const Geometry& g = a.g;
  const long long beg = c * a.chunk_len;
  const long long end = min(beg + a.chunk_len, a.n_vis);
  const long long cand[2] = {beg + (end - beg) / 2, beg};
  int pid = 0;
  for (int t = 0; t < 2; ++t) {
    const double2 x = a.uv[cand[t]];
    int Cu, ru, Cv, rv;
    bool ok = fine_cell(x.x, g.log2O, g.G >> 1, Cu, ru);
    ok = fine_cell(x.y, g.log2O, g.G >> 1, Cv, rv) && ok;
    const int cu0 = Cu - g.h, cv0 = Cv - g.h;
    if (ok && cu0 >= 0 && cv0 >= 0 && cu0 < g.G && cv0 < g.G) {
      pid = (cv0 / patch) * n_pu + (cu0 / patch);
      break;
    }
  }
  chunk_patch[c] = pid;
  chunk_slot[c] = atomicAdd(&patch_count[pid], 1);
}

// Step 2 (one CTA): exclusive scan of patch counts into list offsets, and of
// work items per patch (ceil(count / max_chunks)) into work-item offsets.
// Then write the work items {window u0, window v0, first, last}.
__global__ void patch_scan_kernel(const int* patch_count, int n_patches, int n_pu, int patch, int halo_lo, int max_chunks,
                                  int* patch_off, int4* work, int* n_work, int max_work) {
  extern __shared__ int sh[];  // 2 * blockDim.x
  int* s_cnt = sh;
  int* s_items = sh + blockDim.x;
  __shared__ int carry_cnt, carry_items;
  if (threadIdx.x == 0) { carry_cnt = 0; carry_items = 0; }
  __syncthreads();
  for (int base = 0; base < n_patches; base += blockDim.x) {
    const int p = base + threadIdx.x;
    const int c = p < n_patches ? patch_count[p] : 0;
    const int it = (c + max_chunks - 1) / max_chunks;
    s_cnt[threadIdx.x] = c;
    s_items[threadIdx.x] = it;
    __syncthreads();
    // Hillis-Steele inclusive scan of both arrays
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      int a1 = 0, a2 = 0;
      if ((int)threadIdx.x >= off) { a1 = s_cnt[threadIdx.x - off]; a2 = s_items[threadIdx.x - off]; }
      __syncthreads();
      s_cnt[threadIdx.x] += a1;
      s_items[threadIdx.x] += a2;
      __syncthreads();
    }
    const int excl_cnt = carry_cnt + s_cnt[threadIdx.x] - c;
    const int excl_items = carry_items + s_items[threadIdx.x] - it;
    if (p < n_patches) {
      patch_off[p] = excl_cnt;
      const int pu = p % n_pu, pv = p / n_pu;
      for (int k = 0; k < it; ++k) {
        const int w = excl_items + k;
        if (w < max_work) {
          const int first = excl_cnt + k * max_chunks;
          const int last = min(first + max_chunks, excl_cnt + c);
          work[w] = make_int4(pu * patch - halo_lo, pv * patch - halo_lo, first, last);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) { carry_cnt += s_cnt[threadIdx.x]; carry_items += s_items[threadIdx.x]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    patch_off[n_patches] = carry_cnt;
    *n_work = min(carry_items, max_work);
  }
}

// Step 3: scatter chunk ids into the per-patch lists.
__global__ void chunk_scatter_kernel(long long n_chunks, const int* chunk_patch, const int* chunk_slot, const int* patch_off,
                                     int* chunk_order) {
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  chunk_order[patch_off[chunk_patch[c]] + chunk_slot[c]] = (int)c;
}

cudaError_t launch_kb_table(int S, int O, double beta, int fmt, void* out, cudaStream_t st) {
  const int n = O * S;
  kb_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(S, O, beta, fmt, out);
  return cudaGetLastError();
}

cudaError_t launch_indices(const Args& a, int32_t* cell, int32_t* sub, cudaStream_t st) {
  if (a.n_vis == 0) return cudaSuccess;
  const long long blocks = (a.n_vis + 255) / 256;
  indices_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, cell, sub);
  return cudaGetLastError();
}

cudaError_t launch_patch_binning(const Args& a, const PatchScratch& ps, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(ps.patch_count, 0, sizeof(int) * ps.n_patches, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ps.work_next, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  const unsigned cb = (unsigned)((a.n_chunks + 255) / 256);
  chunk_patch_kernel<<<cb, 256, 0, st>>>(a, ps.patch, ps.n_pu, ps.chunk_patch, ps.chunk_slot, ps.patch_count);
  patch_scan_kernel<<<1, 1024, 2 * 1024 * sizeof(int), st>>>(ps.patch_count, ps.n_patches, ps.n_pu, ps.patch, ps.halo_lo,
                                                             ps.max_chunks, ps.patch_off, ps.work, ps.n_work, ps.max_work);
  chunk_scatter_kernel<<<cb, 256, 0, st>>>(a.n_chunks, ps.chunk_patch, ps.chunk_slot, ps.patch_off, ps.chunk_order);
  return cudaGetLastError();
}

}  // namespace gbg
