// Compression (Merry 2016, Sec. 2.2, last paragraph; the scheme is Muscat's):
// adjacent visibilities on the same point of the oversampled grid meet the
// same GCF samples, so their weighted values are summed into one record
// before gridding. Also the expansion that hands the degridded value of a
// merged record back to each of its members.
//
// Three passes over the records, in tiles of 1024 (one record per thread):
//  1. head flags: record k starts a run unless it and k-1 both have a fine
//     position and the two are equal on both axes. One bit per record (a warp
//     ballot word) and one head count per tile; four records per thread.
//  2. one CTA scans the tile counts: tile offsets and the total.
//  3. each record's run index = tile offset + heads before it in the tile
//     (ballot prefix counts). A head copies its uv. The w*V of a run are
//     summed by a segmented scan across each warp; a run that crosses warps
//     leaves one partial sum per warp.
//  4. the partial sums of runs that cross warps are added in warp order.
// Every sum is taken in a fixed order, so the results are deterministic.
#include "kernels.cuh"
#include "internal.h"

namespace gbg {

namespace {

constexpr int kTile = 1024;

__device__ __forceinline__ void st_stream4(float2* p, float4 v) {
  asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w), "l"(policy_stream())
               : "memory");
}

// Fine position (f_u, f_v) of one record, with the index rule of the
// gridder; false if a coordinate has none.
__device__ __forceinline__ bool fine_pair(double2 x, int log2O, int2& f) {
  int cu, ru, cv, rv;
  const bool ok = fine_cell(x.x, log2O, 0, cu, ru) & fine_cell(x.y, log2O, 0, cv, rv);
  f = make_int2(cu * (1 << log2O) + ru, cv * (1 << log2O) + rv);
  return ok;
}

// Pass 1, 256 threads per tile of kTile records: thread t handles records
// t, t + 256, t + 512 and t + 768 of the tile, so a warp covers 32
// consecutive records at each step and its ballot is one flag word. The four
// uv loads are issued together.
constexpr int kFlagThreads = 256;
constexpr int kFlagSteps = kTile / kFlagThreads;

__global__ void compress_flags_kernel(const double2* __restrict__ uv, long long n, int log2O, unsigned* flags,
                                      int* tile_heads) {
  const long long base = (long long)blockIdx.x * kTile + threadIdx.x;
  const int lane = threadIdx.x & 31;
  double2 x[kFlagSteps];
#pragma unroll
  for (int i = 0; i < kFlagSteps; ++i) {
    const long long k = base + i * kFlagThreads;
    x[i] = k < n ? ld_stream(uv + k) : make_double2(0.0, 0.0);
  }
  int cnt = 0;
#pragma unroll
  for (int i = 0; i < kFlagSteps; ++i) {
    const long long k = base + i * kFlagThreads;
    int2 f = make_int2(0, 0);
    const bool ok = k < n && fine_pair(x[i], log2O, f);
    // the previous record's position: from the lane below, or loaded by lane 0
    int2 fp;
    fp.x = __shfl_up_sync(0xFFFFFFFFu, f.x, 1);
    fp.y = __shfl_up_sync(0xFFFFFFFFu, f.y, 1);
    bool okp = __shfl_up_sync(0xFFFFFFFFu, ok, 1);
    if (lane == 0 && k > 0 && k < n) okp = fine_pair(uv[k - 1], log2O, fp);
    const bool head = k < n && (k == 0 || !ok || !okp || f.x != fp.x || f.y != fp.y);
    const unsigned word = __ballot_sync(0xFFFFFFFFu, head);
    if (lane == 0 && k < n) flags[k >> 5] = word;
    cnt += head ? 1 : 0;
  }
  // head count of the tile
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) cnt += __shfl_down_sync(0xFFFFFFFFu, cnt, d);
  __shared__ int warp_cnt[kFlagThreads / 32];
  if (lane == 0) warp_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
#pragma unroll
    for (int w = 0; w < kFlagThreads / 32; ++w) t += warp_cnt[w];
    tile_heads[blockIdx.x] = t;
  }
}

// Exclusive scan of the tile head counts by one CTA of kTile threads.
__global__ void compress_scan_kernel(const int* __restrict__ tile_heads, long long n_tiles, long long* tile_off,
                                     long long* n_out) {
  __shared__ long long warp_sum[32];
  __shared__ long long carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < n_tiles; base += kTile) {
    const long long t = base + threadIdx.x;
    const long long v = t < n_tiles ? tile_heads[t] : 0;
    long long x = v;  // inclusive scan within the warp
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      long long s = warp_sum[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const long long y = __shfl_up_sync(0xFFFFFFFFu, s, d);
        if (lane >= d) s += y;
      }
      warp_sum[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const long long before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
    if (t < n_tiles) tile_off[t] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_sum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = carry;
}

// Pass 3. Each record's w*V is summed over its run by a segmented inclusive
// scan across the warp (shuffles, a fixed tree order, so the result is
// deterministic). The lane that ends a segment in the warp stores its sum:
//  - into vis_out[run] when the run starts in this warp (it is complete if it
//    also ends here; otherwise pass 4 adds what follows);
//  - into carry[warp] when the run started in an earlier warp.
template <int P>
__global__ void compress_write_kernel(Args a, const unsigned* __restrict__ flags, const long long* __restrict__ tile_off,
                                      double2* __restrict__ uv_out, float2* __restrict__ vis_out,
                                      long long* __restrict__ run_of, float2* __restrict__ carry) {
  __shared__ int warp_prefix[32];
  const long long n = a.n_vis;
  const long long k = (long long)blockIdx.x * kTile + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long wbase = k - lane;
  const unsigned word = wbase < n ? flags[k >> 5] : 0u;
  if (lane == 0) warp_prefix[warp] = __popc(word);
  __syncthreads();
  if (warp == 0) {
    int s = warp_prefix[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xFFFFFFFFu, s, d);
      if (lane >= d) s += y;
    }
    warp_prefix[lane] = s;  // inclusive
  }
  __syncthreads();
  if (wbase >= n) return;  // whole warp past the end (warp-uniform)
  const bool valid = k < n;
  // records past the end act as heads of empty runs, so they stop every segment
  const bool head = valid ? ((word >> lane) & 1u) != 0 : true;
  float2 x[P];
  if (valid) {
    load_vis<P>(a, k, a.weights ? a.weights[k] : 1.f, x);
  } else {
#pragma unroll
    for (int p = 0; p < P; ++p) x[p] = make_float2(0.f, 0.f);
  }
  // segmented inclusive scan: f = "a head lies in (lane - span, lane]"
  bool f = head;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const bool fu = __shfl_up_sync(0xFFFFFFFFu, f, d);
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float yx = __shfl_up_sync(0xFFFFFFFFu, x[p].x, d);
      const float yy = __shfl_up_sync(0xFFFFFFFFu, x[p].y, d);
      if (lane >= d && !f) x[p] = __fadd2_rn(x[p], make_float2(yx, yy));
    }
    if (lane >= d) f = f || fu;
  }
  if (!valid) return;
  const int in_tile = (warp > 0 ? warp_prefix[warp - 1] : 0) + __popc(word & (0xFFFFFFFFu >> (31 - lane)));
  const long long run = tile_off[blockIdx.x] + in_tile - 1;
  if (run_of) run_of[k] = run;
  if (head) uv_out[run] = a.uv[k];
  // does this record end its segment within the warp?
  bool next_head;
  if (lane < 31) next_head = k + 1 >= n || ((word >> (lane + 1)) & 1u);
  else next_head = k + 1 >= n || (flags[(k >> 5) + 1] & 1u);
  if (lane < 31 && !next_head) return;
  if (next_head || lane == 31) {
    if (f) {
#pragma unroll
      for (int p = 0; p < P; ++p) vis_out[run * P + p] = x[p];   // the run starts in this warp
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) carry[(k >> 5) * P + p] = x[p];  // continuation of an earlier run
    }
  }
}

// Pass 4. For each warp whose last run continues into the next warp and
// starts in this warp, add the carries of the following warps, in order,
// up to the warp where the run ends.
template <int P>
__global__ void compress_fixup_kernel(long long n, const unsigned* __restrict__ flags, const long long* __restrict__ tile_off,
                                      float2* __restrict__ vis_out, const float2* __restrict__ carry) {
  const long long n_warps = (n + 31) / 32;
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w + 1 < n_warps;
       w += (long long)gridDim.x * blockDim.x) {
    const unsigned word = flags[w];
    if (word == 0u || (flags[w + 1] & 1u)) continue;  // no run starts here, or the last one ends here
    // the run index of the last head in warp w: heads before warp w plus those in it, minus one
    const long long tile = (w * 32) / kTile;
    long long before = tile_off[tile];
    for (long long u = tile * (kTile / 32); u <= w; ++u) before += __popc(flags[u]);
    const long long run = before - 1;
    float2 s[P];
#pragma unroll
    for (int p = 0; p < P; ++p) s[p] = vis_out[run * P + p];
    for (long long u = w + 1; u < n_warps; ++u) {
      const unsigned fw = flags[u];
      if (fw & 1u) break;  // warp u starts with a head: the run ended with warp u-1 (no carry here)
#pragma unroll
      for (int p = 0; p < P; ++p) s[p] = __fadd2_rn(s[p], carry[u * P + p]);
      if (fw != 0u) break;  // the run ends inside warp u
    }
#pragma unroll
    for (int p = 0; p < P; ++p) vis_out[run * P + p] = s[p];
  }
}

// vis_out[k] = w_k * vis_c[run_of[k]]; a run index outside [0, n_c) gives 0.
template <int P>
__global__ void expand_kernel(long long n, const long long* __restrict__ run_of, long long n_c,
                              const float2* __restrict__ vis_c, const float* __restrict__ weights,
                              float2* __restrict__ vis_out) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const long long r = run_of[k];
    const bool ok = r >= 0 && r < n_c;
    const float w = weights ? weights[k] : 1.f;
    if constexpr (P % 2 == 0) {
#pragma unroll
      for (int p = 0; p < P; p += 2) {
        float4 v = ok ? *(const float4*)(vis_c + r * P + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        st_stream4(vis_out + k * P + p, make_float4(v.x * w, v.y * w, v.z * w, v.w * w));
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const float2 v = ok ? vis_c[r * P + p] : make_float2(0.f, 0.f);
        vis_out[k * P + p] = make_float2(v.x * w, v.y * w);
      }
    }
  }
}

}  // namespace

size_t compress_scratch_bytes(long long n, int P) {
  const long long n_tiles = (n + kTile - 1) / kTile;
  const long long n_warps = n_tiles * (kTile / 32);
  return (size_t)n_warps * sizeof(unsigned) + (size_t)n_tiles * sizeof(int) + (size_t)n_tiles * sizeof(long long) +
         (size_t)n_warps * P * sizeof(float2) + 64;
}

cudaError_t launch_compress(const Args& a, void* scratch, double2* uv_out, float2* vis_out, long long* run_of,
                            long long* n_out, int sm_count, cudaStream_t st) {
  const long long n = a.n_vis;
  const long long n_tiles = (n + kTile - 1) / kTile;
  const long long n_warps = n_tiles * (kTile / 32);
  unsigned* flags = (unsigned*)scratch;
  int* tile_heads = (int*)(flags + n_warps);
  long long* tile_off = (long long*)(((uintptr_t)(tile_heads + n_tiles) + 15) & ~(uintptr_t)15);
  float2* carry = (float2*)(tile_off + n_tiles);
  const long long want = (n_warps + 255) / 256;
  const unsigned fix_blocks = (unsigned)(want < (long long)sm_count * 4 ? want : (long long)sm_count * 4);
  compress_flags_kernel<<<(unsigned)n_tiles, kFlagThreads, 0, st>>>(a.uv, n, a.g.log2O, flags, tile_heads);
  compress_scan_kernel<<<1, kTile, 0, st>>>(tile_heads, n_tiles, tile_off, n_out);
  switch (a.g.P) {
    case 1:
      compress_write_kernel<1><<<(unsigned)n_tiles, kTile, 0, st>>>(a, flags, tile_off, uv_out, vis_out, run_of, carry);
      compress_fixup_kernel<1><<<fix_blocks, 256, 0, st>>>(n, flags, tile_off, vis_out, carry);
      break;
    case 2:
      compress_write_kernel<2><<<(unsigned)n_tiles, kTile, 0, st>>>(a, flags, tile_off, uv_out, vis_out, run_of, carry);
      compress_fixup_kernel<2><<<fix_blocks, 256, 0, st>>>(n, flags, tile_off, vis_out, carry);
      break;
    default:
      compress_write_kernel<4><<<(unsigned)n_tiles, kTile, 0, st>>>(a, flags, tile_off, uv_out, vis_out, run_of, carry);
      compress_fixup_kernel<4><<<fix_blocks, 256, 0, st>>>(n, flags, tile_off, vis_out, carry);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_expand(int P, long long n, const long long* run_of, long long n_c, const float2* vis_c,
                          const float* weights, float2* vis_out, int sm_count, cudaStream_t st) {
  const long long want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < (long long)sm_count * 8 ? want : (long long)sm_count * 8);
  switch (P) {
    case 1: expand_kernel<1><<<blocks, 256, 0, st>>>(n, run_of, n_c, vis_c, weights, vis_out); break;
    case 2: expand_kernel<2><<<blocks, 256, 0, st>>>(n, run_of, n_c, vis_c, weights, vis_out); break;
    default: expand_kernel<4><<<blocks, 256, 0, st>>>(n, run_of, n_c, vis_c, weights, vis_out); break;
  }
  return cudaGetLastError();
}

}  // namespace gbg
