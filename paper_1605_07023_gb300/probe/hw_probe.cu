// GB300 hardware probe: the rates the gridder's design depends on.
//  - FP32 FFMA vs packed FFMA2 (__ffma2_rn) peak, and with independent integer ALU work mixed in;
//  - FP64 DFMA rate (why the index rule avoids FP64 arithmetic);
//  - global vector reductions (atomicAdd float4/float2/float) at random and coalesced addresses
//    over 8 MiB, 128 MiB and 512 MiB (the flush cost of the chunked schedule);
//  - shared-memory f32 atomics and plain read-modify-write (the flush cost of the patch schedule).
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -std=c++17 hw_probe.cu -o hw_probe && ./hw_probe
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

__global__ void ffma_peak(float* out, int iters, float b, float c) {
  float a[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = threadIdx.x * 1e-3f + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void ffma2_peak(float* out, int iters, float b, float c) {
  float2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
  float2 bb = make_float2(b, b), cc = make_float2(c, c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
  }
  float s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 FFMA2 + 8 independent integer ALU ops per iteration
__global__ void ffma2_mixed(float* out, int iters, float b, float c) {
  float2 a[8];
  unsigned x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { a[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f); x[k] = threadIdx.x * 7 + k; }
  float2 bb = make_float2(b, b), cc = make_float2(c, c);
  unsigned y = (unsigned)iters;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) { a[k] = __ffma2_rn(a[k], bb, cc); x[k] = (x[k] ^ y) + 0x9e37u; }
  }
  float s = 0;
  unsigned t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) { s += a[k].x + a[k].y; t ^= x[k]; }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + (float)(t & 1);
}

// 16 FFMA + 8 independent integer ALU ops per iteration
__global__ void ffma_mixed(float* out, int iters, float b, float c) {
  float a[16];
  unsigned x[8];
#pragma unroll
  for (int k = 0; k < 16; ++k) a[k] = threadIdx.x * 1e-3f + k;
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 7 + k;
  unsigned y = (unsigned)iters;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = fmaf(a[k], b, c);
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (x[k] ^ y) + 0x9e37u;
  }
  float s = 0;
  unsigned t = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) s += a[k];
#pragma unroll
  for (int k = 0; k < 8; ++k) t ^= x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + (float)(t & 1);
}

__global__ void dfma_peak(double* out, int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16; x *= 0x7feb352du; x ^= x >> 15; x *= 0x846ca68bu; x ^= x >> 16; return x;
}

// mode 0: random float4 slots; mode 1: coalesced consecutive float4 slots
__global__ void red_v4(float4* g, unsigned nslot_mask, int k_per_thread, int mode) {
  unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned nth = gridDim.x * blockDim.x;
  for (int k = 0; k < k_per_thread; ++k) {
    unsigned idx = mode == 0 ? (hash32(tid * 977u + k) & nslot_mask) : ((tid + (unsigned)k * nth) & nslot_mask);
    atomicAdd(&g[idx], make_float4(1.f, 1.f, 1.f, 1.f));
  }
}

__global__ void red_v2(float2* g, unsigned nslot_mask, int k_per_thread, int mode) {
  unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned nth = gridDim.x * blockDim.x;
  for (int k = 0; k < k_per_thread; ++k) {
    unsigned idx = mode == 0 ? (hash32(tid * 977u + k) & nslot_mask) : ((tid + (unsigned)k * nth) & nslot_mask);
    atomicAdd(&g[idx], make_float2(1.f, 1.f));
  }
}

__global__ void red_f1(float* g, unsigned nslot_mask, int k_per_thread, int mode) {
  unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned nth = gridDim.x * blockDim.x;
  for (int k = 0; k < k_per_thread; ++k) {
    unsigned idx = mode == 0 ? (hash32(tid * 977u + k) & nslot_mask) : ((tid + (unsigned)k * nth) & nslot_mask);
    atomicAdd(&g[idx], 1.f);
  }
}

// 32 KB shared float array per block; 8192 floats
template <int MODE>
__global__ void smem_acc(float* out, int iters) {
  __shared__ float buf[8192];
  for (int i = threadIdx.x; i < 8192; i += blockDim.x) buf[i] = 0.f;
  __syncthreads();
  unsigned base = threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      // conflict-free: lane-consecutive addresses, each thread its own slot per k
      unsigned idx = (base + k * 1024u + (unsigned)it * 7u * 32u) & 8191u;
      if (MODE == 0) atomicAdd(&buf[idx], 1.0f);
      else if (MODE == 1) buf[idx] += 1.0f;  // non-atomic RMW (racy by design across threads? no: idx unique per thread per k within an iteration)
    }
  }
  __syncthreads();
  float s = 0;
  for (int i = threadIdx.x; i < 8192; i += blockDim.x) s += buf[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Shared f32 atomics from warps with only LANES active lanes (a partial flush),
// to see whether the cost is per lane or per instruction.
template <int LANES>
__global__ void smem_atomic_partial(float* out, int iters) {
  __shared__ float buf[8192];
  for (int i = threadIdx.x; i < 8192; i += blockDim.x) buf[i] = 0.f;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  if (lane < LANES) {
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        unsigned idx = (threadIdx.x + k * 1024u + (unsigned)it * 7u * 32u) & 8191u;
        atomicAdd(&buf[idx], 1.0f);
      }
    }
  }
  __syncthreads();
  out[blockIdx.x * blockDim.x + threadIdx.x] = buf[threadIdx.x];
}

// 8 FFMA2 + 2 shared atomics per iteration, to see overlap
__global__ void mix_atomic(float* out, int iters) {
  __shared__ float buf[8192];
  for (int i = threadIdx.x; i < 8192; i += blockDim.x) buf[i] = 0.f;
  __syncthreads();
  float2 a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, k * 0.5f);
  float2 bb = make_float2(0.9999f, 0.9999f), cc = make_float2(1e-4f, 1e-4f);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], bb, cc);
    unsigned idx = (threadIdx.x + (unsigned)it * 32u) & 8191u;
    atomicAdd(&buf[idx], a[0].x);
    atomicAdd(&buf[(idx + 4096u) & 8191u], a[1].y);
  }
  __syncthreads();
  float s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k].x + a[k].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s + buf[threadIdx.x];
}

int main() {
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  int sms = p.multiProcessorCount;
  int clk_khz = 0; cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  printf("device %s SMs %d l2 %d MB clock_attr %d kHz smem/SM %zu regs/SM %d\n", p.name, sms, p.l2CacheSize >> 20, clk_khz,
         p.sharedMemPerMultiprocessor, p.regsPerMultiprocessor);
  const int threads = 256, blocks = sms * 8;
  float* out; CK(cudaMalloc(&out, (size_t)blocks * threads * sizeof(double)));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  auto timeit = [&](auto launch) {
    for (int i = 0; i < 3; ++i) launch();
    cudaDeviceSynchronize();
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
      cudaEventRecord(e0); launch(); cudaEventRecord(e1); cudaEventSynchronize(e1);
      float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
    }
    return best;
  };
  const int iters = 4096;
  double nthr = (double)blocks * threads;
  float ms;
  ms = timeit([&] { ffma_peak<<<blocks, threads>>>(out, iters, 0.9999f, 1e-4f); });
  printf("ffma      : %.3f ms  %.2f TFMA/s (%.2f TFLOP/s)\n", ms, nthr * iters * 16 / ms / 1e9, 2 * nthr * iters * 16 / ms / 1e9);
  ms = timeit([&] { ffma2_peak<<<blocks, threads>>>(out, iters, 0.9999f, 1e-4f); });
  printf("ffma2     : %.3f ms  %.2f TFMA/s (%.2f TFLOP/s)\n", ms, nthr * iters * 16 / ms / 1e9, 2 * nthr * iters * 16 / ms / 1e9);
  ms = timeit([&] { ffma2_mixed<<<blocks, threads>>>(out, iters, 0.9999f, 1e-4f); });
  printf("ffma2+int : %.3f ms  %.2f TFMA/s (8 FFMA2 + 8x2 int per iter)\n", ms, nthr * iters * 16 / ms / 1e9);
  ms = timeit([&] { ffma_mixed<<<blocks, threads>>>(out, iters, 0.9999f, 1e-4f); });
  printf("ffma+int  : %.3f ms  %.2f TFMA/s (16 FFMA + 8x2 int per iter)\n", ms, nthr * iters * 16 / ms / 1e9);
  ms = timeit([&] { dfma_peak<<<blocks, threads>>>((double*)out, iters / 8, 0.9999, 1e-4); });
  printf("dfma      : %.3f ms  %.3f TDFMA/s\n", ms, nthr * (iters / 8) * 8 / ms / 1e9);

  // reductions over a 128 MiB buffer (8M float4 slots)
  size_t bytes = 128ull << 20;
  void* g; CK(cudaMalloc(&g, bytes)); CK(cudaMemset(g, 0, bytes));
  const int K = 64;
  double nops = nthr * K;
  for (int mode = 0; mode < 2; ++mode) {
    ms = timeit([&] { red_v4<<<blocks, threads>>>((float4*)g, (unsigned)(bytes / 16 - 1), K, mode); });
    printf("red.v4 %s: %.3f ms  %.2f Gops/s  %.2f TB/s payload\n", mode ? "seq " : "rand", ms, nops / ms / 1e6, nops * 16 / ms / 1e9);
    ms = timeit([&] { red_v2<<<blocks, threads>>>((float2*)g, (unsigned)(bytes / 8 - 1), K, mode); });
    printf("red.v2 %s: %.3f ms  %.2f Gops/s  %.2f TB/s payload\n", mode ? "seq " : "rand", ms, nops / ms / 1e6, nops * 8 / ms / 1e9);
    ms = timeit([&] { red_f1<<<blocks, threads>>>((float*)g, (unsigned)(bytes / 4 - 1), K, mode); });
    printf("red.f32 %s: %.3f ms  %.2f Gops/s  %.2f TB/s payload\n", mode ? "seq" : "rand", ms, nops / ms / 1e6, nops * 4 / ms / 1e9);
  }
  // 512 MiB buffer: larger than L2
  void* g2; CK(cudaMalloc(&g2, bytes * 4)); CK(cudaMemset(g2, 0, bytes * 4));
  ms = timeit([&] { red_v4<<<blocks, threads>>>((float4*)g2, (unsigned)(bytes * 4 / 16 - 1), K, 0); });
  printf("red.v4 rand 512MiB: %.3f ms  %.2f Gops/s  %.2f TB/s payload\n", ms, nops / ms / 1e6, nops * 16 / ms / 1e9);
  // 8 MiB buffer: hot in L2
  ms = timeit([&] { red_v4<<<blocks, threads>>>((float4*)g2, (unsigned)((8 << 20) / 16 - 1), K, 0); });
  printf("red.v4 rand 8MiB: %.3f ms  %.2f Gops/s  %.2f TB/s payload\n", ms, nops / ms / 1e6, nops * 16 / ms / 1e9);
  {
  const int threads2 = 1024, blocks2 = sms * 2;
  float* out2; CK(cudaMalloc(&out2, (size_t)blocks * threads * 4));
    const int iters2 = 1024;
  double ops = (double)blocks2 * threads2 * iters2 * 8;
  ms = timeit([&] { smem_acc<0><<<blocks2, threads2>>>(out2, iters2); });
  printf("smem atomicAdd f32: %.3f ms %.1f Gops/s  (%.2f per SM per clk @1.9GHz)\n", ms, ops / ms / 1e6, ops / ms / 1e6 / sms / 1.9);
  ms = timeit([&] { smem_acc<1><<<blocks2, threads2>>>(out2, iters2); });
  printf("smem plain RMW f32: %.3f ms %.1f Gops/s  (%.2f per SM per clk @1.9GHz)\n", ms, ops / ms / 1e6, ops / ms / 1e6 / sms / 1.9);
  ms = timeit([&] { smem_atomic_partial<4><<<blocks2, threads2>>>(out2, iters2); });
  printf("smem atomicAdd, 4 of 32 lanes active: %.3f ms %.1f G lane-ops/s %.1f G warp-instr/s\n", ms, ops / 8 / ms / 1e6,
         ops / 32 / ms / 1e6);
  ms = timeit([&] { smem_atomic_partial<32><<<blocks2, threads2>>>(out2, iters2); });
  printf("smem atomicAdd, 32 of 32 lanes active: %.3f ms %.1f G lane-ops/s %.1f G warp-instr/s\n", ms, ops / ms / 1e6,
         ops / 32 / ms / 1e6);
  ms = timeit([&] { mix_atomic<<<blocks2, threads2>>>(out2, iters2); });
  double fma = (double)blocks2 * threads2 * iters2 * 16;
  printf("8 FFMA2 + 2 smem atomics: %.3f ms %.2f TFMA/s\n", ms, fma / ms / 1e9);
  }
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  printf("ok\n");
  return 0;
}
