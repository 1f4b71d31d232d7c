// grid_patch_static(): gridding with the patch schedule for callers that
// cannot allocate device memory.
//
// Who needs it: a real-time imaging pipeline that reserves all of its device
// memory at start-up and must never call the allocator in steady state (an
// allocation can stall or fail half way through an observation), and a host
// framework that owns the device heap through its own allocator, so a library
// allocating behind its back would break its accounting. grid() cannot serve
// them, because plan creation and the patch schedule's first call allocate
// scratch with cudaMalloc.
//
// This entry point takes the plan parameters directly and keeps the patch
// schedule's binning scratch (patch counts and offsets, per-chunk patch ids,
// slots and order, the work items and two counters) in one file-scope device
// array. It calls no cudaMalloc, no cudaFree and no allocating library
// routine; it only enqueues memsets and kernel launches on the caller's
// stream. The kernels are the same ones grid() launches.
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/gridder.h"
#include "internal.h"

using namespace gbg;

namespace {

// Limits of the static scratch. Chunks are 64 visibilities, so up to
// 8,388,608 visibilities per call; up to 16,384 patches (for example G=4096
// with 32-cell patches).
constexpr int kStaticChunkLen = 64;
constexpr long long kStaticMaxChunks = 131072;
constexpr int kStaticMaxPatches = 16384;
constexpr int kStaticMaxChunksPerItem = 128;
constexpr int kStaticMaxWork = kStaticMaxPatches + (int)(kStaticMaxChunks / kStaticMaxChunksPerItem) + 2;

// byte offsets inside the scratch array (all 256-byte aligned)
constexpr size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffPatchCount = 0;
constexpr size_t kOffPatchOff = kOffPatchCount + a256(sizeof(int) * kStaticMaxPatches);
constexpr size_t kOffChunkPatch = kOffPatchOff + a256(sizeof(int) * (kStaticMaxPatches + 1));
constexpr size_t kOffChunkSlot = kOffChunkPatch + a256(sizeof(int) * kStaticMaxChunks);
constexpr size_t kOffChunkOrder = kOffChunkSlot + a256(sizeof(int) * kStaticMaxChunks);
constexpr size_t kOffWork = kOffChunkOrder + a256(sizeof(int) * kStaticMaxChunks);
constexpr size_t kOffNWork = kOffWork + a256(sizeof(int4) * kStaticMaxWork);
constexpr size_t kOffWorkNext = kOffNWork + 256;
constexpr size_t kOffSkipped = kOffWorkNext + 256;
constexpr size_t kScratchBytes = kOffSkipped + 256;  // about 1.9 MB

// The scratch itself. Every GPU that loads this library holds one copy until
// the process exits. Calls share it, so calls that overlap on the GPU race.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// Device address of the scratch, looked up once per device (with that device
// current) on the first call. The name is only a host-side stand-in; kernels
// must get this address. The cached address belongs to the device's current
// context: after cudaDeviceReset it is stale, so the entry point must not be
// used across a reset.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};
int g_sm_count[kMaxDevices] = {};
size_t g_smem_optin[kMaxDevices] = {};

thread_local std::string s_err;
int sfail(int code, const std::string& m) {
  s_err = m;
  return code;
}

const KernelEntry* find_entry(int bu, int bv, int p) {
  int n = 0;
  const KernelEntry* t = p == 1 ? kernels_p1(&n) : p == 2 ? kernels_p2(&n) : p == 4 ? kernels_p4(&n) : nullptr;
  for (int i = 0; t && i < n; ++i)
    if (t[i].bu == bu && t[i].bv == bv) return &t[i];
  return nullptr;
}

}  // namespace

extern "C" {

const char* grid_patch_static_last_error(void) { return s_err.c_str(); }

int grid_patch_static(int G, int S, int oversample, int npol, int Bu, int Bv, int precision, int64_t n_vis,
                      const double* uv, const void* vis, const float* weights, const void* kernel_table, void* grid,
                      cudaStream_t stream) {
  s_err.clear();
  // ---- argument checks (host only)
  if (G < 2 || G > 32768 || (G & 1)) return sfail(GRID_ERR_INVALID, "G must be even, 2..32768");
  if (S < 1 || S > 64 || S > G) return sfail(GRID_ERR_INVALID, "S must be 1..64 and <= G");
  if (oversample < 1 || oversample > 256 || (oversample & (oversample - 1)))
    return sfail(GRID_ERR_INVALID, "oversample must be a power of two <= 256");
  if (npol != 1 && npol != 2 && npol != 4) return sfail(GRID_ERR_UNSUPPORTED, "npol must be 1, 2 or 4");
  if (precision < GRID_PREC_F32 || precision > GRID_PREC_F16) return sfail(GRID_ERR_INVALID, "bad precision");
  if (n_vis < 0) return sfail(GRID_ERR_INVALID, "n_vis < 0");
  if (!kernel_table || !grid || ((uintptr_t)grid % 16)) return sfail(GRID_ERR_INVALID, "null kernel_table, or null or misaligned grid");
  if (n_vis == 0) return GRID_OK;
  if (!uv || !vis || ((uintptr_t)uv % 16)) return sfail(GRID_ERR_INVALID, "null uv or vis, or misaligned uv");
  const size_t vb = (precision == GRID_PREC_F32 ? 8 : 4) * (size_t)npol;
  if ((uintptr_t)vis % (vb >= 16 ? 16 : vb)) return sfail(GRID_ERR_INVALID, "misaligned vis");
  if ((uintptr_t)weights % 4) return sfail(GRID_ERR_INVALID, "weights must be 4-byte aligned");
  const long long n_chunks = (n_vis + kStaticChunkLen - 1) / kStaticChunkLen;
  if (n_chunks > kStaticMaxChunks)
    return sfail(GRID_ERR_INVALID, "n_vis above the static-scratch limit of " +
                                       std::to_string(kStaticMaxChunks * kStaticChunkLen) + " visibilities");
  const KernelEntry* k = find_entry(Bu, Bv, npol);
  if (!k) return sfail(GRID_ERR_UNSUPPORTED, "no kernel built for this (Bu, Bv, npol)");

  // ---- per-device set-up on the first call (no allocation)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return sfail(GRID_ERR_UNSUPPORTED, "device index out of range");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      int sms = 0, optin = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, cudaGetErrorString(e));
      g_sm_count[dev] = sms;
      g_smem_optin[dev] = (size_t)optin;
      g_addr[dev] = (unsigned char*)p;
    }
    scratch = g_addr[dev];
  }

  // ---- geometry (the same rules as grid_plan_create_ex with the patch schedule)
  Geometry g;
  memset(&g, 0, sizeof g);
  g.G = G; g.S = S; g.O = oversample; g.h = (S - 1) / 2; g.P = npol;
  while ((1 << g.log2O) < oversample) ++g.log2O;
  finish_geometry(g, Bu, Bv);
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, k->grid_patch_fn);
  if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  if (g.ts > fa.maxThreadsPerBlock) return sfail(GRID_ERR_UNSUPPORTED, "team does not fit in a CTA");
  g.tpc = 384 / g.ts;
  if (g.tpc < 1) g.tpc = 1;
  while (g.tpc > 1 && g.tpc * g.ts > fa.maxThreadsPerBlock) --g.tpc;
  const int threads = g.tpc * g.ts;
  const size_t smem_max = g_smem_optin[dev];
  const int halo = 12;
  int patch = npol == 4 ? 32 : npol == 2 ? 48 : 96;
  int win = 0;
  for (;;) {
    win = patch + 2 * halo + (g.nbu > g.nbv ? g.nbu : g.nbv);
    win = (win + 15) & ~15;
    if (k->grid_smem(g, threads, win) + fa.sharedSizeBytes + 1024 <= smem_max || patch <= 8) break;
    patch -= 8;
  }
  const size_t smem = k->grid_smem(g, threads, win);
  if (smem + fa.sharedSizeBytes > smem_max) return sfail(GRID_ERR_UNSUPPORTED, "patch window does not fit in shared memory");
  const int n_pu = (G + patch - 1) / patch;
  if (n_pu * n_pu > kStaticMaxPatches)
    return sfail(GRID_ERR_INVALID, "grid has more patches than the static scratch holds (" +
                                       std::to_string(kStaticMaxPatches) + ")");
  e = cudaFuncSetAttribute(k->grid_patch_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(smem_max - fa.sharedSizeBytes));
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k->grid_patch_fn, threads, smem);
  if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  if (occ < 1) return sfail(GRID_ERR_UNSUPPORTED, "gridding kernel cannot be resident with this shape");

  // ---- scratch views into the static array
  PatchScratch ps;
  memset(&ps, 0, sizeof ps);
  ps.patch = patch;
  ps.n_pu = n_pu;
  ps.n_patches = n_pu * n_pu;
  ps.halo_lo = halo;
  ps.win = win;
  ps.max_chunks = kStaticMaxChunksPerItem;
  ps.max_work = kStaticMaxWork;
  ps.patch_count = (int*)(scratch + kOffPatchCount);
  ps.patch_off = (int*)(scratch + kOffPatchOff);
  ps.chunk_patch = (int*)(scratch + kOffChunkPatch);
  ps.chunk_slot = (int*)(scratch + kOffChunkSlot);
  ps.chunk_order = (int*)(scratch + kOffChunkOrder);
  ps.work = (int4*)(scratch + kOffWork);
  ps.n_work = (int*)(scratch + kOffNWork);
  ps.work_next = (int*)(scratch + kOffWorkNext);
  unsigned long long* skipped = (unsigned long long*)(scratch + kOffSkipped);

  Args a;
  memset(&a, 0, sizeof a);
  a.g = g;
  a.n_vis = n_vis;
  a.uv = (const double2*)uv;
  a.vis = vis;
  a.vis_fmt = precision;
  a.weights = weights;
  a.table = kernel_table;
  a.tab_fmt = precision;
  a.grid = (float2*)grid;
  a.chunk_len = kStaticChunkLen;
  a.n_chunks = n_chunks;
  a.warp_sync = (g.ts <= 32 && 32 % g.ts == 0) ? 1 : 0;
  a.skipped = skipped;
  // the counters the previous call left behind must start at zero; the
  // binning launch below also clears the patch counts and the work counter
  e = cudaMemsetAsync(skipped, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  e = launch_patch_binning(a, ps, stream);
  if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, std::string("binning: ") + cudaGetErrorString(e));
  a.chunk_order = ps.chunk_order;
  a.work = ps.work;
  a.n_work = ps.n_work;
  a.work_next = ps.work_next;
  a.win = win;
  long long blocks = (long long)g_sm_count[dev] * occ;
  const long long max_items = ps.n_patches + n_chunks / ps.max_chunks + 1;
  if (blocks > max_items) blocks = max_items;
  void* args[] = {&a};
  e = cudaLaunchKernel(k->grid_patch_fn, dim3((unsigned)blocks), dim3(threads), args, smem, stream);
  if (e != cudaSuccess) return sfail(GRID_ERR_CUDA, std::string("grid kernel launch: ") + cudaGetErrorString(e));
  return GRID_OK;
}

}  // extern "C"
