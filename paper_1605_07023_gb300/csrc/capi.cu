// C ABI of the GB300 gridder: plan management, validation and kernel launch.
// The declarations and their contracts are in include/gridder.h.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "../../include/gridder.h"
#include "internal.h"

using namespace gbg;

struct grid_plan_s {
  grid_plan_desc desc;
  Geometry g;
  int device;
  int sm_count;
  int threads;          // threads per CTA (tpc * ts)
  int chunk_len;
  const KernelEntry* k;
  const void* grid_fn;  // gridding kernel of the plan's schedule
  size_t smem_grid;     // dynamic shared memory of the gridding kernel
  size_t smem_degrid;
  int occ_grid;         // resident gridding CTAs per SM (patch schedule)
  int warp_sync;        // team size divides 32: teams synchronise per warp
  const TileKernel* tile;  // tile schedule: the degridding kernel, its CTA size and shared memory
  TileKernel tile_any;     // the run-time-support kernel's entry, when `tile` points here
  int tile_threads;
  size_t tile_smem;
  int occ_tile;            // resident tile-degridding CTAs per SM
  const void* rot_fn;      // chunked schedule with rotated tables (teams of at most 64 threads), else null
  int rot_tpc;             // its teams per CTA
  int rot_threads;
  size_t rot_smem;
  const LazyEntry* lazy;   // lazy-box schedule: the gridding kernel, its geometry and launch shape
  Geometry gl;             // the widened bin (nu, nv, ts) of the lazy gridder
  int lazy_threads;
  int lazy_teams;          // teams per CTA
  int seg;                 // lanes per team slot
  size_t lazy_smem;
  unsigned long long* d_skipped;
  PatchScratch ps;
  long long ps_chunks_cap;  // chunk capacity of the patch scratch
  void* cs_buf;             // compression scratch (grow-only)
  size_t cs_bytes;
  cudaStream_t cstream;     // copy stream of grid_degrid_host (created on first use)
  cudaStream_t dstream;     // download stream of grid_degrid_host_steps (created on first use)
  cudaEvent_t* evs;         // their events (grow-only)
  int n_evs;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(GRID_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int x) { int r = 0; while ((1 << r) < x) ++r; return r; }
size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

const LazyEntry* find_lazy_kernel(int bu, int bv, int p) {
  int n = 0;
  const LazyEntry* t = p == 1 ? lazy_kernels_p1(&n) : p == 2 ? lazy_kernels_p2(&n) : p == 4 ? lazy_kernels_p4(&n) : nullptr;
  for (int i = 0; t && i < n; ++i)
    if (t[i].bu == bu && t[i].bv == bv) return &t[i];
  return nullptr;
}

const RotEntry* find_rot_kernel(int bu, int bv, int p) {
  int n = 0;
  const RotEntry* t = p == 1 ? rot_kernels_p1(&n) : p == 2 ? rot_kernels_p2(&n) : p == 4 ? rot_kernels_p4(&n) : nullptr;
  for (int i = 0; t && i < n; ++i)
    if (t[i].bu == bu && t[i].bv == bv) return &t[i];
  return nullptr;
}

const KernelEntry* find_kernel(int bu, int bv, int p) {
  int n = 0;
  const KernelEntry* t = p == 1 ? kernels_p1(&n) : p == 2 ? kernels_p2(&n) : p == 4 ? kernels_p4(&n) : nullptr;
  for (int i = 0; t && i < n; ++i)
    if (t[i].bu == bu && t[i].bv == bv) return &t[i];
  return nullptr;
}

size_t tables_bytes(const Geometry& g, int bu, int bv) {
  return a16((size_t)g.O * bu * g.nbu * 8) + a16((size_t)g.O * bv * g.nbv * 8);
}

void free_patch(grid_plan_s* pl) {
  PatchScratch& s = pl->ps;
  cudaFree(s.patch_count); cudaFree(s.patch_off); cudaFree(s.chunk_patch); cudaFree(s.chunk_slot);
  cudaFree(s.chunk_order); cudaFree(s.work); cudaFree(s.n_work); cudaFree(s.work_next);
  s.patch_count = s.patch_off = s.chunk_patch = s.chunk_slot = s.chunk_order = s.n_work = s.work_next = nullptr;
  s.work = nullptr;
  pl->ps_chunks_cap = 0;
}

int ensure_patch_scratch(grid_plan_s* pl, long long n_chunks) {
  if (n_chunks <= pl->ps_chunks_cap) return GRID_OK;
  free_patch(pl);
  PatchScratch& s = pl->ps;
  const long long cap = n_chunks + n_chunks / 4 + 64;
  s.max_work = (int)(s.n_patches + cap / s.max_chunks + 2);
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMalloc(&s.patch_count, sizeof(int) * s.n_patches);
  e = e ? e : cudaMalloc(&s.patch_off, sizeof(int) * (s.n_patches + 1));
  e = e ? e : cudaMalloc(&s.chunk_patch, sizeof(int) * cap);
  e = e ? e : cudaMalloc(&s.chunk_slot, sizeof(int) * cap);
  e = e ? e : cudaMalloc(&s.chunk_order, sizeof(int) * cap);
  e = e ? e : cudaMalloc(&s.work, sizeof(int4) * s.max_work);
  e = e ? e : cudaMalloc(&s.n_work, sizeof(int));
  e = e ? e : cudaMalloc(&s.work_next, sizeof(int));
  if (e != cudaSuccess) {
    free_patch(pl);
    return fail(GRID_ERR_NOMEM, "patch scratch allocation failed: %s", cudaGetErrorString(e));
  }
  pl->ps_chunks_cap = cap;
  return GRID_OK;
}

// Pointer checks: non-null and aligned as the kernels' vector accesses need.
bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

Args make_args(const grid_plan_s* pl, int64_t n_vis, const double* uv) {
  Args a;
  memset(&a, 0, sizeof a);
  a.g = pl->g;
  a.n_vis = n_vis;
  a.uv = (const double2*)uv;
  a.chunk_len = pl->chunk_len;
  a.n_chunks = (n_vis + pl->chunk_len - 1) / pl->chunk_len;
  a.skipped = pl->d_skipped;
  a.vis_fmt = pl->desc.precision;
  a.tab_fmt = pl->desc.precision;
  a.warp_sync = pl->warp_sync;
  return a;
}

// At least n events in the plan's pool (grow-only; created without timing).
int ensure_events(grid_plan_s* pl, int n) {
  if (pl->n_evs >= n) return GRID_OK;
  cudaEvent_t* ev = new cudaEvent_t[n];
  cudaError_t e = cudaSuccess;
  int made = 0;
  for (; made < n; ++made) {
    if (made < pl->n_evs) {
      ev[made] = pl->evs[made];
    } else {
      e = cudaEventCreateWithFlags(&ev[made], cudaEventDisableTiming);
      if (e != cudaSuccess) break;
    }
  }
  if (e != cudaSuccess) {
    for (int i = pl->n_evs; i < made; ++i) cudaEventDestroy(ev[i]);
    delete[] ev;
    return cuda_fail(e, "cudaEventCreateWithFlags");
  }
  delete[] pl->evs;
  pl->evs = ev;
  pl->n_evs = n;
  return GRID_OK;
}

int check_device(const grid_plan_s* pl) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != pl->device) return fail(GRID_ERR_INVALID, "plan was created on device %d, current device is %d", pl->device, dev);
  return GRID_OK;
}

}  // namespace

extern "C" {

const char* grid_last_error(void) { return g_err.c_str(); }

void grid_plan_desc_init(grid_plan_desc* d, int G, int S, int oversample, int npol, int B) {
  if (!d) return;
  memset(d, 0, sizeof *d);
  d->G = G; d->S = S; d->oversample = oversample; d->npol = npol; d->Bu = B; d->Bv = B;
  d->vis_per_chunk = 0; d->threads = 0; d->precision = GRID_PREC_F32; d->schedule = GRID_SCHED_CHUNKED; d->patch = 0;
  d->bin_u = 0; d->bin_v = 0; d->tile_group = 0;
}

int grid_plan_create(grid_plan_t* out, int G, int S, int oversample, int npol, int B) {
  grid_plan_desc d;
  grid_plan_desc_init(&d, G, S, oversample, npol, B);
  return grid_plan_create_ex(out, &d);
}

int grid_plan_create_ex(grid_plan_t* out, const grid_plan_desc* din) {
  g_err.clear();
  if (!out || !din) return fail(GRID_ERR_INVALID, "null argument");
  *out = nullptr;
  grid_plan_desc d = *din;
  if (d.G < 2 || d.G > 32768 || (d.G & 1)) return fail(GRID_ERR_INVALID, "G=%d: must be even, 2..32768", d.G);
  if (d.S < 1 || d.S > 64 || d.S > d.G) return fail(GRID_ERR_INVALID, "S=%d: must be 1..64 and <= G", d.S);
  if (!is_pow2(d.oversample) || d.oversample > 256) return fail(GRID_ERR_INVALID, "oversample=%d: must be a power of two <= 256", d.oversample);
  if (d.npol != 1 && d.npol != 2 && d.npol != 4) return fail(GRID_ERR_INVALID, "npol=%d: must be 1, 2 or 4", d.npol);
  if (d.Bu < 1 || d.Bu > 8 || d.Bv < 1 || d.Bv > 8) return fail(GRID_ERR_INVALID, "B=(%d,%d): must be 1..8", d.Bu, d.Bv);
  if (d.precision < GRID_PREC_F32 || d.precision > GRID_PREC_F16) return fail(GRID_ERR_INVALID, "precision=%d", d.precision);
  if (d.schedule != GRID_SCHED_CHUNKED && d.schedule != GRID_SCHED_PATCH && d.schedule != GRID_SCHED_TILE &&
      d.schedule != GRID_SCHED_LAZY && d.schedule != GRID_SCHED_SORTED)
    return fail(GRID_ERR_INVALID, "schedule=%d", d.schedule);
  if (d.threads % 32 != 0 && (d.schedule == GRID_SCHED_TILE || d.schedule == GRID_SCHED_LAZY))
    return fail(GRID_ERR_INVALID, "threads=%d: the tile and lazy schedules need whole warps", d.threads);
  if (d.schedule != GRID_SCHED_LAZY && (d.bin_u != 0 || d.bin_v != 0))
    return fail(GRID_ERR_INVALID, "bin_u/bin_v apply to the lazy schedule only");
  if (d.tile_group != 0 && (d.schedule != GRID_SCHED_TILE || (d.tile_group != 32 && d.tile_group != 8)))
    return fail(GRID_ERR_INVALID, "tile_group=%d: 32 or 8 (0 = 32), for the tile schedule only", d.tile_group);
  if (d.vis_per_chunk < 0 || d.vis_per_chunk > (1 << 20)) return fail(GRID_ERR_INVALID, "vis_per_chunk=%d", d.vis_per_chunk);
  if (d.threads < 0 || d.threads > 1024) return fail(GRID_ERR_INVALID, "threads=%d", d.threads);
  // the chunked kernels of the plan's shape; a lazy-schedule shape that has none degrids with 2x2 blocks
  int kbu = d.Bu, kbv = d.Bv;
  const KernelEntry* k = find_kernel(kbu, kbv, d.npol);
  if (!k && d.schedule == GRID_SCHED_LAZY) {
    kbu = kbv = 2;
    k = find_kernel(kbu, kbv, d.npol);
  }
  if (!k) return fail(GRID_ERR_UNSUPPORTED, "no kernel built for Bu=%d Bv=%d npol=%d", d.Bu, d.Bv, d.npol);

  grid_plan_s* pl = new grid_plan_s;
  memset(pl, 0, sizeof *pl);
  pl->k = k;
  Geometry& g = pl->g;
  g.G = d.G; g.S = d.S; g.O = d.oversample; g.log2O = ilog2(d.oversample); g.h = (d.S - 1) / 2; g.P = d.npol;
  finish_geometry(g, kbu, kbv);

  cudaError_t e = cudaGetDevice(&pl->device);
  if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaGetDevice"); }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, pl->device);
  if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaGetDeviceProperties"); }
  pl->sm_count = prop.multiProcessorCount;
  pl->grid_fn = d.schedule == GRID_SCHED_PATCH ? k->grid_patch_fn : k->grid_fn;
  cudaFuncAttributes fa_g, fa_d;
  e = cudaFuncGetAttributes(&fa_g, pl->grid_fn);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa_d, k->degrid_fn);
  if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncGetAttributes (is this an sm_103 GPU?)"); }
  const int max_thr = fa_g.maxThreadsPerBlock < fa_d.maxThreadsPerBlock ? fa_g.maxThreadsPerBlock : fa_d.maxThreadsPerBlock;
  if (g.ts > max_thr) {
    const int ts = g.ts;
    delete pl;
    return fail(GRID_ERR_UNSUPPORTED, "team of %d threads exceeds the %d threads per CTA this kernel can run", ts, max_thr);
  }
  const int target = d.threads > 0 ? d.threads : (d.schedule == GRID_SCHED_PATCH ? 384 : 256);
  g.tpc = target / g.ts;
  if (g.tpc < 1) g.tpc = 1;
  while (g.tpc > 1 && g.tpc * g.ts > max_thr) --g.tpc;
  pl->threads = g.tpc * g.ts;
  pl->warp_sync = (g.ts <= 32 && 32 % g.ts == 0) ? 1 : 0;

  if (d.vis_per_chunk == 0) d.vis_per_chunk = d.schedule == GRID_SCHED_PATCH ? 64 : 256;
  pl->chunk_len = d.vis_per_chunk;

  const size_t tb = tables_bytes(g, kbu, kbv);
  if (tb > 96 * 1024) {
    delete pl;
    return fail(GRID_ERR_UNSUPPORTED, "padded GCF tables need %zu bytes of shared memory (> 96 KiB)", tb);
  }
  const size_t smem_max = prop.sharedMemPerBlockOptin;

  int win = 0;
  if (d.schedule == GRID_SCHED_PATCH) {
    PatchScratch& s = pl->ps;
    int patch = d.patch;
    const int halo = 12;
    if (patch <= 0) patch = d.npol == 4 ? 32 : d.npol == 2 ? 48 : 96;
    patch = (patch + 1) & ~1;  // even, so window rows start on 16-byte boundaries
    // shrink the patch until the window fits next to the tables and records
    for (;;) {
      win = patch + 2 * halo + (g.nbu > g.nbv ? g.nbu : g.nbv);
      win = (win + 15) & ~15;  // a multiple of 16 (bank-conflict-free strides)
      if (k->grid_smem(g, pl->threads, win) + fa_g.sharedSizeBytes + 1024 <= smem_max || patch <= 8) break;
      patch -= 8;
    }
    if (patch < 1 || k->grid_smem(g, pl->threads, win) + fa_g.sharedSizeBytes + 1024 > smem_max) {
      delete pl;
      return fail(GRID_ERR_UNSUPPORTED, "patch window does not fit in shared memory");
    }
    d.patch = patch;
    s.patch = patch;
    s.n_pu = (g.G + patch - 1) / patch;
    s.n_patches = s.n_pu * s.n_pu;
    s.halo_lo = halo;
    s.win = win;
    s.max_chunks = 256;
  }
  if (d.schedule != GRID_SCHED_PATCH) {
    // small teams (tiny S and B) put many teams in a CTA: shrink the CTA until
    // its staging buffers fit
    while (g.tpc > 1 && (k->grid_smem(g, g.tpc * g.ts, 0) + fa_g.sharedSizeBytes > smem_max ||
                         k->degrid_smem(g, g.tpc * g.ts, 0) + fa_d.sharedSizeBytes > smem_max))
      --g.tpc;
    pl->threads = g.tpc * g.ts;
  }
  pl->smem_grid = k->grid_smem(g, pl->threads, win);
  pl->smem_degrid = k->degrid_smem(g, pl->threads, 0);
  if (pl->smem_grid + fa_g.sharedSizeBytes > smem_max || pl->smem_degrid + fa_d.sharedSizeBytes > smem_max) {
    delete pl;
    return fail(GRID_ERR_UNSUPPORTED, "kernel needs more shared memory than the device offers");
  }
  // Kernels are shared by every plan with the same (Bu, Bv, P), so each one's dynamic shared
  // memory limit is raised to the device maximum once, not to this plan's need.
  e = cudaFuncSetAttribute(pl->grid_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_max - fa_g.sharedSizeBytes));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k->degrid_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_max - fa_d.sharedSizeBytes));
  if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncSetAttribute"); }
  if (d.schedule == GRID_SCHED_PATCH) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl->occ_grid, pl->grid_fn, pl->threads, pl->smem_grid);
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor"); }
    if (pl->occ_grid < 1) { delete pl; return fail(GRID_ERR_UNSUPPORTED, "gridding kernel cannot be resident with this shape"); }
  }
  if (d.schedule == GRID_SCHED_TILE) {
    if (d.tile_group == 0) d.tile_group = 32;
    const int lpv = 32 / d.tile_group;  // lanes per visibility
    const TileKernel* t = find_tile_kernel(d.S, d.npol, lpv);
    if (!t) {
      // no unrolled kernel for this support: the run-time-support one
      if (tile_kernel_any(d.S, d.npol, lpv, &pl->tile_any)) {
        delete pl;
        return fail(GRID_ERR_UNSUPPORTED, "tile schedule: no kernel for S=%d npol=%d", d.S, d.npol);
      }
      t = &pl->tile_any;
    }
    cudaFuncAttributes fa_t;
    e = cudaFuncGetAttributes(&fa_t, t->fn);
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncGetAttributes (tile)"); }
    int warps = (d.threads > 0 ? d.threads : 256) / 32;
    if (warps * 32 > fa_t.maxThreadsPerBlock) warps = fa_t.maxThreadsPerBlock / 32;
    while (warps > 1 && tile_smem_bytes(*t, g.O, warps) + fa_t.sharedSizeBytes > smem_max) --warps;
    if (warps < 1 || tile_smem_bytes(*t, g.O, warps) + fa_t.sharedSizeBytes > smem_max) {
      delete pl;
      return fail(GRID_ERR_UNSUPPORTED, "tile schedule: one warp's tile does not fit in shared memory");
    }
    e = cudaFuncSetAttribute(t->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_max - fa_t.sharedSizeBytes));
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncSetAttribute (tile)"); }
    pl->tile = t;
    pl->tile_threads = warps * 32;
    pl->tile_smem = tile_smem_bytes(*t, g.O, warps);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pl->occ_tile, t->fn, pl->tile_threads, pl->tile_smem);
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor (tile)"); }
    if (pl->occ_tile < 1) { delete pl; return fail(GRID_ERR_UNSUPPORTED, "tile degridding kernel cannot be resident"); }
  }
  if (d.schedule == GRID_SCHED_LAZY) {
    const LazyEntry* lk = find_lazy_kernel(d.Bu, d.Bv, d.npol);
    if (!lk) { delete pl; return fail(GRID_ERR_UNSUPPORTED, "lazy schedule: no kernel for Bu=%d Bv=%d npol=%d", d.Bu, d.Bv, d.npol); }
    // default bin: the paper's, widened by one block along each axis where it leaves a footprint
    // less than a block of room, while the team stays within a warp
    // the paper's bin for these blocks (Sec. 3): the smallest multiple of B that holds S + B - 1 cells
    const int mbu = ((d.S + 2 * d.Bu - 2) / d.Bu) * d.Bu, mbv = ((d.S + 2 * d.Bv - 2) / d.Bv) * d.Bv;
    if (d.bin_u == 0) d.bin_u = mbu + (mbu - d.S < d.Bu && (mbu / d.Bu + 1) * (mbv / d.Bv) <= 32 ? d.Bu : 0);
    if (d.bin_v == 0) d.bin_v = mbv + (mbv - d.S < d.Bv && (d.bin_u / d.Bu) * (mbv / d.Bv + 1) <= 32 ? d.Bv : 0);
    if (d.bin_u % d.Bu || d.bin_v % d.Bv || d.bin_u < mbu || d.bin_v < mbv || d.bin_u > 1024 || d.bin_v > 1024) {
      const int bu = d.bin_u, bv = d.bin_v, mu = mbu, mv = mbv;
      delete pl;
      return fail(GRID_ERR_INVALID, "bin %dx%d: sides must be multiples of (Bu, Bv) and at least %dx%d", bu, bv, mu, mv);
    }
    Geometry& gl = pl->gl;
    gl = g;
    gl.nu = d.bin_u / d.Bu;
    gl.nv = d.bin_v / d.Bv;
    gl.nbu = d.bin_u;
    gl.nbv = d.bin_v;
    gl.ts = gl.nu * gl.nv;
    gl.nuB = gl.nbu;
    gl.nvB = gl.nbv;
    gl.mu = (unsigned)((1ull << 31) / (unsigned)gl.nu + 1);
    gl.mv = (unsigned)((1ull << 31) / (unsigned)gl.nv + 1);
    gl.mbu = (unsigned)((1ull << 31) / (unsigned)gl.nbu + 1);
    gl.mbv = (unsigned)((1ull << 31) / (unsigned)gl.nbv + 1);
    if (gl.ts > 32) {
      const int ts = gl.ts;  // gl belongs to the plan
      delete pl;
      return fail(GRID_ERR_UNSUPPORTED, "lazy schedule: %d threads per team (more than a warp)", ts);
    }
    int seg = 1;
    while (seg < gl.ts) seg <<= 1;
    cudaFuncAttributes fa_l;
    e = cudaFuncGetAttributes(&fa_l, lk->fn);
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncGetAttributes (lazy)"); }
    int warps = (d.threads > 0 ? d.threads : 128) / 32;
    if (warps * 32 > fa_l.maxThreadsPerBlock) warps = fa_l.maxThreadsPerBlock / 32;
    while (warps > 1 && lk->smem(gl, warps * (32 / seg)) + fa_l.sharedSizeBytes > smem_max) --warps;
    const size_t sm = lk->smem(gl, warps * (32 / seg));
    if (warps < 1 || sm + fa_l.sharedSizeBytes > smem_max) {
      delete pl;
      return fail(GRID_ERR_UNSUPPORTED, "lazy schedule: tables and records do not fit in shared memory");
    }
    e = cudaFuncSetAttribute(lk->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_max - fa_l.sharedSizeBytes));
    if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncSetAttribute (lazy)"); }
    gl.tpc = warps * (32 / seg);
    pl->lazy = lk;
    pl->seg = seg;
    pl->lazy_threads = warps * 32;
    pl->lazy_teams = gl.tpc;
    pl->lazy_smem = sm;
  }
  if (d.schedule == GRID_SCHED_SORTED) {
    // box-ordered batches and rotated tables: teams of at most 64 threads whose CTA fits in
    // shared memory
    const RotEntry* re = find_rot_kernel(kbu, kbv, d.npol);
    if (!re || g.ts > 64) {
      const int ts = g.ts;
      delete pl;
      return fail(GRID_ERR_UNSUPPORTED, "sorted schedule: %d threads per team (at most 64)", ts);
    }
    {
      const void* fn = g.ts <= 32 ? re->fn : re->fn_wide;
      cudaFuncAttributes fa_r;
      e = cudaFuncGetAttributes(&fa_r, fn);
      if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncGetAttributes (rotated)"); }
      Geometry gr = g;
      const int target = d.threads > 0 ? d.threads : 256;
      gr.tpc = target / g.ts;
      if (gr.tpc < 1) gr.tpc = 1;
      while (gr.tpc > 1 && gr.tpc * g.ts > fa_r.maxThreadsPerBlock) --gr.tpc;
      size_t (*const smem_of)(const Geometry&) = g.ts <= 32 ? re->smem : re->smem_wide;
      while (gr.tpc > 1 && smem_of(gr) + fa_r.sharedSizeBytes > smem_max) --gr.tpc;
      if (g.ts <= fa_r.maxThreadsPerBlock && smem_of(gr) + fa_r.sharedSizeBytes <= smem_max) {
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_max - fa_r.sharedSizeBytes));
        if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaFuncSetAttribute (rotated)"); }
        pl->rot_fn = fn;
        pl->rot_tpc = gr.tpc;
        pl->rot_threads = gr.tpc * g.ts;
        pl->rot_smem = smem_of(gr);
      }
    }
    if (!pl->rot_fn) {
      delete pl;
      return fail(GRID_ERR_UNSUPPORTED, "sorted schedule: tables and records do not fit in shared memory");
    }
  }
  // word 0: skipped visibilities; word 1: status flags of the lazy gridder
  e = cudaMalloc(&pl->d_skipped, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) { delete pl; return fail(GRID_ERR_NOMEM, "cudaMalloc: %s", cudaGetErrorString(e)); }
  e = cudaMemset(pl->d_skipped, 0, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) { cudaFree(pl->d_skipped); delete pl; return cuda_fail(e, "cudaMemset"); }
  pl->desc = d;
  *out = pl;
  return GRID_OK;
}

void grid_plan_destroy(grid_plan_t pl) {
  if (!pl) return;
  free_patch(pl);
  cudaFree(pl->cs_buf);
  for (int i = 0; i < pl->n_evs; ++i) cudaEventDestroy(pl->evs[i]);
  delete[] pl->evs;
  if (pl->cstream) cudaStreamDestroy(pl->cstream);
  if (pl->dstream) cudaStreamDestroy(pl->dstream);
  cudaFree(pl->d_skipped);
  delete pl;
}

int grid_plan_describe(grid_plan_t pl, grid_plan_desc* desc, int* bin_u, int* bin_v, int* team_size) {
  if (!pl) return fail(GRID_ERR_INVALID, "null plan");
  const Geometry& g = pl->lazy ? pl->gl : pl->g;
  if (desc) { *desc = pl->desc; desc->threads = pl->lazy ? pl->lazy_threads : pl->threads; }
  if (bin_u) *bin_u = g.nbu;
  if (bin_v) *bin_v = g.nbv;
  if (team_size) *team_size = g.ts;
  return GRID_OK;
}

int grid(grid_plan_t pl, int64_t n_vis, const double* uv, const void* vis, const float* weights, const void* kernel_table,
         void* grid_out, cudaStream_t stream) {
  g_err.clear();
  if (!pl) return fail(GRID_ERR_INVALID, "null plan");
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis=%lld out of range", (long long)n_vis);
  if (!kernel_table || !grid_out) return fail(GRID_ERR_INVALID, "null kernel_table or grid");
  if (!aligned(grid_out, 16)) return fail(GRID_ERR_INVALID, "grid must be 16-byte aligned");
  if (n_vis == 0) return GRID_OK;
  if (!uv || !vis) return fail(GRID_ERR_INVALID, "null uv or vis");
  if (!aligned(uv, 16)) return fail(GRID_ERR_INVALID, "uv must be 16-byte aligned");
  const size_t vbytes = (pl->desc.precision == GRID_PREC_F32 ? 8 : 4) * (size_t)pl->g.P;
  if (!aligned(vis, vbytes >= 16 ? 16 : vbytes)) return fail(GRID_ERR_INVALID, "vis must be %zu-byte aligned", vbytes >= 16 ? (size_t)16 : vbytes);
  if (weights && !aligned(weights, 4)) return fail(GRID_ERR_INVALID, "weights must be 4-byte aligned");
  int rc = check_device(pl);
  if (rc) return rc;
  if (pl->chunk_len > 0 && (n_vis + pl->chunk_len - 1) / pl->chunk_len > 0x7FFFFFFFLL)
    return fail(GRID_ERR_INVALID, "too many chunks");

  Args a = make_args(pl, n_vis, uv);
  a.vis = vis;
  a.weights = weights;
  a.table = kernel_table;
  a.grid = (float2*)grid_out;
  cudaError_t e;
  if (pl->lazy) {
    a.g = pl->gl;
    a.seg = pl->seg;
    a.status = (unsigned*)(pl->d_skipped + 1);
    const long long blocks = (a.n_chunks + pl->lazy_teams - 1) / pl->lazy_teams;
    if (blocks > 0x7FFFFFFFLL) return fail(GRID_ERR_INVALID, "too many chunks");
    void* args[] = {&a};
    e = cudaLaunchKernel(pl->lazy->fn, dim3((unsigned)blocks), dim3(pl->lazy_threads), args, pl->lazy_smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid (lazy) kernel launch");
    return GRID_OK;
  }
  if (pl->rot_fn) {
    a.g.tpc = pl->rot_tpc;
    const long long blocks = (a.n_chunks + pl->rot_tpc - 1) / pl->rot_tpc;
    if (blocks > 0x7FFFFFFFLL) return fail(GRID_ERR_INVALID, "too many chunks");
    void* args[] = {&a};
    e = cudaLaunchKernel(pl->rot_fn, dim3((unsigned)blocks), dim3(pl->rot_threads), args, pl->rot_smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid (rotated) kernel launch");
    return GRID_OK;
  }
  if (pl->desc.schedule != GRID_SCHED_PATCH) {
    const long long blocks = (a.n_chunks + pl->g.tpc - 1) / pl->g.tpc;
    void* args[] = {&a};
    e = cudaLaunchKernel(pl->grid_fn, dim3((unsigned)blocks), dim3(pl->threads), args, pl->smem_grid, stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid kernel launch");
    return GRID_OK;
  }
  rc = ensure_patch_scratch(pl, a.n_chunks);
  if (rc) return rc;
  const PatchScratch& s = pl->ps;
  e = launch_patch_binning(a, s, stream);
  if (e != cudaSuccess) return cuda_fail(e, "patch binning");
  a.chunk_order = s.chunk_order;
  a.work = s.work;
  a.n_work = s.n_work;
  a.work_next = s.work_next;
  a.win = s.win;
  long long blocks = (long long)pl->sm_count * pl->occ_grid;
  const long long max_items = s.n_patches + a.n_chunks / s.max_chunks + 1;
  if (blocks > max_items) blocks = max_items;
  void* args[] = {&a};
  e = cudaLaunchKernel(pl->grid_fn, dim3((unsigned)blocks), dim3(pl->threads), args, pl->smem_grid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "grid kernel launch");
  return GRID_OK;
}

int degrid(grid_plan_t pl, int64_t n_vis, const double* uv, const void* grid_in, const void* kernel_table, void* vis,
           cudaStream_t stream) {
  return degrid_weighted(pl, n_vis, uv, grid_in, kernel_table, nullptr, vis, stream);
}

int degrid_weighted(grid_plan_t pl, int64_t n_vis, const double* uv, const void* grid_in, const void* kernel_table,
                    const float* weights, void* vis, cudaStream_t stream) {
  g_err.clear();
  if (!pl) return fail(GRID_ERR_INVALID, "null plan");
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis=%lld out of range", (long long)n_vis);
  if (!kernel_table || !grid_in) return fail(GRID_ERR_INVALID, "null kernel_table or grid");
  if (!aligned(grid_in, 16)) return fail(GRID_ERR_INVALID, "grid must be 16-byte aligned");
  if (n_vis == 0) return GRID_OK;
  if (!uv || !vis) return fail(GRID_ERR_INVALID, "null uv or vis");
  if (!aligned(uv, 16) || !aligned(vis, 8)) return fail(GRID_ERR_INVALID, "uv must be 16-byte and vis 8-byte aligned");
  if (weights && !aligned(weights, 4)) return fail(GRID_ERR_INVALID, "weights must be 4-byte aligned");
  if ((n_vis + pl->chunk_len - 1) / pl->chunk_len > 0x7FFFFFFFLL) return fail(GRID_ERR_INVALID, "too many chunks");
  int rc = check_device(pl);
  if (rc) return rc;
  Args a = make_args(pl, n_vis, uv);
  a.weights = weights;
  a.table = kernel_table;
  a.grid = (float2*)grid_in;
  a.vis_out = (float2*)vis;
  a.status = (unsigned*)(pl->d_skipped + 1);
  void* args[] = {&a};
  cudaError_t e;
  if (pl->tile) {
    // the tensor maps of this grid (host-side encoding, passed by value)
    TileMaps maps;
    tile_maps(*pl->tile, grid_in, pl->g.G, pl->g.P, &maps);  // on failure maps.ok = 0: direct reads
    void* targs[] = {&a, &maps};
    // persistent warps, one group of 32 (or 8) visibilities at a time: one wave of resident CTAs
    const long long gs = 32 / pl->tile->lpv;
    const long long groups = (n_vis + gs - 1) / gs, wpc = pl->tile_threads / 32;
    long long blocks = (groups + wpc - 1) / wpc;
    if (blocks > (long long)pl->sm_count * pl->occ_tile) blocks = (long long)pl->sm_count * pl->occ_tile;
    e = cudaLaunchKernel(pl->tile->fn, dim3((unsigned)blocks), dim3(pl->tile_threads), targs, pl->tile_smem, stream);
    if (e != cudaSuccess) return cuda_fail(e, "degrid (tile) kernel launch");
    return GRID_OK;
  }
  const long long blocks = (a.n_chunks + pl->g.tpc - 1) / pl->g.tpc;
  e = cudaLaunchKernel(pl->k->degrid_fn, dim3((unsigned)blocks), dim3(pl->threads), args, pl->smem_degrid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "degrid kernel launch");
  return GRID_OK;
}

int grid_make_kernel_table(int S, int oversample, double beta, int precision, void* table_out, cudaStream_t stream) {
  g_err.clear();
  if (S < 1 || S > 64 || !is_pow2(oversample) || oversample > 256) return fail(GRID_ERR_INVALID, "S=%d oversample=%d", S, oversample);
  if (!(beta >= 0.0) || beta > 700.0) return fail(GRID_ERR_INVALID, "beta=%g out of range", beta);
  if (precision < GRID_PREC_F32 || precision > GRID_PREC_F16) return fail(GRID_ERR_INVALID, "precision=%d", precision);
  if (!table_out) return fail(GRID_ERR_INVALID, "null table_out");
  cudaError_t e = launch_kb_table(S, oversample, beta, precision, table_out, stream);
  if (e != cudaSuccess) return cuda_fail(e, "kb_table kernel launch");
  return GRID_OK;
}

int grid_compute_indices(grid_plan_t pl, int64_t n_vis, const double* uv, int32_t* cell, int32_t* sub, cudaStream_t stream) {
  g_err.clear();
  if (!pl) return fail(GRID_ERR_INVALID, "null plan");
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis out of range");
  if (n_vis == 0) return GRID_OK;
  if (!uv || !cell || !sub) return fail(GRID_ERR_INVALID, "null pointer");
  if (!aligned(uv, 16) || !aligned(cell, 8) || !aligned(sub, 8)) return fail(GRID_ERR_INVALID, "misaligned pointer");
  if ((n_vis + 255) / 256 > 0x7FFFFFFFLL) return fail(GRID_ERR_INVALID, "too many visibilities for one launch");
  int rc = check_device(pl);
  if (rc) return rc;
  Args a = make_args(pl, n_vis, uv);
  cudaError_t e = launch_indices(a, cell, sub, stream);
  if (e != cudaSuccess) return cuda_fail(e, "indices kernel launch");
  return GRID_OK;
}

int grid_plan_skipped(grid_plan_t pl, int64_t* n_skipped, int reset) {
  if (!pl || !n_skipped) return fail(GRID_ERR_INVALID, "null argument");
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpy(&v, pl->d_skipped, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  *n_skipped = (int64_t)v;
  if (reset) {
    e = cudaMemset(pl->d_skipped, 0, sizeof v);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  }
  return GRID_OK;
}

const char* grid_plan_gridder(grid_plan_t pl) {
  if (!pl) return "";
  if (pl->lazy) return "lazy";
  if (pl->rot_fn) return pl->g.ts <= 32 ? "sorted" : "sorted-wide";
  return pl->desc.schedule == GRID_SCHED_PATCH ? "patch" : "chunked";
}

int grid_plan_status(grid_plan_t pl, unsigned* flags, int reset) {
  g_err.clear();
  if (!pl || !flags) return fail(GRID_ERR_INVALID, "null argument");
  int rc = check_device(pl);
  if (rc) return rc;
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpy(&v, pl->d_skipped + 1, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (status)");
  *flags = (unsigned)v;
  if (reset) {
    e = cudaMemset(pl->d_skipped + 1, 0, sizeof v);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (status)");
  }
  return GRID_OK;
}

int grid_compress(grid_plan_t pl, int64_t n_vis, const double* uv, const void* vis, const float* weights,
                  double* uv_out, void* vis_out, int64_t* run_of, int64_t* n_out, cudaStream_t stream) {
  g_err.clear();
  if (!pl) return fail(GRID_ERR_INVALID, "null plan");
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis=%lld out of range", (long long)n_vis);
  if (!n_out || !aligned(n_out, 8)) return fail(GRID_ERR_INVALID, "n_out must be a non-null 8-byte aligned device pointer");
  int rc = check_device(pl);
  if (rc) return rc;
  if (n_vis == 0) {
    cudaError_t e = cudaMemsetAsync(n_out, 0, sizeof(int64_t), stream);
    return e == cudaSuccess ? GRID_OK : cuda_fail(e, "cudaMemsetAsync");
  }
  if (!uv || !vis || !uv_out || !vis_out) return fail(GRID_ERR_INVALID, "null uv, vis, uv_out or vis_out");
  if (!aligned(uv, 16) || !aligned(uv_out, 16)) return fail(GRID_ERR_INVALID, "uv and uv_out must be 16-byte aligned");
  const size_t vbytes = (pl->desc.precision == GRID_PREC_F32 ? 8 : 4) * (size_t)pl->g.P;
  if (!aligned(vis, vbytes >= 16 ? 16 : vbytes)) return fail(GRID_ERR_INVALID, "vis must be %zu-byte aligned", vbytes >= 16 ? (size_t)16 : vbytes);
  if (!aligned(vis_out, 8)) return fail(GRID_ERR_INVALID, "vis_out must be 8-byte aligned");
  if (weights && !aligned(weights, 4)) return fail(GRID_ERR_INVALID, "weights must be 4-byte aligned");
  if (run_of && !aligned(run_of, 8)) return fail(GRID_ERR_INVALID, "run_of must be 8-byte aligned");
  const size_t need = compress_scratch_bytes(n_vis, pl->g.P);
  if (need > pl->cs_bytes) {
    cudaFree(pl->cs_buf);
    pl->cs_buf = nullptr;
    pl->cs_bytes = 0;
    cudaError_t e = cudaMalloc(&pl->cs_buf, need + need / 4);
    if (e != cudaSuccess) return fail(GRID_ERR_NOMEM, "compression scratch allocation failed: %s", cudaGetErrorString(e));
    pl->cs_bytes = need + need / 4;
  }
  Args a = make_args(pl, n_vis, uv);
  a.vis = vis;
  a.weights = weights;
  cudaError_t e = launch_compress(a, pl->cs_buf, (double2*)uv_out, (float2*)vis_out, (long long*)run_of,
                                  (long long*)n_out, pl->sm_count, stream);
  if (e != cudaSuccess) return cuda_fail(e, "compression kernel launch");
  return GRID_OK;
}

int degrid_expand(grid_plan_t pl, int64_t n_vis, const int64_t* run_of, int64_t n_compressed, const void* vis_compressed,
                  const float* weights, void* vis_out, cudaStream_t stream) {
  g_err.clear();
  if (!pl) return fail(GRID_ERR_INVALID, "null plan");
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis=%lld out of range", (long long)n_vis);
  if (n_compressed < 0 || n_compressed > n_vis) return fail(GRID_ERR_INVALID, "n_compressed=%lld out of range", (long long)n_compressed);
  if (n_vis == 0) return GRID_OK;
  if (!run_of || !vis_out || (n_compressed > 0 && !vis_compressed)) return fail(GRID_ERR_INVALID, "null run_of, vis_compressed or vis_out");
  const size_t va = pl->g.P % 2 == 0 ? 16 : 8;  // even P moves two complex values per vector access
  if (!aligned(run_of, 8) || !aligned(vis_out, va) || (vis_compressed && !aligned(vis_compressed, va)))
    return fail(GRID_ERR_INVALID, "run_of must be 8-byte, vis_compressed and vis_out %zu-byte aligned", va);
  if (weights && !aligned(weights, 4)) return fail(GRID_ERR_INVALID, "weights must be 4-byte aligned");
  int rc = check_device(pl);
  if (rc) return rc;
  cudaError_t e = launch_expand(pl->g.P, n_vis, (const long long*)run_of, n_compressed, (const float2*)vis_compressed,
                                weights, (float2*)vis_out, pl->sm_count, stream);
  if (e != cudaSuccess) return cuda_fail(e, "expand kernel launch");
  return GRID_OK;
}

int grid_degrid_host(grid_plan_t gp, grid_plan_t dp, int64_t n_vis, const double* uv_host, const void* vis_host,
                     const float* weights_host, double* uv_dev, void* vis_dev, float* weights_dev, void* vis_out_dev,
                     const void* kernel_table, void* grid_dev, void* vis_out_host, void* grid_host, int64_t chunk,
                     cudaStream_t stream) {
  g_err.clear();
  if (!gp || !dp) return fail(GRID_ERR_INVALID, "null plan");
  const Geometry &a = gp->g, &b = dp->g;
  if (a.G != b.G || a.S != b.S || a.O != b.O || a.P != b.P || gp->desc.precision != dp->desc.precision)
    return fail(GRID_ERR_INVALID, "the two plans differ in G, S, oversample, npol or precision");
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis=%lld out of range", (long long)n_vis);
  if (!kernel_table || !grid_dev) return fail(GRID_ERR_INVALID, "null kernel_table or grid");
  if (n_vis > 0 && (!uv_host || !vis_host || !uv_dev || !vis_dev || !vis_out_dev || !vis_out_host))
    return fail(GRID_ERR_INVALID, "null uv, vis or vis_out buffer");
  if (weights_host && !weights_dev) return fail(GRID_ERR_INVALID, "weights_host needs weights_dev");
  if (chunk < 0) return fail(GRID_ERR_INVALID, "chunk=%lld", (long long)chunk);
  int rc = check_device(gp);
  if (rc) return rc;
  if (chunk == 0) chunk = 1 << 20;
  const long long nc = n_vis > 0 ? (n_vis + chunk - 1) / chunk : 0;
  if (nc > 4096) return fail(GRID_ERR_INVALID, "%lld chunks: use a larger chunk", nc);
  const int need_ev = (int)(2 * nc + 3);
  cudaError_t e = cudaSuccess;
  if (!gp->cstream) e = cudaStreamCreateWithFlags(&gp->cstream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
  rc = ensure_events(gp, need_ev);
  if (rc) return rc;
  cudaStream_t cs = gp->cstream;
  cudaEvent_t* ev = gp->evs;  // [0] start, [1] gridded, [2] end, [3 + c] chunk c uploaded, [3 + nc + c] chunk c degridded
  const size_t vb = (gp->desc.precision == GRID_PREC_F32 ? 8 : 4) * (size_t)a.P;
  const size_t ob = 8 * (size_t)a.P;
  const size_t grid_bytes = (size_t)a.P * a.G * a.G * 8;
#define GB_TRY(x) do { e = (x); if (e != cudaSuccess) return cuda_fail(e, #x); } while (0)
  GB_TRY(cudaEventRecord(ev[0], stream));
  GB_TRY(cudaStreamWaitEvent(cs, ev[0], 0));
  GB_TRY(cudaMemsetAsync(grid_dev, 0, grid_bytes, stream));
  // upload chunk c on the copy stream while chunk c-1 is gridded on the caller's stream
  for (long long c = 0; c < nc; ++c) {
    const long long k0 = c * chunk, n = std::min<long long>(chunk, n_vis - k0);
    GB_TRY(cudaMemcpyAsync(uv_dev + 2 * k0, uv_host + 2 * k0, (size_t)n * 16, cudaMemcpyHostToDevice, cs));
    GB_TRY(cudaMemcpyAsync((char*)vis_dev + k0 * vb, (const char*)vis_host + k0 * vb, (size_t)n * vb,
                           cudaMemcpyHostToDevice, cs));
    if (weights_host)
      GB_TRY(cudaMemcpyAsync(weights_dev + k0, weights_host + k0, (size_t)n * 4, cudaMemcpyHostToDevice, cs));
    GB_TRY(cudaEventRecord(ev[3 + c], cs));
    GB_TRY(cudaStreamWaitEvent(stream, ev[3 + c], 0));
    rc = grid(gp, n, uv_dev + 2 * k0, (const char*)vis_dev + k0 * vb, weights_host ? weights_dev + k0 : nullptr,
              kernel_table, grid_dev, stream);
    if (rc) return rc;
  }
  // the grid goes down while it is degridded
  GB_TRY(cudaEventRecord(ev[1], stream));
  if (grid_host) {
    GB_TRY(cudaStreamWaitEvent(cs, ev[1], 0));
    GB_TRY(cudaMemcpyAsync(grid_host, grid_dev, grid_bytes, cudaMemcpyDeviceToHost, cs));
  }
  // degrid chunk c, then bring it down on the copy stream while chunk c+1 is degridded
  for (long long c = 0; c < nc; ++c) {
    const long long k0 = c * chunk, n = std::min<long long>(chunk, n_vis - k0);
    rc = degrid(dp, n, uv_dev + 2 * k0, grid_dev, kernel_table, (char*)vis_out_dev + k0 * ob, stream);
    if (rc) return rc;
    GB_TRY(cudaEventRecord(ev[3 + nc + c], stream));
    GB_TRY(cudaStreamWaitEvent(cs, ev[3 + nc + c], 0));
    GB_TRY(cudaMemcpyAsync((char*)vis_out_host + k0 * ob, (const char*)vis_out_dev + k0 * ob, (size_t)n * ob,
                           cudaMemcpyDeviceToHost, cs));
  }
  // later work on the caller's stream comes after every copy
  GB_TRY(cudaEventRecord(ev[2], cs));
  GB_TRY(cudaStreamWaitEvent(stream, ev[2], 0));
#undef GB_TRY
  return GRID_OK;
}

int grid_degrid_host_steps(grid_plan_t gp, grid_plan_t dp, int n_steps, const grid_host_step* steps, int64_t n_vis,
                           double* const* uv_dev, void* const* vis_dev, float* const* weights_dev,
                           void* const* vis_out_dev, const void* kernel_table, void* grid_dev, int64_t chunk,
                           cudaStream_t stream) {
  g_err.clear();
  if (!gp || !dp) return fail(GRID_ERR_INVALID, "null plan");
  const Geometry &a = gp->g, &b = dp->g;
  if (a.G != b.G || a.S != b.S || a.O != b.O || a.P != b.P || gp->desc.precision != dp->desc.precision)
    return fail(GRID_ERR_INVALID, "the two plans differ in G, S, oversample, npol or precision");
  if (n_steps < 0 || n_steps > 64 || (n_steps > 0 && !steps)) return fail(GRID_ERR_INVALID, "n_steps=%d (0..64)", n_steps);
  if (n_vis < 0 || n_vis > ((int64_t)1 << 40)) return fail(GRID_ERR_INVALID, "n_vis=%lld out of range", (long long)n_vis);
  if (!kernel_table || !grid_dev) return fail(GRID_ERR_INVALID, "null kernel_table or grid");
  if (chunk < 0) return fail(GRID_ERR_INVALID, "chunk=%lld", (long long)chunk);
  if (n_steps == 0) return GRID_OK;
  if (!uv_dev || !vis_dev || !vis_out_dev) return fail(GRID_ERR_INVALID, "null work-buffer arrays");
  bool weighted = false;
  for (int st = 0; st < n_steps; ++st) {
    const grid_host_step& h = steps[st];
    if (n_vis > 0 && (!h.uv_host || !h.vis_host || !h.vis_out_host)) return fail(GRID_ERR_INVALID, "step %d: null host buffer", st);
    if (st > 0 && (h.weights_host != nullptr) != weighted) return fail(GRID_ERR_INVALID, "steps must all have weights or none");
    weighted = h.weights_host != nullptr;
  }
  for (int w = 0; w < 2; ++w)
    if (n_vis > 0 && (!uv_dev[w] || !vis_dev[w] || !vis_out_dev[w] || (weighted && (!weights_dev || !weights_dev[w]))))
      return fail(GRID_ERR_INVALID, "null device work buffer in set %d", w);
  int rc = check_device(gp);
  if (rc) return rc;
  if (chunk == 0) chunk = 1 << 22;  // across steps the copies overlap anyway: fewer, larger pieces measured faster
  const long long nc = n_vis > 0 ? (n_vis + chunk - 1) / chunk : 0;
  if (nc > 64) return fail(GRID_ERR_INVALID, "%lld chunks: use a larger chunk (at most 64 per step)", nc);
  cudaError_t e = cudaSuccess;
  if (!gp->cstream) e = cudaStreamCreateWithFlags(&gp->cstream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !gp->dstream) e = cudaStreamCreateWithFlags(&gp->dstream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreateWithFlags");
  // events per step: uploaded chunks, degridded chunks, gridded, grid down, inputs free, outputs down; plus start
  const int per = (int)(2 * nc + 4);
  rc = ensure_events(gp, 1 + per * n_steps);
  if (rc) return rc;
  cudaEvent_t* ev = gp->evs;
  auto E = [&](int st, int k) { return ev[1 + st * per + k]; };  // k: 0..nc-1 up, nc..2nc-1 degridded, then 4 more
  const int kG = (int)(2 * nc), kGD = kG + 1, kFree = kG + 2, kDown = kG + 3;
  cudaStream_t up = gp->cstream, down = gp->dstream;
  const size_t vb = (gp->desc.precision == GRID_PREC_F32 ? 8 : 4) * (size_t)a.P;
  const size_t ob = 8 * (size_t)a.P;
  const size_t grid_bytes = (size_t)a.P * a.G * a.G * 8;
#define GB_TRY(x) do { e = (x); if (e != cudaSuccess) return cuda_fail(e, #x); } while (0)
  GB_TRY(cudaEventRecord(ev[0], stream));
  GB_TRY(cudaStreamWaitEvent(up, ev[0], 0));
  GB_TRY(cudaStreamWaitEvent(down, ev[0], 0));
  for (int st = 0; st < n_steps; ++st) {
    const grid_host_step& h = steps[st];
    const int w = st & 1;
    // uploads into work set w once step st-2 no longer reads it
    if (st >= 2) GB_TRY(cudaStreamWaitEvent(up, E(st - 2, kFree), 0));
    for (long long c = 0; c < nc; ++c) {
      const long long k0 = c * chunk, n = std::min<long long>(chunk, n_vis - k0);
      GB_TRY(cudaMemcpyAsync(uv_dev[w] + 2 * k0, h.uv_host + 2 * k0, (size_t)n * 16, cudaMemcpyHostToDevice, up));
      GB_TRY(cudaMemcpyAsync((char*)vis_dev[w] + k0 * vb, (const char*)h.vis_host + k0 * vb, (size_t)n * vb,
                             cudaMemcpyHostToDevice, up));
      if (weighted)
        GB_TRY(cudaMemcpyAsync(weights_dev[w] + k0, h.weights_host + k0, (size_t)n * 4, cudaMemcpyHostToDevice, up));
      GB_TRY(cudaEventRecord(E(st, (int)c), up));
    }
    // the grid is reused: wait until the previous step's grid went down
    if (st >= 1) GB_TRY(cudaStreamWaitEvent(stream, E(st - 1, kGD), 0));
    GB_TRY(cudaMemsetAsync(grid_dev, 0, grid_bytes, stream));
    for (long long c = 0; c < nc; ++c) {
      const long long k0 = c * chunk, n = std::min<long long>(chunk, n_vis - k0);
      GB_TRY(cudaStreamWaitEvent(stream, E(st, (int)c), 0));
      rc = grid(gp, n, uv_dev[w] + 2 * k0, (const char*)vis_dev[w] + k0 * vb, weighted ? weights_dev[w] + k0 : nullptr,
                kernel_table, grid_dev, stream);
      if (rc) return rc;
    }
    GB_TRY(cudaEventRecord(E(st, kG), stream));
    GB_TRY(cudaStreamWaitEvent(down, E(st, kG), 0));
    if (h.grid_host) GB_TRY(cudaMemcpyAsync(h.grid_host, grid_dev, grid_bytes, cudaMemcpyDeviceToHost, down));
    GB_TRY(cudaEventRecord(E(st, kGD), down));
    // degrid into output set w once step st-2's outputs went down
    if (st >= 2) GB_TRY(cudaStreamWaitEvent(stream, E(st - 2, kDown), 0));
    for (long long c = 0; c < nc; ++c) {
      const long long k0 = c * chunk, n = std::min<long long>(chunk, n_vis - k0);
      rc = degrid(dp, n, uv_dev[w] + 2 * k0, grid_dev, kernel_table, (char*)vis_out_dev[w] + k0 * ob, stream);
      if (rc) return rc;
      GB_TRY(cudaEventRecord(E(st, (int)(nc + c)), stream));
      GB_TRY(cudaStreamWaitEvent(down, E(st, (int)(nc + c)), 0));
      GB_TRY(cudaMemcpyAsync((char*)h.vis_out_host + k0 * ob, (const char*)vis_out_dev[w] + k0 * ob, (size_t)n * ob,
                             cudaMemcpyDeviceToHost, down));
    }
    GB_TRY(cudaEventRecord(E(st, kFree), stream));
    GB_TRY(cudaEventRecord(E(st, kDown), down));
  }
  // later work on the caller's stream comes after every copy
  GB_TRY(cudaStreamWaitEvent(stream, E(n_steps - 1, kDown), 0));
  GB_TRY(cudaEventRecord(ev[0], up));
  GB_TRY(cudaStreamWaitEvent(stream, ev[0], 0));
#undef GB_TRY
  return GRID_OK;
}

int grid_tap_form(int Bu, int Bv, int npol, int* form, int* multiplies) {
  if (!form && !multiplies) return fail(GRID_ERR_INVALID, "grid_tap_form: both outputs are null");
  if (Bu < 1 || Bv < 1 || !(npol == 1 || npol == 2 || npol == 4))
    return fail(GRID_ERR_INVALID, "grid_tap_form: Bu=%d Bv=%d npol=%d out of range", Bu, Bv, npol);
  const KernelEntry* k = find_kernel(Bu, Bv, npol);
  if (!k) return fail(GRID_ERR_UNSUPPORTED, "grid_tap_form: no kernel for Bu=%d Bv=%d npol=%d", Bu, Bv, npol);
  // Sec. 6: B*B (or B*P) multiplies before the products, then one per (cell, polarization)
  static_assert((int)TAP_PRODUCT == (int)GRID_TAPS_PRODUCT && (int)TAP_FACTOR_V == (int)GRID_TAPS_FACTOR_V &&
                (int)TAP_FACTOR_U == (int)GRID_TAPS_FACTOR_U, "tap form codes");
  const int pre = k->form == TAP_PRODUCT ? Bu * Bv : (k->form == TAP_FACTOR_V ? Bv * npol : Bu * npol);
  if (form) *form = k->form;
  if (multiplies) *multiplies = pre + Bu * Bv * npol;
  return GRID_OK;
}

int grid_measure_fma_peak(int iters, double* tflops, cudaStream_t stream) {
  g_err.clear();
  if (!tflops || iters < 1 || iters > (1 << 24)) return fail(GRID_ERR_INVALID, "iters=%d must be 1 .. 2^24, tflops not null", iters);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice / attribute");
  const int threads = 256, blocks = sms * 8;  // 64 warps per SM: every FMA pipe kept busy
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  if (e == cudaSuccess) e = launch_fma_peak(blocks, threads, iters, stream);  // warm-up (clocks up)
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], stream);
  if (e == cudaSuccess) e = launch_fma_peak(blocks, threads, iters, stream);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "FMA peak measurement");
  *tflops = fma_peak_flops_per_launch(blocks, threads, iters) / (ms * 1e-3) / 1e12;
  return GRID_OK;
}

int grid_device_info(int* sm_count, int* fma_lanes_per_sm, int* max_clock_khz) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  int sms = 0, clk = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
  if (sm_count) *sm_count = sms;
  if (fma_lanes_per_sm) *fma_lanes_per_sm = 128;
  if (max_clock_khz) *max_clock_khz = clk;
  return GRID_OK;
}

}  // extern "C"
