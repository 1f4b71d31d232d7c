// Batched gridding: the C ABI (grid_batch_*) and its kernel instantiations.
// Many grids of the same size, with uneven visibility counts and per-grid
// GCF support, are gridded by persistent kernel launches: one launch per
// block shape (items with S >= S_split may use a second shape, Sec. 5: the
// best coarsening depends on the bin size), each compiled for its own shape
// so that the larger shape's registers do not bind the smaller one. The
// launches can be captured in a CUDA graph because grid_batch_execute()
// allocates nothing and only enqueues a counter reset and the kernels.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gridder.h"
#include "internal.h"

using namespace gbg;

namespace gbg {

#define GB_BATCH(BU, BV, P) \
  {BU, BV, BU, BV, P, (const void*)&grid_batch_kernel<BU, BV, BU, BV, P>, &batch_smem_bytes<BU, BV, BU, BV, P>}

static const BatchKernelEntry kBatchKernels[] = {
    GB_BATCH(1, 1, 1), GB_BATCH(2, 1, 1), GB_BATCH(1, 2, 1), GB_BATCH(2, 2, 1), GB_BATCH(3, 3, 1), GB_BATCH(4, 2, 1),
    GB_BATCH(2, 4, 1), GB_BATCH(4, 4, 1), GB_BATCH(1, 1, 4), GB_BATCH(2, 1, 4), GB_BATCH(2, 2, 4), GB_BATCH(4, 2, 4),
};

}  // namespace gbg

// One block shape of a batch: its kernel and launch shape.
struct BatchShape {
  const BatchKernelEntry* k = nullptr;
  int bu = 0, bv = 0;
  int threads = 0, nb_max = 0, tpc_max = 0, occ = 0;
  size_t smem = 0;
  int first_unit = 0, n_units = 0;  // this shape's work units in d_units
};

struct grid_batch_s {
  int G, O, P, S_split, max_S, precision, chunk_len, device;
  int n_shapes;  // 1, or 2 when items with S >= S_split use the second shape
  BatchShape shape[2];
  int sm_count;
  // device state
  BatchItem* d_items = nullptr;
  int4* d_units = nullptr;
  int* d_next = nullptr;  // one work counter per shape
  unsigned long long* d_skipped = nullptr;
  int n_items = 0, n_units = 0, cap_items = 0, cap_units = 0;
};

namespace {
thread_local std::string b_err;
int bfail(int code, const char* msg) {
  b_err = msg;
  return code;
}
int nb_of(int S, int B) { return ((S + B - 1 + B - 1) / B) * B; }

// Kernel, CTA size, record buffers and residency of one shape for supports up to max_S.
const BatchKernelEntry* find_batch_kernel(int bu, int bv, int P) {
  for (const auto& e : kBatchKernels)
    if (e.bu == bu && e.bv == bv && e.bu2 == bu && e.bv2 == bv && e.p == P) return &e;
  return nullptr;
}

int setup_shape(BatchShape& sh, int bu, int bv, int P, int O, int max_S, int threads, const cudaDeviceProp& prop) {
  sh.k = find_batch_kernel(bu, bv, P);
  if (!sh.k) return bfail(GRID_ERR_UNSUPPORTED, "no batched kernel built for this block shape and npol");
  sh.bu = bu;
  sh.bv = bv;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, sh.k->fn);
  if (e != cudaSuccess) return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  sh.nb_max = std::max(nb_of(max_S, bu), nb_of(max_S, bv));
  const int ts_max = (nb_of(max_S, bu) / bu) * (nb_of(max_S, bv) / bv);
  int thr = threads ? threads : 256;
  thr = std::max(thr, ts_max);
  thr = std::min(thr, fa.maxThreadsPerBlock);
  if (ts_max > thr) return bfail(GRID_ERR_UNSUPPORTED, "largest team does not fit in a CTA");
  sh.threads = thr;
  // record buffers for at most 32 teams per CTA (small-S items use part of the CTA)
  const int ts_min = (nb_of(1, bu) / bu) * (nb_of(1, bv) / bv);
  sh.tpc_max = std::min(32, thr / ts_min);
  sh.smem = sh.k->smem(O, sh.nb_max, sh.tpc_max);
  const size_t smem_max = prop.sharedMemPerBlockOptin;
  if (sh.smem + fa.sharedSizeBytes > smem_max) return bfail(GRID_ERR_UNSUPPORTED, "batched kernel needs too much shared memory");
  e = cudaFuncSetAttribute(sh.k->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem_max - fa.sharedSizeBytes));
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sh.occ, sh.k->fn, sh.threads, sh.smem);
  if (e == cudaSuccess && sh.occ < 1) e = cudaErrorInvalidConfiguration;
  if (e != cudaSuccess) return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  return GRID_OK;
}
}  // namespace

extern "C" {

const char* grid_batch_last_error(void) { return b_err.c_str(); }

int grid_batch_create(grid_batch_t* out, int G, int oversample, int npol, int Bu, int Bv, int max_S, int precision,
                      int vis_per_chunk, int threads) {
  return grid_batch_create_ex(out, G, oversample, npol, Bu, Bv, Bu, Bv, 0, max_S, precision, vis_per_chunk, threads);
}

int grid_batch_create_ex(grid_batch_t* out, int G, int oversample, int npol, int Bu, int Bv, int Bu2, int Bv2,
                         int S_split, int max_S, int precision, int vis_per_chunk, int threads) {
  b_err.clear();
  if (!out) return bfail(GRID_ERR_INVALID, "null out");
  *out = nullptr;
  if (G < 2 || G > 32768 || (G & 1)) return bfail(GRID_ERR_INVALID, "G must be even, 2..32768");
  if (oversample < 1 || oversample > 256 || (oversample & (oversample - 1))) return bfail(GRID_ERR_INVALID, "bad oversample");
  if (max_S < 1 || max_S > 64 || max_S > G) return bfail(GRID_ERR_INVALID, "max_S must be 1..64 and <= G");
  if (precision < GRID_PREC_F32 || precision > GRID_PREC_F16) return bfail(GRID_ERR_INVALID, "bad precision");
  if (vis_per_chunk < 0 || vis_per_chunk > (1 << 20) || threads < 0 || threads > 1024)
    return bfail(GRID_ERR_INVALID, "bad vis_per_chunk or threads");
  if (Bu2 == Bu && Bv2 == Bv) S_split = 0;
  if (S_split < 0 || S_split > 64) return bfail(GRID_ERR_INVALID, "S_split must be 0..64");
  if (!find_batch_kernel(Bu, Bv, npol) || !find_batch_kernel(Bu2, Bv2, npol))
    return bfail(GRID_ERR_UNSUPPORTED, "no batched kernel built for these block shapes and npol");
  cudaDeviceProp prop;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  grid_batch_s* b = new grid_batch_s;
  b->G = G; b->O = oversample; b->P = npol; b->S_split = S_split;
  b->max_S = max_S; b->precision = precision;
  b->chunk_len = vis_per_chunk ? vis_per_chunk : 256;
  b->device = dev;
  b->sm_count = prop.multiProcessorCount;
  b->n_shapes = S_split > 0 ? 2 : 1;
  // the first shape serves supports below S_split, the second the rest (up to max_S)
  int rc = setup_shape(b->shape[0], Bu, Bv, npol, oversample, S_split > 0 ? std::min(max_S, S_split - 1) : max_S,
                       threads, prop);
  if (rc == GRID_OK && b->n_shapes == 2) rc = setup_shape(b->shape[1], Bu2, Bv2, npol, oversample, max_S, threads, prop);
  if (rc != GRID_OK) {
    delete b;
    return rc;
  }
  e = cudaMalloc(&b->d_next, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_skipped, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(b->d_skipped, 0, sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaFree(b->d_next);
    cudaFree(b->d_skipped);
    delete b;
    return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = b;
  return GRID_OK;
}

void grid_batch_destroy(grid_batch_t b) {
  if (!b) return;
  cudaFree(b->d_items);
  cudaFree(b->d_units);
  cudaFree(b->d_next);
  cudaFree(b->d_skipped);
  delete b;
}

int grid_batch_set(grid_batch_t b, int n_items, const grid_batch_item* items) {
  b_err.clear();
  if (!b || n_items < 0 || (n_items > 0 && !items)) return bfail(GRID_ERR_INVALID, "bad arguments");
  std::vector<BatchItem> hi(n_items);
  struct U { int item; int first; int n; double cost; };
  std::vector<U> units[2];
  for (int i = 0; i < n_items; ++i) {
    const grid_batch_item& s = items[i];
    if (s.n_vis < 0 || s.S < 1 || s.S > b->max_S) return bfail(GRID_ERR_INVALID, "item S out of range or negative n_vis");
    if (s.n_vis > 0 && (!s.uv || !s.vis || !s.kernel_table || !s.grid))
      return bfail(GRID_ERR_INVALID, "null pointer in a non-empty item");
    if (((uintptr_t)s.uv % 16) || ((uintptr_t)s.grid % 16) || ((uintptr_t)s.vis % 4) || ((uintptr_t)s.weights % 4))
      return bfail(GRID_ERR_INVALID, "misaligned item pointer");
    const size_t vb = (b->precision == GRID_PREC_F32 ? 8 : 4) * (size_t)b->P;
    if ((uintptr_t)s.vis % (vb >= 16 ? 16 : vb)) return bfail(GRID_ERR_INVALID, "misaligned vis pointer");
    const int cls = (b->n_shapes == 2 && s.S >= b->S_split) ? 1 : 0;
    const BatchShape& sh = b->shape[cls];
    hi[i] = BatchItem{(const double2*)s.uv, s.vis, s.weights, s.kernel_table, (float2*)s.grid, (long long)s.n_vis, s.S, 0};
    const int nbu = nb_of(s.S, sh.bu), nbv = nb_of(s.S, sh.bv);
    const int ts = (nbu / sh.bu) * (nbv / sh.bv);
    const int tpc = std::min(sh.tpc_max, sh.threads / ts);
    const long long nch = (s.n_vis + b->chunk_len - 1) / b->chunk_len;
    if (nch > 0x7FFFFFFFLL) return bfail(GRID_ERR_INVALID, "item too large");
    for (long long c = 0; c < nch; c += tpc) {
      const int n = (int)std::min<long long>(tpc, nch - c);
      const long long nv = std::min<long long>((long long)n * b->chunk_len, s.n_vis - c * b->chunk_len);
      units[cls].push_back(U{i, (int)c, n, (double)nv * nbu * nbv});
    }
  }
  // per shape, most expensive units first (longest-processing-time order for the persistent CTAs)
  std::vector<int4> hu;
  for (int k = 0; k < b->n_shapes; ++k) {
    std::stable_sort(units[k].begin(), units[k].end(), [](const U& x, const U& y) { return x.cost > y.cost; });
    b->shape[k].first_unit = (int)hu.size();
    b->shape[k].n_units = (int)units[k].size();
    for (const U& u : units[k]) hu.push_back(make_int4(u.item, u.first, u.n, 0));
  }
  cudaError_t e = cudaSuccess;
  if (n_items > b->cap_items) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    e = cudaMalloc(&b->d_items, sizeof(BatchItem) * n_items);
    b->cap_items = e == cudaSuccess ? n_items : 0;
  }
  if (e == cudaSuccess && (int)hu.size() > b->cap_units) {
    cudaFree(b->d_units);
    b->d_units = nullptr;
    e = cudaMalloc(&b->d_units, sizeof(int4) * hu.size());
    b->cap_units = e == cudaSuccess ? (int)hu.size() : 0;
  }
  if (e == cudaSuccess && n_items) e = cudaMemcpy(b->d_items, hi.data(), sizeof(BatchItem) * n_items, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !hu.empty()) e = cudaMemcpy(b->d_units, hu.data(), sizeof(int4) * hu.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bfail(e == cudaErrorMemoryAllocation ? GRID_ERR_NOMEM : GRID_ERR_CUDA, cudaGetErrorString(e));
  b->n_items = n_items;
  b->n_units = (int)hu.size();
  return GRID_OK;
}

int grid_batch_execute(grid_batch_t b, cudaStream_t stream) {
  b_err.clear();
  if (!b) return bfail(GRID_ERR_INVALID, "null batch");
  if (b->n_units == 0) return GRID_OK;
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, 2 * sizeof(int), stream);
  if (e != cudaSuccess) return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  // one launch per shape, back to back on the stream (the second kernel's CTAs start as the
  // first kernel's finish)
  for (int k = 0; k < b->n_shapes; ++k) {
    const BatchShape& sh = b->shape[k];
    if (sh.n_units == 0) continue;
    BatchArgs a;
    memset(&a, 0, sizeof a);
    a.G = b->G; a.O = b->O;
    a.log2O = 0;
    while ((1 << a.log2O) < b->O) ++a.log2O;
    a.P = b->P; a.fmt = b->precision; a.chunk_len = b->chunk_len; a.nb_max = sh.nb_max; a.tpc_max = sh.tpc_max;
    a.items = b->d_items; a.units = b->d_units + sh.first_unit; a.n_units = sh.n_units; a.unit_next = b->d_next + k;
    a.skipped = b->d_skipped;
    const int blocks = std::min(b->sm_count * sh.occ, sh.n_units);
    void* args[] = {&a};
    e = cudaLaunchKernel(sh.k->fn, dim3(blocks), dim3(sh.threads), args, sh.smem, stream);
    if (e != cudaSuccess) return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  }
  return GRID_OK;
}

int grid_batch_skipped(grid_batch_t b, int64_t* n_skipped, int reset) {
  if (!b || !n_skipped) return bfail(GRID_ERR_INVALID, "null argument");
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpy(&v, b->d_skipped, sizeof v, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(b->d_skipped, 0, sizeof v);
  if (e != cudaSuccess) return bfail(GRID_ERR_CUDA, cudaGetErrorString(e));
  *n_skipped = (int64_t)v;
  return GRID_OK;
}

int grid_batch_describe(grid_batch_t b, int* threads, int* n_units, int* ctas) {
  if (!b) return bfail(GRID_ERR_INVALID, "null batch");
  if (threads) *threads = b->shape[0].threads;
  if (n_units) *n_units = b->n_units;
  if (ctas) {
    int c = 0;
    for (int k = 0; k < b->n_shapes; ++k) c += std::min(b->sm_count * b->shape[k].occ, b->shape[k].n_units);
    *ctas = c;
  }
  return GRID_OK;
}

}  // extern "C"
