// Chunked gridder with phase-rotated tap tables, box-ordered batches and
// staged move masks.
//
// The work distribution of the chunked schedule (Sec. 3, Fig. 2; Sec. 4: one
// chunk of consecutive visibilities per team, records staged through shared
// memory), with the per-visibility work of a team thread cut to a record
// load, two tap loads, the value loads, one bit test and the Bu*Bv*P packed
// FMAs. Three changes make that possible.
//
//  - Rotated tables. Thread (au, av) owns the cells whose position modulo the
//    bin is au*Bu + i (i < Bu) along u. For a visibility whose footprint starts
//    at cell c0 with fine row r, the tap of such a cell depends only on r,
//    ph = c0 mod nbu and the cell's position c modulo the bin:
//        R[r][ph][c] = T[r][(c - ph) mod nbu]  if that index is < S, else 0
//    (a cell of the box before the footprint has index >= nbu - Bu + 1 >= S
//    because the bin holds S + Bu - 1 cells). The staging thread stores the
//    offset of row (r, ph); a team thread adds its own constant au*Bu and
//    reads its Bu taps as one aligned vector, with no wrap-around test.
//  - Box order. A batch of staged visibilities is processed in the order of
//    its footprints' first block (v, then u) instead of the input order. The
//    sum does not depend on the order, and visibilities that share a box
//    become neighbours: on baseline-ordered tracks whose channels interleave,
//    the footprint steps back and forth across block edges, and each such
//    step costs a flush in input order.
//  - Move masks. The box of a visibility is the run of nu blocks starting at
//    the footprint's first block q. When q changes from the previous
//    visibility's p, the threads whose block leaves the box are those of the
//    block residues p .. q-1 (or q .. p-1) modulo nu, along each axis. The
//    staging threads compute that set as a bit mask over the team once per
//    visibility; a team thread tests its bit, and only when it is set
//    flushes its block (Sec. 3) and computes the block it owns next.
// Invalid visibilities sort last, with zero values and an empty mask, so the
// record loop has no branch for them.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace gbg {

// Shared memory: the two rotated tables, then one area per team: the record
// buffer in box order (records, values), the staging area in input order
// (records, values), the sort keys, the first blocks in box order and, for
// teams of more than 32 threads, the upper mask words. Offsets inside a
// team's area are compile-time constants.
template <int P, bool WIDE>
struct RotTeamLayout {
  static constexpr unsigned meta = 0;                          // int4 {u row, v row, first block, mask}
  static constexpr unsigned vals = meta + kRB * 16;            // float2 [kRB][P]
  static constexpr unsigned tmeta = vals + kRB * P * 8;        // input order
  static constexpr unsigned tvals = tmeta + kRB * 16;
  static constexpr unsigned keys = tvals + kRB * P * 8;        // u32 [kRB]
  static constexpr unsigned sortK = keys + kRB * 4;            // u32 [kRB], box order
  static constexpr unsigned mhi = sortK + kRB * 4;             // WIDE: u32 every 16 bytes, box order
  // Team areas are 16 bytes past a multiple of 128, so the broadcast 16-byte loads of the
  // (up to 8) teams of one warp fall in different shared-memory banks.
  static constexpr unsigned bytes = (mhi + (WIDE ? kRB * 16 : 0) + 127) / 128 * 128 + 16;
};

struct RotLayout {
  unsigned tabU, tabV, colT, rowT, teams, total;
};

template <int P, bool WIDE>
__host__ __device__ inline RotLayout rot_layout(const Geometry& g) {
  RotLayout L{};
  size_t off = 0;
  L.tabU = (unsigned)off; off += align16((size_t)g.O * g.nbu * g.nbu * 4);
  L.tabV = (unsigned)off; off += align16((size_t)g.O * g.nbv * g.nbv * 4);
  L.colT = (unsigned)off; off += align16((size_t)g.nu * (g.nu + 1) * 8);
  L.rowT = (unsigned)off; off += align16((size_t)g.nv * (g.nv + 1) * 8);
  L.teams = (unsigned)off; off += (size_t)g.tpc * RotTeamLayout<P, WIDE>::bytes;
  L.total = (unsigned)off;
  return L;
}

template <int P>
size_t rot_smem_bytes(const Geometry& g) {
  return rot_layout<P, false>(g).total;
}

template <int P>
size_t rot_smem_bytes_wide(const Geometry& g) {
  return rot_layout<P, true>(g).total;
}

// R[(r*nb + ph)*nb + c] = T[r][(c - ph) mod nb] for indices < S, else 0.
__device__ __forceinline__ void build_rotated_table(float* tab, const Args& a, int nb) {
  const Geometry& g = a.g;
  // one (row, phase) line of nb entries per step: the rotation is a cyclic
  // shift of the zero-padded row T[r][0..S), nb >= S
  for (int line = threadIdx.x; line < g.O * nb; line += blockDim.x) {
    const int r = line / nb, ph = line - r * nb;
    float* out = tab + (size_t)line * nb;
    int k = nb - ph;  // tap index of entry c = 0, modulo nb
    for (int c = 0; c < nb; ++c, ++k) {
      if (k == nb) k = 0;
      out[c] = k < g.S ? load_tap(a.table, a.tab_fmt, r * g.S + k) : 0.f;
    }
  }
}

// Move-mask tables. When the box's first block moves from p to q along an
// axis of n blocks, the blocks that leave it are those of the residues
// min(p, q), ..., min(p, q) + d - 1 (mod n), d = min(|q - p|, n). colT[s][d]
// is the team mask (thread l = au + av*nu) of the threads whose column au is
// one of those residues from s; rowT[s][d] the same for rows av.
__device__ __forceinline__ void build_move_tables(unsigned long long* colT, unsigned long long* rowT, const Geometry& g) {
  for (int idx = threadIdx.x; idx < g.nu * (g.nu + 1); idx += blockDim.x) {
    const int st = idx / (g.nu + 1), d = idx % (g.nu + 1);
    unsigned long long m = 0;
    for (int k = 0; k < d; ++k) {
      const int au = (st + k) % g.nu;
      for (int av = 0; av < g.nv; ++av) m |= 1ull << (au + av * g.nu);
    }
    colT[idx] = m;
  }
  for (int idx = threadIdx.x; idx < g.nv * (g.nv + 1); idx += blockDim.x) {
    const int st = idx / (g.nv + 1), d = idx % (g.nv + 1);
    unsigned long long m = 0;
    for (int k = 0; k < d; ++k) {
      const int av = (st + k) % g.nv;
      for (int au = 0; au < g.nu; ++au) m |= 1ull << (au + av * g.nu);
    }
    rowT[idx] = m;
  }
}

// Row (start residue, count) of the move tables for a move from p to q.
__device__ __forceinline__ int move_row(int p, int q, int n, unsigned mag) {
  const int d = q > p ? q - p : p - q;
  return mod_small(q < p ? q : p, n, mag) * (n + 1) + (d < n ? d : n);
}

// Sort key of a record: its first block (v, then u; 13 bits each, which
// only matters for the order, not for correctness) above its index in the
// batch, so that keys are distinct. Invalid records sort last.
__device__ __forceinline__ unsigned sort_key(unsigned K, int r) {
  if (K == kInvalid) return 0xFFFFFFE0u | (unsigned)r;
  return (((K >> 16) & 0x1FFFu) << 18) | ((K & 0x1FFFu) << 5) | (unsigned)r;
}

template <int P>
__device__ __forceinline__ void load_vals(const float2* p, float2 (&v)[P]) {
  if constexpr (P % 2 == 0) {
#pragma unroll
    for (int i = 0; i < P; i += 2) {
      const float4 q = *(const float4*)(p + i);
      v[i] = make_float2(q.x, q.y);
      v[i + 1] = make_float2(q.z, q.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < P; ++i) v[i] = p[i];
  }
}

template <int P>
__device__ __forceinline__ void store_vals(float2* p, const float2 (&v)[P]) {
  if constexpr (P % 2 == 0) {
#pragma unroll
    for (int i = 0; i < P; i += 2) *(float4*)(p + i) = make_float4(v[i].x, v[i].y, v[i + 1].x, v[i + 1].y);
  } else {
#pragma unroll
    for (int i = 0; i < P; ++i) p[i] = v[i];
  }
}

template <typename T>
__device__ __forceinline__ T* sm(unsigned char* smem, unsigned off) {
  return (T*)(smem + off);
}

// Phase 1: stage batch b of a team's chunk in input order (each team thread
// takes records l, l+ts, ...): the exact index rule, the rotated-table row
// offsets (bytes from the start of shared memory), the footprint's first
// block, the weighted values and the sort key.
template <int BU, int BV, int P>
__device__ __forceinline__ void rot_stage(const Args& a, unsigned char* smem, unsigned tb, unsigned tabV, long long kb,
                                          long long vend, int l) {
  using TL = RotTeamLayout<P, false>;
  const Geometry& g = a.g;
  for (int r = l; r < kRB; r += g.ts) {
    const bool h = kb + r < vend;
    double2 x = make_double2(0.0, 0.0);
    float w = 1.f;
    VisWords<P> q;
    if (h) {
      x = a.uv[kb + r];
      if (a.weights) w = a.weights[kb + r];
      load_vis_words<P>(a, kb + r, q);
    }
    if (kb + kRB + r < vend) {
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a.uv + kb + kRB + r));
      asm volatile("prefetch.global.L1 [%0];" ::"l"((const char*)a.vis + (kb + kRB + r) * (long long)P * (a.vis_fmt == FMT_F32 ? 8 : 4)));
    }
    int Cu, ru, Cv, rv;
    bool ok = fine_cell(x.x, g.log2O, g.G >> 1, Cu, ru);
    ok = fine_cell(x.y, g.log2O, g.G >> 1, Cv, rv) && ok;
    const int cu0 = Cu - g.h, cv0 = Cv - g.h;
    ok = ok && cu0 >= 0 && cu0 + g.S <= g.G && cv0 >= 0 && cv0 + g.S <= g.G;
    if (h && !ok) atomicAdd(a.skipped, 1ULL);
    ok = ok && h;
    int4 m;
    float2 val[P];
    if (ok) {
      const int phu = mod_small(cu0, g.nbu, g.mbu), phv = mod_small(cv0, g.nbv, g.mbv);
      m.x = (int)((unsigned)((ru * g.nbu + phu) * g.nbu) * 4u);  // the u table starts at offset 0
      m.y = (int)(tabV + (unsigned)((rv * g.nbv + phv) * g.nbv) * 4u);
      m.z = (cu0 / BU) | ((cv0 / BV) << 16);
      vis_values<P>(a, q, w, val);
    } else {
      m.x = 0;
      m.y = (int)tabV;
      m.z = (int)kInvalid;
#pragma unroll
      for (int p = 0; p < P; ++p) val[p] = make_float2(0.f, 0.f);
    }
    m.w = 0;
    sm<int4>(smem, tb + TL::tmeta)[r] = m;
    store_vals<P>(sm<float2>(smem, tb + TL::tvals) + r * P, val);
    sm<unsigned>(smem, tb + TL::keys)[r] = sort_key((unsigned)m.z, r);
  }
}

// Phase 2: each record's rank among the batch's keys is its slot in box
// order; the record moves there.
template <int P>
__device__ __forceinline__ void rot_sort(const Geometry& g, unsigned char* smem, unsigned tb, int l) {
  using TL = RotTeamLayout<P, false>;
  const unsigned* keys = sm<unsigned>(smem, tb + TL::keys);
  for (int r = l; r < kRB; r += g.ts) {
    const unsigned k = keys[r];
    int rank = 0;
#pragma unroll
    for (int s = 0; s < kRB; s += 4) {
      const uint4 q = *(const uint4*)(keys + s);
      rank += (q.x < k) + (q.y < k) + (q.z < k) + (q.w < k);
    }
    const int4 m = sm<int4>(smem, tb + TL::tmeta)[r];
    float2 v[P];
    load_vals<P>(sm<float2>(smem, tb + TL::tvals) + r * P, v);
    sm<int4>(smem, tb + TL::meta)[rank] = m;
    store_vals<P>(sm<float2>(smem, tb + TL::vals) + rank * P, v);
    sm<unsigned>(smem, tb + TL::sortK)[rank] = (unsigned)m.z;
  }
}

// Phase 3: move masks in box order, against the previous record (the last
// valid record of the earlier batches for slot 0; every thread moves on the
// chunk's first valid record). lastK then advances to this batch's last
// valid record.
template <int P, bool WIDE>
__device__ __forceinline__ void rot_masks(const Args& a, unsigned char* smem, unsigned tb, int l, unsigned& lastK,
                                          unsigned colT_off, unsigned rowT_off) {
  using TL = RotTeamLayout<P, false>;
  using M = typename std::conditional<WIDE, unsigned long long, unsigned>::type;
  const Geometry& g = a.g;
  const unsigned* sortK = sm<unsigned>(smem, tb + TL::sortK);
  for (int s = l; s < kRB; s += g.ts) {
    const unsigned K = sortK[s];
    M mask = 0;
    if (K != kInvalid) {
      const unsigned Kp = s > 0 ? sortK[s - 1] : lastK;  // valid records precede invalid ones
      if (Kp == kInvalid) {
        mask = g.ts >= (int)(8 * sizeof(M)) ? ~(M)0 : (((M)1 << g.ts) - 1);  // the chunk's first record
      } else {
        const int iu = move_row((int)(Kp & 0xFFFFu), (int)(K & 0xFFFFu), g.nu, g.mu);
        const int iv = move_row((int)(Kp >> 16), (int)(K >> 16), g.nv, g.mv);
        const unsigned long long* colT = sm<unsigned long long>(smem, colT_off);
        const unsigned long long* rowT = sm<unsigned long long>(smem, rowT_off);
        mask = (M)(colT[iu] | rowT[iv]);
      }
    }
    sm<int4>(smem, tb + TL::meta)[s].w = (int)(unsigned)mask;
    if constexpr (WIDE) sm<int4>(smem, tb + TL::mhi)[s].x = (int)(unsigned)((unsigned long long)mask >> 32);
  }
  for (int s = kRB - 1; s >= 0; --s) {
    const unsigned K = sortK[s];
    if (K != kInvalid) { lastK = K; break; }
  }
}

// The chunked schedule with rotated tables: teams of at most 32 threads, or
// with WIDE at most 64 (a thread in lanes 32..63 of its team reads its mask
// word from the second array).
template <int BU, int BV, int P, bool WIDE>
__global__ void grid_rot_kernel(Args a) {
  using TL = RotTeamLayout<P, WIDE>;
  extern __shared__ __align__(16) unsigned char smem[];
  const Geometry& g = a.g;
  const RotLayout L = rot_layout<P, WIDE>(g);
  build_rotated_table(sm<float>(smem, L.tabU), a, g.nbu);
  build_rotated_table(sm<float>(smem, L.tabV), a, g.nbv);
  build_move_tables(sm<unsigned long long>(smem, L.colT), sm<unsigned long long>(smem, L.rowT), g);

  const int team = threadIdx.x / g.ts;
  const int l = threadIdx.x - team * g.ts;
  const int au = l % g.nu, av = l / g.nu;
  const unsigned tb = L.teams + (unsigned)team * TL::bytes;
  const unsigned myU = (unsigned)(au * BU * 4), myV = (unsigned)(av * BV * 4);
  const unsigned mybit = 1u << (l & 31);
  const unsigned mword = (WIDE && l >= 32) ? tb + TL::mhi : tb + TL::meta + 12;  // + r*16
  const int nb = (a.chunk_len + kRB - 1) / kRB;
  const unsigned wmask = warp_lane_mask();

  float2 acc[P][BV][BU];
#pragma unroll
  for (int p = 0; p < P; ++p)
#pragma unroll
    for (int j = 0; j < BV; ++j)
#pragma unroll
      for (int i = 0; i < BU; ++i) acc[p][j][i] = make_float2(0.f, 0.f);

  const long long chunk = (long long)blockIdx.x * g.tpc + team;
  const long long vbeg = chunk * a.chunk_len;
  const long long vend = chunk < a.n_chunks ? min(vbeg + a.chunk_len, a.n_vis) : vbeg;
  __syncthreads();  // tables ready
  unsigned cur = kInvalid, lastK = kInvalid;
  for (int b = 0; b < nb; ++b) {
    // the staging area is not read by the record loop, so it is refilled
    // while slower lanes finish the previous batch
    rot_stage<BU, BV, P>(a, smem, tb, L.tabV, vbeg + (long long)b * kRB, vend, l);
    group_sync(a, wmask);
    rot_sort<P>(g, smem, tb, l);
    group_sync(a, wmask);
    rot_masks<P, WIDE>(a, smem, tb, l, lastK, L.colT, L.rowT);
    group_sync(a, wmask);
#pragma unroll 1
    for (int r = 0; r < kRB; ++r) {
      const int4 m = sm<int4>(smem, tb + TL::meta)[r];
      const unsigned mw = WIDE ? *sm<unsigned>(smem, mword + (unsigned)r * 16u) : (unsigned)m.w;
      const bool moved = (mw & mybit) != 0u;
      if (moved) {
        // this thread's block leaves the box: flush and clear it, and take the
        // block of its residue in the new box
        if (cur != kInvalid) {
          flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
          // Cleared by a multiply by zero, so that moved and staying lanes
          // run the same packed FMAs below. Measured 4% faster than giving
          // the moved lanes their own assigning multiplies; clearing with
          // zero constants raised the kernel to 128 registers.
#pragma unroll
          for (int p = 0; p < P; ++p)
#pragma unroll
            for (int j = 0; j < BV; ++j)
#pragma unroll
              for (int i = 0; i < BU; ++i) acc[p][j][i] = __fmul2_rn(acc[p][j][i], make_float2(0.f, 0.f));
        }
        const int qu = m.z & 0xFFFF, qv = (int)((unsigned)m.z >> 16);
        int du = au - mod_small(qu, g.nu, g.mu);
        int dv = av - mod_small(qv, g.nv, g.mv);
        if (du < 0) du += g.nu;
        if (dv < 0) dv += g.nv;
        cur = (unsigned)(qu + du) | ((unsigned)(qv + dv) << 16);
      }
      float wu[BU], wv[BV];
      load_taps<BU>(sm<float>(smem, (unsigned)m.x + myU), wu);
      load_taps<BV>(sm<float>(smem, (unsigned)m.y + myV), wv);
      float2 v[P];
      load_vals<P>(sm<float2>(smem, tb + TL::vals) + r * P, v);
      Contribution<BU, BV, P> c;
      c.from_taps(wu, wv, v);
      c.template apply<true>(acc);
    }
  }
  if (cur != kInvalid) flush_global<BU, BV, P, false>(acc, cur, a.grid, g.G);
}

// Function table entry for one (Bu, Bv, P): the kernel for teams of at most
// 32 threads and the one for 33..64.
struct RotEntry {
  int bu, bv, p;
  const void* fn;
  const void* fn_wide;
  size_t (*smem)(const Geometry&);
  size_t (*smem_wide)(const Geometry&);
};

}  // namespace gbg
