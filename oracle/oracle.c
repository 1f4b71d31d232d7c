/*
 * Plain FP64 reference for convolutional gridding and degridding.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the correctness oracle. Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it. The
 * product path (the CUDA library) never calls it and shares no code with it.
 *
 * What it computes (Merry 2016, Sec. 2.2 "Convolutional Gridding"): every
 * visibility is a Dirac delta at its (u, v) position. The delta is convolved
 * with a gridding convolution function (GCF) and the result is sampled on the
 * regular grid. Contributions from different visibilities add. The GCF is
 * tabulated with oversampling (Sec. 2.2), is separable, G_ij = G^u_i G^v_j
 * (Sec. 4), and is the same for every polarization (Sec. 4).
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *  - uv are in grid-pixel units relative to the grid centre. Cell G/2 holds
 *    u = 0.
 *  - The oversample factor O is a power of two.
 *  - The fine position is f = floor(u*O + 1/2), evaluated exactly on the
 *    FP64 input value.
 *  - The nearest cell is c = floor((f + O/2) / O). The sub-offset is
 *    s = f - c*O, in [-O/2, O/2). The table row is r = s + O/2.
 *  - The footprint half-width is h = (S-1)/2 (integer division). The
 *    footprint covers cells C-h .. C-h+S-1, where C = c + G/2.
 *  - If a visibility's footprint is not wholly inside [0,G)^2, or its
 *    coordinates are not finite, it is skipped (counted, not gridded).
 *  - Weights multiply the visibility when gridding ("pre-weighted values",
 *    Sec. 4). Degridding applies no weight.
 *  - Degridding is the Hermitian adjoint of gridding with unit weights. The
 *    taps are real, so conj(tap) = tap.
 *  - The Kaiser-Bessel GCF is T(d) = I0(beta*sqrt(1-(2d/S)^2)) / I0(beta) for
 *    |d| <= S/2, and 0 otherwise. Row r, tap i sits at d = i - h - (r-O/2)/O.
 *
 * Arrays:
 *  - uv: [n][2] doubles (u, v).
 *  - vis: [n][P] complex, stored as interleaved (re, im) doubles.
 *  - grid: [P][G][G] complex, interleaved, row index v, column index u.
 *  - table: [O][S] doubles.
 *
 * Compile with -ffp-contract=off, so that no multiply-add is fused and every
 * product and sum is one correctly rounded FP64 operation.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

/* Largest |u*O| handled. Beyond it a visibility is off any supported grid. */
#define ORACLE_MAX_FINE 1099511627776.0 /* 2^40 */

static int is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

/*
 * Fine position f = floor(y + 1/2), y = u*O, in exact arithmetic.
 * y is exact because O is a power of two and |y| <= 2^40. The rounding rule
 * comes from the readings above. Write fl = floor(y). Then frac = y - fl is
 * exact whenever it matters for the comparison with 1/2 (Sterbenz's lemma for
 * |y| >= 1/2), so f = fl + (frac >= 1/2).
 * Returns 0 on success, -1 if u is not finite or out of range.
 */
int oracle_fine_position(double u, int O, int64_t* f) {
  if (!isfinite(u) || !is_pow2(O)) return -1;
  double y = u * (double)O;
  if (fabs(y) > ORACLE_MAX_FINE) return -1;
  double fl = floor(y);
  double frac = y - fl;
  *f = (int64_t)fl + (frac >= 0.5 ? 1 : 0);
  return 0;
}

/* Floor division for a positive divisor. */
static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
  return q;
}

/*
 * Per-visibility indices along one axis: absolute centre cell C and table row r.
 * Returns 0 if the footprint C-h .. C-h+S-1 lies in [0, G), else -1.
 */
static int axis_index(double u, int G, int S, int O, int64_t* C, int* r) {
  int64_t f;
  if (oracle_fine_position(u, O, &f) != 0) return -1;
  int64_t c = floor_div(f + O / 2, O);
  int64_t s = f - c * O; /* in [-O/2, O/2) */
  int h = (S - 1) / 2;
  *C = c + G / 2;
  *r = (int)(s + O / 2);
  if (*C - h < 0 || *C - h + S > G) return -1;
  return 0;
}

/*
 * Indices for n visibilities.
 *  - cell: [n][2] (C_u, C_v) absolute centre cells.
 *  - sub: [n][2] (r_u, r_v) table rows.
 * An invalid visibility gets cell = sub = (-1, -1).
 * Returns the number of invalid (skipped) visibilities, or -1 on bad
 * arguments.
 */
int64_t oracle_indices(int G, int S, int O, int64_t n, const double* uv, int32_t* cell, int32_t* sub) {
  if (G <= 0 || (G & 1) || S <= 0 || S > G || !is_pow2(O)) return -1;
  int64_t skipped = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t Cu, Cv;
    int ru, rv;
    int ok = axis_index(uv[2 * k], G, S, O, &Cu, &ru) == 0 && axis_index(uv[2 * k + 1], G, S, O, &Cv, &rv) == 0;
    if (ok) {
      cell[2 * k] = (int32_t)Cu;
      cell[2 * k + 1] = (int32_t)Cv;
      sub[2 * k] = ru;
      sub[2 * k + 1] = rv;
    } else {
      cell[2 * k] = cell[2 * k + 1] = -1;
      sub[2 * k] = sub[2 * k + 1] = -1;
      ++skipped;
    }
  }
  return skipped;
}

/*
 * Modified Bessel function of the first kind, order 0, from its power series
 * I0(x) = sum_k ((x/2)^k / k!)^2. All terms are positive, so there is no
 * cancellation. Terms are added until they no longer change the sum.
 */
double oracle_bessel_i0(double x) {
  double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 2000; ++k) {
    term *= q / ((double)k * (double)k);
    double next = sum + term;
    if (next == sum) break;
    sum = next;
  }
  return sum;
}

/*
 * Oversampled Kaiser-Bessel table, [O][S] doubles.
 * Row r, tap i: T(d) with d = i - h - (r - O/2)/O, following the readings
 * above. Returns 0, or -1 on bad arguments.
 */
int oracle_kb_table(int S, int O, double beta, double* table) {
  if (S <= 0 || O <= 0) return -1;
  int h = (S - 1) / 2;
  double norm = oracle_bessel_i0(beta);
  for (int r = 0; r < O; ++r) {
    for (int i = 0; i < S; ++i) {
      double d = (double)(i - h) - (double)(r - O / 2) / (double)O;
      double x = 2.0 * d / (double)S;
      double val = 0.0;
      if (fabs(x) <= 1.0) val = oracle_bessel_i0(beta * sqrt(1.0 - x * x)) / norm;
      table[(size_t)r * S + i] = val;
    }
  }
  return 0;
}

/*
 * Gridding (Sec. 2.2): for every valid visibility k, every polarization p and
 * every footprint tap (i, j):
 *   grid[p][C_v-h+j][C_u-h+i] += w_k * V_{k,p} * T[r_u][i] * T[r_v][j]
 * This is a direct scatter in visibility order, with no bins, tiles or
 * atomics. It accumulates into grid; the caller zeroes it.
 * Returns the number of skipped visibilities, or -1 on bad arguments.
 */
int64_t oracle_grid(int G, int S, int O, int P, int64_t n, const double* uv, const double* vis,
                    const double* weights, const double* table, double* grid) {
  if (G <= 0 || (G & 1) || S <= 0 || S > G || !is_pow2(O) || P <= 0) return -1;
  int h = (S - 1) / 2;
  int64_t skipped = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t Cu, Cv;
    int ru, rv;
    if (axis_index(uv[2 * k], G, S, O, &Cu, &ru) != 0 || axis_index(uv[2 * k + 1], G, S, O, &Cv, &rv) != 0) {
      ++skipped;
      continue;
    }
    double w = weights ? weights[k] : 1.0;
    const double* tu = table + (size_t)ru * S;
    const double* tv = table + (size_t)rv * S;
    for (int p = 0; p < P; ++p) {
      double vre = w * vis[2 * ((size_t)k * P + p)];
      double vim = w * vis[2 * ((size_t)k * P + p) + 1];
      for (int j = 0; j < S; ++j) {
        size_t row = ((size_t)p * G + (size_t)(Cv - h + j)) * G;
        for (int i = 0; i < S; ++i) {
          double t = tu[i] * tv[j];
          size_t cellidx = row + (size_t)(Cu - h + i);
          grid[2 * cellidx] += t * vre;
          grid[2 * cellidx + 1] += t * vim;
        }
      }
    }
  }
  return skipped;
}

/*
 * Degridding, the Hermitian adjoint of gridding with unit weights. For every
 * valid visibility k and polarization p:
 *   V_{k,p} = sum_{i,j} conj(T[r_u][i] * T[r_v][j]) * grid[p][C_v-h+j][C_u-h+i]
 * A skipped visibility gets V = 0. Overwrites vis.
 * Returns the number of skipped visibilities, or -1 on bad arguments.
 */
int64_t oracle_degrid(int G, int S, int O, int P, int64_t n, const double* uv, const double* grid,
                      const double* table, double* vis) {
  if (G <= 0 || (G & 1) || S <= 0 || S > G || !is_pow2(O) || P <= 0) return -1;
  int h = (S - 1) / 2;
  int64_t skipped = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t Cu, Cv;
    int ru, rv;
    int ok = axis_index(uv[2 * k], G, S, O, &Cu, &ru) == 0 && axis_index(uv[2 * k + 1], G, S, O, &Cv, &rv) == 0;
    if (!ok) ++skipped;
    for (int p = 0; p < P; ++p) {
      double sre = 0.0, sim = 0.0;
      if (ok) {
        const double* tu = table + (size_t)ru * S;
        const double* tv = table + (size_t)rv * S;
        for (int j = 0; j < S; ++j) {
          size_t row = ((size_t)p * G + (size_t)(Cv - h + j)) * G;
          for (int i = 0; i < S; ++i) {
            double t = tu[i] * tv[j]; /* real taps: conj(t) == t */
            size_t cellidx = row + (size_t)(Cu - h + i);
            sre += t * grid[2 * cellidx];
            sim += t * grid[2 * cellidx + 1];
          }
        }
      }
      vis[2 * ((size_t)k * P + p)] = sre;
      vis[2 * ((size_t)k * P + p) + 1] = sim;
    }
  }
  return skipped;
}

/*
 * Compression (Sec. 2.2, last paragraph; the scheme is Muscat's). Visibilities
 * that are adjacent and sit on the same point of the oversampled grid meet
 * the same GCF samples, so their weighted values can be added and gridded as
 * one visibility. The grid is unchanged up to rounding.
 * Readings:
 *  - "adjacent" means consecutive in the given order. A run is a maximal
 *    sequence of consecutive visibilities whose fine positions (f_u, f_v) are
 *    equal. Equal fine positions on both axes mean the same cell and the same
 *    GCF sample row.
 *  - A visibility with no fine position is a run of its own. Such a run is
 *    skipped when gridded, as before compression. A coordinate has no fine
 *    position here when it is not finite or |u*O| >= 2^26. That is far
 *    outside any supported grid (G <= 32768 and O <= 256 keep |u*O| < 2^22).
 *  - A merged record carries the first member's uv and the sum over the run
 *    of w_k V_k. Its weight is 1.
 * Outputs: uv_out [m][2], vis_out [m][P] complex (interleaved), and run_of
 * [n] (the run holding visibility k). Returns m, or -1 on bad arguments.
 */
int64_t oracle_compress(int O, int P, int64_t n, const double* uv, const double* vis, const double* weights,
                        double* uv_out, double* vis_out, int64_t* run_of) {
  if (!is_pow2(O) || P <= 0 || n < 0) return -1;
  int64_t m = 0;
  int prev_ok = 0;
  int64_t pfu = 0, pfv = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t fu = 0, fv = 0;
    int ok = oracle_fine_position(uv[2 * k], O, &fu) == 0 && oracle_fine_position(uv[2 * k + 1], O, &fv) == 0 &&
             fabs(uv[2 * k] * (double)O) < 67108864.0 && fabs(uv[2 * k + 1] * (double)O) < 67108864.0;
    int same = ok && prev_ok && fu == pfu && fv == pfv;
    if (!same) {
      uv_out[2 * m] = uv[2 * k];
      uv_out[2 * m + 1] = uv[2 * k + 1];
      for (int p = 0; p < 2 * P; ++p) vis_out[(size_t)m * 2 * P + p] = 0.0;
      ++m;
    }
    double w = weights ? weights[k] : 1.0;
    for (int p = 0; p < 2 * P; ++p) vis_out[(size_t)(m - 1) * 2 * P + p] += w * vis[(size_t)k * 2 * P + p];
    run_of[k] = m - 1;
    prev_ok = ok;
    pfu = fu;
    pfv = fv;
  }
  return m;
}
