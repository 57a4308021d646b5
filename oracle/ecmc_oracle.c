/*
 * ecmc_oracle.c -- reference (oracle) implementation of the parallel event
 * chain (PEC) Monte Carlo sweep for two-dimensional hard disks, after
 * Kampmann, Boltz, Kierfeld, arXiv:1409.6948.
 *
 * TEST INFRASTRUCTURE ONLY: this file is compiled into liboracle.so, which
 * the tests, the smoke check and the benchmark's CPU-baseline leg load.  The
 * CUDA library is a separate implementation that shares no code with it.
 *
 * Plain, sequential FP64 C, compiled with -O2 -ffp-contract=off (no fused
 * multiply-add), one disk at a time and one candidate at a time, so that a
 * reader can check it against the paper step by step:
 *
 *   Sec. 2, eq. (1)      hard disks of diameter sigma in a periodic L x L box.
 *   Sec. 3.2             straight event chain: the moving disk advances along
 *                        d until it touches another disk; the rest of the
 *                        displacement budget ell is passed to that disk.
 *   Sec. 3.4, steps 1-7  the sweep: square cells on a randomly shifted
 *                        lattice, 2x2 blocks with four colours, one random
 *                        colour order per sweep, n_m chain starts per cell
 *                        drawn WITH replacement, disks outside the active
 *                        cell frozen.
 *   Sec. 3.4 (Fig. 1)    a chain that would leave its cell or that hits a
 *                        frozen disk is reflected, angle of incidence equal to
 *                        angle of reflection.
 *   Sec. 3.4 (Fig. 2)    why the start list is drawn with replacement; the
 *                        shuffled list of distinct members is kept only as a
 *                        negative control (ORC_LIST_WITHOUT_REPL).
 *   Sec. 3.4 (Fig. 3)    the rejecting boundary rule the paper compares
 *                        against (ORC_BOUNDARY_REJECT): a chain that reaches
 *                        a wall or a frozen disk is rejected as a whole.
 *   Sec. 2               pair-correlation histogram with the centred-bin rule.
 *   Sec. 4, eq. (nm)     default number of chains per cell.
 *
 * Readings where the paper is silent, ambiguous or garbled:
 *   - direction: axis x on even sweeps and y on odd sweeps, sign +/- drawn
 *     per chain (the "+x/+y only" variant is not reversible, Sec. 3.2);
 *   - shift uniform on [0,w) x [0,h); colour order uniform over the 24
 *     orders, shared by all blocks; colour = (cx mod 2) + 2 (cy mod 2);
 *   - a disk belongs to the cell holding its centre (half-open cells),
 *     cx = floor((x - s_x mod L) * (1/w)) clamped to the grid.  The paper
 *     fixes no rounding rule at cell walls; the reciprocal is multiplied
 *     (one rounded product, as the CUDA binning computes it) rather than
 *     divided, so both sides put a disk lying on a wall to rounding in the
 *     same cell;
 *     start disk = member number floor(v n_c / 2^64) in ascending-id order;
 *   - geometry is done in the frame of the active cell: the cell occupies
 *     [0,w] x [0,h]; its members and every periodic image of every other
 *     disk whose centre lies in (-sigma, w+sigma) x (-sigma, h+sigma) are
 *     placed in that frame (this is exact for any even number of cells >= 2
 *     with w, h > sigma, including two cells per side, where a
 *     minimum-image convention would pick the wrong image);
 *   - ties: equal hit distances are broken by the smaller (id, image) key;
 *     at equal distance the chain end beats a contact, and a contact beats
 *     a wall; a corner reflects both components;
 *   - reflection (Fig. 1, angle of incidence equal to angle of reflection):
 *     a chain along an axis turns back along that axis at a frozen disk, as
 *     it does at a wall -- the reflection about the contact's tangent taken
 *     with respect to the chain axis.  This keeps every chain its own
 *     reverse (the detailed-balance argument around Fig. 2); a specular
 *     reflection about the line of centres would leave the axes, so the
 *     reverse chain would never be proposed (kept as ORC_FLAG_SPECULAR_AXIS,
 *     which the exact three-disk law rejects).  Isotropic chains reflect
 *     specularly about the line of centres; a wall flips the normal
 *     component of d;
 *   - pressure estimator, the collision form of eq. (pressure) that the
 *     paper names as an extension: the projected separation b of every
 *     contact (lifts and frozen-disk reflections) is summed per cell, and
 *     each cell's sum and displacement are weighted by its member count n_c:
 *     beta P / rho = 1 + sum_cells n_c sum_b / sum_cells n_c n_m ell.  Every
 *     cell receives the same displacement n_m ell whatever n_c, so the
 *     unweighted ratio over-weights sparse cells and reads low (the
 *     low-density virial series shows it); the unweighted sums are kept in
 *     sum_b, sum_disp.
 */
#include "ecmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x64-10, written from the description in Salmon et al., "Parallel  */
/* random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 64x64->128 */
/* multiplications, a word permutation and a key xor, with a Weyl-sequence   */
/* key schedule.                                                             */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ull
#define PHILOX_M1 0xCA5A826395121157ull
#define PHILOX_W0 0x9E3779B97F4A7C15ull /* golden ratio                */
#define PHILOX_W1 0xBB67AE8584CAA73Bull /* sqrt(3) - 1                 */

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t hi0, lo0, hi1, lo1;
    mul_hi_lo(PHILOX_M0, c0, &hi0, &lo0);
    mul_hi_lo(PHILOX_M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c3 ^ k1;
    uint64_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += PHILOX_W0;
    k1 += PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw4(const orc_params* p, uint64_t t, uint64_t purpose, uint64_t a, uint64_t b,
                  uint64_t out[4]) {
  uint64_t ctr[4] = {t, purpose, a, b};
  uint64_t key[2] = {p->seed, p->replica};
  orc_philox4x64_10(ctr, key, out);
}

/* uniform double in [0,1) from the top 53 bits */
static double unit53(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0,n): high word of the 128-bit product v*n */
static uint64_t below(uint64_t v, uint64_t n) {
  uint64_t hi, lo;
  mul_hi_lo(v, n, &hi, &lo);
  return hi;
}

/* ------------------------------------------------------------------------ */
/* Per-sweep draws (Sec. 3.4 steps 1-3)                                      */
/* ------------------------------------------------------------------------ */
void orc_sweep_draws(const orc_params* p, int64_t t, double* shift_x, double* shift_y,
                     int perm[4]) {
  uint64_t u[4];
  draw4(p, (uint64_t)t, ORC_PURPOSE_SWEEP, 0, 0, u);
  double w = p->L / (double)p->cells_x;
  double h = p->L / (double)p->cells_y;
  if (p->flags & ORC_FLAG_NO_SHIFT) {
    *shift_x = 0.0;
    *shift_y = 0.0;
  } else {
    *shift_x = unit53(u[0]) * w;
    *shift_y = unit53(u[1]) * h;
  }
  /* the colour order is permutation number below(u2, 24) of 0,1,2,3 in
   * lexicographic order (Lehmer code with factorial digits 6, 2, 1) */
  int code = (int)below(u[2], 24);
  if (p->flags & ORC_FLAG_FIXED_COLOURS) code = 0;
  int pool[4] = {0, 1, 2, 3};
  int left = 4;
  const int fact[4] = {6, 2, 1, 1};
  for (int i = 0; i < 4; ++i) {
    int digit = code / fact[i];
    code = code % fact[i];
    perm[i] = pool[digit];
    for (int j = digit; j < left - 1; ++j) pool[j] = pool[j + 1];
    --left;
  }
}

/* ------------------------------------------------------------------------ */
/* Cell decomposition (Sec. 3.4 step 1)                                      */
/* ------------------------------------------------------------------------ */
static int cell_index_1d(double v, double shift, double L, double w, int cells) {
  double u = v - shift;
  if (u < 0.0) u += L;
  const double inv_w = 1.0 / w;
  int c = (int)(u * inv_w);
  if (c >= cells) c = cells - 1;
  if (c < 0) c = 0;
  return c;
}

int orc_bin(const orc_params* p, int64_t t, const double* x, const double* y, int32_t* cell) {
  double sx, sy;
  int perm[4];
  orc_sweep_draws(p, t, &sx, &sy, perm);
  double w = p->L / (double)p->cells_x;
  double h = p->L / (double)p->cells_y;
  for (int64_t i = 0; i < p->N; ++i) {
    int cx = cell_index_1d(x[i], sx, p->L, w, p->cells_x);
    int cy = cell_index_1d(y[i], sy, p->L, h, p->cells_y);
    cell[i] = cy * p->cells_x + cx;
  }
  return 0;
}

int orc_default_nm(int64_t N, double L, double sigma, int cells_x, int cells_y, double ell) {
  const double pi = 3.14159265358979323846;
  double eta = (double)N * pi * sigma * sigma / (4.0 * L * L);       /* eq. (1)  */
  double eta_hcp = pi / (2.0 * sqrt(3.0));                            /* Sec. 2   */
  double lambda0 = sigma * (eta_hcp - eta) / (2.0 * eta_hcp);         /* Sec. 4   */
  double per_cell = (double)N / ((double)cells_x * (double)cells_y);  /* N / 4n   */
  double nm = per_cell * lambda0 / ell;                               /* eq. (nm) */
  int r = (int)floor(nm + 0.5);
  return r < 1 ? 1 : r;
}

/* The strategy that closes Sec. 4 for the degree of parallelisation, the
 * displacement and the chain starts, on a square grid of an even number of
 * cells per side (n = h^2 blocks of 2x2 cells, h blocks per side):
 *   1) h as large as possible with N / (eta n) > 100, which keeps the
 *      displacement of step 2 above 10 lambda0; then, while the cell side
 *      L / (2h) is not above max(sigma, min_cell_side), one block per side
 *      less (at least one);
 *   2) ell = lambda0 (N / (eta n))^(1/2), the second form of eq. (criterion),
 *      so that a chain spans about one cell;
 *   3) n_m from eq. (nm) (orc_default_nm).
 * Returns 0, or -1 if eta is at or above close packing or 2x2 cells of side
 * above the minimum do not fit. */
int orc_suggest_parameters(int64_t N, double L, double sigma, double min_cell_side,
                           int* cells_per_side, double* ell, int* n_m) {
  const double pi = 3.14159265358979323846;
  double eta = (double)N * pi * sigma * sigma / (4.0 * L * L); /* eq. (1) */
  double eta_hcp = pi / (2.0 * sqrt(3.0));
  double lambda0 = sigma * (eta_hcp - eta) / (2.0 * eta_hcp); /* Sec. 4 */
  if (!(lambda0 > 0.0) || N < 1) return -1;
  double side_min = min_cell_side > sigma ? min_cell_side : sigma;
  int64_t h = 1;
  while ((double)N / (eta * (double)((h + 1) * (h + 1))) > 100.0) h++;
  while (h > 1 && !(L / (double)(2 * h) > side_min)) h--;
  if (!(L / (double)(2 * h) > side_min)) return -1;
  double n = (double)(h * h);
  *cells_per_side = (int)(2 * h);
  *ell = lambda0 * sqrt((double)N / (eta * n));
  *n_m = orc_default_nm(N, L, sigma, (int)(2 * h), (int)(2 * h), *ell);
  return 0;
}

/* Uniformly distributed unit vector for chain k of cell c in sweep t: the
 * first point (u, v) of the sequence of Philox pairs, uniform on
 * [-1,1)^2, that falls inside the unit disc (and not at its centre),
 * divided by its length.  No trigonometric function is involved, so the
 * direction is reproducible to the last bit. */
static void isotropic_direction(const orc_params* p, int64_t t, int c, int k, double* dx,
                                double* dy) {
  for (uint64_t attempt = 0;; ++attempt) {
    uint64_t q[4];
    uint64_t ctr[4] = {(uint64_t)t, ORC_PURPOSE_DIRECTION, (uint64_t)c,
                       ((uint64_t)k << 32) | attempt};
    uint64_t key[2] = {p->seed, p->replica};
    orc_philox4x64_10(ctr, key, q);
    for (int h = 0; h < 2; ++h) {
      double u = 2.0 * unit53(q[2 * h]) - 1.0;
      double v = 2.0 * unit53(q[2 * h + 1]) - 1.0;
      double n2 = u * u + v * v;
      if (n2 > 0.0 && n2 <= 1.0) {
        double n = sqrt(n2);
        *dx = u / n;
        *dy = v / n;
        return;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One active cell in its own frame                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n;        /* objects in the frame                        */
  int n_mem;    /* the first n_mem objects are the members      */
  int cap;
  double* X;    /* frame coordinates                            */
  double* Y;
  int64_t* key; /* id*9 + image code (tie-break order)          */
  int64_t* id;
} frame_t;

static void frame_reserve(frame_t* f, int need) {
  if (need <= f->cap) return;
  int cap = f->cap ? f->cap : 256;
  while (cap < need) cap *= 2;
  f->X = (double*)realloc(f->X, sizeof(double) * cap);
  f->Y = (double*)realloc(f->Y, sizeof(double) * cap);
  f->key = (int64_t*)realloc(f->key, sizeof(int64_t) * cap);
  f->id = (int64_t*)realloc(f->id, sizeof(int64_t) * cap);
  f->cap = cap;
}

static void frame_push(frame_t* f, double X, double Y, int64_t id, int img) {
  frame_reserve(f, f->n + 1);
  f->X[f->n] = X;
  f->Y[f->n] = Y;
  f->key[f->n] = id * 9 + img;
  f->id[f->n] = id;
  f->n++;
}

/* periodic wrap into [-L/2, L/2) of a value known to lie in (-3L/2, 3L/2) */
static double wrap_centered(double v, double L) {
  if (v >= 0.5 * L) return v - L;
  if (v < -0.5 * L) return v + L;
  return v;
}

/* periodic wrap into [0, L) of a value known to lie in (-L, 2L) */
static double wrap_box(double v, double L) {
  if (v < 0.0) v += L;
  if (v >= L) v -= L;
  return v;
}

/* Add every image of disk j whose centre lies within the open strip of
 * width sigma around the cell rectangle [0,w] x [0,h]. */
static void add_frozen_images(frame_t* f, double X0, double Y0, int64_t id, double L,
                              double w, double h, double sigma) {
  for (int kx = -1; kx <= 1; ++kx) {
    double X = (kx == 0) ? X0 : (kx > 0 ? X0 + L : X0 - L);
    if (!(X > -sigma && X < w + sigma)) continue;
    for (int ky = -1; ky <= 1; ++ky) {
      double Y = (ky == 0) ? Y0 : (ky > 0 ? Y0 + L : Y0 - L);
      if (!(Y > -sigma && Y < h + sigma)) continue;
      frame_push(f, X, Y, id, (kx + 1) * 3 + (ky + 1));
    }
  }
}

typedef struct {
  double w, h, sigma, sig2;
  orc_stats* st;
  unsigned char* touched; /* per member: was the active disk of a chain */
  int specular;           /* frozen-disk contact: 1 specular, 0 reversal */
  int reject;             /* ORC_BOUNDARY_REJECT                         */
  double* X0;             /* reject: members' coordinates at chain start */
  double* Y0;
  unsigned char* touched0;
} chain_ctx;

/*
 * One straight event chain inside the frame (Sec. 3.2 with the boundary rule
 * of Sec. 3.4): object m (a member) starts with direction (dx, dy) and
 * budget ell.  Each step finds the first of
 *   - the end of the budget r,
 *   - the first contact with another object (brute force over the frame),
 *   - the first wall of the cell rectangle,
 * moves the active disk there and lifts (member hit), reflects specularly
 * (frozen disk hit) or flips the normal component of d (wall).
 *
 * Under the rejecting rule the members' coordinates are saved at the start;
 * the first wall or frozen-disk event restores them and ends the chain
 * (return value 1), and the chain's contact sum is dropped.  Otherwise the
 * chain's contact sum is added to the statistics as it accrues.
 */
static int run_chain(frame_t* f, const chain_ctx* cx, int m, double dx, double dy, double ell,
                     orc_chain_rec* rec) {
  const double w = cx->w, h = cx->h, sig2 = cx->sig2;
  double r = ell;
  int64_t nev = 0, nwall = 0;
  int rejected = 0;
  double chain_b = 0.0; /* reject: the chain's contact sum until it is accepted */
  if (cx->reject) {
    memcpy(cx->X0, f->X, sizeof(double) * (size_t)f->n_mem);
    memcpy(cx->Y0, f->Y, sizeof(double) * (size_t)f->n_mem);
    if (cx->touched) memcpy(cx->touched0, cx->touched, (size_t)f->n_mem);
  }
  if (cx->touched) cx->touched[m] = 1;
  for (int64_t iter = 0;; ++iter) {
    if (iter >= ORC_MAX_EVENTS_PER_CHAIN) {
      if (cx->st) cx->st->capped++;
      break;
    }
    const double Xm = f->X[m], Ym = f->Y[m];

    /* distance to the cell walls along d */
    double swx = INFINITY, swy = INFINITY;
    if (dx > 0.0) swx = (w - Xm) / fabs(dx);
    else if (dx < 0.0) swx = Xm / fabs(dx);
    if (dy > 0.0) swy = (h - Ym) / fabs(dy);
    else if (dy < 0.0) swy = Ym / fabs(dy);
    if (swx < 0.0) swx = 0.0;
    if (swy < 0.0) swy = 0.0;
    double swall = swx < swy ? swx : swy;

    /* first contact along d, brute force over every object of the frame */
    double best_s = INFINITY, best_b = 0.0;
    int best = -1;
    for (int j = 0; j < f->n; ++j) {
      if (j == m) continue;
      double ddx = f->X[j] - Xm;
      double ddy = f->Y[j] - Ym;
      double b = ddx * dx + ddy * dy;      /* separation along d            */
      if (!(b > 0.0)) continue;            /* disks behind are never hit    */
      double c = ddx * dy - ddy * dx;      /* separation across d           */
      double c2 = c * c;
      if (!(c2 < sig2)) continue;          /* passes beside                 */
      double s = b - sqrt(sig2 - c2);      /* travel until |separation|=sigma */
      if (s < 0.0) s = 0.0;
      if (s < best_s || (s == best_s && f->key[j] < f->key[best])) {
        best_s = s;
        best_b = b;
        best = j;
      }
    }

    if (r <= best_s && r <= swall) { /* budget used up: the chain ends */
      f->X[m] = Xm + r * dx;
      f->Y[m] = Ym + r * dy;
      if (cx->reject && cx->st) cx->st->sum_b += chain_b;
      break;
    }
    if (cx->reject && !(best_s <= swall && best < f->n_mem)) {
      /* the chain reaches a wall or a frozen disk: rejected as a whole */
      if (best_s <= swall) {
        nev++;
        if (cx->st) {
          cx->st->events++;
          cx->st->frozen_hits++;
        }
      } else {
        nwall++;
        if (cx->st) cx->st->wall_hits++;
      }
      memcpy(f->X, cx->X0, sizeof(double) * (size_t)f->n_mem);
      memcpy(f->Y, cx->Y0, sizeof(double) * (size_t)f->n_mem);
      if (cx->touched) memcpy(cx->touched, cx->touched0, (size_t)f->n_mem);
      if (cx->st) cx->st->rejected++;
      rejected = 1;
      break;
    }
    if (best_s <= swall) { /* contact */
      const double s = best_s;
      double nX = Xm + s * dx, nY = Ym + s * dy;
      f->X[m] = nX;
      f->Y[m] = nY;
      r = r - s;
      nev++;
      if (cx->st) {
        cx->st->events++;
        if (cx->reject) chain_b += best_b - s;
        else cx->st->sum_b += best_b - s;
      }
      if (best < f->n_mem) { /* lift: the hit member moves on along d */
        if (cx->st) cx->st->lifts++;
        m = best;
        if (cx->touched) cx->touched[m] = 1;
      } else if (cx->specular) { /* frozen disk: specular reflection about
                                    * the line of centres at contact */
        double nx = f->X[best] - nX;
        double ny = f->Y[best] - nY;
        double nn = nx * nx + ny * ny;
        double k = 2.0 * (dx * nx + dy * ny) / nn;
        dx = dx - k * nx;
        dy = dy - k * ny;
        if (cx->st) cx->st->frozen_hits++;
      } else { /* frozen disk, chain along a coordinate axis: the chain turns
                * back along the same axis */
        dx = -dx;
        dy = -dy;
        if (cx->st) cx->st->frozen_hits++;
      }
    } else { /* wall: move onto the wall, flip the normal component(s) */
      const double s = swall;
      double nX, nY;
      int flip_x = (swx == swall), flip_y = (swy == swall);
      if (flip_x) nX = (dx > 0.0) ? w : 0.0;
      else nX = Xm + s * dx;
      if (flip_y) nY = (dy > 0.0) ? h : 0.0;
      else nY = Ym + s * dy;
      f->X[m] = nX;
      f->Y[m] = nY;
      if (flip_x) dx = -dx;
      if (flip_y) dy = -dy;
      r = r - s;
      nwall++;
      if (cx->st) cx->st->wall_hits++;
    }
  }
  if (rec) {
    rec->end_id = f->id[m];
    rec->events = nev;
    rec->walls = nwall;
  }
  return rejected;
}

static int check_params(const orc_params* p) {
  if (p->N <= 0 || !(p->L > 0.0) || !(p->sigma > 0.0)) return -1;
  if (p->cells_x < 2 || p->cells_y < 2 || (p->cells_x & 1) || (p->cells_y & 1)) return -1;
  if (!(p->L / p->cells_x > p->sigma) || !(p->L / p->cells_y > p->sigma)) return -1;
  if (!(p->ell >= 0.0) || p->n_m < 1) return -1;
  if (p->boundary != ORC_BOUNDARY_REFLECT && p->boundary != ORC_BOUNDARY_REJECT) return -1;
  return 0;
}

int orc_sweeps(const orc_params* p, double* x, double* y, int64_t t0, int64_t n_sweeps,
               orc_stats* st, orc_chain_rec* recs) {
  if (check_params(p)) return -1;
  const int64_t N = p->N;
  const double L = p->L, sigma = p->sigma;
  const int ncx = p->cells_x, ncy = p->cells_y, ncell = ncx * ncy;
  const double w = L / (double)ncx, h = L / (double)ncy;
  chain_ctx ctx = {w, h, sigma, sigma * sigma, st, NULL,
                   p->dir_mode == ORC_DIR_ISOTROPIC || (p->flags & ORC_FLAG_SPECULAR_AXIS),
                   p->boundary == ORC_BOUNDARY_REJECT, NULL, NULL, NULL};

  int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * N);
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (ncell + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (ncell + 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * N);
  unsigned char* touched = NULL;
  int cap0 = 0;
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (p->n_m > 0 ? p->n_m : 1));
  int64_t* perm_buf = NULL;
  int64_t perm_cap = 0;
  frame_t f;
  memset(&f, 0, sizeof(f));

  for (int64_t s = 0; s < n_sweeps; ++s) {
    const int64_t t = t0 + s;
    double sx, sy;
    int perm[4];
    orc_sweep_draws(p, t, &sx, &sy, perm);

    /* step 1: every disk to the cell holding its centre; members of each
     * cell listed in ascending id (counting sort by cell, stable in id) */
    orc_bin(p, t, x, y, cell);
    memset(start, 0, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < N; ++i) start[cell[i] + 1]++;
    for (int c = 0; c < ncell; ++c) start[c + 1] += start[c];
    memcpy(fill, start, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < N; ++i) order[fill[cell[i]]++] = i;

    /* steps 2-6: colours in the drawn order; inside a colour the cells are
     * independent, visited row by row */
    for (int ci = 0; ci < 4; ++ci) {
      const int colour = perm[ci];
      const int colour_x = colour & 1, colour_y = colour >> 1;
      for (int k = 0; k < ncell; ++k) {
        int c = (p->flags & ORC_FLAG_REVERSE_CELLS) ? (ncell - 1 - k) : k;
        int cx = c % ncx, cy = c / ncx;
        if ((cx & 1) != colour_x || (cy & 1) != colour_y) continue;

        const double ox = sx + (double)cx * w; /* cell origin in box coordinates */
        const double oy = sy + (double)cy * h;
        const int64_t nc = start[c + 1] - start[c];

        /* frame: members first (ascending id), then frozen images */
        f.n = 0;
        for (int64_t q = start[c]; q < start[c + 1]; ++q) {
          int64_t i = order[q];
          frame_push(&f, wrap_centered(x[i] - ox, L), wrap_centered(y[i] - oy, L), i, 4);
        }
        f.n_mem = f.n;
        if (p->flags & ORC_FLAG_BRUTE_FROZEN) {
          for (int64_t j = 0; j < N; ++j) {
            if (cell[j] == c) continue;
            add_frozen_images(&f, wrap_centered(x[j] - ox, L), wrap_centered(y[j] - oy, L), j, L,
                              w, h, sigma);
          }
        } else {
          /* distinct neighbour cells of the 3x3 block (with two cells per
           * side the left and right neighbour coincide) */
          int nb[8], nnb = 0;
          for (int oyc = -1; oyc <= 1; ++oyc)
            for (int oxc = -1; oxc <= 1; ++oxc) {
              int qx = ((cx + oxc) % ncx + ncx) % ncx;
              int qy = ((cy + oyc) % ncy + ncy) % ncy;
              int q = qy * ncx + qx;
              if (q == c) continue;
              int dup = 0;
              for (int e = 0; e < nnb; ++e) dup |= (nb[e] == q);
              if (!dup) nb[nnb++] = q;
            }
          for (int e = 0; e < nnb; ++e)
            for (int64_t q = start[nb[e]]; q < start[nb[e] + 1]; ++q) {
              int64_t j = order[q];
              add_frozen_images(&f, wrap_centered(x[j] - ox, L), wrap_centered(y[j] - oy, L), j,
                                L, w, h, sigma);
            }
        }
        if (f.n_mem > cap0) {
          cap0 = f.n_mem;
          touched = (unsigned char*)realloc(touched, (size_t)cap0);
          ctx.X0 = (double*)realloc(ctx.X0, sizeof(double) * (size_t)cap0);
          ctx.Y0 = (double*)realloc(ctx.Y0, sizeof(double) * (size_t)cap0);
          ctx.touched0 = (unsigned char*)realloc(ctx.touched0, (size_t)cap0);
        }
        memset(touched, 0, (size_t)f.n_mem);
        ctx.touched = touched;

        /* step 5: the start list */
        if (nc > 0) {
          if (p->list_mode == ORC_LIST_WITHOUT_REPL) {
            /* negative control: first entry as drawn with replacement, the
             * others a uniformly shuffled list of the remaining members,
             * cycled if n_m > n_c */
            if (nc > perm_cap) {
              perm_cap = nc;
              perm_buf = (int64_t*)realloc(perm_buf, sizeof(int64_t) * perm_cap);
            }
            uint64_t v[4];
            draw4(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)c, 0, v);
            int64_t first = (int64_t)below(v[0], (uint64_t)nc);
            int64_t nrest = 0;
            perm_buf[nrest++] = first;
            for (int64_t q = 0; q < nc; ++q)
              if (q != first) perm_buf[nrest++] = q;
            /* Fisher-Yates on perm_buf[1..nc-1] */
            for (int64_t i = nc - 1; i >= 2; --i) {
              uint64_t u[4];
              draw4(p, (uint64_t)t, ORC_PURPOSE_SHUFFLE, (uint64_t)c, (uint64_t)(i >> 2), u);
              int64_t j = 1 + (int64_t)below(u[i & 3], (uint64_t)i);
              int64_t tmp = perm_buf[i];
              perm_buf[i] = perm_buf[j];
              perm_buf[j] = tmp;
            }
            for (int k2 = 0; k2 < p->n_m; ++k2) list[k2] = perm_buf[k2 % nc];
          } else {
            for (int k2 = 0; k2 < p->n_m; ++k2) {
              uint64_t v[4];
              draw4(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)c, (uint64_t)k2, v);
              list[k2] = (int64_t)below(v[0], (uint64_t)nc);
            }
          }
        }

        /* step 6: one chain per list entry, in list order */
        const double sum_b_before = st ? st->sum_b : 0.0;
        int accepted = 0;
        for (int k2 = 0; k2 < p->n_m; ++k2) {
          orc_chain_rec* rec = recs ? &recs[(s * ncell + c) * p->n_m + k2] : NULL;
          if (rec) {
            rec->start_id = -1;
            rec->end_id = -1;
            rec->events = 0;
            rec->walls = 0;
          }
          if (nc == 0) continue;
          uint64_t v[4];
          draw4(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)c, (uint64_t)k2, v);
          double dx, dy;
          if (p->dir_mode == ORC_DIR_ISOTROPIC) {
            isotropic_direction(p, t, c, k2, &dx, &dy);
          } else {
            int axis = (int)(t & 1);
            double sign = (p->dir_mode == ORC_DIR_POS_ONLY) ? 1.0 : ((v[1] >> 63) ? -1.0 : 1.0);
            dx = axis == 0 ? sign : 0.0;
            dy = axis == 0 ? 0.0 : sign;
          }
          int m = (int)list[k2];
          if (rec) rec->start_id = f.id[m];
          const int rej = run_chain(&f, &ctx, m, dx, dy, p->ell, rec);
          if (st) {
            st->chains++;
            if (!rej) st->sum_disp += p->ell;
          }
          accepted += rej ? 0 : 1;
        }

        /* member-weighted pressure sums: the cell's contact sum and its
         * displacement, each weighted by the number of members n_c */
        if (st && nc > 0) {
          st->sum_b_w += (double)nc * (st->sum_b - sum_b_before);
          st->sum_disp_w += (double)nc * ((double)accepted * p->ell);
        }

        /* write back, in box coordinates, every member that was the active
         * disk of a chain; the others keep their coordinates untouched */
        for (int q = 0; q < f.n_mem; ++q) {
          if (!touched[q]) continue;
          int64_t i = f.id[q];
          x[i] = wrap_box(f.X[q] + ox, L);
          y[i] = wrap_box(f.Y[q] + oy, L);
        }
      }
    }
    if (st) st->sweeps++;
  }

  free(cell);
  free(start);
  free(fill);
  free(order);
  free(touched);
  free(ctx.X0);
  free(ctx.Y0);
  free(ctx.touched0);
  free(list);
  free(perm_buf);
  free(f.X);
  free(f.Y);
  free(f.key);
  free(f.id);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sequential straight event chain on the whole periodic box (Sec. 3.2)      */
/* ------------------------------------------------------------------------ */
int orc_seq_sweeps(int64_t N, double L, double sigma, double ell, int64_t n_chains,
                   uint64_t seed, uint64_t replica, double* x, double* y, int64_t t0,
                   int64_t n_sweeps, orc_stats* st) {
  if (N <= 0 || !(L > 4.0 * sigma) || !(ell >= 0.0)) return -1;
  orc_params p;
  memset(&p, 0, sizeof(p));
  p.seed = seed;
  p.replica = replica;
  const double sig2 = sigma * sigma;
  /* longest single step: every disk within reach is then its own minimum image */
  const double seg = 0.25 * L;
  for (int64_t s = 0; s < n_sweeps; ++s) {
    const int64_t t = t0 + s;
    for (int64_t k = 0; k < n_chains; ++k) {
      uint64_t v[4];
      draw4(&p, (uint64_t)t, ORC_PURPOSE_CHAIN, 0, (uint64_t)k, v);
      int64_t m = (int64_t)below(v[0], (uint64_t)N);
      double sign = (v[1] >> 63) ? -1.0 : 1.0;
      int axis = (int)(t & 1);
      double dx = axis == 0 ? sign : 0.0, dy = axis == 0 ? 0.0 : sign;
      double r = ell;
      for (int64_t iter = 0;; ++iter) {
        if (iter >= ORC_MAX_EVENTS_PER_CHAIN) {
          if (st) st->capped++;
          break;
        }
        double best_s = INFINITY, best_b = 0.0;
        int64_t best = -1;
        for (int64_t j = 0; j < N; ++j) {
          if (j == m) continue;
          double ddx = wrap_centered(x[j] - x[m], L);
          double ddy = wrap_centered(y[j] - y[m], L);
          double b = ddx * dx + ddy * dy;
          if (!(b > 0.0)) continue;
          double c = ddx * dy - ddy * dx;
          double c2 = c * c;
          if (!(c2 < sig2)) continue;
          double sj = b - sqrt(sig2 - c2);
          if (sj < 0.0) sj = 0.0;
          if (sj < best_s || (sj == best_s && j < best)) {
            best_s = sj;
            best_b = b;
            best = j;
          }
        }
        /* free flight of at most seg; the chain ends when the budget does */
        double step = r < seg ? r : seg;
        if (step <= best_s) {
          x[m] = wrap_box(x[m] + step * dx, L);
          y[m] = wrap_box(y[m] + step * dy, L);
          r = r - step;
          if (!(r > 0.0)) break;
          continue;
        }
        x[m] = wrap_box(x[m] + best_s * dx, L);
        y[m] = wrap_box(y[m] + best_s * dy, L);
        r = r - best_s;
        if (st) {
          st->events++;
          st->lifts++;
          st->sum_b += best_b - best_s;
        }
        m = best;
      }
      if (st) {
        st->chains++;
        st->sum_disp += ell;
      }
    }
    if (st) st->sweeps++;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Pair-correlation histogram (Sec. 2)                                       */
/* ------------------------------------------------------------------------ */
void orc_gr_counts(int64_t N, double L, const double* x, const double* y, double sigma,
                   double dr, int nbins, int64_t i_begin, int64_t i_end, int64_t* counts) {
  for (int64_t i = i_begin; i < i_end; ++i) {
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue;
      double ddx = wrap_centered(x[j] - x[i], L);
      double ddy = wrap_centered(y[j] - y[i], L);
      double d = sqrt(ddx * ddx + ddy * ddy);
      double q = (d - sigma) / dr;
      if (!(q >= 0.0)) continue;
      if (!(q < (double)nbins)) continue;
      int bin = (int)q;
      counts[bin]++;
    }
  }
}

/* The same histogram with the pairs found through a cell list: the box is
 * cut into nc x nc square cells of side at least r_max (1 + 1e-6), r_max =
 * sigma + nbins dr, so that a pair within r_max (minimum image) lies in the
 * same or in adjacent cells; with nc >= 3 the nine cells around a disk are
 * distinct and no pair is seen twice.  Every pair is then tested with exactly
 * the expressions of orc_gr_counts, so the counts are identical; with nc < 3
 * this is orc_gr_counts.  Needs positions in [0, L). */
void orc_gr_counts_cells(int64_t N, double L, const double* x, const double* y, double sigma,
                         double dr, int nbins, int64_t* counts) {
  const double rmax = sigma + dr * (double)nbins;
  const int64_t nc = (int64_t)floor(L / (rmax * (1.0 + 1e-6)));
  if (nc < 3 || N < 2) {
    orc_gr_counts(N, L, x, y, sigma, dr, nbins, 0, N, counts);
    return;
  }
  const double cs = L / (double)nc;
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc * nc));
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  for (int64_t c = 0; c < nc * nc; ++c) head[c] = -1;
  for (int64_t i = 0; i < N; ++i) {
    int64_t cx = (int64_t)(x[i] / cs), cy = (int64_t)(y[i] / cs);
    if (cx < 0) cx = 0;
    if (cx > nc - 1) cx = nc - 1;
    if (cy < 0) cy = 0;
    if (cy > nc - 1) cy = nc - 1;
    cell[i] = cy * nc + cx;
    next[i] = head[cell[i]];
    head[cell[i]] = i;
  }
  for (int64_t i = 0; i < N; ++i) {
    const int64_t cx = cell[i] % nc, cy = cell[i] / nc;
    for (int64_t oy = -1; oy <= 1; ++oy) {
      for (int64_t ox = -1; ox <= 1; ++ox) {
        const int64_t c = ((cy + oy + nc) % nc) * nc + (cx + ox + nc) % nc;
        for (int64_t j = head[c]; j >= 0; j = next[j]) {
          if (j == i) continue;
          double ddx = wrap_centered(x[j] - x[i], L);
          double ddy = wrap_centered(y[j] - y[i], L);
          double d = sqrt(ddx * ddx + ddy * ddy);
          double q = (d - sigma) / dr;
          if (!(q >= 0.0)) continue;
          if (!(q < (double)nbins)) continue;
          counts[(int)q]++;
        }
      }
    }
  }
  free(head);
  free(next);
  free(cell);
}

/* ------------------------------------------------------------------------ */
/* Hexatic order parameter (Sec. 2, eq. Psi)                                 */
/* ------------------------------------------------------------------------ */
/* Next neighbours are the Delaunay neighbours.  Disk l (relative position
 * d_l from disk k, minimum image) is a Delaunay neighbour of k when the
 * perpendicular bisector of k and l keeps a piece of positive length after it
 * is cut by the half-planes p.d_m <= |d_m|^2 / 2 of every other disk m within
 * rs of k: that piece is the Voronoi edge between k and l.  The result is the
 * exact Delaunay graph when every Voronoi vertex of k lies within rs/2 of k
 * (a disk beyond rs cannot cut the cell then); disks for which that check
 * fails are counted in the return value.  Psi_k = sum over neighbours of
 * exp(6 i phi_kl) / n_k, exp(6 i phi) = (dx + i dy)^6 / |d|^6 with no
 * trigonometric function.  Returns -1 if L <= 2 rs. */
int orc_hexatic(int64_t N, double L, const double* x, const double* y, double rs,
                double* psi_k, int32_t* n_nb, double* psi) {
  if (!(L > 2.0 * rs) || N < 1) return -1;
  int cap = 64;
  double* cx = (double*)malloc(sizeof(double) * cap);
  double* cy = (double*)malloc(sizeof(double) * cap);
  const double rs2 = rs * rs, v2max = 0.25 * rs * rs;
  double sre = 0.0, sim = 0.0;
  int bad = 0;
  for (int64_t k = 0; k < N; ++k) {
    int nc = 0;
    for (int64_t j = 0; j < N; ++j) {
      if (j == k) continue;
      double ddx = wrap_centered(x[j] - x[k], L);
      double ddy = wrap_centered(y[j] - y[k], L);
      if (!(ddx * ddx + ddy * ddy < rs2)) continue;
      if (nc == cap) {
        cap *= 2;
        cx = (double*)realloc(cx, sizeof(double) * cap);
        cy = (double*)realloc(cy, sizeof(double) * cap);
      }
      cx[nc] = ddx;
      cy[nc] = ddy;
      nc++;
    }
    double re = 0.0, im = 0.0;
    int n = 0, ok = 1;
    for (int l = 0; l < nc; ++l) {
      const double ux = -cy[l], uy = cx[l];          /* along the bisector   */
      const double px0 = 0.5 * cx[l], py0 = 0.5 * cy[l]; /* its midpoint    */
      double tlo = -INFINITY, thi = INFINITY;
      for (int m = 0; m < nc && tlo < thi; ++m) {
        if (m == l) continue;
        const double a = ux * cx[m] + uy * cy[m];
        const double b = 0.5 * (cx[m] * cx[m] + cy[m] * cy[m]) - (px0 * cx[m] + py0 * cy[m]);
        if (a > 0.0) {
          const double t = b / a;
          if (t < thi) thi = t;
        } else if (a < 0.0) {
          const double t = b / a;
          if (t > tlo) tlo = t;
        } else if (b < 0.0) {
          thi = -INFINITY;
        }
      }
      if (!(tlo < thi)) continue;
      if (!(tlo > -INFINITY) || !(thi < INFINITY)) {
        ok = 0;
      } else {
        const double vx0 = px0 + tlo * ux, vy0 = py0 + tlo * uy;
        const double vx1 = px0 + thi * ux, vy1 = py0 + thi * uy;
        if (!(vx0 * vx0 + vy0 * vy0 < v2max) || !(vx1 * vx1 + vy1 * vy1 < v2max)) ok = 0;
      }
      /* exp(6 i phi) = z^6 / |z|^6 */
      const double zx = cx[l], zy = cy[l];
      const double z2x = zx * zx - zy * zy, z2y = 2.0 * zx * zy;
      const double z3x = z2x * zx - z2y * zy, z3y = z2x * zy + z2y * zx;
      const double z6x = z3x * z3x - z3y * z3y, z6y = 2.0 * z3x * z3y;
      const double r2 = zx * zx + zy * zy;
      const double r6 = r2 * r2 * r2;
      re += z6x / r6;
      im += z6y / r6;
      n++;
    }
    if (!ok) bad++;
    const double pk_re = n > 0 ? re / (double)n : 0.0, pk_im = n > 0 ? im / (double)n : 0.0;
    if (psi_k) {
      psi_k[2 * k] = pk_re;
      psi_k[2 * k + 1] = pk_im;
    }
    if (n_nb) n_nb[k] = n;
    sre += pk_re;
    sim += pk_im;
  }
  free(cx);
  free(cy);
  if (psi) {
    psi[0] = sre / (double)N;
    psi[1] = sim / (double)N;
  }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Smallest pair distance (overlap check), plain uniform grid                */
/* ------------------------------------------------------------------------ */
double orc_min_dist2(int64_t N, double L, const double* x, const double* y, double rcut) {
  int g = (int)(L / rcut);
  if (g < 3) {
    double best = rcut * rcut;
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = i + 1; j < N; ++j) {
        double ddx = wrap_centered(x[j] - x[i], L);
        double ddy = wrap_centered(y[j] - y[i], L);
        double d2 = ddx * ddx + ddy * ddy;
        if (d2 < best) best = d2;
      }
    return best;
  }
  double gs = L / (double)g;
  int64_t ng = (int64_t)g * g;
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * ng);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * N);
  for (int64_t q = 0; q < ng; ++q) head[q] = -1;
  for (int64_t i = 0; i < N; ++i) {
    int gx = (int)(wrap_box(x[i], L) / gs), gy = (int)(wrap_box(y[i], L) / gs);
    if (gx >= g) gx = g - 1;
    if (gy >= g) gy = g - 1;
    int64_t q = (int64_t)gy * g + gx;
    next[i] = head[q];
    head[q] = i;
  }
  double best = rcut * rcut;
  for (int gy = 0; gy < g; ++gy)
    for (int gx = 0; gx < g; ++gx)
      for (int64_t i = head[(int64_t)gy * g + gx]; i >= 0; i = next[i])
        for (int oy = -1; oy <= 1; ++oy)
          for (int ox = -1; ox <= 1; ++ox) {
            int qx = ((gx + ox) % g + g) % g, qy = ((gy + oy) % g + g) % g;
            for (int64_t j = head[(int64_t)qy * g + qx]; j >= 0; j = next[j]) {
              if (j <= i) continue;
              double ddx = wrap_centered(x[j] - x[i], L);
              double ddy = wrap_centered(y[j] - y[i], L);
              double d2 = ddx * ddx + ddy * ddy;
              if (d2 < best) best = d2;
            }
          }
  free(head);
  free(next);
  return best;
}

/* ------------------------------------------------------------------------ */
/* One chain on a caller-built frame (geometry tests)                        */
/* ------------------------------------------------------------------------ */
int orc_run_chain_frame(int n, int n_mem, double* X, double* Y, const int64_t* id,
                        const int32_t* img, double w, double h, double sigma, int m, double dx,
                        double dy, double ell, int mode, orc_stats* st,
                        orc_chain_rec* rec) {
  if (n < 1 || n_mem < 1 || n_mem > n || m < 0 || m >= n_mem) return -1;
  frame_t f;
  memset(&f, 0, sizeof(f));
  for (int q = 0; q < n; ++q) frame_push(&f, X[q], Y[q], id[q], img[q]);
  f.n_mem = n_mem;
  const int reject = (mode & 2) != 0;
  double* X0 = reject ? (double*)malloc(sizeof(double) * (size_t)n_mem) : NULL;
  double* Y0 = reject ? (double*)malloc(sizeof(double) * (size_t)n_mem) : NULL;
  chain_ctx ctx = {w, h, sigma, sigma * sigma, st, NULL, mode & 1, reject, X0, Y0, NULL};
  if (rec) rec->start_id = id[m];
  const int rej = run_chain(&f, &ctx, m, dx, dy, ell, rec);
  if (st) {
    st->chains++;
    if (!rej) st->sum_disp += ell;
  }
  free(X0);
  free(Y0);
  for (int q = 0; q < n; ++q) {
    X[q] = f.X[q];
    Y[q] = f.Y[q];
  }
  free(f.X);
  free(f.Y);
  free(f.key);
  free(f.id);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sweeps with a copy of the configuration after every sweep (sampling)     */
/* ------------------------------------------------------------------------ */
int orc_sweeps_snap(const orc_params* p, double* x, double* y, int64_t t0, int64_t n_sweeps,
                    orc_stats* st, double* snap_x, double* snap_y) {
  for (int64_t s = 0; s < n_sweeps; ++s) {
    int rc = orc_sweeps(p, x, y, t0 + s, 1, st, NULL);
    if (rc) return rc;
    memcpy(snap_x + s * p->N, x, sizeof(double) * p->N);
    memcpy(snap_y + s * p->N, y, sizeof(double) * p->N);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Autocorrelation time of the hexatic order parameter (Sec. 2, eq. tau)     */
/* ------------------------------------------------------------------------ */
/* R series (replicas) of n samples, series r in re[r*n .. r*n+n), im[...]:
 * C(dt) = Re <conj(Psi_r(t)) Psi_r(t+dt)> / <|Psi_r(t)|^2>, each average over
 * all the terms available (R (n - dt) pairs at lag dt, R n samples for the
 * norm), the mean of Psi taken as zero as the definition says.  tau = the
 * first lag with C < 1/e, moved back linearly towards the lag before it;
 * INFINITY if there is none up to max_lag.  c[] (may be NULL) receives
 * C(0..max_lag).  Returns 0, or -1 for a bad argument. */
int orc_autocorrelation_time(const double* re, const double* im, int64_t n, int R,
                             int64_t max_lag, double* tau, double* c) {
  if (n < 2 || R < 1 || max_lag < 1 || max_lag >= n) return -1;
  double power = 0.0;
  for (int r = 0; r < R; ++r)
    for (int64_t t = 0; t < n; ++t) {
      const int64_t i = (int64_t)r * n + t;
      power += re[i] * re[i] + im[i] * im[i];
    }
  power = power / ((double)n * (double)R);
  if (!(power > 0.0)) return -1;
  double threshold = exp(-1.0);
  double c_prev = 0.0;
  *tau = INFINITY;
  for (int64_t lag = 0; lag <= max_lag; ++lag) {
    double sum = 0.0;
    int64_t pairs = n - lag;
    for (int r = 0; r < R; ++r) {
      const double* a_re = re + (int64_t)r * n;
      const double* a_im = im + (int64_t)r * n;
      for (int64_t t = 0; t < pairs; ++t) {
        /* real part of conj(a) * b */
        sum += a_re[t] * a_re[t + lag] + a_im[t] * a_im[t + lag];
      }
    }
    double c_lag = (sum / ((double)pairs * (double)R)) / power;
    if (c) c[lag] = c_lag;
    if (c_lag < threshold && isinf(*tau)) {
      if (lag == 0)
        *tau = 0.0;
      else
        *tau = (double)(lag - 1) + (c_prev - threshold) / (c_prev - c_lag);
    }
    c_prev = c_lag;
  }
  return 0;
}
