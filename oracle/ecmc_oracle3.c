/*
 * ecmc_oracle3.c -- oracle of the parallel event-chain sweep for hard
 * spheres in three dimensions (Kampmann, Boltz, Kierfeld, arXiv:1409.6948,
 * Sec. 3.4, the three-dimensional generalisation of the seven steps).
 *
 * TEST INFRASTRUCTURE ONLY (see ecmc_oracle3.h).  Plain sequential FP64 C,
 * compiled with -ffp-contract=off, one sphere and one candidate at a time.
 *
 * The two-dimensional readings carry over, with these choices for the third
 * dimension:
 *   - cells: the box is cut into cells^3 cubes of side w = L / cells on a
 *     lattice shifted by s uniform on [0,w)^3; a sphere belongs to the cube
 *     holding its centre; colour = (cx mod 2) + 2 (cy mod 2) + 4 (cz mod 2);
 *     one uniformly random order of the eight colours per sweep;
 *   - chains run along a coordinate axis, x, y, z in turn by sweep
 *     (axis = t mod 3), sign drawn per chain; like the two-dimensional axis
 *     chains they turn back along the axis at a cell wall or a frozen
 *     sphere, which keeps each chain its own reverse;
 *   - frozen spheres: every periodic image of a sphere of the 26 neighbour
 *     cells whose centre lies in the open slab (-sigma, w+sigma)^3;
 *   - hit test for direction +-e_a: b = +-(x_a(j) - x_a(m)),
 *     c^2 = dp*dp + dq*dq over the two other axes in increasing order,
 *     hit iff b > 0 and c^2 < sigma^2, s = max(0, b - sqrt(sigma^2 - c^2));
 *   - ties, event order and the member-weighted pressure sums as in two
 *     dimensions.  The collision form beta P / rho = 1 + sum b / sum ell
 *     carries over unchanged: per unit displacement a mover meets contacts
 *     at rate rho g(sigma+) pi sigma^2, with mean b = 2 sigma / 3 over the
 *     disc of impact parameters, which is the excess term
 *     (2 pi / 3) rho sigma^3 g(sigma+) of the pressure equation.
 */
#include "ecmc_oracle3.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* same Philox words as the two-dimensional oracle: key (seed, replica),
 * counter (t, purpose, a, b) */
static void draw4_3(const orc3_params* p, uint64_t t, uint64_t purpose, uint64_t a, uint64_t b,
                    uint64_t out[4]) {
  uint64_t ctr[4] = {t, purpose, a, b};
  uint64_t key[2] = {p->seed, p->replica};
  orc_philox4x64_10(ctr, key, out);
}

static uint64_t below3(uint64_t v, uint64_t n) {
  /* uniform integer in [0,n): high word of the 128-bit product v*n */
  return (uint64_t)(((unsigned __int128)v * (unsigned __int128)n) >> 64);
}

static double unit53_3(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

static double wrapc(double v, double L) {
  if (v >= 0.5 * L) return v - L;
  if (v < -0.5 * L) return v + L;
  return v;
}

static double wrapb(double v, double L) {
  if (v < 0.0) v += L;
  if (v >= L) v -= L;
  return v;
}

static int check3(const orc3_params* p) {
  if (p->N <= 0 || !(p->L > 0.0) || !(p->sigma > 0.0)) return -1;
  if (p->cells < 2 || (p->cells & 1)) return -1;
  if (!(p->L / p->cells > p->sigma)) return -1;
  if (!(p->ell >= 0.0) || p->n_m < 1) return -1;
  return 0;
}

void orc3_sweep_draws(const orc3_params* p, int64_t t, double shift[3], int perm[8]) {
  uint64_t u[4];
  draw4_3(p, (uint64_t)t, ORC_PURPOSE_SWEEP, 0, 0, u);
  const double w = p->L / (double)p->cells;
  for (int a = 0; a < 3; ++a)
    shift[a] = (p->flags & ORC_FLAG_NO_SHIFT) ? 0.0 : unit53_3(u[a]) * w;
  /* permutation number below(u3, 8!) in lexicographic order, decoded with
   * factorial digits 7!, 6!, ..., 0! */
  int code = (int)below3(u[3], 40320);
  if (p->flags & ORC_FLAG_FIXED_COLOURS) code = 0;
  int pool[8] = {0, 1, 2, 3, 4, 5, 6, 7};
  int left = 8;
  const int fact[8] = {5040, 720, 120, 24, 6, 2, 1, 1};
  for (int i = 0; i < 8; ++i) {
    const int digit = code / fact[i];
    code = code % fact[i];
    perm[i] = pool[digit];
    for (int j = digit; j < left - 1; ++j) pool[j] = pool[j + 1];
    --left;
  }
}

static int cell1(double v, double shift, double L, double w, int cells) {
  double u = v - shift;
  if (u < 0.0) u += L;
  const double inv_w = 1.0 / w;
  int c = (int)(u * inv_w);
  if (c >= cells) c = cells - 1;
  if (c < 0) c = 0;
  return c;
}

int orc3_bin(const orc3_params* p, int64_t t, const double* x, const double* y, const double* z,
             int32_t* cell) {
  if (check3(p)) return -1;
  double s[3];
  int perm[8];
  orc3_sweep_draws(p, t, s, perm);
  const int nc = p->cells;
  const double w = p->L / (double)nc;
  for (int64_t i = 0; i < p->N; ++i) {
    const int cx = cell1(x[i], s[0], p->L, w, nc);
    const int cy = cell1(y[i], s[1], p->L, w, nc);
    const int cz = cell1(z[i], s[2], p->L, w, nc);
    cell[i] = (cz * nc + cy) * nc + cx;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Frame of one active cell                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n, n_mem, cap;
  double* C[3];  /* frame coordinates x, y, z        */
  int64_t* key;  /* id * 27 + image code              */
  int64_t* id;
} frame3;

static void f3_push(frame3* f, double X, double Y, double Z, int64_t id, int img) {
  if (f->n + 1 > f->cap) {
    int cap = f->cap ? 2 * f->cap : 256;
    for (int a = 0; a < 3; ++a) f->C[a] = (double*)realloc(f->C[a], sizeof(double) * cap);
    f->key = (int64_t*)realloc(f->key, sizeof(int64_t) * cap);
    f->id = (int64_t*)realloc(f->id, sizeof(int64_t) * cap);
    f->cap = cap;
  }
  f->C[0][f->n] = X;
  f->C[1][f->n] = Y;
  f->C[2][f->n] = Z;
  f->key[f->n] = id * 27 + img;
  f->id[f->n] = id;
  f->n++;
}

static void f3_free(frame3* f) {
  for (int a = 0; a < 3; ++a) free(f->C[a]);
  free(f->key);
  free(f->id);
}

/* every image of sphere id whose centre lies in the open slab around [0,w]^3 */
static void add_images3(frame3* f, const double X0[3], int64_t id, double L, double w,
                        double sigma) {
  for (int kx = -1; kx <= 1; ++kx) {
    const double X = X0[0] + (double)kx * L;
    if (!(X > -sigma && X < w + sigma)) continue;
    for (int ky = -1; ky <= 1; ++ky) {
      const double Y = X0[1] + (double)ky * L;
      if (!(Y > -sigma && Y < w + sigma)) continue;
      for (int kz = -1; kz <= 1; ++kz) {
        const double Z = X0[2] + (double)kz * L;
        if (!(Z > -sigma && Z < w + sigma)) continue;
        f3_push(f, X, Y, Z, id, (kx + 1) * 9 + (ky + 1) * 3 + (kz + 1));
      }
    }
  }
}

/*
 * One chain along axis a with sign sg and budget ell (Sec. 3.2 in three
 * dimensions with the boundary rule of Sec. 3.4): each step finds the first
 * of the end of the budget, the first contact (brute force over the frame)
 * and the wall ahead; a member contact lifts, a frozen contact or a wall
 * turns the chain back along its axis.
 */
static void chain3(frame3* f, double w, double sig2, int m, int a, int sg, double ell,
                   orc_stats* st, unsigned char* touched, orc_chain_rec* rec) {
  const int p = a == 0 ? 1 : 0, q = a == 2 ? 1 : 2;
  double r = ell;
  int64_t nev = 0, nwall = 0;
  if (touched) touched[m] = 1;
  for (int64_t iter = 0;; ++iter) {
    if (iter >= ORC_MAX_EVENTS_PER_CHAIN) {
      if (st) st->capped++;
      break;
    }
    const double P = f->C[a][m];
    double sw = sg > 0 ? w - P : P;
    if (sw < 0.0) sw = 0.0;
    double best_s = INFINITY, best_b = 0.0;
    int best = -1;
    for (int j = 0; j < f->n; ++j) {
      if (j == m) continue;
      const double da = f->C[a][j] - P;
      const double b = sg > 0 ? da : -da;
      if (!(b > 0.0)) continue;
      const double dp = f->C[p][j] - f->C[p][m];
      const double dq = f->C[q][j] - f->C[q][m];
      const double c2 = dp * dp + dq * dq;
      if (!(c2 < sig2)) continue;
      double s = b - sqrt(sig2 - c2);
      if (s < 0.0) s = 0.0;
      if (s < best_s || (s == best_s && f->key[j] < f->key[best])) {
        best_s = s;
        best_b = b;
        best = j;
      }
    }
    if (r <= best_s && r <= sw) { /* budget used up */
      f->C[a][m] = P + (sg > 0 ? r : -r);
      break;
    }
    if (best_s <= sw) { /* contact */
      f->C[a][m] = P + (sg > 0 ? best_s : -best_s);
      r = r - best_s;
      nev++;
      if (st) {
        st->events++;
        st->sum_b += best_b - best_s;
      }
      if (best < f->n_mem) { /* lift */
        if (st) st->lifts++;
        m = best;
        if (touched) touched[m] = 1;
      } else { /* frozen sphere: back along the axis */
        sg = -sg;
        if (st) st->frozen_hits++;
      }
    } else { /* wall: onto the wall, back along the axis */
      f->C[a][m] = sg > 0 ? w : 0.0;
      r = r - sw;
      sg = -sg;
      nwall++;
      if (st) st->wall_hits++;
    }
  }
  if (rec) {
    rec->end_id = f->id[m];
    rec->events = nev;
    rec->walls = nwall;
  }
}

int orc3_sweeps(const orc3_params* p, double* x, double* y, double* z, int64_t t0,
                int64_t n_sweeps, orc_stats* st, orc_chain_rec* recs) {
  if (check3(p)) return -1;
  const int64_t N = p->N;
  const double L = p->L, sigma = p->sigma, sig2 = sigma * sigma;
  const int nc = p->cells, ncell = nc * nc * nc;
  const double w = L / (double)nc;
  double* pos[3] = {x, y, z};

  int32_t* cell = (int32_t*)malloc(sizeof(int32_t) * N);
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (ncell + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (ncell + 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * N);
  unsigned char* touched = NULL;
  int cap0 = 0;
  frame3 f;
  memset(&f, 0, sizeof(f));

  for (int64_t s = 0; s < n_sweeps; ++s) {
    const int64_t t = t0 + s;
    double sh[3];
    int perm[8];
    orc3_sweep_draws(p, t, sh, perm);
    const int axis = (int)(t % 3);

    /* step 1: cells, members in ascending id */
    orc3_bin(p, t, x, y, z, cell);
    memset(start, 0, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < N; ++i) start[cell[i] + 1]++;
    for (int c = 0; c < ncell; ++c) start[c + 1] += start[c];
    memcpy(fill, start, sizeof(int64_t) * (ncell + 1));
    for (int64_t i = 0; i < N; ++i) order[fill[cell[i]]++] = i;

    for (int ci = 0; ci < 8; ++ci) {
      const int colour = perm[ci];
      for (int k = 0; k < ncell; ++k) {
        const int c = (p->flags & ORC_FLAG_REVERSE_CELLS) ? (ncell - 1 - k) : k;
        const int cx = c % nc, cy = (c / nc) % nc, cz = c / (nc * nc);
        if ((cx & 1) + 2 * (cy & 1) + 4 * (cz & 1) != colour) continue;
        const double o[3] = {sh[0] + (double)cx * w, sh[1] + (double)cy * w,
                             sh[2] + (double)cz * w};
        const int64_t ncm = start[c + 1] - start[c];

        /* frame: members first (ascending id), then frozen images */
        f.n = 0;
        for (int64_t qq = start[c]; qq < start[c + 1]; ++qq) {
          const int64_t i = order[qq];
          f3_push(&f, wrapc(x[i] - o[0], L), wrapc(y[i] - o[1], L), wrapc(z[i] - o[2], L), i,
                  13);
        }
        f.n_mem = f.n;
        if (p->flags & ORC_FLAG_BRUTE_FROZEN) {
          for (int64_t j = 0; j < N; ++j) {
            if (cell[j] == c) continue;
            const double X0[3] = {wrapc(x[j] - o[0], L), wrapc(y[j] - o[1], L),
                                  wrapc(z[j] - o[2], L)};
            add_images3(&f, X0, j, L, w, sigma);
          }
        } else {
          int nb[26], nnb = 0;
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int qx = ((cx + dx) % nc + nc) % nc;
                const int qy = ((cy + dy) % nc + nc) % nc;
                const int qz = ((cz + dz) % nc + nc) % nc;
                const int qc = (qz * nc + qy) * nc + qx;
                if (qc == c) continue;
                int dup = 0;
                for (int e = 0; e < nnb; ++e) dup |= (nb[e] == qc);
                if (!dup) nb[nnb++] = qc;
              }
          for (int e = 0; e < nnb; ++e)
            for (int64_t qq = start[nb[e]]; qq < start[nb[e] + 1]; ++qq) {
              const int64_t j = order[qq];
              const double X0[3] = {wrapc(x[j] - o[0], L), wrapc(y[j] - o[1], L),
                                    wrapc(z[j] - o[2], L)};
              add_images3(&f, X0, j, L, w, sigma);
            }
        }
        if (f.n_mem > cap0) {
          cap0 = f.n_mem;
          touched = (unsigned char*)realloc(touched, (size_t)cap0);
        }
        if (f.n_mem > 0) memset(touched, 0, (size_t)f.n_mem);

        /* steps 5-6: n_m chains, starts drawn with replacement */
        const double sum_b_before = st ? st->sum_b : 0.0;
        for (int k2 = 0; k2 < p->n_m; ++k2) {
          orc_chain_rec* rec = recs ? &recs[(s * ncell + c) * p->n_m + k2] : NULL;
          if (rec) {
            rec->start_id = -1;
            rec->end_id = -1;
            rec->events = 0;
            rec->walls = 0;
          }
          if (ncm == 0) continue;
          uint64_t v[4];
          draw4_3(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)c, (uint64_t)k2, v);
          const int m = (int)below3(v[0], (uint64_t)ncm);
          const int sg = (v[1] >> 63) ? -1 : 1;
          if (rec) rec->start_id = f.id[m];
          chain3(&f, w, sig2, m, axis, sg, p->ell, st, touched, rec);
          if (st) {
            st->chains++;
            st->sum_disp += p->ell;
          }
        }
        if (st && ncm > 0) {
          st->sum_b_w += (double)ncm * (st->sum_b - sum_b_before);
          st->sum_disp_w += (double)ncm * ((double)p->n_m * p->ell);
        }
        /* write back the members that moved */
        for (int qq = 0; qq < f.n_mem; ++qq) {
          if (!touched[qq]) continue;
          const int64_t i = f.id[qq];
          for (int a = 0; a < 3; ++a) pos[a][i] = wrapb(f.C[a][qq] + o[a], L);
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
  f3_free(&f);
  return 0;
}

int orc3_run_chain_frame(int n, int n_mem, double* X, double* Y, double* Z, const int64_t* id,
                         const int32_t* img, double w, double sigma, int m, int axis, int sign,
                         double ell, orc_stats* st, orc_chain_rec* rec) {
  if (n < 1 || n_mem < 1 || n_mem > n || m < 0 || m >= n_mem || axis < 0 || axis > 2 ||
      (sign != 1 && sign != -1))
    return -1;
  frame3 f;
  memset(&f, 0, sizeof(f));
  for (int qq = 0; qq < n; ++qq) f3_push(&f, X[qq], Y[qq], Z[qq], id[qq], img[qq]);
  f.n_mem = n_mem;
  if (rec) rec->start_id = id[m];
  chain3(&f, w, sigma * sigma, m, axis, sign, ell, st, NULL, rec);
  if (st) {
    st->chains++;
    st->sum_disp += ell;
  }
  for (int qq = 0; qq < n; ++qq) {
    X[qq] = f.C[0][qq];
    Y[qq] = f.C[1][qq];
    Z[qq] = f.C[2][qq];
  }
  f3_free(&f);
  return 0;
}

double orc3_min_dist2(int64_t N, double L, const double* x, const double* y, const double* z,
                      double rcut) {
  double best = rcut * rcut;
  int g = (int)(L / rcut);
  if (g < 3) {
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = i + 1; j < N; ++j) {
        const double dx = wrapc(x[j] - x[i], L), dy = wrapc(y[j] - y[i], L),
                     dz = wrapc(z[j] - z[i], L);
        const double d2 = dx * dx + dy * dy + dz * dz;
        if (d2 < best) best = d2;
      }
    return best;
  }
  const double gs = L / (double)g;
  const int64_t ng = (int64_t)g * g * g;
  int64_t* head = (int64_t*)malloc(sizeof(int64_t) * ng);
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * N);
  for (int64_t qq = 0; qq < ng; ++qq) head[qq] = -1;
  for (int64_t i = 0; i < N; ++i) {
    int gx = (int)(wrapb(x[i], L) / gs), gy = (int)(wrapb(y[i], L) / gs),
        gz = (int)(wrapb(z[i], L) / gs);
    if (gx >= g) gx = g - 1;
    if (gy >= g) gy = g - 1;
    if (gz >= g) gz = g - 1;
    const int64_t qq = ((int64_t)gz * g + gy) * g + gx;
    next[i] = head[qq];
    head[qq] = i;
  }
  for (int64_t i = 0; i < N; ++i) {
    int gx = (int)(wrapb(x[i], L) / gs), gy = (int)(wrapb(y[i], L) / gs),
        gz = (int)(wrapb(z[i], L) / gs);
    if (gx >= g) gx = g - 1;
    if (gy >= g) gy = g - 1;
    if (gz >= g) gz = g - 1;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int qx = ((gx + dx) % g + g) % g, qy = ((gy + dy) % g + g) % g,
                    qz = ((gz + dz) % g + g) % g;
          for (int64_t j = head[((int64_t)qz * g + qy) * g + qx]; j >= 0; j = next[j]) {
            if (j <= i) continue;
            const double ex = wrapc(x[j] - x[i], L), ey = wrapc(y[j] - y[i], L),
                         ez = wrapc(z[j] - z[i], L);
            const double d2 = ex * ex + ey * ey + ez * ez;
            if (d2 < best) best = d2;
          }
        }
  }
  free(head);
  free(next);
  return best;
}
