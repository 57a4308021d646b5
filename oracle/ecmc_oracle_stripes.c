/*
 * ecmc_oracle_stripes.c -- oracle of the striped decomposition of Sec. 3.4
 * (Fig. 3, "stripes"); the readings are listed in ecmc_oracle_stripes.h.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain sequential FP64 C, compiled like the rest
 * of the oracle with -ffp-contract=off, brute force over every object of a
 * stripe's frame at every step.
 */
#include "ecmc_oracle_stripes.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Philox words of the sweep's counter (t, purpose, a, b) under the key
 * (seed, replica), as for the cells */
static void draw4_s(const orc_params* p, uint64_t t, uint64_t purpose, uint64_t a, uint64_t b,
                    uint64_t out[4]) {
  uint64_t ctr[4] = {t, purpose, a, b};
  uint64_t key[2] = {p->seed, p->replica};
  orc_philox4x64_10(ctr, key, out);
}

/* uniform integer in [0,n): high word of the 128-bit product v*n */
static uint64_t below_s(uint64_t v, uint64_t n) {
  return (uint64_t)(((unsigned __int128)v * (unsigned __int128)n) >> 64);
}

static double unit53_s(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

static int check_stripes(const orc_params* p) {
  if (p->N <= 0 || !(p->L > 0.0) || !(p->sigma > 0.0)) return -1;
  if (p->cells_x < 2 || (p->cells_x & 1)) return -1;
  if (!(p->L / p->cells_x > p->sigma)) return -1;
  if (!(p->ell >= 0.0) || p->n_m < 1) return -1;
  if (p->dir_mode != ORC_DIR_PM_AXIS_ALT && p->dir_mode != ORC_DIR_POS_ONLY) return -1;
  if (p->boundary != ORC_BOUNDARY_REFLECT && p->boundary != ORC_BOUNDARY_REJECT) return -1;
  return 0;
}

void orc_stripe_draws(const orc_params* p, int64_t t, double* shift, int* first_colour) {
  uint64_t u[4];
  draw4_s(p, (uint64_t)t, ORC_PURPOSE_SWEEP, 0, 0, u);
  const double w = p->L / (double)p->cells_x;
  *shift = (p->flags & ORC_FLAG_NO_SHIFT) ? 0.0 : unit53_s(u[0]) * w;
  *first_colour = (p->flags & ORC_FLAG_FIXED_COLOURS) ? 0 : (int)below_s(u[2], 2);
}

/* stripe index of a coordinate across the axis, as the cells' index */
static int stripe_of(double v, double shift, double L, double w, int stripes) {
  double u = v - shift;
  if (u < 0.0) u += L;
  int k = (int)(u * (1.0 / w));
  if (k >= stripes) k = stripes - 1;
  if (k < 0) k = 0;
  return k;
}

int orc_stripe_bin(const orc_params* p, int64_t t, const double* x, const double* y,
                   int32_t* stripe) {
  if (check_stripes(p)) return -1;
  double shift;
  int first;
  orc_stripe_draws(p, t, &shift, &first);
  const double w = p->L / (double)p->cells_x;
  const double* across = (t & 1) ? x : y; /* axis x on even sweeps: stripes cut y */
  for (int64_t i = 0; i < p->N; ++i) stripe[i] = stripe_of(across[i], shift, p->L, w, p->cells_x);
  return 0;
}

/* position reduced into [0, L) after a move along the periodic axis */
static double wrap_along(double v, double L) {
  v = fmod(v, L);
  if (v < 0.0) v += L;
  if (v >= L) v -= L;
  return v;
}

/*
 * One chain (Sec. 3.2) in a stripe: each step takes the nearest of the
 * budget's end and the first contact along the axis.  The forward distance
 * to object j is its along-axis separation in the direction of motion,
 * taken in (0, L] around the periodic stripe; j is hit if its across offset
 * c satisfies c^2 < sigma^2, after a travel b - sqrt(sigma^2 - c^2).  A
 * member hit is lifted; a frozen disk hit rejects the chain (every member
 * back at its start, the contact sum dropped) or turns it back.
 */
int orc_run_chain_stripe(int n, int n_mem, double* U, const double* V, const int64_t* key,
                         double L, double sigma, int m, int sign, double ell, int reject,
                         orc_stats* st, orc_chain_rec* rec) {
  if (n < 1 || n_mem < 1 || n_mem > n || m < 0 || m >= n_mem || !(L > 0.0) ||
      !(sigma > 0.0) || !(ell >= 0.0))
    return -1;
  const double sig2 = sigma * sigma;
  double* U0 = NULL;
  if (reject) {
    U0 = (double*)malloc(sizeof(double) * (size_t)(n_mem > 0 ? n_mem : 1));
    memcpy(U0, U, sizeof(double) * (size_t)n_mem);
  }
  double d = sign > 0 ? 1.0 : -1.0;
  double r = ell, chain_b = 0.0;
  int64_t nev = 0;
  int rejected = 0;
  for (int64_t iter = 0;; ++iter) {
    if (iter >= ORC_MAX_EVENTS_PER_CHAIN) {
      if (st) st->capped++;
      break;
    }
    const double Um = U[m], Vm = V[m];
    double best_s = INFINITY, best_b = 0.0;
    int best = -1;
    for (int j = 0; j < n; ++j) {
      if (j == m) continue;
      double c = V[j] - Vm;
      double c2 = c * c;
      if (!(c2 < sig2)) continue; /* passes beside */
      double b = d * (U[j] - Um);
      if (b <= 0.0) b += L;       /* ahead around the periodic stripe */
      double s = b - sqrt(sig2 - c2);
      if (s < 0.0) s = 0.0;
      if (s < best_s || (s == best_s && key[j] < key[best])) {
        best_s = s;
        best_b = b;
        best = j;
      }
    }
    if (r <= best_s) { /* budget used up: the chain ends */
      U[m] = wrap_along(Um + d * r, L);
      if (st) st->sum_b += chain_b;
      break;
    }
    nev++;
    if (st) st->events++;
    if (best >= n_mem && reject) { /* frozen disk: the chain is rejected */
      memcpy(U, U0, sizeof(double) * (size_t)n_mem);
      if (st) {
        st->frozen_hits++;
        st->rejected++;
      }
      rejected = 1;
      break;
    }
    U[m] = wrap_along(Um + d * best_s, L);
    r = r - best_s;
    chain_b += best_b - best_s;
    if (best < n_mem) { /* lift */
      if (st) st->lifts++;
      m = best;
    } else { /* frozen disk under the reflecting rule: back along the axis */
      if (st) st->frozen_hits++;
      d = -d;
    }
  }
  if (rec) {
    rec->end_id = m;
    rec->events = nev;
    rec->walls = 0;
  }
  free(U0);
  return rejected;
}

int orc_stripe_sweeps(const orc_params* p, double* x, double* y, int64_t t0, int64_t n_sweeps,
                      orc_stats* st, orc_chain_rec* recs) {
  if (check_stripes(p)) return -1;
  const int64_t N = p->N;
  const int S = p->cells_x;
  const double L = p->L, sigma = p->sigma, w = L / (double)S;
  int32_t* stripe = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S + 1));
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (size_t)p->n_m);
  /* frame of one stripe: members first (ascending id), then frozen images */
  double* U = (double*)malloc(sizeof(double) * (size_t)(3 * N));
  double* V = (double*)malloc(sizeof(double) * (size_t)(3 * N));
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * N));
  int64_t* fid = (int64_t*)malloc(sizeof(int64_t) * (size_t)(3 * N));
  int64_t* perm_buf = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);

  for (int64_t s = 0; s < n_sweeps; ++s) {
    const int64_t t = t0 + s;
    double shift;
    int first;
    orc_stripe_draws(p, t, &shift, &first);
    double* along = (t & 1) ? y : x;
    double* across = (t & 1) ? x : y;
    orc_stripe_bin(p, t, x, y, stripe);
    memset(start, 0, sizeof(int64_t) * (size_t)(S + 1));
    for (int64_t i = 0; i < N; ++i) start[stripe[i] + 1]++;
    for (int k = 0; k < S; ++k) start[k + 1] += start[k];
    memcpy(fill, start, sizeof(int64_t) * (size_t)(S + 1));
    for (int64_t i = 0; i < N; ++i) order[fill[stripe[i]]++] = i;

    for (int ci = 0; ci < 2; ++ci) {
      const int colour = ci == 0 ? first : 1 - first;
      for (int kk = 0; kk < S / 2; ++kk) {
        /* the stripes of one colour are independent: visited in increasing
         * index, or in reverse under ORC_FLAG_REVERSE_CELLS */
        const int k = colour + 2 * ((p->flags & ORC_FLAG_REVERSE_CELLS) ? (S / 2 - 1 - kk) : kk);
        const double origin = shift + (double)k * w; /* lower edge across */
        const int64_t nc = start[k + 1] - start[k];
        int n = 0;
        for (int64_t q = start[k]; q < start[k + 1]; ++q) {
          const int64_t i = order[q];
          double v = across[i] - origin;
          if (v >= 0.5 * L) v -= L;
          if (v < -0.5 * L) v += L;
          U[n] = along[i];
          V[n] = v;
          key[n] = i * 3 + 1;
          fid[n] = i;
          n++;
        }
        const int n_mem = n;
        /* every image across (shifts -L, 0, +L) of every other disk whose
         * centre lies within sigma of the stripe's band [0, w] */
        for (int64_t j = 0; j < N; ++j) {
          if (stripe[j] == k) continue;
          double v0 = across[j] - origin;
          if (v0 >= 0.5 * L) v0 -= L;
          if (v0 < -0.5 * L) v0 += L;
          for (int im = -1; im <= 1; ++im) {
            const double v = im == 0 ? v0 : (im > 0 ? v0 + L : v0 - L);
            if (!(v > -sigma && v < w + sigma)) continue;
            U[n] = along[j];
            V[n] = v;
            key[n] = j * 3 + (im + 1);
            fid[n] = j;
            n++;
          }
        }

        /* start list: with replacement, or the shuffled list of distinct
         * members (negative control), drawn as for a cell */
        if (nc > 0) {
          if (p->list_mode == ORC_LIST_WITHOUT_REPL) {
            uint64_t v[4];
            draw4_s(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)k, 0, v);
            const int64_t fst = (int64_t)below_s(v[0], (uint64_t)nc);
            int64_t nrest = 0;
            perm_buf[nrest++] = fst;
            for (int64_t q = 0; q < nc; ++q)
              if (q != fst) perm_buf[nrest++] = q;
            for (int64_t i = nc - 1; i >= 2; --i) { /* Fisher-Yates on entries 1.. */
              uint64_t u[4];
              draw4_s(p, (uint64_t)t, ORC_PURPOSE_SHUFFLE, (uint64_t)k, (uint64_t)(i >> 2), u);
              const int64_t j = 1 + (int64_t)below_s(u[i & 3], (uint64_t)i);
              const int64_t tmp = perm_buf[i];
              perm_buf[i] = perm_buf[j];
              perm_buf[j] = tmp;
            }
            for (int c = 0; c < p->n_m; ++c) list[c] = perm_buf[c % nc];
          } else {
            for (int c = 0; c < p->n_m; ++c) {
              uint64_t v[4];
              draw4_s(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)k, (uint64_t)c, v);
              list[c] = (int64_t)below_s(v[0], (uint64_t)nc);
            }
          }
        }

        const double sum_b_before = st ? st->sum_b : 0.0;
        int accepted = 0;
        for (int c = 0; c < p->n_m; ++c) {
          orc_chain_rec* rec = recs ? &recs[(s * S + k) * p->n_m + c] : NULL;
          if (rec) {
            rec->start_id = -1;
            rec->end_id = -1;
            rec->events = 0;
            rec->walls = 0;
          }
          if (nc == 0) continue;
          uint64_t v[4];
          draw4_s(p, (uint64_t)t, ORC_PURPOSE_CHAIN, (uint64_t)k, (uint64_t)c, v);
          const int sign = (p->dir_mode == ORC_DIR_POS_ONLY) ? 1 : ((v[1] >> 63) ? -1 : 1);
          const int m = (int)list[c];
          if (rec) rec->start_id = fid[m];
          const int rej = orc_run_chain_stripe(n, n_mem, U, V, key, L, sigma, m, sign, p->ell,
                                               p->boundary == ORC_BOUNDARY_REJECT, st, rec);
          if (rec) rec->end_id = fid[rec->end_id];
          if (st) {
            st->chains++;
            if (!rej) st->sum_disp += p->ell;
          }
          accepted += rej ? 0 : 1;
        }
        if (st && nc > 0) {
          st->sum_b_w += (double)nc * (st->sum_b - sum_b_before);
          st->sum_disp_w += (double)nc * ((double)accepted * p->ell);
        }
        /* write back the along-axis coordinate of every member */
        for (int q = 0; q < n_mem; ++q) along[fid[q]] = U[q];
      }
    }
    if (st) st->sweeps++;
  }
  free(stripe);
  free(start);
  free(fill);
  free(order);
  free(list);
  free(U);
  free(V);
  free(key);
  free(fid);
  free(perm_buf);
  return 0;
}
