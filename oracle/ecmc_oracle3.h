/*
 * ecmc_oracle3.h -- oracle of the parallel event-chain sweep for hard
 * spheres in three dimensions, the generalisation that Sec. 3.4 of
 * Kampmann, Boltz, Kierfeld (arXiv:1409.6948) mentions without details:
 * cubic cells on a randomly shifted lattice, 2x2x2 blocks with eight
 * colours, n_m chains per cell started at members drawn with replacement,
 * the other cells frozen.
 *
 * TEST INFRASTRUCTURE ONLY, like ecmc_oracle.h: the CUDA library never
 * includes, links or calls anything declared here.
 */
#ifndef ECMC_ORACLE3_H
#define ECMC_ORACLE3_H

#include <stdint.h>

#include "ecmc_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int64_t N;       /* number of spheres                                */
  double L;        /* side of the periodic cubic box                   */
  double sigma;    /* sphere diameter                                  */
  int cells;       /* cells per side, the same on all three axes (even, >= 2) */
  double ell;      /* total displacement of one chain                  */
  int n_m;         /* chains started per cell and sweep                */
  uint64_t seed;   /* Philox key word 0                                */
  uint64_t replica;/* Philox key word 1                                */
  unsigned flags;  /* ORC_FLAG_NO_SHIFT, ORC_FLAG_BRUTE_FROZEN,
                      ORC_FLAG_REVERSE_CELLS, ORC_FLAG_FIXED_COLOURS    */
} orc3_params;

/* Per-sweep draws: the shift of the cell lattice (uniform on [0,w)^3) and the
 * order of the eight colours (permutation number below(u3, 8!) of 0..7 in
 * lexicographic order). */
void orc3_sweep_draws(const orc3_params* p, int64_t t, double shift[3], int perm[8]);

/* Cell of every sphere for sweep t: cell = (cz * cells + cy) * cells + cx. */
int orc3_bin(const orc3_params* p, int64_t t, const double* x, const double* y, const double* z,
             int32_t* cell);

/* Sweeps t0 .. t0+n_sweeps-1 in place (sphere-id order, wrapped to [0,L)).
 * Statistics as orc_sweeps (member-weighted pressure sums); recs, if not
 * NULL, receives one record per (sweep, cell, chain), indexed
 * [(s*cells^3 + cell)*n_m + k].  Returns 0 or -1 on invalid parameters. */
int orc3_sweeps(const orc3_params* p, double* x, double* y, double* z, int64_t t0,
                int64_t n_sweeps, orc_stats* st, orc_chain_rec* recs);

/* One chain on a caller-built frame: objects 0..n_mem-1 are members of the
 * active cell [0,w]^3, the rest frozen (img: image code 0..26 for the
 * tie-break key id*27 + img).  Object m starts along axis (0, 1, 2) with
 * sign +-1 and budget ell.  X, Y, Z are updated in place. */
int orc3_run_chain_frame(int n, int n_mem, double* X, double* Y, double* Z, const int64_t* id,
                         const int32_t* img, double w, double sigma, int m, int axis, int sign,
                         double ell, orc_stats* st, orc_chain_rec* rec);

/* Smallest squared minimum-image distance over all pairs closer than rcut
 * (rcut*rcut if none), by a uniform grid. */
double orc3_min_dist2(int64_t N, double L, const double* x, const double* y, const double* z,
                      double rcut);

#ifdef __cplusplus
}
#endif
#endif
