/*
 * ecmc_oracle.h -- interface of the reference (oracle) implementation of the
 * parallel event-chain Monte Carlo sweep for two-dimensional hard disks
 * (Kampmann, Boltz, Kierfeld, "Parallelized event chain algorithm for dense
 * hard sphere and polymer systems", arXiv:1409.6948).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and ecmc_oracle.c are used by the
 * test suite, by the smoke check and by the benchmark's CPU-baseline leg.
 * The CUDA library never includes, links or calls anything declared here;
 * the two implementations share no code.
 */
#ifndef ECMC_ORACLE_H
#define ECMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Direction rule of the chains (reading of Sec. 3.2 and of the sweep of
 * Sec. 3.4; the irreversible "+x/+y only" variant breaks detailed balance
 * once cells have walls, Sec. 3.2).  Chains along an axis turn back at a
 * frozen disk; isotropic chains are reflected specularly (Fig. 1). */
#define ORC_DIR_PM_AXIS_ALT 0 /* axis x on even sweeps, y on odd; sign +/- per chain */
#define ORC_DIR_POS_ONLY 1    /* axis alternates, sign always + (negative control)   */
#define ORC_DIR_ISOTROPIC 2   /* direction uniform on the circle, drawn per chain    */

/* Start-list rule (Sec. 3.4 step 5 and the discussion of Fig. 2). */
#define ORC_LIST_WITH_REPL 0    /* n_m draws with replacement (the paper's rule)   */
#define ORC_LIST_WITHOUT_REPL 1 /* shuffled distinct members (negative control)    */

/* Boundary rule (Sec. 3.4, discussion of Fig. 3). */
#define ORC_BOUNDARY_REFLECT 0 /* reflect at walls and frozen disks (the paper's rule) */
#define ORC_BOUNDARY_REJECT 1  /* reject the whole chain when it reaches a wall or a
                                  frozen disk: every disk it moved returns to its
                                  position at the chain's start                      */

/* flags */
#define ORC_FLAG_NO_SHIFT 1u       /* grid shift forced to (0,0) (closed-form tests) */
#define ORC_FLAG_BRUTE_FROZEN 2u   /* frozen set from ALL disks, not neighbour cells */
#define ORC_FLAG_REVERSE_CELLS 4u  /* cells of one colour visited in reverse order   */
#define ORC_FLAG_FIXED_COLOURS 8u  /* colour order 0,1,2,3 instead of the drawn one  */
#define ORC_FLAG_SPECULAR_AXIS 16u /* axis chains reflect specularly at frozen disks
                                      (breaks detailed balance: negative control)   */

/* Philox counter "purpose" words. */
#define ORC_PURPOSE_SWEEP 0u
#define ORC_PURPOSE_CHAIN 1u
#define ORC_PURPOSE_SHUFFLE 2u
#define ORC_PURPOSE_DIRECTION 3u

/* Hard cap on events of one chain; a chain that reaches it stops and is
 * counted in orc_stats.capped. */
#define ORC_MAX_EVENTS_PER_CHAIN (1 << 22)

typedef struct {
  int64_t N;       /* number of disks                                  */
  double L;        /* side of the periodic square box                  */
  double sigma;    /* disk diameter                                    */
  int cells_x;     /* cells per side along x (even, >= 2)              */
  int cells_y;     /* cells per side along y (even, >= 2)              */
  double ell;      /* total displacement of one chain                  */
  int n_m;         /* chains started per cell and sweep                */
  uint64_t seed;   /* Philox key word 0                                */
  uint64_t replica;/* Philox key word 1                                */
  int dir_mode;    /* ORC_DIR_*                                        */
  int list_mode;   /* ORC_LIST_*                                       */
  unsigned flags;  /* ORC_FLAG_*                                       */
  int boundary;    /* ORC_BOUNDARY_*                                   */
} orc_params;

typedef struct {
  int64_t sweeps;      /* sweeps performed                                   */
  int64_t chains;      /* chains run (cells with no member start none)       */
  int64_t events;      /* contacts: lifts + reflections at frozen disks      */
  int64_t lifts;       /* contacts with an active disk (displacement passed) */
  int64_t frozen_hits; /* contacts with a frozen disk (chain reflected)      */
  int64_t wall_hits;   /* reflections at a cell wall                         */
  int64_t capped;      /* chains stopped by ORC_MAX_EVENTS_PER_CHAIN         */
  double sum_b;        /* sum over contacts of the separation projected on d */
  double sum_disp;     /* sum over chains of the displacement budget ell     */
  double sum_b_w;      /* sum over cells of n_c * (contact sum of the cell)  */
  double sum_disp_w;   /* sum over cells of n_c * (accepted chains) * ell    */
  int64_t rejected;    /* chains rejected under ORC_BOUNDARY_REJECT; their
                          contacts are counted in events, lifts, frozen_hits
                          and wall_hits but not in sum_b, and their budget is
                          not in sum_disp                                      */
} orc_stats;

/* Optional per-chain record (debugging and parity tests). */
typedef struct {
  int64_t start_id;  /* disk that started the chain                */
  int64_t end_id;    /* disk that was moving when the budget ran out */
  int64_t events;    /* contacts in this chain                      */
  int64_t walls;     /* wall reflections in this chain              */
} orc_chain_rec;

/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* Per-sweep random numbers: grid shift and colour order (Sec. 3.4 steps 1-3). */
void orc_sweep_draws(const orc_params* p, int64_t t, double* shift_x, double* shift_y, int perm[4]);

/* Cell of every disk for sweep t (Sec. 3.4 step 1): cell = cy*cells_x + cx. */
int orc_bin(const orc_params* p, int64_t t, const double* x, const double* y, int32_t* cell);

/* Default n_m from eq. (nm) with the mean free path estimate of Sec. 4. */
int orc_default_nm(int64_t N, double L, double sigma, int cells_x, int cells_y, double ell);

/* The paper's closing strategy of Sec. 4 on square grids: the largest number
 * of 2x2 blocks n = h^2 with N / (eta n) > 100 (cell side above
 * max(sigma, min_cell_side)), ell = lambda0 (N / (eta n))^(1/2) (eq.
 * criterion), n_m from eq. (nm).  Returns 0 or -1 (no such grid). */
int orc_suggest_parameters(int64_t N, double L, double sigma, double min_cell_side,
                           int* cells_per_side, double* ell, int* n_m);

/* Run sweeps t0 .. t0+n_sweeps-1 in place on positions x[N], y[N] (disk-id
 * order, wrapped to [0,L)).  Statistics are accumulated into *st (may be
 * NULL).  If recs is not NULL it receives one record per (sweep, cell, chain)
 * slot, indexed [(s*ncells + cell)*n_m + k]; cells without members leave
 * start_id = -1.  Returns 0, or a negative code on invalid parameters. */
int orc_sweeps(const orc_params* p, double* x, double* y, int64_t t0, int64_t n_sweeps,
               orc_stats* st, orc_chain_rec* recs);

/* Textbook sequential straight event chain on the periodic box without any
 * cell decomposition (Sec. 3.2): n_chains chains per sweep, start disk
 * uniform with replacement, direction +/-x or +/-y.  Used as a special-case
 * cross-check of the cell-decomposed sweep. */
int orc_seq_sweeps(int64_t N, double L, double sigma, double ell, int64_t n_chains,
                   uint64_t seed, uint64_t replica, double* x, double* y, int64_t t0,
                   int64_t n_sweeps, orc_stats* st);

/* Ordered-pair counts of the pair-correlation histogram (Sec. 2): bin i
 * counts minimum-image distances d with sigma + i*dr <= d < sigma+(i+1)*dr.
 * Only disks i in [i_begin, i_end) are taken as first member of a pair (so a
 * sample of disks can be used); counts[] is accumulated, not cleared. */
void orc_gr_counts(int64_t N, double L, const double* x, const double* y, double sigma,
                   double dr, int nbins, int64_t i_begin, int64_t i_end, int64_t* counts);

/* The same counts over all disks, with the pairs found through a cell list
 * of cells no smaller than sigma + nbins dr (each pair tested with the
 * expressions of orc_gr_counts, so the counts are identical); positions in
 * [0, L).  counts[] is accumulated. */
void orc_gr_counts_cells(int64_t N, double L, const double* x, const double* y, double sigma,
                         double dr, int nbins, int64_t* counts);

/* Hexatic order parameter (Sec. 2, eq. Psi) with Delaunay next neighbours,
 * decided by clipping bisectors with the disks within rs (exact when every
 * Voronoi vertex lies within rs/2; the number of disks failing that check is
 * returned, -1 if L <= 2 rs).  psi_k[2N] (per disk, re/im), n_nb[N] and
 * psi[2] (the mean) may each be NULL. */
int orc_hexatic(int64_t N, double L, const double* x, const double* y, double rs,
                double* psi_k, int32_t* n_nb, double* psi);

/* Smallest minimum-image pair distance squared among all pairs closer than
 * rcut (returns rcut*rcut if there is none), by a plain uniform grid. */
double orc_min_dist2(int64_t N, double L, const double* x, const double* y, double rcut);

/* orc_sweeps one sweep at a time, copying x, y after each sweep s into
 * snap_x[s*N ..], snap_y[s*N ..]. */
int orc_sweeps_snap(const orc_params* p, double* x, double* y, int64_t t0, int64_t n_sweeps,
                    orc_stats* st, double* snap_x, double* snap_y);

/* Run one chain on a caller-built frame: objects 0..n_mem-1 are members of
 * the active cell [0,w] x [0,h], the rest frozen (img = image code used only
 * for tie-breaks).  Object m starts with direction (dx,dy) and budget ell.
 * mode bit 0: reflect specularly at frozen objects (else turn the chain
 * back); bit 1: the rejecting boundary rule (ORC_BOUNDARY_REJECT).
 * X, Y are updated in place. */
int orc_run_chain_frame(int n, int n_mem, double* X, double* Y, const int64_t* id,
                        const int32_t* img, double w, double h, double sigma, int m, double dx,
                        double dy, double ell, int mode, orc_stats* st,
                        orc_chain_rec* rec);

/* Autocorrelation time of R complex series of n samples (Sec. 2, eq. tau;
 * series r at re[r n ..], im[r n ..]): C(dt) = Re <conj(Psi_r(t))
 * Psi_r(t+dt)> / <|Psi_r|^2> over t and r, with the mean of Psi taken as
 * zero, tau = the 1/e lag, interpolated linearly; INFINITY if C stays above
 * 1/e up to max_lag.  c (may be NULL) receives C(0..max_lag).  Returns 0 or
 * -1. */
int orc_autocorrelation_time(const double* re, const double* im, int64_t n, int R,
                             int64_t max_lag, double* tau, double* c);

#ifdef __cplusplus
}
#endif
#endif
