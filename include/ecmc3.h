/*
 * ecmc3.h -- C ABI of the parallel event-chain sweep for hard spheres in
 * three dimensions: the generalisation of the two-dimensional sweep of
 * Kampmann, Boltz, Kierfeld, arXiv:1409.6948, Sec. 3.4, which the paper
 * mentions as straightforward and leaves without details.
 *
 * One sweep (Sec. 3.4 steps 1-7 in three dimensions):
 *   1. cubic cells of side w = L / cells on a lattice shifted by a random
 *      vector (uniform on [0,w)^3, Philox words 0-2 of (t, 0, 0, 0));
 *   2. 2x2x2 blocks, colour = (cx mod 2) + 2 (cy mod 2) + 4 (cz mod 2);
 *   3. one random order of the eight colours per sweep (permutation number
 *      floor(u3 * 8! / 2^64) in lexicographic order);
 *   4-6. every cell of the current colour runs n_m chains, each started at a
 *      member drawn with replacement; the other cells are frozen; chains run
 *      along axis t mod 3 with a sign drawn per chain and turn back along
 *      the axis at a cell wall or a frozen sphere (the reading that keeps
 *      every chain its own reverse, as for the two-dimensional axis chains);
 *   7. repeat with a new decomposition.
 * Contacts, ties (smaller id*27 + image code first; chain end before contact
 * before wall) and the member-weighted collision pressure follow the
 * two-dimensional library (ecmc.h); beta P / rho = 1 + sum_b_w / sum_disp_w
 * holds in three dimensions unchanged.
 *
 * Conventions: every call returns ECMC_OK (0) or a negative ECMC_ERR_* code
 * from ecmc.h, with a message in ecmc_last_error_message().  Positions are
 * interleaved [x0, y0, z0, x1, ...] in sphere-id order, wrapped to [0, L).
 * Host pointers are copied before the call returns; device pointers (flag
 * on_device = 1) must stay valid until the handle's stream has passed the
 * call.  Sweeps are asynchronous on the handle's stream; getters synchronise
 * it.  A handle is not thread-safe.
 */
#ifndef ECMC3_H
#define ECMC3_H

#include <stdint.h>

#include "ecmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ecmc3_ctx* ecmc3_t;

/* Parameters for ecmc3_set_param / ecmc3_get_param. */
#define ECMC3_PARAM_N_CHAINS 1   /* chains per cell and sweep, n_m >= 1 (default 1) */
#define ECMC3_PARAM_REPLICA 4    /* Philox key word 1, integer in [0, 9e15] (default 0) */
/* 1 (default): one persistent launch per sweep, in which each cell waits
 * (bounded, ECMC_ERR_TIMEOUT after 5 s) for the neighbours of earlier colours
 * of the sweep; 0: one launch per colour phase.  Same results bit for bit;
 * reading it back gives the schedule in use. */
#define ECMC3_PARAM_PERSISTENT 15
/* Limit of one dependency wait of the persistent sweep in ms (default 5000). */
#define ECMC3_PARAM_WAIT_LIMIT_MS 16
/* Failure test: 1 makes the persistent sweep's dependency waits look for a
 * value nobody writes, so that they run out after the wait limit and the
 * sweep reports ECMC_ERR_TIMEOUT (no device fault; the handle recovers when
 * positions are set again). */
#define ECMC3_PARAM_WAIT_TEST 17
/* 1 (default): a chain found to rattle periodically (after a turn-back, the
 * state the next leg starts from equals the one 2, 4, ... or 16 legs
 * earlier, with every sphere moved in between back in place, bit for bit)
 * repeats the recorded legs without searching for contacts until the budget
 * runs out; 0: every leg searched.  Same results bit for bit; the replayed
 * legs are counted in ecmc_counters_t.replayed_legs. */
#define ECMC3_PARAM_REPLAY 14

/* N spheres of diameter sigma in a periodic cube of side L, cells^3 cubic
 * cells (cells even, >= 2, L / cells > sigma), chains of total displacement
 * ell, Philox key (seed, 0).  Start: the simple cubic lattice, sphere
 * (iz k + iy) k + ix at ((ix + 1/2) a, (iy + 1/2) a, (iz + 1/2) a),
 * a = L / k, N = k^3 (ECMC_ERR_ARG unless a > sigma).  ECMC_ERR_UNSUPPORTED
 * if one cell's frame does not fit in shared memory. */
ECMC_API int ecmc3_create(ecmc3_t* out, int64_t N, double L, double sigma, int cells,
                          double ell, uint64_t seed);
/* Release the handle (NULL: nothing to do, ECMC_OK). */
ECMC_API int ecmc3_destroy(ecmc3_t h);

ECMC_API int ecmc3_set_param(ecmc3_t h, int key, double value);
ECMC_API int ecmc3_get_param(ecmc3_t h, int key, double* value);

/* Stream for every later call (a cudaStream_t; NULL = the handle's own). */
ECMC_API int ecmc3_set_stream(ecmc3_t h, void* stream);

/* Load 3N coordinates (host or device) and set the sweep counter to t0; the
 * statistics are reset.  ECMC_ERR_OVERLAP if two spheres are closer than
 * sigma (1 - 1e-9); the state is then invalid until positions are set. */
ECMC_API int ecmc3_set_positions(ecmc3_t h, const double* xyz, int on_device, int64_t t0);

/* Copy the 3N coordinates out (host or device memory of the caller). */
ECMC_API int ecmc3_positions(ecmc3_t h, double* xyz, int on_device);

/* Enqueue n sweeps (asynchronous). */
ECMC_API int ecmc3_sweep(ecmc3_t h, int64_t n_sweeps);

/* Wait for the handle's stream; reports device-side errors
 * (ECMC_ERR_CAPACITY: a cell or frame exceeded its bound; ECMC_ERR_CHAIN_CAP). */
ECMC_API int ecmc3_synchronize(ecmc3_t h);

/* Sweep counter t of the next sweep. */
ECMC_API int ecmc3_sweep_index(ecmc3_t h, int64_t* t);

/* Counters since the last reset (rejected_chains is 0). */
ECMC_API int ecmc3_counters(ecmc3_t h, ecmc_counters_t* out);

/* beta P sigma^3 = rho sigma^3 (1 + sum_b_w / sum_disp_w) over the sweeps
 * since the last reset, and its batch-means standard error (20 batches). */
ECMC_API int ecmc3_pressure(ecmc3_t h, double* betaP_sigma3, double* stderr_out);
ECMC_API int ecmc3_reset_stats(ecmc3_t h);

/* Smallest pair distance if below rcut = min(2 sigma, w), else rcut. */
ECMC_API int ecmc3_min_distance(ecmc3_t h, double* dmin);

/* Cell of every sphere in the last binning ((cz * cells + cy) * cells + cx). */
ECMC_API int ecmc3_last_cells(ecmc3_t h, int32_t* cell_of_id);

/* Chain records of the last sweep, 4 int32 per (cell, chain): start id, end
 * id (the sphere moving when the budget ran out), contacts, wall turns;
 * cells without members hold start id -1.  out holds cells^3 * n_m * 4. */
ECMC_API int ecmc3_chain_records(ecmc3_t h, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif
