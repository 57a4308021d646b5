/*
 * ecmc_stripes.h -- C ABI of the striped decomposition that Kampmann, Boltz,
 * Kierfeld (arXiv:1409.6948) test beside their checkerboard in Sec. 3.4
 * (Fig. 3, "stripes", the parallelisation proposed by Kapfer and Krauth):
 * chains of event-chain moves run inside stripes that span the periodic box
 * along the chain axis, and a chain that touches a disk of a neighbouring
 * stripe is rejected as a whole.
 *
 * One sweep t (the paper names the variant without further detail; this is
 * the reading):
 *   - axis a = x on even t, y on odd t; each chain moves along +a or -a, the
 *     sign drawn per chain (Philox word 1 of (t, 1, stripe, k), top bit set:
 *     -a);
 *   - S stripes parallel to a (S even, w = L / S > sigma), each spanning the
 *     box along a, on a lattice shifted across a by unit53(u0) * w, u the
 *     Philox words of (t, 0, 0, 0); a disk belongs to the stripe holding its
 *     centre, index floor((v - shift mod L) * (1 / w)) clamped to [0, S-1],
 *     v the disk's coordinate across a;
 *   - colour = stripe index mod 2; colour floor(u2 * 2 / 2^64) runs first,
 *     then the other;
 *   - every stripe of the running colour starts n_m chains, one after the
 *     other, at members drawn with replacement: member number
 *     floor(v0 * n_c / 2^64) in ascending id, v the Philox words of
 *     (t, 1, stripe, k); all other stripes are frozen;
 *   - a stripe is periodic along a: a disk ahead is found round the end of
 *     the box, and there are no walls;
 *   - a contact with a frozen disk rejects the chain (ECMC_BOUNDARY_REJECT,
 *     the default and the paper's stripes: every disk the chain moved goes
 *     back to its position at the chain's start) or turns it back along the
 *     axis (ECMC_BOUNDARY_REFLECT);
 *   - ties as in ecmc.h: the smaller (id, image) key first, the chain's end
 *     before a contact at equal distance.
 * Contacts are evaluated with the same FP64 expressions, without
 * contraction, as the plain sequential definition of the variant, so a run
 * is reproducible bit for bit from (seed, replica, t).
 *
 * Conventions as ecmc.h: every call returns ECMC_OK (0) or a negative
 * ECMC_ERR_* code with a message in ecmc_last_error_message(); positions are
 * interleaved [x0, y0, x1, y1, ...] in disk-id order, wrapped to [0, L);
 * host buffers are copied before the call returns, device buffers
 * (on_device = 1) must stay valid until the handle's stream has passed the
 * call; sweeps are asynchronous on the handle's stream and getters
 * synchronise it; a handle is not thread-safe.
 */
#ifndef ECMC_STRIPES_H
#define ECMC_STRIPES_H

#include <stdint.h>

#include "ecmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ecmc_stripes_ctx* ecmc_stripes_t;

/* Parameters for ecmc_stripes_set_param / ecmc_stripes_get_param. */
#define ECMC_STRIPES_PARAM_N_CHAINS 1 /* chains per stripe and sweep, n_m >= 1 (default 1) */
#define ECMC_STRIPES_PARAM_REPLICA 4  /* Philox key word 1, integer in [0, 9e15] (default 0) */
/* ECMC_BOUNDARY_REJECT (default) or ECMC_BOUNDARY_REFLECT. */
#define ECMC_STRIPES_PARAM_BOUNDARY 21
/* Start lists (Sec. 3.4 step 5, Fig. 3): ECMC_LIST_WITH_REPL (default), each
 * start disk drawn among the stripe's members; ECMC_LIST_WITHOUT_REPL, the
 * negative control: the first start as drawn, then a Fisher-Yates shuffle of
 * the other members with Philox draws, cycled.  The shuffled list needs the
 * sorted-frame kernel (ECMC_ERR_UNSUPPORTED from ecmc_stripes_sweep when a
 * stripe's frame does not fit in shared memory). */
#define ECMC_STRIPES_PARAM_LIST_MODE 19
/* Chain kernel: 1 (default) = the sorted-frame kernel when a stripe's frame
 * fits in shared memory (one warp per stripe; strips of width sigma/2 across
 * the axis, each sorted along it once per phase -- two disks of one strip
 * cannot pass each other -- and per contact only a short window ahead of the
 * mover in the five strips within sigma tested); 0 = the block-wide scan of
 * the whole frame in global memory.  Reading it returns the kernel the next
 * sweep uses.  Both give the same trajectories bit for bit. */
#define ECMC_STRIPES_PARAM_KERNEL 24

/* N disks of diameter sigma in a periodic square of side L, `stripes`
 * stripes (even, >= 2, L / stripes > sigma), chains of total displacement
 * ell, Philox key (seed, 0).  Start: the square lattice of ecmc_create (N a
 * perfect square, L / sqrt(N) > sigma).  Errors: ECMC_ERR_ARG, ECMC_ERR_OOM,
 * ECMC_ERR_CUDA. */
ECMC_API int ecmc_stripes_create(ecmc_stripes_t* out, int64_t N, double L, double sigma,
                                 int stripes, double ell, uint64_t seed);
/* Release the handle (NULL: nothing to do, ECMC_OK). */
ECMC_API int ecmc_stripes_destroy(ecmc_stripes_t h);

ECMC_API int ecmc_stripes_set_param(ecmc_stripes_t h, int key, double value);
ECMC_API int ecmc_stripes_get_param(ecmc_stripes_t h, int key, double* value);

/* Stream for every later call (a cudaStream_t; NULL = the handle's own). */
ECMC_API int ecmc_stripes_set_stream(ecmc_stripes_t h, void* stream);

/* Load 2N coordinates (host or device), each reduced into [0, L), and set
 * the sweep counter to t0; the statistics are reset.  The configuration is
 * not checked for overlaps (ecmc_set_positions of a two-dimensional handle
 * does that). */
ECMC_API int ecmc_stripes_set_positions(ecmc_stripes_t h, const double* xy, int on_device,
                                        int64_t t0);
/* Copy the 2N coordinates out (host or device memory of the caller). */
ECMC_API int ecmc_stripes_positions(ecmc_stripes_t h, double* xy, int on_device);

/* Enqueue n sweeps (asynchronous). */
ECMC_API int ecmc_stripes_sweep(ecmc_stripes_t h, int64_t n_sweeps);

/* Wait for the handle's stream; reports device-side errors
 * (ECMC_ERR_CAPACITY: a stripe's frame exceeded its packing bound;
 * ECMC_ERR_CHAIN_CAP: a chain reached 2^22 contacts). */
ECMC_API int ecmc_stripes_synchronize(ecmc_stripes_t h);

/* Sweep counter t of the next sweep. */
ECMC_API int ecmc_stripes_sweep_index(ecmc_stripes_t h, int64_t* t);

/* Counters since the last reset (wall_hits and replayed_legs are 0). */
ECMC_API int ecmc_stripes_counters(ecmc_stripes_t h, ecmc_counters_t* out);

/* beta P sigma^2 = rho sigma^2 (1 + sum_b_w / sum_disp_w), the
 * member-weighted collision estimator of ecmc_pressure over the sweeps since
 * the last reset, with its batch-means standard error (20 batches).  It
 * holds under ECMC_BOUNDARY_REFLECT; under the rejecting rule the pressure
 * is read from the contact value of g(r) instead. */
ECMC_API int ecmc_stripes_pressure(ecmc_stripes_t h, double* betaP_sigma2, double* stderr_out);
ECMC_API int ecmc_stripes_reset_stats(ecmc_stripes_t h);

/* Stripe of every disk in the last sweep. */
ECMC_API int ecmc_stripes_last_stripes(ecmc_stripes_t h, int32_t* stripe_of_id);

/* Chain records of the last sweep, 4 int32 per (stripe, chain): start id,
 * end id (the disk moving when the chain ended or was rejected), contacts,
 * 0; stripes without members hold start id -1.  out holds
 * stripes * n_m * 4. */
ECMC_API int ecmc_stripes_chain_records(ecmc_stripes_t h, int32_t* out);

#ifdef __cplusplus
}
#endif
#endif
