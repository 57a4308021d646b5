/*
 * ecmc.h -- C ABI of the GB300 parallel event-chain Monte Carlo library
 * (libecmc.so) for two-dimensional hard disks.
 *
 * Method: Kampmann, Boltz, Kierfeld, "Parallelized event chain algorithm for
 * dense hard sphere and polymer systems", arXiv:1409.6948.
 *   Sec. 2 (eq. 1)   N hard disks of diameter sigma in a periodic L x L box.
 *   Sec. 3.2         straight event chain: the active disk moves along d until
 *                    it touches another disk, the rest of the displacement
 *                    budget ell passes to the disk it hit.
 *   Sec. 3.4         one sweep: cells on a randomly shifted square lattice,
 *                    2x2 blocks coloured in four colours, the colours visited
 *                    in a random order, n_m chain starts per cell drawn with
 *                    replacement, chains reflected at the cell walls and at
 *                    frozen disks (Fig. 1).
 *   Sec. 2 (eq. pressure) and the collision form of the pressure noted at the
 *                    end of Sec. 3.4: the pressure estimators.
 *
 * Conventions for every function:
 *   - returns ECMC_OK (0) or a negative ECMC_ERR_* code; ecmc_strerror()
 *     gives a message and ecmc_last_error_message() the detail of the most
 *     recent failure on the calling thread;
 *   - a handle is used by one host thread at a time;
 *   - "host" pointers are ordinary (pageable or pinned) host memory,
 *     "device" pointers are CUDA device memory of the handle's device; the
 *     library never takes ownership of caller memory;
 *   - positions are exchanged in disk-id order as interleaved pairs
 *     xy[2*i] = x_i, xy[2*i+1] = y_i (float64), wrapped into [0, L).
 *   - work is enqueued on the handle's stream (ecmc_set_stream; default: a
 *     stream the library creates); functions that return data to the host
 *     synchronise that stream.
 */
#ifndef ECMC_H
#define ECMC_H

#include <stdint.h>

#if defined(__GNUC__)
#define ECMC_API __attribute__((visibility("default")))
#else
#define ECMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define ECMC_OK 0
#define ECMC_ERR_ARG -1         /* invalid argument or parameter combination     */
#define ECMC_ERR_CUDA -2        /* a CUDA runtime call failed                    */
#define ECMC_ERR_OOM -3         /* device or host allocation failed              */
#define ECMC_ERR_OVERLAP -4     /* two disks closer than sigma (beyond rounding) */
#define ECMC_ERR_TIMEOUT -5     /* a bounded device-side wait gave up            */
#define ECMC_ERR_STATE -6       /* call not valid in the handle's current state  */
#define ECMC_ERR_CAPACITY -7    /* a cell frame exceeded its capacity            */
#define ECMC_ERR_UNSUPPORTED -8 /* option not supported for these parameters    */
#define ECMC_ERR_CHAIN_CAP -9   /* a chain hit the per-chain event cap           */

/* ---- parameters (ecmc_set_param / ecmc_get_param) ---------------------- */
/* Chains started per cell and sweep, n_m (Sec. 3.4 step 5).  Default:
 * eq. (nm) of Sec. 4, n_m = max(1, round((N / cells) lambda0 / ell)) with
 * lambda0 = sigma (eta_hcp - eta) / (2 eta_hcp). */
#define ECMC_PARAM_N_CHAINS 1
/* Direction rule: ECMC_DIR_PM_AXIS_ALT (default) = axis x on even sweeps and
 * y on odd sweeps, sign drawn per chain; ECMC_DIR_POS_ONLY = sign always +
 * (a variant that is not reversible, Sec. 3.2; kept for negative tests);
 * ECMC_DIR_ISOTROPIC = a uniform unit direction per chain (rejection-sampled
 * point of the unit disc divided by its length), specular reflection at
 * frozen disks (Fig. 1, Sec. 3.4); candidates screened in FP32 with rigorous
 * bounds (ECMC_PARAM_PRECISION 1) or all tested in FP64 (0), the same
 * trajectory either way. */
#define ECMC_PARAM_DIR_MODE 2
/* Candidate geometry: ECMC_PREC_FP64 = every candidate tested in FP64;
 * ECMC_PREC_FP32_GEOM (default) = candidates screened in FP32 cell-relative
 * coordinates with rigorous error bounds, the contact decided in FP64.  Both
 * give bit-identical trajectories. */
#define ECMC_PARAM_PRECISION 3
/* Replica number: second word of the Philox key (seed, replica); an integer
 * in [0, 9e15], so that the double passed to set_param holds it exactly. */
#define ECMC_PARAM_REPLICA 4
/* Lanes cooperating on one cell in the sweep kernel: 1, 2, 4, 8, 16, 32, or
 * 0 = automatic (default). */
#define ECMC_PARAM_LANES_PER_CELL 5
/* Pair-correlation histogram: bin width (default 0.01 sigma) and upper edge
 * (default 5 sigma); changing either clears the accumulated histogram. */
#define ECMC_PARAM_GR_DR 6
#define ECMC_PARAM_GR_RMAX 7
/* 1 = record per-kernel CUDA-event times (ecmc_kernel_times), 0 = off. */
#define ECMC_PARAM_TIMING 8
/* Width of the candidate strips across the chain axis, in units of sigma
 * (0.125 .. 2; default 0.5).  Changes only the speed, never the result. */
#define ECMC_PARAM_STRIP_WIDTH 9
/* 1 = keep per-chain records of the most recent sweep (ecmc_chain_records). */
#define ECMC_PARAM_RECORD_CHAINS 10
/* Warps per block of the chain kernel (1 .. 8, 0 = automatic). */
#define ECMC_PARAM_WARPS_PER_BLOCK 11
/* 1 = capture each sweep in a CUDA graph and replay it (default 1). */
#define ECMC_PARAM_USE_GRAPH 12
/* Where the chain kernel keeps the cell frames: 0 = shared memory, 1 = FP32
 * screening data in shared memory and FP64 coordinates in global memory,
 * 2 = global memory (cells too large for shared memory), -1 = automatic
 * (default).  The persistent sweep kernel uses 0 or 1 (automatic: 0; with 1
 * its FP64 coordinates live in a per-warp scratch area).  Changes only the
 * speed, never the result. */
#define ECMC_PARAM_FRAME_MODE 13
/* 1 = replay the legs of a chain that rattles between two reflectors
 * (frozen disks or walls) once its position after a reflection repeats bit
 * for bit, without searching for candidates again (default 1); 0 = search on
 * every leg.  Changes only the speed, never the result. */
#define ECMC_PARAM_REPLAY 14
/* 1 = run the four colour phases of a sweep in one persistent launch when a
 * warp's frames fit in shared memory (default 1): warps take cell groups from
 * a work list ordered by phase, wait until the neighbours of earlier phases
 * have finished (bounded waits), build the frames themselves and run the
 * chains; 0 = one frame-builder and one chain launch per phase.  Reading it
 * returns the mode in use.  Changes only the speed, never the result. */
#define ECMC_PARAM_PERSISTENT 15
/* Limit of one dependency wait of the persistent kernel, in ms (default
 * 5000).  A wait that exceeds it abandons the sweep: ecmc_sweep or the next
 * call reports ECMC_ERR_TIMEOUT and the positions must be set again. */
#define ECMC_PARAM_WAIT_LIMIT_MS 16
/* 1 = the persistent kernel's dependency waits look for a value that no cell
 * ever writes, so every wait runs into the limit (a test of the failure path
 * that faults nothing; default 0). */
#define ECMC_PARAM_WAIT_TEST 17
/* Read-only: kernel launches per sweep of the current configuration (5 with
 * the persistent kernel, 12 with per-phase launches). */
#define ECMC_PARAM_KERNELS_PER_SWEEP 18
/* Start lists (Sec. 3.4 step 5): ECMC_LIST_WITH_REPL (default), every start
 * disk drawn independently among the members (the paper's correct rule);
 * ECMC_LIST_WITHOUT_REPL, a negative control: the first start as drawn, then a
 * uniformly shuffled list of the other members (Fisher-Yates with Philox
 * draws), cycled when n_m exceeds the members -- the list form the paper shows
 * to bias the pressure (Fig. 3).  Needs cells of at most 128 disks
 * (ECMC_ERR_UNSUPPORTED otherwise); disables the replay of rattling chains. */
#define ECMC_PARAM_LIST_MODE 19
/* Read-only: cells whose chains run at the same time with the current launch
 * shape -- the persistent kernel's grid (all blocks resident) times the cells
 * a warp serves (32 / lanes per cell); 0 with per-phase launches, whose
 * residency the hardware scheduler decides. */
#define ECMC_PARAM_CHAINS_IN_FLIGHT 20
/* Boundary rule (Sec. 3.4 and the comparison of Fig. 3):
 * ECMC_BOUNDARY_REFLECT (default), chains reflect at cell walls and frozen
 * disks (the paper's rule); ECMC_BOUNDARY_REJECT, a chain that reaches a cell
 * wall or a frozen disk is rejected as a whole -- every disk it moved returns
 * to its position at the chain's start, its contacts are counted in events,
 * lifts, frozen_hits and wall_hits but not in sum_b, and its budget is not in
 * sum_disp (ecmc_pressure then averages over accepted chains only, an
 * estimator not derived for this rule; the paper reads the pressure of this
 * variant from g(sigma+)).  Axis chains only (ECMC_ERR_UNSUPPORTED with
 * isotropic directions); allocates an undo log of 32 bytes per bucket slot
 * (ECMC_ERR_OOM if that fails). */
#define ECMC_PARAM_BOUNDARY 21
#define ECMC_BOUNDARY_REFLECT 0
#define ECMC_BOUNDARY_REJECT 1
#define ECMC_LIST_WITH_REPL 0
#define ECMC_LIST_WITHOUT_REPL 1

#define ECMC_DIR_PM_AXIS_ALT 0
#define ECMC_DIR_POS_ONLY 1
#define ECMC_DIR_ISOTROPIC 2
#define ECMC_PREC_FP64 0
#define ECMC_PREC_FP32_GEOM 1

typedef struct ecmc_ctx* ecmc_t;

typedef struct {
  int64_t sweeps;      /* sweeps since the last reset                           */
  int64_t chains;      /* chains run (a cell without members starts none)       */
  int64_t events;      /* contacts: lifts + reflections at frozen disks         */
  int64_t lifts;       /* contacts with an active disk (budget passed on)       */
  int64_t frozen_hits; /* contacts with a frozen disk (chain reflected)         */
  int64_t wall_hits;   /* reflections at a cell wall (not counted as events)    */
  int64_t fp64_evals;  /* candidates evaluated in FP64 (FP32_GEOM screening)    */
  double sum_b;        /* sum over contacts of the separation along d           */
  double sum_disp;     /* sum over chains of the displacement budget ell        */
  int64_t replayed_legs; /* reflection legs (frozen disk or wall) of a chain that
                          * repeated the two legs before them bit for bit and were
                          * replayed without a candidate search; included in
                          * frozen_hits / wall_hits                             */
  int64_t rejected_chains; /* chains rejected under ECMC_BOUNDARY_REJECT          */
} ecmc_counters_t;

typedef struct {
  double bin_ms;       /* per-sweep draws and the cell binning pass            */
  double frame_ms;     /* frame builders (active cell + frozen halo staging)   */
  double phase_ms;     /* the chain kernels of the four colour phases          */
  double other_ms;     /* end-of-sweep reduction                               */
  int64_t bin_launches;
  int64_t frame_launches;
  int64_t phase_launches;
  int64_t other_launches;
} ecmc_timing_t;

typedef struct {
  int64_t start_id; /* disk that started the chain                          */
  int64_t end_id;   /* disk that was moving when the budget ran out        */
  int64_t events;   /* contacts of the chain                                */
  int64_t walls;    /* wall reflections of the chain                        */
} ecmc_chain_rec_t;

/* Create a system of N disks of diameter sigma in the periodic L x L box,
 * started on a k x k square lattice (k = sqrt(N); disk iy*k + ix at
 * ((ix + 1/2) L/k, (iy + 1/2) L/k)), with cells_x x cells_y cells (both
 * even and >= 2; w = L/cells_x and h = L/cells_y must exceed sigma), total
 * chain displacement ell, Philox seed `seed`.  Sec. 2 and Sec. 3.4.
 * Errors: ECMC_ERR_ARG (N not a perfect square or < 1, cells odd or < 2,
 * w or h <= sigma, L/k <= sigma so the lattice would overlap, ell < 0,
 * sigma outside [2^-40, 2^40] or L >= 2^40 sigma),
 * ECMC_ERR_CUDA, ECMC_ERR_OOM.  *out receives the handle (owned by the
 * library until ecmc_destroy). */
ECMC_API int ecmc_create(ecmc_t* out, int64_t N, double L, double sigma, int cells_x, int cells_y,
                double ell, uint64_t seed);

/* One replica of a batch: an independent system (Sec. 3.4's sweep applied to
 * each), advanced together with the others in the same launches.  The paper
 * runs 30 independent simulations to estimate errors (Sec. 3.4, Fig. 4);
 * here many replicas of different N and packing fraction share the GPU. */
typedef struct {
  int64_t N;        /* disks (a perfect square: square-lattice start)        */
  double L;         /* box side                                             */
  double sigma;     /* disk diameter                                        */
  int cells_x;      /* cells per side (even, >= 2, side > sigma)            */
  int cells_y;
  double ell;       /* chain displacement                                   */
  int n_m;          /* chains per cell and sweep; 0 = eq. (nm) default      */
  uint64_t seed;    /* Philox key word 0                                    */
  uint64_t replica; /* Philox key word 1                                    */
} ecmc_replica_desc_t;

/* Create a handle holding R independent replicas, each started on its own
 * square lattice.  Positions of the whole handle (ecmc_positions,
 * ecmc_set_positions) are the replicas' id-ordered pairs concatenated in
 * replica order.  Sweeps advance every replica by one sweep in the same
 * launches (one graph per sweep).  Errors as ecmc_create, for any replica;
 * ECMC_ERR_ARG if R < 1. */
ECMC_API int ecmc_create_batch(ecmc_t* out, const ecmc_replica_desc_t* desc, int R);

/* Number of replicas of the handle. */
ECMC_API int ecmc_num_replicas(ecmc_t h, int* R);

/* Parameters of replica r as used (n_m resolved). */
ECMC_API int ecmc_replica_desc(ecmc_t h, int r, ecmc_replica_desc_t* out);

/* Pressure (as ecmc_pressure) and counters (as ecmc_counters) of replica r.
 * ecmc_pressure itself reports replica 0, ecmc_counters the sum over all
 * replicas. */
ECMC_API int ecmc_replica_pressure(ecmc_t h, int r, double* betaP_sigma2, double* stderr_out);
ECMC_API int ecmc_replica_counters(ecmc_t h, int r, ecmc_counters_t* out);

/* The paper's strategy for the degree of parallelisation (Sec. 4, final
 * paragraph), for a system of N disks of diameter sigma in an L x L box:
 *   1) n, the number of 2x2 blocks (4n cells), is the largest with
 *      N / (eta n) > 100, so that the chain displacement of step 2 stays
 *      above 10 lambda0; cells per side = 2 floor(sqrt(n)), at least 2, and
 *      reduced until the cell side exceeds min_cell_side (>= sigma);
 *   2) ell = lambda0 (N / (eta n))^(1/2), the second form of eq. (criterion);
 *   3) n_m from eq. (nm),
 * with lambda0 = sigma (eta_hcp - eta) / (2 eta_hcp) (Sec. 4).  Fills the
 * geometry fields of *out (seed and replica are left as given).
 * ECMC_ERR_ARG if the system is too small for 2x2 cells of side > sigma. */
ECMC_API int ecmc_suggest_parameters(int64_t N, double L, double sigma, double min_cell_side,
                                     ecmc_replica_desc_t* out);

/* ---- measured choice of cells and ell (Sec. 4, Figs. 5-6) ---------------- */
/* Sampling proxies ecmc_tune_geometry can maximise. */
#define ECMC_TUNE_EVENTS 0 /* collision events per second                          */
#define ECMC_TUNE_MSD 1    /* mean square displacement per disk per second         */
#define ECMC_TUNE_TAU 2    /* sweeps per second / tau of Psi in sweeps (eq. tau)    */

/* One trial of ecmc_tune_geometry. */
typedef struct {
  int cells;            /* cells per side                                        */
  int n_m;              /* chains per cell and sweep, eq. (nm)                   */
  double ell;           /* chain displacement                                    */
  int status;           /* ECMC_OK, or why the trial did not run (ECMC_ERR_ARG:  */
                        /* cell side not above 2 sigma, ell <= 0, ...)           */
  int64_t sweeps;       /* timed sweeps                                          */
  double ms_per_sweep;  /* CUDA-event time per timed sweep                       */
  double events_per_s;
  double sweeps_per_s;
  double lambda0;       /* measured mean free path: displacement over contacts,  */
                        /* wall reflections and chain ends                       */
  double ell_star;      /* eq. (criterion) with that lambda0: L lambda0 / (sqrt(n) sigma), */
                        /* n = cells^2 / 4 blocks                                */
  double msd_per_sweep; /* ECMC_TUNE_MSD: mean square displacement per disk and sweep */
  double tau_sweeps;    /* ECMC_TUNE_TAU: autocorrelation time of Psi in sweeps  */
  double score;         /* the proxy (-1 if the trial did not run)                */
} ecmc_geom_trial_t;

/* The degree of parallelisation chosen by measurement: the paper's strategy
 * (Sec. 4; ecmc_suggest_parameters) picks cells and ell from eqs. (nm),
 * (lambda0) and (criterion); this entry point times the alternatives instead.
 * For every pair (cells[i], ells[j]) -- trial index i * n_ells + j -- it
 * builds a system with base's N, L, sigma, seed and replica, n_m from eq. (nm),
 * starting from xy (host memory, 2N values in id order; NULL = the square
 * lattice), runs warm_sweeps sweeps, then sweeps timed with CUDA events in
 * batches of trial_sweeps until at least min_seconds have passed, and scores
 * it by `proxy` (ECMC_TUNE_*; MSD and TAU run trial_sweeps further sweeps to
 * measure it).  trials (n_cells * n_ells entries) receives every trial, *best
 * the index of the largest score.  Cells whose side is not above 2 sigma are
 * skipped (status ECMC_ERR_ARG).  Each trial is a separate handle: the
 * caller's handles are not touched.  Errors: ECMC_ERR_ARG (bad arguments, no
 * candidate ran), ECMC_ERR_OOM, ECMC_ERR_CUDA. */
ECMC_API int ecmc_tune_geometry(const ecmc_replica_desc_t* base, const double* xy,
                                const int* cells, int n_cells, const double* ells, int n_ells,
                                int warm_sweeps, int trial_sweeps, double min_seconds, int proxy,
                                ecmc_geom_trial_t* trials, int* best);

/* One launch shape and its measured time per sweep. */
typedef struct {
  int lanes_per_cell;
  int warps_per_block; /* per-phase kernels only                              */
  int frame_mode;      /* per-phase kernels only                              */
  int persistent;      /* 1 = the persistent sweep kernel (ECMC_PARAM_PERSISTENT) */
  double ms_per_sweep;
} ecmc_tune_result_t;

/* Time trial_sweeps sweeps (after one warm-up sweep) for every launch shape
 * that fits (the persistent sweep kernel with lanes per cell 1..32; the
 * per-phase kernels with lanes per cell 1..32, warps per block 1 and 2, frame
 * modes 0 and 1, or 2 when nothing else fits), keep the
 * fastest, and put the handle back exactly where it was (positions, sweep
 * counter, statistics): every shape gives bit-identical trajectories, so the
 * tuning does not change the simulation.  best receives the chosen shape;
 * all (may be NULL) up to max_all measured shapes, *n_all their number. */
ECMC_API int ecmc_autotune(ecmc_t h, int trial_sweeps, ecmc_tune_result_t* best,
                           ecmc_tune_result_t* all, int max_all, int* n_all);

/* Release the handle and all its device memory.  NULL is accepted. */
ECMC_API int ecmc_destroy(ecmc_t h);

/* Set / query one ECMC_PARAM_* value.  ECMC_ERR_ARG for an unknown key or a
 * value out of range. */
ECMC_API int ecmc_set_param(ecmc_t h, int key, double value);
ECMC_API int ecmc_get_param(ecmc_t h, int key, double* value);

/* Use the caller's CUDA stream (a cudaStream_t passed as void*, or NULL for
 * the library's own stream) for all later work.  The caller keeps ownership
 * of the stream and must keep it alive while the handle uses it. */
ECMC_API int ecmc_set_stream(ecmc_t h, void* stream);

/* Replace the configuration by the 2N values at xy (interleaved, id order;
 * device memory if on_device != 0, else host memory) and set the sweep
 * counter to t0 (the Philox counter of the next sweep).  Values are wrapped
 * into [0, L).  Errors: ECMC_ERR_ARG (NULL, t0 < 0). */
ECMC_API int ecmc_set_positions(ecmc_t h, const double* xy, int on_device, int64_t t0);

/* Enqueue n_sweeps sweeps (Sec. 3.4 steps 1-7) on the handle's stream.
 * Asynchronous: errors raised on the device (ECMC_ERR_CAPACITY,
 * ECMC_ERR_CHAIN_CAP) are reported by the next synchronising call. */
ECMC_API int ecmc_sweep(ecmc_t h, int64_t n_sweeps);

/* Wait for the handle's stream; report device-side errors. */
ECMC_API int ecmc_synchronize(ecmc_t h);

/* Copy the configuration out (2N doubles, interleaved, id order) into
 * caller memory (device if on_device != 0). */
ECMC_API int ecmc_positions(ecmc_t h, double* xy_out, int on_device);

/* Current sweep counter (the Philox counter of the next sweep). */
ECMC_API int ecmc_sweep_index(ecmc_t h, int64_t* t);

/* Counters accumulated since creation or the last ecmc_reset_stats. */
ECMC_API int ecmc_counters(ecmc_t h, ecmc_counters_t* out);

/* Clear counters, pressure accumulators and the pair histogram. */
ECMC_API int ecmc_reset_stats(ecmc_t h);

/* Pressure from the collision sums since the last reset, the collision form
 * of eq. (pressure) of Sec. 2: beta P sigma^2 = rho sigma^2 (1 + B / D) with
 * B = sum over cells of n_c * (sum over the cell's contacts of the centre
 * separation along d at contact) and D = sum over cells of n_c * n_m * ell,
 * n_c the number of members of the cell.  (Each cell gets the same
 * displacement whatever n_c; weighting by n_c removes the bias this causes.)
 * stderr_out (may be NULL) is the standard error from batch means over the
 * sweeps since the reset (0 if fewer than 2 sweeps).
 * ECMC_ERR_STATE if no sweep has run since the reset. */
ECMC_API int ecmc_pressure(ecmc_t h, double* betaP_sigma2, double* stderr_out);

/* Add the pair histogram of the current configuration (replica 0) to the
 * accumulated one: ordered pairs with sigma + i dr <= d < sigma + (i+1) dr
 * (Sec. 2). */
ECMC_API int ecmc_gr_measure(ecmc_t h);

/* Accumulated counts (int64[nbins]) and number of measurements.
 * ECMC_ERR_ARG if nbins differs from the configured bin count. */
ECMC_API int ecmc_gr_counts(ecmc_t h, int64_t* counts, int nbins, int64_t* n_meas);

/* Normalised g(R_i) = <n(r_i)> / (N rho 2 pi R_i dr) with the area-weighted
 * radius R_i = 2 (e1^3 - e0^3) / (3 (e1^2 - e0^2)) of each bin (Sec. 2);
 * r_out (may be NULL) receives R_i. */
ECMC_API int ecmc_gr(ecmc_t h, double* g_out, double* r_out, int nbins);

/* Number of histogram bins for the current GR_DR / GR_RMAX. */
ECMC_API int ecmc_gr_nbins(ecmc_t h, int* nbins);

/* The same three for replica r of a batch (ecmc_gr_measure, ecmc_gr_counts
 * and ecmc_gr are these with r = 0).  Every replica has its own histogram of
 * ecmc_gr_nbins bins [sigma_r + i dr, sigma_r + (i+1) dr) and its own
 * measurement count; ecmc_replica_gr_measure with r = -1 adds the current
 * configuration of every replica to its histogram (one launch per replica,
 * enqueued on the stream).  ECMC_ERR_ARG if r is out of range. */
ECMC_API int ecmc_replica_gr_measure(ecmc_t h, int r);
ECMC_API int ecmc_replica_gr_counts(ecmc_t h, int r, int64_t* counts, int nbins,
                                    int64_t* n_meas);
ECMC_API int ecmc_replica_gr(ecmc_t h, int r, double* g_out, double* r_out, int nbins);

/* Smallest minimum-image pair distance of the current configuration among
 * pairs closer than 2 sigma (2 sigma if none), over all replicas. */
ECMC_API int ecmc_min_distance(ecmc_t h, double* dmin);

/* Cell of every disk (by id, replicas concatenated) in the most recent
 * binning, cy*cells_x+cx within its replica. */
ECMC_API int ecmc_last_cells(ecmc_t h, int32_t* cell_of_id);

/* Per-kernel times accumulated while ECMC_PARAM_TIMING is 1. */
ECMC_API int ecmc_kernel_times(ecmc_t h, ecmc_timing_t* out);

/* Per-chain records of the most recent sweep (requires
 * ECMC_PARAM_RECORD_CHAINS = 1 during that sweep) of replica 0:
 * out[cell * n_m + k] for cell = cy * cells_x + cx; cells without members
 * hold start_id = -1.  n must equal cells_x * cells_y * n_m. */
ECMC_API int ecmc_chain_records(ecmc_t h, ecmc_chain_rec_t* out, int64_t n);

/* Measure, on the current device, the shared-memory load bandwidth (GB/s,
 * 16-byte loads from every SM) and the FP64 fused multiply-add throughput
 * (GFLOP/s); the roofline denominators of the chain kernel.  No handle is
 * needed; takes a few milliseconds. */
ECMC_API int ecmc_device_peaks(double* smem_gbs, double* fp64_gflops);

/* Hexatic order parameter of every replica (Sec. 2, eq. Psi): Psi = N^-1 sum_k
 * Psi_k, Psi_k = sum over the next neighbours l of exp(6 i phi_kl) / n_k, phi
 * the angle of the vector k -> l to the x axis, next neighbours = Delaunay
 * neighbours (the paper triangulates with a library).  Disk l within rs of k
 * (minimum image) is a neighbour when the perpendicular bisector of k and l
 * keeps a piece of positive length after the half-planes of every other disk
 * within rs cut it (the Voronoi edge); the result is the exact Delaunay graph
 * when every Voronoi vertex of k lies within rs/2, and *n_bad counts the
 * disks for which that check fails (0 in dense fluids with the default rs).
 *   rs     neighbour radius (<= 0: 3.5 sigma of each replica); L must exceed 2 rs
 *   psi    [2R] receives Re, Im of Psi of replica r at [2r], [2r+1] (summed
 *          in disk-id order)
 *   psi_k  [2N] per-disk Re, Im, disks of all replicas concatenated in id
 *          order (as ecmc_positions), or NULL
 *   n_nb   [N] neighbour counts, same order, or NULL
 *   n_bad  number of uncertified disks, or NULL
 * Errors: ECMC_ERR_ARG, ECMC_ERR_STATE, ECMC_ERR_CAPACITY (more than 64
 * disks within rs of one disk), ECMC_ERR_CUDA.  Synchronises the stream. */
ECMC_API int ecmc_hexatic(ecmc_t h, double rs, double* psi, double* psi_k, int32_t* n_nb,
                          int64_t* n_bad);

/* Autocorrelation time of the hexatic order parameter (Sec. 2, eq. tau),
 * from R independent series (replicas of one system) of n samples each:
 * C(dt) = Re <Psi_r*(t) Psi_r(t + dt)>_{t,r} / <|Psi_r(t)|^2>_{t,r}, the
 * numerator averaged over the R (n - dt) pairs at lag dt, the denominator over
 * all R n samples, with the mean of Psi taken as zero as the definition
 * prescribes (its phase depends on the arbitrary reference axis); tau is the
 * lag at which C first falls below 1/e, interpolated linearly between the lags
 * around it, in units of the sampling interval (+infinity if C stays at or
 * above 1/e up to max_lag).
 *   psi     host memory, 2 n R doubles, sample-major: Re, Im of series r at
 *           sample t at [2 (t R + r)], [2 (t R + r) + 1]
 *   n       samples per series (>= 2); R series (>= 1)
 *   max_lag largest lag evaluated (<= 0: n / 4); must be below n
 *   tau     receives tau
 *   c_out   host memory for C(0 .. max_lag), or NULL (then the scan stops at
 *           the 1/e crossing)
 * Host arithmetic, no device work.  Errors: ECMC_ERR_ARG (NULL psi or tau,
 * n < 2, R < 1, max_lag >= n, series without positive finite power). */
ECMC_API int ecmc_autocorrelation_time(const double* psi, int64_t n, int R, int64_t max_lag,
                                       double* tau, double* c_out);

/* The square root of the chain kernel's hit distance (Sec. 3.2: the
 * distance to contact s = b - sqrt(sigma^2 - c^2) is formed in FP64 with the
 * square root correctly rounded to nearest, as IEEE 754 sqrt).  The kernel
 * takes it on the integer pipes (an FP32 reciprocal-square-root estimate,
 * two fixed-point Newton steps, an exact integer remainder for the
 * rounding); this entry evaluates that routine on n inputs:
 *   where = 0  host memory, on the host, with the estimate replaced by the
 *              exact reciprocal square root of the float seed times
 *              (1 + rel_error), |rel_error| <= 2^-20; tests the Newton steps
 *              and the rounding against estimates far worse than the SFU's
 *   where = 1  device memory x, out; on the device exactly as the chain
 *              kernel evaluates it; stream = cudaStream_t (NULL = legacy
 *              default); returns after the kernel has finished
 * Inputs that are not positive normal doubles give NaN.  Errors:
 * ECMC_ERR_ARG (NULL pointers with n > 0, n < 0, bad where or rel_error),
 * ECMC_ERR_CUDA. */
ECMC_API int ecmc_sqrt_rn(const double* x, double* out, int64_t n, int where, double rel_error,
                          void* stream);

/* Size of the static scratch array behind ecmc_sweep_noalloc (16 MiB). */
#define ECMC_NOALLOC_SCRATCH_BYTES (16u << 20)

/* ecmc_sweep_noalloc: n_sweeps sweeps of a system whose positions the caller
 * keeps in its own device memory, with no device allocation at all.  The
 * paper has no counterpart: this is for callers that cannot call cudaMalloc,
 * such as an application whose device memory is owned by its own pool (every
 * allocation outside it is forbidden) or code that must not allocate after
 * its set-up.  The scratch (cell buckets, frame records, per-cell results)
 * comes from one static device array of ECMC_NOALLOC_SCRATCH_BYTES compiled
 * into the library, held by every GPU that loads the library until exit.
 *   xy         device memory, 2N float64 interleaved in disk-id order; read,
 *              then overwritten with the positions after the sweeps
 *   N ... ell  as for ecmc_create; n_m chains per cell; seed, replica the
 *              Philox key; t0 the Philox counter of the first sweep
 *   stream     cudaStream_t (NULL = legacy default stream)
 * The sweeps are the same as those of a handle with the same parameters
 * (ecmc_set_positions(xy, t0), ecmc_sweep(n_sweeps)), screening in FP32: the
 * same argument checks (except that N need not be a perfect square), the
 * same geometry and the same overlap check of the input.  The call returns
 * after the work on `stream` has finished.  Errors, each leaving xy as it
 * was passed in:
 *   ECMC_ERR_ARG         as ecmc_create (N >= 1 any size below 2^27), or
 *                        n_m < 1, t0 < 0, n_sweeps < 0, xy NULL;
 *   ECMC_ERR_OVERLAP     two input disks closer than sigma (1 - 1e-9)^(1/2);
 *   ECMC_ERR_CAPACITY    the system needs more scratch than the array holds
 *                        (roughly N <= 64k disks at eta 0.7), or a cell of
 *                        the input holds more disks than its packing bound;
 *   ECMC_ERR_UNSUPPORTED cell frames too large for shared memory (the handle
 *                        would use frames in global memory instead);
 *   ECMC_ERR_CHAIN_CAP   a chain reached the per-chain event cap;
 *   ECMC_ERR_CUDA        a CUDA call failed.
 * The first call on a device looks up the array's device address and caches
 * it; make it before any stream capture, and do not call this entry point on
 * a device after cudaDeviceReset in the same process (the cached address is
 * then stale).  Every call shares the array: calls that overlap on the GPU
 * race and must be serialised by the caller. */
ECMC_API int ecmc_sweep_noalloc(double* xy, int64_t N, double L, double sigma, int cells_x,
                                int cells_y, double ell, int n_m, uint64_t seed, uint64_t replica,
                                int64_t t0, int64_t n_sweeps, void* stream);

/* Message for an error code (static string). */
ECMC_API const char* ecmc_strerror(int code);

/* Detail of the most recent failure on the calling thread (static buffer). */
ECMC_API const char* ecmc_last_error_message(void);

/* Library version string. */
ECMC_API const char* ecmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ECMC_H */
