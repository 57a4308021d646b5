/*
 * ecmc_oracle_stripes.h -- oracle of the striped decomposition that the
 * paper tests beside its checkerboard in Sec. 3.4 (Fig. 3, "stripes", the
 * parallelisation proposed by Kapfer and Krauth): chains of rejection-free
 * event-chain moves run inside stripes that span the box along the chain
 * axis; a chain that would touch a disk of a neighbouring stripe is
 * rejected as a whole (or, for comparison, turns back).
 *
 * TEST INFRASTRUCTURE ONLY, like ecmc_oracle.h: the CUDA library never
 * includes, links or calls anything declared here.
 *
 * The sweep t (reading of the paper's one-sentence description; the paper
 * gives no further detail):
 *   - axis a = x on even t, y on odd t; the chains of the sweep move along
 *     +-a, the sign drawn per chain (the same direction rule as the cells);
 *   - the box is cut into S = p->cells_x stripes (S even, L / S > sigma),
 *     each spanning the whole box along a and of width w = L / S across it,
 *     on a lattice shifted across by unit53(u0) * w, u = Philox words of
 *     (t, SWEEP, 0, 0);
 *   - colour = stripe index mod 2; colour below(u2, 2) runs first
 *     (ORC_FLAG_NO_SHIFT, ORC_FLAG_FIXED_COLOURS and ORC_FLAG_REVERSE_CELLS
 *     act as for the cells);
 *   - every stripe of the running colour starts n_m chains at members
 *     chosen by p->list_mode exactly as a cell does (counter words
 *     (t, CHAIN, stripe, k) and (t, SHUFFLE, stripe, .)), one after the
 *     other, the disks of all other stripes frozen;
 *   - a stripe is periodic along a (its members meet each other's images
 *     around the box); there are no walls;
 *   - a contact with a frozen disk rejects the whole chain
 *     (ORC_BOUNDARY_REJECT, the paper's stripes) or turns it back along the
 *     axis (ORC_BOUNDARY_REFLECT);
 *   - ties as for the cells: smaller (id, image) key first, and the chain's
 *     end before a contact at equal distance;
 *   - pressure sums as for the cells (member-weighted per stripe).
 */
#ifndef ECMC_ORACLE_STRIPES_H
#define ECMC_ORACLE_STRIPES_H

#include <stdint.h>

#include "ecmc_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Shift of the stripe lattice across the axis, and the colour that runs
 * first in sweep t. */
void orc_stripe_draws(const orc_params* p, int64_t t, double* shift, int* first_colour);

/* Stripe of every disk in sweep t (the index across the axis of sweep t). */
int orc_stripe_bin(const orc_params* p, int64_t t, const double* x, const double* y,
                   int32_t* stripe);

/* Sweeps t0 .. t0+n_sweeps-1 in place.  p->cells_x is the number of
 * stripes; p->cells_y is not used; p->dir_mode must be ORC_DIR_PM_AXIS_ALT
 * or ORC_DIR_POS_ONLY.  recs, if not NULL, receives one record per (sweep,
 * stripe, chain) at [(s * stripes + stripe) * n_m + k].  Returns 0 or -1 on
 * invalid parameters. */
int orc_stripe_sweeps(const orc_params* p, double* x, double* y, int64_t t0, int64_t n_sweeps,
                      orc_stats* st, orc_chain_rec* recs);

/* One chain in a caller-built stripe frame: U is the coordinate along the
 * axis (periodic with period L), V the coordinate across it; objects
 * 0..n_mem-1 are members, the rest frozen; key orders ties.  Object m moves
 * with sign +-1 and budget ell; reject selects the rejecting rule.  U is
 * updated in place (V never changes).  Returns 1 if the chain was rejected,
 * 0 if not, -1 on invalid arguments; rec->end_id is the frame index of the
 * object moving when the chain ended or was rejected. */
int orc_run_chain_stripe(int n, int n_mem, double* U, const double* V, const int64_t* key,
                         double L, double sigma, int m, int sign, double ell, int reject,
                         orc_stats* st, orc_chain_rec* rec);

#ifdef __cplusplus
}
#endif
#endif
