// ecmc_chain.cuh -- the event-chain loop of one group of cells, shared by the
// per-phase chain kernel (ecmc_phase.cu) and the persistent sweep kernel
// (ecmc_sweep.cu).
//
// Sec. 3.4 steps 5-6 with the straight event chain of Sec. 3.2: in every
// active cell, n_m chains start at members drawn WITH replacement (member
// number floor(v n_c / 2^64) in ascending-id order, v from Philox keyed by
// (seed, replica) and counter (sweep, chain purpose, cell, chain)).  The
// active disk moves along +/- the sweep's axis until the first of
//   - the end of the displacement budget,
//   - a contact with another member (the rest of the budget passes to it),
//   - a contact with a frozen disk (the chain turns back along its axis),
//   - the cell wall (the chain turns back; Fig. 1).
// Ties: the budget end beats a contact, a contact beats a wall, equal hit
// distances go to the smaller (disk id, image) key.
//
// Work layout: one warp serves cpw = 32/TPC cells; TPC lanes share one cell.
// The warp copies its group's frame record into shared memory; every lane
// group then runs its cell's chains.  Candidates come from the strip of
// width 2 sigma across the chain axis around the active disk.  With FP32
// screening, each candidate's hit distance is bracketed in FP32 by rigorous
// error bounds, and only candidates that can be the first hit (in practice
// one) are evaluated in FP64 with the reference arithmetic, so the decision
// and the new position are exactly those of a full FP64 search.
#pragma once
#include <climits>

#include "ecmc_device.cuh"
#include "ecmc_internal.cuh"

namespace ecmc {

// Legs of the current chain kept for cycle detection (a power of two): a
// chain that rattles through a row of up to kHist/2 disks between two
// reflectors repeats with a period of at most kHist legs.
constexpr int kHist = 32;
constexpr size_t kHistLegBytes = 32;  // P, step, contact sum (FP64); disk, flags

struct LegHist {
  double* P;     // start position along the axis
  double* step;  // length of the leg
  double* addb;  // contribution to the contact sum (contacts)
  int* m;        // active disk (frame index)
  int* flags;    // bit 0: moving in -d; bit 1: frozen disk; bit 2: wall; 0 in both: lift
};

struct Frame {
  const int* bst;
  const int* mrank;
  const int* mslot;
  float* a32;
  float* b32;  // written only by isotropic chains
  double* a64;
  double* b64;  // written only by isotropic chains (axis chains keep the cross coordinate)
  const int* key;
  const int* info;
  unsigned char* touched;
  int cpw;
};

// FP64 hit test and hit distance along an axis direction of sign sg,
// written as the general expressions reduce for d = (+-1, 0):
//   b = (x_j - x_m) . d,  c = (x_j - x_m) x d,  hit iff b > 0 and c^2 < sigma^2,
//   s = max(0, b - sqrt(sigma^2 - c^2)).
// The arithmetic is exactly the reference's; comparisons, sign changes and
// the correctly rounded square root run on the integer pipes (ecmc_device.cuh),
// and the square root is taken of a positive placeholder when the candidate
// misses, so there is no branch.  sigma^2 - c^2 > 0 is a normal number for
// every hit (sigma is restricted to [2^-40, 2^40]), as sqrt_rn requires.
__device__ __forceinline__ bool exact_hit(double aj, double bj, double P, double Q, int sg,
                                          double sig2, double& s, double& b) {
  const double da = aj - P;
  const double db = bj - Q;
  const long long bda = dbits(da);
  const bool ahead = (sg > 0) ? (bda > 0) : (bda < 0 && bda != (long long)0x8000000000000000ull);
  b = flip_if(da, sg < 0);
  const double c2 = db * db;
  const bool hit = ahead && lt_nn(c2, sig2);
  const double x = sig2 - c2;
  const double sq = sqrt_rn(hit ? x : 1.0);
  s = clamp0(b - sq);
  return hit;
}

__device__ __forceinline__ bool better(double s, int key, double bs, int bkey) {
  return s < bs || (s == bs && key < bkey);
}

// Start list without replacement (the negative control of Sec. 3.4): entry 0
// is the member drawn for chain 0, entries 1..n-1 the other members in
// ascending rank, shuffled by Fisher-Yates from the top: position i (n-1 down
// to 2) swaps with 1 + floor(u n_i / 2^64), u word i mod 4 of the Philox draw
// (sweep, shuffle purpose, cell, i / 4).  pl holds up to kHist * 8 entries per
// group, interleaved [entry][group].
__device__ __forceinline__ void shuffled_list(int* pl, int CPW, int gi, int n, int first,
                                              int64_t t, int lc, uint64_t seed,
                                              uint64_t replica) {
  int q = 0;
  pl[gi] = first;
  for (int i = 0; i < n; ++i)
    if (i != first) pl[(++q) * CPW + gi] = i;
  U64x4 u;
  int cur = -1;
  for (int i = n - 1; i >= 2; --i) {
    if ((i >> 2) != cur) {
      cur = i >> 2;
      u = philox((uint64_t)t, kPurposeShuffle, (uint64_t)lc, (uint64_t)cur, seed, replica);
    }
    const int j = 1 + (int)below_n(u.v[i & 3], (uint64_t)i);
    const int a = pl[i * CPW + gi];
    pl[i * CPW + gi] = pl[j * CPW + gi];
    pl[j * CPW + gi] = a;
  }
}

// Cycle replay.  Called after a reflection, with the state (m, sg, P) the next
// leg starts from.  If for some even K <= kHist the configuration equals the
// one K legs earlier -- the same active disk, direction and position bit for
// bit, and every other disk that moved in those K legs back where it was --
// then nothing else distinguishes the two moments (frozen disks and walls do
// not move, the decision depends on the budget only through its end), so the
// next legs repeat those K legs exactly, step for step, as long as the budget
// exceeds the step.  They are replayed from the history with one subtraction
// each; at the leg where the budget runs out the disks are put where the
// recorded legs left them and the full search resumes (and ends the chain).
// The smallest such K is used.  The TPC lanes of the group share the search:
// lane sub tests K = 2 (sub + 1), 2 (sub + 1) + 2 TPC, ..., and the group
// takes the minimum (every lane of the group arrives here with the same
// state, so all TPC lanes take part in the shuffles).
template <int TPC>
__device__ __forceinline__ void replay_cycle(const Frame& f, const LegHist& hs, int gi, int sub,
                                             int& n_leg, int& m, int& sg, double& P,
                                             float& P32, double& Q, float& Q32, double& r,
                                             int64_t& n_iter, double& sum_b, int& n_events,
                                             int& n_lifts, int& n_frozen, int& n_walls,
                                             int& ch_events, int& ch_walls, int& n_replayed) {
  const int CPW = f.cpw;
  int Kf = INT_MAX;
  // the loops stay rolled: the check runs at every reflection, and unrolled
  // it grows the sweep kernel beyond what its instruction cache holds
#pragma unroll 1
  for (int K = 2 * (sub + 1); K <= kHist && K <= n_leg; K += 2 * TPC) {
    const int s0 = ((n_leg - K) & (kHist - 1)) * CPW + gi;
    if (hs.m[s0] != m || dbits(hs.P[s0]) != dbits(P) || ((hs.flags[s0] & 1) != (sg < 0 ? 1 : 0)))
      continue;
    bool same = true;
#pragma unroll 1
    for (int i = n_leg - K; i < n_leg && same; ++i) {
      const int si = (i & (kHist - 1)) * CPW + gi;
      const int D = hs.m[si];
      if (D == m) continue;
      bool first = true;  // D's first leg in the window starts where D was
#pragma unroll 1
      for (int j = n_leg - K; j < i; ++j) first &= (hs.m[(j & (kHist - 1)) * CPW + gi] != D);
      if (first) same = dbits(f.a64[D * CPW + gi]) == dbits(hs.P[si]);
    }
    if (same) {
      Kf = K;
      break;
    }
  }
  if (TPC > 1) {
    const unsigned gmask = TPC == 32 ? 0xffffffffu : (((1u << TPC) - 1u) << (gi * TPC));
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) {
      const int ok = __shfl_xor_sync(gmask, Kf, o);
      Kf = ok < Kf ? ok : Kf;
    }
  }
  if (Kf == INT_MAX) return;
  const int base = n_leg - Kf;
  int o = 0;
  for (;;) {
    const int si = ((base + o) & (kHist - 1)) * CPW + gi;
    const double sl = hs.step[si];
    if (n_iter >= kMaxEventsPerChain || le_nn(r, sl)) break;
    const int fl = hs.flags[si];
    const bool wall = (fl & 4) != 0, frozen = (fl & 2) != 0;
    r = r - sl;
    n_iter += 1;
    n_replayed += 1;
    n_walls += wall ? 1 : 0;
    ch_walls += wall ? 1 : 0;
    n_events += wall ? 0 : 1;
    ch_events += wall ? 0 : 1;
    n_frozen += frozen ? 1 : 0;
    n_lifts += (wall || frozen) ? 0 : 1;
    if (!wall) sum_b += hs.addb[si];
    o = (o + 1 == Kf) ? 0 : o + 1;
  }
  // the configuration at offset o of the cycle: disks that stopped in the
  // first o legs stand where those legs left them
  for (int i = 0; i < o; ++i) {
    const int si = ((base + i) & (kHist - 1)) * CPW + gi;
    const int fl = hs.flags[si];
    if ((fl & 6) == 0) {
      const double end = hs.P[si] + flip_if(hs.step[si], (fl & 1) != 0);
      const int D = hs.m[si];
      f.a64[D * CPW + gi] = end;
      f.a32[D * CPW + gi] = to_float_trunc(end);
    }
  }
  const int so = ((base + o) & (kHist - 1)) * CPW + gi;
  m = hs.m[so];
  sg = (hs.flags[so] & 1) ? -1 : 1;
  P = hs.P[so];
  P32 = to_float_trunc(P);
  Q = f.b64[m * CPW + gi];
  Q32 = f.b32[m * CPW + gi];
  n_leg = 0;
}

// The chains of one group of cells (Sec. 3.4 steps 5-6), their write-back
// and per-cell statistics.  Lane group gi of the warp works on global active
// cell a (valid: a exists) of colour phase colour_index, whose frame is column
// gi of f.
// Rejecting boundary rule: log the frame state of member m before it moves
// (entry e of cell c's undo log), and restore a whole log, newest first.
// Every lane of the group writes and reads the same values.
__device__ __forceinline__ void undo_push(const Geom& g, int c, int e, const Frame& f, int m,
                                          int gi) {
  const int i = m * f.cpw + gi;
  UndoEntry u;
  u.a = f.a64[i];
  u.b = f.b64[i];
  u.a32 = f.a32[i];
  u.b32 = f.b32[i];
  u.m = m;
  u.touched = f.touched[i];
  g.undo[(int64_t)c * g.undo_stride + e] = u;
}

__device__ __forceinline__ void undo_restore(const Geom& g, int c, int n, const Frame& f,
                                             int gi) {
  for (int e = n - 1; e >= 0; --e) {
    const UndoEntry u = g.undo[(int64_t)c * g.undo_stride + e];
    const int i = u.m * f.cpw + gi;
    f.a64[i] = u.a;
    f.b64[i] = u.b;
    f.a32[i] = u.a32;
    f.b32[i] = u.b32;
    f.touched[i] = (unsigned char)u.touched;
  }
}

template <int TPC, bool SCREEN, bool REJECT>
__device__ __forceinline__ void run_group(const Frame& f, const LegHist& hs, const int* hdr,
                                          const Geom* __restrict__ rg,
                                          const SweepState* __restrict__ sts, int rep, int a,
                                          bool valid, int colour_index, RecLayout lay,
                                          double* __restrict__ px, double* __restrict__ py,
                                          CellStats* __restrict__ cs,
                                          ChainRec* __restrict__ recs, int rec_stride, int replay,
                                          int* err) {
  constexpr int CPW = 32 / TPC;
  const int lane = threadIdx.x & 31;
  const int gi = lane / TPC, sub = lane - gi * TPC;
  const Geom& g = rg[rep];
  const SweepState* st = sts + rep;
  const int colour = st->perm[colour_index];
  const int hx = g.cells_x >> 1;
  const int la = a - g.act_off;
  const int cx = 2 * (la % hx) + (colour & 1);
  const int cy = 2 * (la / hx) + (colour >> 1);
  const int lc = cy * g.cells_x + cx;  // cell within the replica (Philox counter word)
  const int c = g.cell_off + lc;       // global cell
  const int axis = st->axis;
  const int64_t t = st->t;
  const double E = axis == 0 ? g.w : g.h;  // cell extent along the chain axis
  const int nmem = valid ? hdr[CPW + gi] : 0;

  double sum_b = 0.0;
  int n_events = 0, n_lifts = 0, n_frozen = 0, n_walls = 0, n_fp64 = 0, n_chains = 0;
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  const unsigned FULL = 0xffffffffu;

  // Chain state, identical in the TPC lanes of a group.  The loop is
  // warp-uniform: every lane runs the same instruction stream each event
  // (lanes whose cell is finished are masked), so one FP64 instruction
  // serves every cell of the warp.
  int k = 0;
  bool active = false;
  int m = 0, sg = 1;
  double P = 0.0, Q = 0.0, r = 0.0;
  float P32 = 0.f, Q32 = 0.f;
  int64_t n_iter = 0;
  int ch_events = 0, ch_walls = 0, start_key = 0;
  int n_leg = 0;  // legs of the current chain recorded in the history
  int n_replayed = 0;
  // rejecting boundary rule: movers logged, the chain's contact sum until
  // the chain is accepted, chains rejected
  constexpr bool reject_rule = REJECT;
  int n_undo = 0, n_rejected = 0;
  double ch_b = 0.0;
  if (reject_rule) replay = 0;
  bool done = (!valid) || nmem == 0;

  for (;;) {
    if (!done && !active) {
      if (k >= g.n_m) {
        done = true;
      } else {
        // start disk drawn with replacement among the members, sign of d
        const U64x4 v = philox((uint64_t)t, kPurposeChain, (uint64_t)lc, (uint64_t)k, g.seed,
                               g.replica);
        int idx = (int)below_n(v.v[0], (uint64_t)nmem);
        if (g.list_mode == 1) {
          // negative control: the first start as drawn, then a uniformly
          // shuffled list of the other members, cycled (kept in the leg
          // history's space: no replay in this mode)
          int* pl = (int*)hs.P;
          if (k == 0) shuffled_list(pl, CPW, gi, nmem, idx, t, lc, g.seed, g.replica);
          idx = pl[(k % nmem) * CPW + gi];
        }
        m = f.mrank[idx * CPW + gi];
        sg = (g.dir_mode == 1) ? 1 : ((v.v[1] >> 63) ? -1 : 1);
        P = f.a64[m * CPW + gi];
        Q = f.b64[m * CPW + gi];
        P32 = f.a32[m * CPW + gi];
        Q32 = f.b32[m * CPW + gi];
        r = g.ell;
        if (reject_rule) {
          undo_push(g, c, 0, f, m, gi);
          n_undo = 1;
          ch_b = 0.0;
        }
        f.touched[m * CPW + gi] = 1;
        start_key = f.key[m * CPW + gi];
        n_iter = 0;
        ch_events = 0;
        ch_walls = 0;
        n_leg = 0;
        active = true;
        ++k;
        ++n_chains;
      }
    }
    if (__all_sync(FULL, done)) break;
    const bool live = !done;
    const bool capped = live && (n_iter >= kMaxEventsPerChain);
    if (capped) atomicCAS(err, DEV_OK, DEV_CHAIN_CAP);
    const bool go = live && !capped;

    // distance to the wall ahead (the axis direction has |d| = 1)
    const double sw = clamp0((sg > 0) ? (E - P) : P);

    // candidate strip across the axis
    int jbeg = 0, jend = 0;
    if (go) {
      const float qlo = Q32 - g.sig_plus - g.strip_margin;
      const float qhi = Q32 + g.sig_plus + g.strip_margin;
      int klo = (int)((qlo + g.sigf) * g.inv_bin_w);
      int khi = (int)((qhi + g.sigf) * g.inv_bin_w);
      klo = klo < 0 ? 0 : (klo >= lay.nbin ? lay.nbin - 1 : klo);
      khi = khi < 0 ? 0 : (khi >= lay.nbin ? lay.nbin - 1 : khi);
      jbeg = f.bst[klo * CPW + gi];
      jend = f.bst[(khi + 1) * CPW + gi];
    }

    double best_s = INF, best_b = 0.0;
    int best_key = INT_MAX, best_j = m;
    if (SCREEN) {
      const float eps = g.eps_d, smarg = g.s_margin;
      float U = __int_as_float(0x7f800000), L1 = U, L2 = U;
      int j1 = m;
      for (int j = jbeg + sub; j < jend; j += TPC) {
        if (j == m) continue;
        const float da = f.a32[j * CPW + gi] - P32;
        const float db = f.b32[j * CPW + gi] - Q32;
        const float bb = sg > 0 ? da : -da;
        if (!(bb > -eps)) continue;
        const float adb = fabsf(db);
        if (!(adb < g.sig_plus)) continue;
        const float x = fmaxf(fmaf(-adb, adb, g.sig2f), 0.0f);
        const float sc = bb - x * rsqrtf(fmaxf(x, 1e-30f));
        const float lo = sc - smarg;
        if (lo < L1) {
          L2 = L1;
          L1 = lo;
          j1 = j;
        } else if (lo < L2) {
          L2 = lo;
        }
        if (bb > eps && adb < g.sig_minus) U = fminf(U, fmaxf(sc + smarg, 0.0f));
      }
      if (TPC > 1) {
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) {
          const float oU = __shfl_xor_sync(FULL, U, o);
          const float oL1 = __shfl_xor_sync(FULL, L1, o);
          const float oL2 = __shfl_xor_sync(FULL, L2, o);
          const int oj1 = __shfl_xor_sync(FULL, j1, o);
          U = fminf(U, oU);
          const float nL2 = fminf(fmaxf(L1, oL1), fminf(L2, oL2));
          if (oL1 < L1 || (oL1 == L1 && oj1 < j1)) {
            L1 = oL1;
            j1 = oj1;
          }
          L2 = nL2;
        }
      }
      // exact FP64 evaluation of the candidates that can be the first hit:
      // those whose lower bound reaches min(smallest certain upper bound,
      // budget, wall distance)
      const float Lam = fminf(U, to_float_up_nn(min_nn(r, sw)));
      const bool need = go && (L1 <= Lam);
      const bool multi = need && (L2 <= Lam);
      const bool single = need && !multi;
      const int jj = single ? j1 : m;
      double s1, b1;
      const bool h1 = exact_hit(f.a64[jj * CPW + gi], f.b64[jj * CPW + gi], P, Q, sg, g.sig2,
                                s1, b1);
      if (single && h1) {
        best_s = s1;
        best_b = b1;
        best_j = jj;
      }
      n_fp64 += single ? 1 : 0;
      if (__any_sync(FULL, multi)) {
        int nev = 0;
        if (multi) {
          for (int j = jbeg + sub; j < jend; j += TPC) {
            if (j == m) continue;
            const float da = f.a32[j * CPW + gi] - P32;
            const float db = f.b32[j * CPW + gi] - Q32;
            const float bb = sg > 0 ? da : -da;
            if (!(bb > -eps)) continue;
            const float adb = fabsf(db);
            if (!(adb < g.sig_plus)) continue;
            const float x = fmaxf(fmaf(-adb, adb, g.sig2f), 0.0f);
            const float lo = (bb - x * rsqrtf(fmaxf(x, 1e-30f))) - smarg;
            if (!(lo <= Lam)) continue;
            ++nev;
            double s, b;
            if (exact_hit(f.a64[j * CPW + gi], f.b64[j * CPW + gi], P, Q, sg, g.sig2, s, b)) {
              const int kj = f.key[j * CPW + gi];
              if (better(s, kj, best_s, best_key)) {
                best_s = s;
                best_b = b;
                best_key = kj;
                best_j = j;
              }
            }
          }
        }
        if (TPC > 1) {
#pragma unroll
          for (int o = 1; o < TPC; o <<= 1) {
            const double os = __shfl_xor_sync(FULL, best_s, o);
            const double ob = __shfl_xor_sync(FULL, best_b, o);
            const int ok = __shfl_xor_sync(FULL, best_key, o);
            const int oj = __shfl_xor_sync(FULL, best_j, o);
            nev += __shfl_xor_sync(FULL, nev, o);
            if (better(os, ok, best_s, best_key)) {
              best_s = os;
              best_b = ob;
              best_key = ok;
              best_j = oj;
            }
          }
        }
        n_fp64 += nev;
      }
    } else {
      // every strip candidate in FP64
      int nev = 0;
      for (int j = jbeg + sub; j < jend; j += TPC) {
        if (j == m) continue;
        ++nev;
        double s, b;
        if (exact_hit(f.a64[j * CPW + gi], f.b64[j * CPW + gi], P, Q, sg, g.sig2, s, b)) {
          const int kj = f.key[j * CPW + gi];
          if (better(s, kj, best_s, best_key)) {
            best_s = s;
            best_b = b;
            best_key = kj;
            best_j = j;
          }
        }
      }
      if (TPC > 1) {
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) {
          const double os = __shfl_xor_sync(FULL, best_s, o);
          const double ob = __shfl_xor_sync(FULL, best_b, o);
          const int ok = __shfl_xor_sync(FULL, best_key, o);
          const int oj = __shfl_xor_sync(FULL, best_j, o);
          nev += __shfl_xor_sync(FULL, nev, o);
          if (better(os, ok, best_s, best_key)) {
            best_s = os;
            best_b = ob;
            best_key = ok;
            best_j = oj;
          }
        }
      }
      n_fp64 += nev;
    }

    // event decision in FP64 (budget end < contact < wall on ties), as
    // selects so that all lanes share one instruction stream
    const bool is_end = le_nn(r, best_s) && le_nn(r, sw);
    const bool is_contact = !is_end && le_nn(best_s, sw);
    const bool is_wall = !is_end && !is_contact;
    const double step = is_end ? r : (is_contact ? best_s : sw);
    const double Pstep = P + flip_if(step, sg < 0);
    const double Pnew = is_wall ? ((sg > 0) ? E : 0.0) : Pstep;
    const double rnew = r - step;
    const double addb = best_b - best_s;
    const float P32n = to_float_trunc(Pnew);
    bool end_chain = capped;
    bool rejected_now = false;
    if (go) {
      if (is_contact) {
        if (reject_rule) ch_b += addb;
        else sum_b += addb;
      }
      r = rnew;
      const bool is_lift = is_contact && (f.info[best_j * CPW + gi] >= 0);
      n_events += is_contact ? 1 : 0;
      ch_events += is_contact ? 1 : 0;
      n_lifts += is_lift ? 1 : 0;
      n_frozen += (is_contact && !is_lift) ? 1 : 0;
      n_walls += is_wall ? 1 : 0;
      ch_walls += is_wall ? 1 : 0;
      n_iter += (is_contact || is_wall) ? 1 : 0;
      rejected_now = reject_rule && (is_wall || (is_contact && !is_lift));
      if (rejected_now) {
        // the chain reached a wall or a frozen disk: every disk it moved
        // returns to its position at the chain's start
        undo_restore(g, c, n_undo < g.cap_mem ? n_undo : g.cap_mem, f, gi);
        ++n_rejected;
      } else if (replay && g.list_mode == 0 && !is_end) {
        // every lane of the group writes the same values, so each lane reads
        // back its own writes
        const int hl = (n_leg & (kHist - 1)) * CPW + gi;
        hs.P[hl] = P;
        hs.step[hl] = step;
        hs.addb[hl] = addb;
        hs.m[hl] = m;
        hs.flags[hl] = (sg < 0 ? 1 : 0) | (is_lift ? 0 : (is_wall ? 4 : 2));
        ++n_leg;
      }
      if (rejected_now) {
      } else if (is_lift) {
        // the hit member carries on with the rest of the budget
        f.a64[m * CPW + gi] = Pnew;
        f.a32[m * CPW + gi] = P32n;
        m = best_j;
        P = f.a64[m * CPW + gi];
        Q = f.b64[m * CPW + gi];
        P32 = f.a32[m * CPW + gi];
        Q32 = f.b32[m * CPW + gi];
        if (reject_rule) {
          if (n_undo < g.cap_mem) undo_push(g, c, n_undo, f, m, gi);
          else atomicCAS(err, DEV_OK, DEV_CAPACITY);
          ++n_undo;
        }
        f.touched[m * CPW + gi] = 1;
      } else {
        P = Pnew;
        P32 = P32n;
        if (!is_end) {
          // frozen disk or wall: the chain turns back along its axis
          sg = -sg;
          if (replay && g.list_mode == 0) replay_cycle<TPC>(f, hs, gi, sub, n_leg, m, sg, P, P32, Q, Q32, r, n_iter, sum_b,
                                   n_events, n_lifts, n_frozen, n_walls, ch_events, ch_walls,
                                   n_replayed);
        }
      }
      end_chain = is_end || rejected_now;
      if (reject_rule && is_end) sum_b += ch_b;
    }
    if (end_chain) {
      if (!rejected_now) {
        f.a64[m * CPW + gi] = P;
        f.a32[m * CPW + gi] = P32;
      }
      if (recs != nullptr && sub == 0) {
        ChainRec rc;
        rc.start_id = start_key >> 4;
        rc.end_id = f.key[m * CPW + gi] >> 4;
        rc.events = ch_events;
        rc.walls = ch_walls;
        recs[(int64_t)c * rec_stride + (k - 1)] = rc;
      }
      active = false;
    }
  }

  __syncwarp();
  if (!valid) return;
  // write the members that were active in a chain back in box coordinates
  const double ox = st->sx + (double)cx * g.w;
  const double oy = st->sy + (double)cy * g.h;
  for (int q = sub; q < nmem; q += TPC) {
    const int j = f.mrank[q * CPW + gi];
    if (!f.touched[j * CPW + gi]) continue;
    const double A = f.a64[j * CPW + gi], B = f.b64[j * CPW + gi];
    const double X = axis == 0 ? A : B, Y = axis == 0 ? B : A;
    const int slot = f.mslot[q * CPW + gi];
    px[slot] = wrap_box0(X + ox, g.L);
    py[slot] = wrap_box0(Y + oy, g.L);
  }
  if (sub == 0) {
    CellStats s;
    s.sum_b = sum_b;
    s.events = n_events;
    s.lifts = n_lifts;
    s.frozen = n_frozen;
    s.walls = n_walls;
    s.fp64_evals = n_fp64;
    s.chains = n_chains;
    s.n_mem = nmem;
    s.replayed = n_replayed;
    s.rejected = n_rejected;
    cs[c] = s;
  }
}


}  // namespace ecmc
