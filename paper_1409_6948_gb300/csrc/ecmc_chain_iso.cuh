// ecmc_chain_iso.cuh -- the event-chain loop with isotropic directions.
//
// The variant the paper prefers for its applications (Sec. 3.2-3.4): every
// chain draws its own unit direction d, uniform on the circle; the active
// disk moves along d until the first of
//   - the end of the displacement budget,
//   - a contact with another member (the rest of the budget passes to it,
//     d unchanged),
//   - a contact with a frozen disk: specular reflection about the line of
//     centres at contact, d <- d - 2 (d.n) n / (n.n) (Fig. 1),
//   - a cell wall: the component of d normal to it flips (both at a corner).
// Ties as for axis chains: budget end < contact < wall; equal hit distances
// go to the smaller (disk id, image) key.
//
// The direction of chain k of cell c in sweep t is the first point (u, v) of
// the Philox pairs keyed (seed, replica), counter (t, direction purpose, c,
// k * 2^32 + attempt), uniform on [-1,1)^2, that lies in the unit disc and not
// at its centre, divided by its length: square root and division are IEEE
// operations, so the direction is reproducible to the last bit.
//
// SCREEN = false: every candidate of the frame is tested in FP64 with the
// expressions of the reference arithmetic (no contraction).  SCREEN = true:
// the projections b = D.d and c = D x d of every candidate are first computed
// in FP32 from the frame's FP32 coordinates and bracketed by rigorous error
// bounds, giving an interval for its hit distance; only candidates whose lower
// bound reaches the smallest certain upper bound (or the budget and wall
// distance) are tested in FP64, so the first hit and the new position are
// those of the full FP64 search.  Either way trajectories are bit-identical to
// the reference.  Frames are built with axis 0 (frame coordinates a = x, b = y).
#pragma once

#include "ecmc_chain.cuh"

namespace ecmc {

constexpr uint64_t kPurposeDirection = 3;

__device__ __forceinline__ void iso_direction(int64_t t, int lc, int k, uint64_t seed,
                                              uint64_t replica, double& dx, double& dy) {
  for (uint64_t attempt = 0; attempt < 4096; ++attempt) {
    const U64x4 q = philox((uint64_t)t, kPurposeDirection, (uint64_t)lc,
                           ((uint64_t)k << 32) | attempt, seed, replica);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double u = 2.0 * unit_double(q.v[2 * h]) - 1.0;
      const double v = 2.0 * unit_double(q.v[2 * h + 1]) - 1.0;
      const double n2 = u * u + v * v;
      if (n2 > 0.0 && n2 <= 1.0) {
        const double n = sqrt(n2);
        dx = u / n;
        dy = v / n;
        return;
      }
    }
  }
  // unreachable in practice (each attempt succeeds with probability
  // 1 - (1 - pi/4)^2 > 0.95); a fixed direction keeps the loop bounded
  dx = 1.0;
  dy = 0.0;
}

// FP64 hit test of candidate j along d, the reference expressions
__device__ __forceinline__ bool iso_hit(const Frame& f, int j, int CPW, int gi, double X, double Y,
                                        double dx, double dy, double sig2, double& s, double& b) {
  const double ddx = f.a64[j * CPW + gi] - X;
  const double ddy = f.b64[j * CPW + gi] - Y;
  b = ddx * dx + ddy * dy;
  if (!(b > 0.0)) return false;
  const double cc = ddx * dy - ddy * dx;
  const double c2 = cc * cc;
  if (!(c2 < sig2)) return false;
  s = b - sqrt_rn(sig2 - c2);
  if (s < 0.0) s = 0.0;
  return true;
}

// FP32 bracket [lo, hi] of the hit distance of candidate j (certain: j hits
// for sure, so hi bounds the first hit); false when j certainly misses
__device__ __forceinline__ bool iso_bracket(const Frame& f, const Geom& g, int j, int CPW, int gi,
                                            float X32, float Y32, float dx32, float dy32,
                                            float& lo, float& hi, bool& certain) {
  const float ex = __fsub_rn(f.a32[j * CPW + gi], X32);
  const float ey = __fsub_rn(f.b32[j * CPW + gi], Y32);
  const float b32 = __fadd_rn(__fmul_rn(ex, dx32), __fmul_rn(ey, dy32));
  const float e = g.iso_e;
  if (!(b32 > -e)) return false;
  const float c32 = __fsub_rn(__fmul_rn(ex, dy32), __fmul_rn(ey, dx32));
  const float ac = fabsf(c32);
  if (!(ac < __fadd_rn(g.iso_sig_hi, e))) return false;
  const float cl = fmaxf(__fsub_rn(ac, e), 0.0f), ch = __fadd_rn(ac, e);
  const float xhi = fmaxf(__fsub_rn(g.sig2f, __fmul_rn(cl, cl)), 0.0f);
  const float xlo = fmaxf(__fsub_rn(g.sig2f, __fmul_rn(ch, ch)), 0.0f);
  const float sq_hi = __fadd_rn(__fsqrt_rn(xhi), g.iso_sq);
  const float sq_lo = fmaxf(__fsub_rn(__fsqrt_rn(xlo), g.iso_sq), 0.0f);
  lo = __fsub_rn(__fsub_rn(__fsub_rn(b32, e), sq_hi), g.iso_r);
  hi = fmaxf(__fadd_rn(__fsub_rn(__fadd_rn(b32, e), sq_lo), g.iso_r), 0.0f);
  certain = __fsub_rn(b32, e) > 0.0f && __fadd_rn(ch, e) < g.iso_sig_lo;
  return true;
}

template <int TPC, bool SCREEN>
__device__ __forceinline__ void run_group_iso(const Frame& f, const int* hdr, void* hl,
                                              const Geom* __restrict__ rg,
                                              const SweepState* __restrict__ sts, int rep, int a,
                                              bool valid, int colour_index,
                                              double* __restrict__ px, double* __restrict__ py,
                                              CellStats* __restrict__ cs,
                                              ChainRec* __restrict__ recs, int rec_stride,
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
  const int lc = cy * g.cells_x + cx;
  const int c = g.cell_off + lc;
  const int64_t t = st->t;
  const double W = g.w, H = g.h, sig2 = g.sig2;
  const int nmem = valid ? hdr[CPW + gi] : 0;
  const int nobj = valid ? hdr[gi] : 0;
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  const unsigned FULL = 0xffffffffu;

  double sum_b = 0.0;
  int n_events = 0, n_lifts = 0, n_frozen = 0, n_walls = 0, n_fp64 = 0, n_chains = 0;
  int k = 0;
  bool active = false;
  int m = 0;
  double X = 0.0, Y = 0.0, dx = 1.0, dy = 0.0, r = 0.0;
  int64_t n_iter = 0;
  int ch_events = 0, ch_walls = 0, start_key = 0;
  bool done = (!valid) || nmem == 0;

  for (;;) {
    if (!done && !active) {
      if (k >= g.n_m) {
        done = true;
      } else {
        const U64x4 v = philox((uint64_t)t, kPurposeChain, (uint64_t)lc, (uint64_t)k, g.seed,
                               g.replica);
        int idx = (int)below_n(v.v[0], (uint64_t)nmem);
        if (g.list_mode == 1) {
          int* pl = (int*)hl;
          if (k == 0) shuffled_list(pl, CPW, gi, nmem, idx, t, lc, g.seed, g.replica);
          idx = pl[(k % nmem) * CPW + gi];
        }
        m = f.mrank[idx * CPW + gi];
        iso_direction(t, lc, k, g.seed, g.replica, dx, dy);
        X = f.a64[m * CPW + gi];
        Y = f.b64[m * CPW + gi];
        r = g.ell;
        f.touched[m * CPW + gi] = 1;
        start_key = f.key[m * CPW + gi];
        n_iter = 0;
        ch_events = 0;
        ch_walls = 0;
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

    // distances to the walls along d
    double swx = INF, swy = INF;
    if (dx > 0.0) swx = (W - X) / fabs(dx);
    else if (dx < 0.0) swx = X / fabs(dx);
    if (dy > 0.0) swy = (H - Y) / fabs(dy);
    else if (dy < 0.0) swy = Y / fabs(dy);
    if (swx < 0.0) swx = 0.0;
    if (swy < 0.0) swy = 0.0;
    const double swall = swx < swy ? swx : swy;

    // first contact along d
    double best_s = INF, best_b = 0.0;
    int best_key = INT_MAX, best_j = m;
    int nev = 0;
    auto consider = [&](int j) {
      double s, b;
      ++nev;
      if (iso_hit(f, j, CPW, gi, X, Y, dx, dy, sig2, s, b)) {
        const int kj = f.key[j * CPW + gi];
        if (better(s, kj, best_s, best_key)) {
          best_s = s;
          best_b = b;
          best_key = kj;
          best_j = j;
        }
      }
    };
    if (SCREEN) {
      // FP32 brackets; the candidates that can be the first hit go to FP64
      const float X32 = to_float_trunc(X), Y32 = to_float_trunc(Y);
      const float dx32 = __double2float_rn(dx), dy32 = __double2float_rn(dy);
      float U = __int_as_float(0x7f800000), L1 = U, L2 = U;
      int j1 = m;
      if (go) {
        for (int j = sub; j < nobj; j += TPC) {
          if (j == m) continue;
          float lo, hi;
          bool certain;
          if (!iso_bracket(f, g, j, CPW, gi, X32, Y32, dx32, dy32, lo, hi, certain)) continue;
          if (lo < L1) {
            L2 = L1;
            L1 = lo;
            j1 = j;
          } else if (lo < L2) {
            L2 = lo;
          }
          if (certain) U = fminf(U, hi);
        }
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
      const float Lam = fminf(U, to_float_up_nn(r < swall ? r : swall));
      const bool need = go && (L1 <= Lam);
      const bool multi = need && (L2 <= Lam);
      if (need && !multi && sub == 0) consider(j1);
      if (__any_sync(FULL, multi)) {
        if (multi) {
          for (int j = sub; j < nobj; j += TPC) {
            if (j == m) continue;
            float lo, hi;
            bool certain;
            if (!iso_bracket(f, g, j, CPW, gi, X32, Y32, dx32, dy32, lo, hi, certain)) continue;
            if (lo <= Lam) consider(j);
          }
        }
      }
    } else if (go) {
      for (int j = sub; j < nobj; j += TPC)
        if (j != m) consider(j);
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
    n_fp64 += go ? nev : 0;

    bool end_chain = capped;
    if (go) {
      if (r <= best_s && r <= swall) {
        // budget used up: the chain ends
        X = X + r * dx;
        Y = Y + r * dy;
        end_chain = true;
      } else if (best_s <= swall) {
        const double s = best_s;
        const double nX = X + s * dx, nY = Y + s * dy;
        r = r - s;
        sum_b += best_b - s;
        ++n_events;
        ++ch_events;
        ++n_iter;
        if (f.info[best_j * CPW + gi] >= 0) {
          // lift: the hit member moves on along d
          ++n_lifts;
          // the stopped disk, in FP64 and in the FP32 copy the screen reads
          f.a64[m * CPW + gi] = nX;
          f.b64[m * CPW + gi] = nY;
          f.a32[m * CPW + gi] = to_float_trunc(nX);
          f.b32[m * CPW + gi] = to_float_trunc(nY);
          m = best_j;
          X = f.a64[m * CPW + gi];
          Y = f.b64[m * CPW + gi];
          f.touched[m * CPW + gi] = 1;
        } else {
          // frozen disk: specular reflection about the line of centres
          ++n_frozen;
          const double nx = f.a64[best_j * CPW + gi] - nX;
          const double ny = f.b64[best_j * CPW + gi] - nY;
          const double nn = nx * nx + ny * ny;
          const double kk = 2.0 * (dx * nx + dy * ny) / nn;
          dx = dx - kk * nx;
          dy = dy - kk * ny;
          X = nX;
          Y = nY;
        }
      } else {
        // wall: onto the wall, flip the normal component(s)
        const double s = swall;
        const bool flip_x = swx == swall, flip_y = swy == swall;
        const double nX = flip_x ? (dx > 0.0 ? W : 0.0) : X + s * dx;
        const double nY = flip_y ? (dy > 0.0 ? H : 0.0) : Y + s * dy;
        X = nX;
        Y = nY;
        if (flip_x) dx = -dx;
        if (flip_y) dy = -dy;
        r = r - s;
        ++n_walls;
        ++ch_walls;
        ++n_iter;
      }
    }
    if (end_chain) {
      f.a64[m * CPW + gi] = X;
      f.b64[m * CPW + gi] = Y;
      f.a32[m * CPW + gi] = to_float_trunc(X);
      f.b32[m * CPW + gi] = to_float_trunc(Y);
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
  const double ox = st->sx + (double)cx * g.w;
  const double oy = st->sy + (double)cy * g.h;
  for (int q = sub; q < nmem; q += TPC) {
    const int j = f.mrank[q * CPW + gi];
    if (!f.touched[j * CPW + gi]) continue;
    const int slot = f.mslot[q * CPW + gi];
    px[slot] = wrap_box0(f.a64[j * CPW + gi] + ox, g.L);
    py[slot] = wrap_box0(f.b64[j * CPW + gi] + oy, g.L);
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
    s.replayed = 0;
    s.rejected = 0;
    cs[c] = s;
  }
}

}  // namespace ecmc
